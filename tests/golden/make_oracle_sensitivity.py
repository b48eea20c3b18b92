"""Writes oracle_sensitivity.txt: how far the oracle's own trajectory moves
when every step's populations and history are perturbed at the level of one
rounding of the arithmetic.

This calls only the oracle (and the seeded input generators): no value here
comes from the CUDA path.  It fixes the bars of the parity tests that run the
paper's workloads with a small regularisation of the interface normal
(Eq. (8), n = grad phi / |grad phi|).  There the scheme itself amplifies any
rounding difference: where lambda != 0 but grad phi is at rounding level, the
direction of n, and with it the flux lambda n of Eq. (7), is set by
rounding.  Two implementations of the same scheme that round differently
then part at the rate the scheme amplifies rounding, which this record
measures on the oracle alone.

Cases: the paper's six workloads at n_delta = 1e-5 and 1e-9, and the rough
stress cases (seeded noise on phi, u and p) at the default regularisation
(recorded with n_delta 0).

Model of a second implementation: after every step, each population f_i,
g_i (g_0 without the constant rho0) and each history value is multiplied by
(1 + eps xi), xi uniform in [-1, 1) from SplitMix64 (seed 7 + step), with
eps = 2^-53 (an FP64 implementation) or 2^-24 (FP32 storage).  Recorded per
case, n_delta and arithmetic, every 10 steps to 100: max |delta f| and
max |delta g| (FP64: absolute; FP32: relative to the array's maximum, the
form of the FP32 bar).  For the paper's workloads also "onestep": the
largest departure after a single step from the oracle's state at
t0 = 0, 25, 50, 75, 99 perturbed once in the same way.

Run: python tests/golden/make_oracle_sensitivity.py  (about a minute)
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_sensitivity.txt")
N_DELTAS = (1e-5, 1e-9)
EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


def trajectory(case, eps, steps=100, every=10):
    o = oracle.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    rho0 = case.params.rho0
    out = {}
    for t in range(1, steps + 1):
        o.step(1)
        if eps:
            n = case.params.nx * case.params.ny
            xi = 2.0 * W.uniform_array(7 + t, 23 * n) - 1.0
            f = o.fields(oracle.F_POP)
            g = o.fields(oracle.G_POP)
            h = o.fields(oracle.HIST)
            f *= 1.0 + eps * xi[: 9 * n].reshape(f.shape)
            g[0] -= rho0
            g *= 1.0 + eps * xi[9 * n: 18 * n].reshape(g.shape)
            g[0] += rho0
            h *= 1.0 + eps * xi[18 * n:].reshape(h.shape)
            o.set_fields(oracle.F_POP, f)
            o.set_fields(oracle.G_POP, g)
            o.set_fields(oracle.HIST, h)
        if t % every == 0:
            out[t] = (o.fields(oracle.F_POP), o.fields(oracle.G_POP))
    o.close()
    return out


ONE_STEP_TIMES = (0, 25, 50, 75, 99)


def one_step(case, eps):
    """max over t0 in ONE_STEP_TIMES of the oracle's departure after one step
    from its state at t0 perturbed once at one rounding (as above)."""
    o = oracle.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    rho0 = case.params.rho0
    n = case.params.nx * case.params.ny
    worst = [0.0, 0.0]
    t = 0
    for t0 in ONE_STEP_TIMES:
        o.step(t0 - t)
        t = t0
        f, g, h = o.fields(oracle.F_POP), o.fields(oracle.G_POP), o.fields(oracle.HIST)
        outs = []
        for e in (0.0, eps):
            xi = 2.0 * W.uniform_array(1000 + t0, 23 * n) - 1.0
            fp = f * (1.0 + e * xi[: 9 * n].reshape(f.shape))
            gp = g.copy()
            gp[0] -= rho0
            gp *= 1.0 + e * xi[9 * n: 18 * n].reshape(g.shape)
            gp[0] += rho0
            hp = h * (1.0 + e * xi[18 * n:].reshape(h.shape))
            q = oracle.Oracle(case.params)
            q.init_fields(case.phi, case.ux, case.uy, case.p)
            q.set_fields(oracle.F_POP, fp)
            q.set_fields(oracle.G_POP, gp)
            q.set_fields(oracle.HIST, hp)
            q.step(1)
            outs.append((q.fields(oracle.F_POP), q.fields(oracle.G_POP)))
            q.close()
        for k in range(2):
            d = np.abs(outs[1][k] - outs[0][k]).max()
            worst[k] = max(worst[k], d)
    o.close()
    return worst


def main():
    oracle.set_threads(os.cpu_count() or 1)
    lines = ["# Oracle response to per-step rounding-level perturbations (see make_oracle_sensitivity.py).",
             "# case n_delta arith step df dg   (fp64: absolute max; fp32: max relative to the array max)"]
    runs = [(name, nd, W.paper_parity_case(name, W.PREC_FP64, n_delta=nd))
            for name in W.PAPER_PARITY_CASES for nd in N_DELTAS]
    runs += [(name, 0.0, W.stress_case(name, W.PREC_FP64)) for name in W.STRESS_CASES]
    for name, nd, case in runs:
        ref = trajectory(case, 0.0)
        for arith, eps in EPS.items():
            per = trajectory(case, eps)
            for t in sorted(per):
                df = np.abs(per[t][0] - ref[t][0]).max()
                dg = np.abs(per[t][1] - ref[t][1]).max()
                if arith == "fp32":
                    df /= np.abs(ref[t][0]).max()
                    dg /= np.abs(ref[t][1]).max()
                lines.append(f"{name} {nd:g} {arith} {t} {df:.3e} {dg:.3e}")
            print(lines[-1], flush=True)
            if nd > 0:
                df, dg = one_step(case, eps)
                if arith == "fp32":
                    df /= np.abs(ref[100][0]).max()
                    dg /= np.abs(ref[100][1]).max()
                lines.append(f"{name} {nd:g} {arith} onestep {df:.3e} {dg:.3e}")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
