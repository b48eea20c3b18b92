"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Grids span several x-strips and y-segments of the marching kernel and end in
ragged tails; cases cover periodic, wall and wetting boundaries, both phase
models, every gravity mode and both viscosity laws.  Tolerances (from the
method's specification): FP64 max |delta f|, |delta g| <= 1e-12 after 100
steps; FP32 max |delta| / max |ref| <= 1e-5 per population array; total phi
conserved to 1e-12 relative in FP64.  Every comparison prints its measured
error.
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


def _both(pk, oracle_mod, case, steps):
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    o = oracle_mod.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    if steps:
        sim.step(steps)
        o.step(steps)
    return sim, o


def rel_err(a, b, rho0=None):
    """max |a - b| / max |b|; with rho0 given, the constant rho0 of g_0 is
    taken out of both first (the dynamic part of g)."""
    if rho0 is not None:
        a = a.copy()
        b = b.copy()
        a[0] -= rho0
        b[0] -= rho0
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# FP32: the stated bar is max|delta| / max|ref| <= 1e-5 per population array
# (g as the scheme defines it, g_0 carrying rho0).  The dynamic part of g
# (rho0 removed) is printed beside it and held to TOL32_GDYN: it is driven by
# mu_phi grad phi, and mu_phi = psi'(phi) - k lap phi differences phi values
# that FP32 storage of the nine f_i rounds at ~5e-8, a ~1e-5 relative
# effect on mu (measured on GB300: at most 1.3e-5, the layered channel).
TOL32 = 1e-5
TOL32_GDYN = 5e-5


def _cmp_pops(pk, oracle_mod, sim, o, fp64, tol64=1e-12, tol32=(TOL32, TOL32), label=""):
    out = {}
    for k, (which_g, which_o, name) in enumerate(((pk.LBM_F_POP, oracle_mod.F_POP, "f"),
                                                  (pk.LBM_G_POP, oracle_mod.G_POP, "g"))):
        a = sim.fields(which_g)
        b = o.fields(which_o)
        assert np.isfinite(a).all()
        if fp64:
            err = np.abs(a - b).max()
            bar = tol64[k] if isinstance(tol64, tuple) else tol64
            print(f"\n[parity] {label} fp64 {name}: max|d| {err:.2e} (bar {bar:.1e})")
            assert err <= bar, (name, err, bar)
        else:
            err = rel_err(a, b)
            print(f"\n[parity] {label} fp32 {name}: max|d|/max|ref| {err:.2e} (bar {tol32[k]:.1e})", end="")
            assert err <= tol32[k], (name, err)
            if name == "g":
                e2 = rel_err(a, b, sim.params.rho0)
                print(f"; dynamic part of g {e2:.2e} (bar {TOL32_GDYN:.0e})", end="")
                assert e2 <= TOL32_GDYN, ("g dynamic part", e2)
        out[name] = err
    return out


# ---- the paper's workloads, small enough for the oracle, several tiles wide
@pytest.mark.parametrize("name", W.PAPER_PARITY_CASES)
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_paper_workload_parity(pk, oracle_mod, name, prec):
    """The stated bar on the paper's workloads (Sec. 4), 100 steps, with the
    library's default regularisation of n (the normal as the paper writes
    it is the subject of test_gpu_parity_paper_normal.py)."""
    case = W.paper_parity_case(name, prec)
    sim, o = _both(pk, oracle_mod, case, 100)
    _cmp_pops(pk, oracle_mod, sim, o, prec == W.PREC_FP64, label=name)


# ---- stress cases: rough seeded inputs, every boundary / model / rate path
SENSITIVITY = os.path.join(os.path.dirname(__file__), "golden", "oracle_sensitivity.txt")


def _stress_bars(name, prec):
    """Fixed bars of a stress case after 100 steps: the stated bar, or 10 x
    the oracle's own departure when every step is perturbed at one rounding
    of the arithmetic, where that is larger (tests/golden/oracle_sensitivity.txt,
    written from the oracle alone by make_oracle_sensitivity.py)."""
    arith = "fp64" if prec == W.PREC_FP64 else "fp32"
    stated = 1e-12 if prec == W.PREC_FP64 else TOL32
    with open(SENSITIVITY) as fh:
        for line in fh:
            f = line.split()
            if len(f) == 6 and f[0] == name and f[2] == arith and f[3] == "100":
                return (max(stated, 10.0 * float(f[4])), max(stated, 10.0 * float(f[5])))
    raise KeyError((name, arith))


@pytest.mark.parametrize("name", list(W.STRESS_CASES))
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_stress_parity(pk, oracle_mod, name, prec):
    """Rough inputs (seeded noise on phi, u, p) excite grid-scale dynamics
    that amplify any rounding difference.  The CUDA path must agree with the
    oracle within fixed bars: the stated one, or, where the case itself
    amplifies rounding more, 10x the oracle's own recorded response."""
    case = W.stress_case(name, prec)
    sim, o = _both(pk, oracle_mod, case, 100)
    bars = _stress_bars(name, prec)
    if prec == W.PREC_FP64:
        _cmp_pops(pk, oracle_mod, sim, o, True, tol64=bars, label=name)
    else:
        _cmp_pops(pk, oracle_mod, sim, o, False, tol32=bars, label=name)


@pytest.mark.parametrize("nx,ny", [(3, 3), (129, 65), (131, 130), (4, 256), (260, 66)])
@pytest.mark.parametrize("walls", ["none", "y", "all"])
@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
def test_edge_sizes(pk, oracle_mod, nx, ny, walls, model):
    """Smallest grid, a 1-column last strip, a 1-row and a 2-row last
    segment, the Poiseuille channel shape."""
    case = W.noisy_drop(nx, ny, precision=W.PREC_FP64, walls=walls, theta=(80, 100, 60, 120),
                        gravity=(W.GRAV_RHO, 1e-6, -1e-6), model=model)
    sim, o = _both(pk, oracle_mod, case, 30)
    _cmp_pops(pk, oracle_mod, sim, o, True)


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_macroscopic_fields_and_history(pk, oracle_mod, prec):
    case = W.noisy_drop(200, 140, precision=prec, walls="y", theta=(90, 90, 45, 135), noise=0.005,
                        u_amp=0.002, gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -1e-5))
    sim, o = _both(pk, oracle_mod, case, 0)
    P = case.params
    dphi = P.phiA - P.phiB
    beta = 12 * P.sigma / (P.width * dphi**4)
    # scales of the terms whose difference some fields are:
    # mu = psi'(phi) - k lap phi ~ beta dphi^3 ; m^{phi C} = -(drho/dphi) M (grad phi - lambda n)
    # with |grad phi| ~ dphi / W
    mu_scale = beta * dphi**3
    m_scale = abs(P.rhoA - P.rhoB) / dphi * P.mobility / P.width * dphi
    for step in (0, 37):
        if step:
            sim.step(step)
            o.step(step)
        umax = np.abs(o.fields(oracle_mod.UX)).max() + np.abs(o.fields(oracle_mod.UY)).max()
        for wg, wo in ((pk.LBM_PHI, oracle_mod.PHI), (pk.LBM_UX, oracle_mod.UX),
                       (pk.LBM_UY, oracle_mod.UY), (pk.LBM_P, oracle_mod.P),
                       (pk.LBM_RHO, oracle_mod.RHO), (pk.LBM_MU, oracle_mod.MU),
                       (pk.LBM_MCX, oracle_mod.MCX), (pk.LBM_MCY, oracle_mod.MCY),
                       (pk.LBM_HIST, oracle_mod.HIST)):
            a, b = sim.fields(wg), o.fields(wo)
            scale = np.abs(b).max()
            if wg == pk.LBM_MU:
                scale = max(scale, mu_scale)
            elif wg in (pk.LBM_MCX, pk.LBM_MCY):
                scale = max(scale, m_scale)
            if wg == pk.LBM_HIST:
                a, b = a.copy(), b.copy()
                a[2:] /= max(m_scale * umax, 1e-300)
                b[2:] /= max(m_scale * umax, 1e-300)
                a[:2] /= np.abs(b[:2]).max()
                b[:2] /= np.abs(b[:2]).max()
                scale = 1.0
            tol = 1e-12 if prec == W.PREC_FP64 else 1e-5
            err = np.abs(a - b).max() / scale
            print(f"\n[fields] step {step} field {wg}: {err:.2e} (bar {tol:.0e})", end="")
            assert err <= tol, (step, wg, err)


def test_total_phi_conservation_fp64(pk, oracle_mod):
    case = W.noisy_drop(256, 192, precision=W.PREC_FP64, walls="all", theta=(50, 130, 60, 120),
                        gravity=(W.GRAV_RHO, 0.0, -1e-5))
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    s0 = sim.fields(pk.LBM_PHI).sum()
    sim.step(500)
    s1 = sim.fields(pk.LBM_PHI).sum()
    assert abs(s1 - s0) <= 1e-12 * abs(s0)


def test_total_phi_drift_fp32_is_small(pk):
    case = W.noisy_drop(256, 192, precision=W.PREC_FP32, walls="y")
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    s0 = sim.diag()["sum_phi"]
    sim.step(500)
    s1 = sim.diag()["sum_phi"]
    assert abs(s1 - s0) <= 1e-5 * abs(s0)


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_diagnostics(pk, oracle_mod, prec):
    case = W.square_droplet(n=160, D=80, precision=prec, steps=60)
    case.params.diag_every = 20
    sim, o = _both(pk, oracle_mod, case, 60)
    a, b = sim.diag(), o.diag()
    assert a["t"] == b["t"] == 60
    assert a["n_avg"] == b["n_avg"]
    rt = 1e-11 if prec == W.PREC_FP64 else 1e-3
    assert a["sum_phi"] == pytest.approx(b["sum_phi"], rel=1e-12 if prec == W.PREC_FP64 else 1e-6)
    for k in ("Du_rms", "Sm_rms", "umax"):
        assert a[k] == pytest.approx(b[k], rel=rt), k


def test_set_fields_resume(pk, oracle_mod):
    """Populations and history written through lbm_set_fields continue
    exactly like the oracle's state."""
    case = W.noisy_drop(150, 100, precision=W.PREC_FP64, walls="y", theta=(90, 90, 70, 110))
    o = oracle_mod.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    o.step(13)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    sim.set_fields(pk.LBM_F_POP, o.fields(oracle_mod.F_POP))
    sim.set_fields(pk.LBM_G_POP, o.fields(oracle_mod.G_POP))
    sim.set_fields(pk.LBM_HIST, o.fields(oracle_mod.HIST))
    assert np.array_equal(sim.fields(pk.LBM_F_POP), o.fields(oracle_mod.F_POP))
    o.step(20)
    sim.step(20)
    _cmp_pops(pk, oracle_mod, sim, o, True)


def test_unstable_run_is_reported(pk):
    """A run driven far past the Mach limit returns LBM_EUNSTABLE at the
    next diagnostic point (no abort, handle still usable)."""
    case = W.noisy_drop(128, 64, precision=W.PREC_FP32, u_amp=0.0,
                        gravity=(W.GRAV_CONST, 0.05, 0.0))
    case.params.diag_every = 50
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    with pytest.raises(pk.LbmError) as ei:
        sim.step(5000)
    assert ei.value.code == pk.LBM_EUNSTABLE
    sim.init_fields(case.phi)  # still usable
    assert sim.t == 0


def _window(full_phi, y0, y1, x0, x1):
    return np.ascontiguousarray(full_phi[y0:y1, x0:x1])


@pytest.mark.parametrize("n", [16384])
def test_full_size_sampled_windows(pk, oracle_mod, n):
    """The throughput workload (RTI, n x n, FP32, the launch configuration the
    benchmark times), checked on sampled windows: after k steps a node depends
    only on nodes within 2k, so the oracle run on a window with a 2k margin
    reproduces the window's interior exactly (up to rounding).  k = 100
    steps, the horizon of the stated FP32 bar."""
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        pytest.skip("needs ~50 GB of device memory")
    case = W.rti_multimode(n, precision=W.PREC_FP32)
    k = 100
    m = 2 * k + 6
    wy = 48
    x0 = n // 3
    windows = (0, n // 2 - wy // 2, n - wy)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    sim.step(k)
    got = {y0: (sim.fields(pk.LBM_F_POP, region=(x0, y0, wy, wy)),
                sim.fields(pk.LBM_G_POP, region=(x0, y0, wy, wy))) for y0 in windows}
    sim.close()
    ref = {}
    for y0 in windows:
        ylo = max(0, y0 - m)
        yhi = min(n, y0 + wy + m)
        sub = case.params.with_(nx=wy + 2 * m, ny=yhi - ylo, bc=(0, 0, 1, 1))
        phi = _window(case.phi, ylo, yhi, x0 - m, x0 + wy + m)
        o = oracle_mod.Oracle(sub)
        o.init_fields(phi)
        o.step(k)
        iy0 = y0 - ylo
        sl = (slice(None), slice(iy0, iy0 + wy), slice(m, m + wy))
        ref[y0] = (o.fields(oracle_mod.F_POP)[sl], o.fields(oracle_mod.G_POP)[sl])
    # relative to the array maximum over the sampled windows (g_0 without rho0)
    rho0 = case.params.rho0
    gmax = max(np.abs(np.concatenate([ref[y][1][:1] - rho0, ref[y][1][1:]])).max() for y in windows)
    fmax = max(np.abs(ref[y][0]).max() for y in windows)
    for y0 in windows:
        fa, ga = got[y0]
        fo, go = ref[y0]
        ef = np.abs(fa - fo).max() / fmax
        eg = np.abs(ga - go).max() / gmax
        print(f"\n[full size {n}^2, {k} steps] window y0={y0}: f {ef:.2e} g {eg:.2e} (bar 1e-05)", end="")
        assert ef <= 1e-5, (y0, ef)
        assert eg <= 1e-5, (y0, eg)


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
@pytest.mark.parametrize("walls", ["none", "y", "x", "all"])
@pytest.mark.parametrize("nx,ny", [(300, 150), (16, 70), (257, 129), (129, 200)])
def test_tma_kernel_matches_register_kernel(pk, prec, walls, nx, ny, model):
    """The TMA-staged steps (Allen-Cahn and Cahn-Hilliard) and the
    register-pipelined step compute the same update from the same pulled
    values (the TMA kernels relax the unit-rate moments as m^eq + m_src/2
    instead of m + (m^eq - m) + m_src/2).  After one step they agree to
    rounding, after 20 steps to the parity bar.  129 columns leave a last
    strip of one column; 200 rows several segments and a ragged one."""
    case = W.noisy_drop(nx, ny, precision=prec, walls=walls, noise=0.005, u_amp=0.002, model=model,
                        theta=(60, 120, 45, 135), gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    sims = []
    for flags in (0, pk.LBM_FLAG_NO_TMA):
        sim = pk.Simulation(case.params.with_(flags=flags))
        sim.init_fields(case.phi, case.ux, case.uy, case.p)
        sims.append(sim)
    for steps, tol in ((1, 1e-14 if prec == W.PREC_FP64 else 1e-6), (19, 1e-12 if prec == W.PREC_FP64 else 1e-5)):
        for sim in sims:
            sim.step(steps)
        for which in (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST):
            a, b = sims[0].fields(which), sims[1].fields(which)
            d = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
            assert d <= tol, (steps, which, d, int((a != b).sum()))
