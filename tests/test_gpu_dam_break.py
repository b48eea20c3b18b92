"""The dam break of Sec. 4.5 at the reduced-precision configuration's size
(4096 x 2048, density ratio 1000, viscosity ratio 100, a = 1024 square
water column at the left wall, gravity 1e-5, 90-degree walls), run until
the surge reaches the far wall.

Parameters: nu_B = 0.5, so nu_A = 0.05 and the heavy phase's viscous rate
s_g^{7,8} = 1/(3 nu_A + 1/2) = 1.54.  With nu_B = 0.1 (nu_A = 0.01,
s = 1.89) the scheme goes unstable at the surge front after about 8000
steps in FP64 and FP32 alike, and the FP64 oracle does the same on a reduced
case (the design notes give the sweep); the viscosity ratio the
configuration names is kept either way.

The front is measured two ways: the last phi = 1/2 crossing on the bottom
row (what the paper plots; an air film under the surge tip makes it lag)
and the last column holding at least one cell of water (sum over y of
phi >= 1), which follows the tip.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

NX, NY, A = 4096, 2048, 1024


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.mem_get_info()[0] < 8e9:
        pytest.skip("needs ~5 GB of device memory")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


def bottom_front(phi):
    row = phi[0]
    idx = np.nonzero(row >= 0.5)[0]
    i = int(idx.max())
    if i + 1 >= len(row):
        return float(i)
    a, b = row[i], row[i + 1]
    return i + (a - 0.5) / (a - b)


def tip(phi):
    col = phi.sum(axis=0)
    idx = np.nonzero(col >= 1.0)[0]
    i = int(idx.max())
    if i + 1 >= len(col):
        return float(i)
    a, b = col[i], col[i + 1]
    return i + (a - 1.0) / (a - b)


def _run(pk, prec, steps, every, n_delta=0.0):
    case = W.dam_break(nx=NX, ny=NY, col_w=A, col_h=A, nuB=0.5, precision=prec)
    prm = case.params.with_(diag_every=500, n_delta=n_delta)
    sim = pk.Simulation(prm)
    sim.init_fields(case.phi)
    s0 = sim.diag()["sum_phi"]
    rows = []
    while sim.t < steps:
        sim.step(every)  # LBM_EUNSTABLE (non-finite or |u| > 0.4) raises
        phi = sim.fields(pk.LBM_PHI)
        d = sim.diag()
        rows.append((sim.t, bottom_front(phi), tip(phi), d["umax"], (d["sum_phi"] - s0) / s0))
    sim.close()
    return rows


def test_surge_reaches_the_far_wall(pk, capsys):
    """FP64, FP32 and FP16 deviation storage run 24000 steps, until the
    surge tip is within about 130 cells of the far wall (x = 4096), with no
    instability.  Total phi: FP64 drifts by rounding only (about 1e-16 per
    step, bound 5e-12 over the run; measured 1.3e-12); FP32 and the 16-bit
    codec by FP32 rounding of the sums (bound 5e-4; measured 2.1e-4 in FP32).
    The FP32 tip follows FP64 to within 2 % of the distance run, the FP16
    one to within 5 %."""
    steps, every = 24000, 2000
    r64 = _run(pk, W.PREC_FP64, steps, every)
    r32 = _run(pk, W.PREC_FP32, steps, every)
    r16 = _run(pk, W.PREC_FP16_DEV, steps, every)
    with capsys.disabled():
        print("\n[dam break 4096x2048, a = 1024, nu_B = 0.5, g = 1e-5]  t: bottom-row front / tip, "
              "FP64 | FP32 | FP16 deviations")
        for a, b, c in zip(r64, r32, r16):
            print(f"  {a[0]:6d}: {a[1]:8.1f} / {a[2]:8.1f} | {b[1]:8.1f} / {b[2]:8.1f} | {c[1]:8.1f} / {c[2]:8.1f}"
                  f"   max|u| {a[3]:.3f}   phi drift {a[4]:+.1e} | {b[4]:+.1e} | {c[4]:+.1e}")
    assert r64[-1][2] > 3900 and r32[-1][2] > 3900 and r16[-1][2] > 3900
    assert max(abs(r[4]) for r in r64) <= 5e-12
    assert max(abs(r[4]) for r in r32) <= 5e-4
    assert max(abs(r[4]) for r in r16) <= 5e-4
    for a, b, c in zip(r64, r32, r16):
        assert abs(a[2] - b[2]) <= 0.02 * (a[2] - A) + 2.0, (a, b)
        assert abs(a[2] - c[2]) <= 0.05 * (a[2] - A) + 2.0, (a, c)


@pytest.mark.parametrize("n_delta", [0.0, 1e-5], ids=["default", "paper_normal"])
def test_front_after_4000_steps(pk, n_delta, capsys):
    """The front after 4000 steps (FP64) with the library's default
    regularisation of n and with the paper's normal (n_delta = 1e-5): the
    regularisation moves it by a small fraction of a cell."""
    r = _run(pk, W.PREC_FP64, 4000, 4000, n_delta=n_delta)[-1]
    with capsys.disabled():
        print(f"\n[dam break front, 4000 steps, n_delta {'default' if n_delta == 0 else n_delta}] "
              f"bottom row {r[1]:.3f}, tip {r[2]:.3f}")
    assert r[2] > A + 40
