"""Physics of the CUDA path on the paper's benchmark where an analytic answer
exists: the layered Poiseuille flow at the density ratios of Table 2
(Sec. 4.2), run on the GPU to steady state in FP64."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


def _table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_layered_poiseuille.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return {int(r[0]): float(r[1]) for r in rows}


def poiseuille_err(pk, ratio, ny=100, W_=4.0, steps=170000, nu=0.1, G=1e-6):
    """Err_u (Eq. (47)) of the steady layered channel at the paper's grid
    height (ny = 100, W = 4, nu_A = nu_B = 0.1, M = 0.1, sigma = 1e-3) against
    the analytic profile of Eq. (46), and the ratio of the computed to the
    analytic peak speed.  The flow does not depend on x; 16 columns let the
    TMA step run it (segments of 8 rows, one launch per step)."""
    muA, muB = nu * ratio, nu
    case = W.layered_poiseuille(nx=16, ny=ny, rhoA=float(ratio), muA=muA, muB=muB, Gx=G, W=W_)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    sim.step(steps)
    u = sim.fields(pk.LBM_UX)[:, 1]
    ue = W.layered_poiseuille_exact(ny, W_, muA, muB, G)
    return float(np.abs(u - ue).sum() / np.abs(ue).sum()), float(u.max() / ue.max())


@pytest.mark.parametrize("ratio", [10, 1000])
def test_layered_poiseuille_density_ratios(pk, ratio):
    """The lowest and highest density ratios of Table 2 on the GPU, at the
    oracle's bars: Err_u below 10 x (ratio 10) and 2.5 x (ratio 1000) the
    table's value (the oracle measures 1.06e-2 and 1.03e-2), and the peak
    speed within 2 % of the analytic one."""
    err, peak = poiseuille_err(pk, ratio)
    assert np.isfinite(err)
    assert err < (10 if ratio == 10 else 2.5) * _table2()[ratio], (ratio, err)
    assert abs(peak - 1.0) < 0.02, (ratio, peak)
