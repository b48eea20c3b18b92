"""The failure path of the step kernels, exercised without a fault: one
bounded device wait on a barrier that nothing arrives on gives up, the
handle's device flag reports it at the next synchronising call as
LBM_ECUDA, and the handle and its state stay usable."""
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


def test_bounded_wait_timeout_is_reported_and_the_handle_recovers(pk):
    case = W.noisy_drop(64, 48, precision=W.PREC_FP32, walls="y")
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    sim.step(5)
    f5 = sim.fields(pk.LBM_F_POP)
    pk.lbm_selftest_wait_timeout(sim.handle)
    with pytest.raises(pk.LbmError) as ei:
        sim.fields(pk.LBM_PHI)
    assert ei.value.code == pk.LBM_ECUDA
    assert "gave up waiting" in str(ei.value)
    # reported once, state untouched, stepping continues as before
    assert np.array_equal(sim.fields(pk.LBM_F_POP), f5)
    ref = pk.Simulation(case.params)
    ref.init_fields(case.phi, case.ux, case.uy, case.p)
    ref.step(10)
    sim.step(5)
    assert np.array_equal(sim.fields(pk.LBM_F_POP), ref.fields(pk.LBM_F_POP))
