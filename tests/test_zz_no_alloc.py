"""lbm_fields_noalloc: the population / history export that allocates no
device memory, for callers that cannot let the library allocate (with all
device memory reserved up front, or with the device full).  Its output must
equal what lbm_fields returns.

This file is collected last on purpose, and every test in it works both in
a fresh process and after the rest of the suite."""
import ctypes as C

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


def _noalloc(pk, sim, which, shape):
    out = np.empty(shape)
    rc = pk.load().lbm_fields_noalloc(sim.handle, which, out.ctypes.data_as(C.POINTER(C.c_double)))
    return rc, out


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_noalloc_export_matches_lbm_fields_twice(pk, prec):
    case = W.noisy_drop(200, 120, precision=prec, walls="y", theta=(90, 90, 60, 120),
                        noise=0.005, u_amp=0.002)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    for _ in range(2):  # two calls in a row, with steps in between
        sim.step(7)
        for which, planes in ((pk.LBM_F_POP, 9), (pk.LBM_G_POP, 9), (pk.LBM_HIST, 5)):
            bytes_before = sim.device_bytes
            rc, got = _noalloc(pk, sim, which, (planes, case.params.ny, case.params.nx))
            assert rc == pk.LBM_OK, pk.lbm_last_error(sim.handle)
            assert sim.device_bytes == bytes_before
            ref = sim.fields(which)
            assert np.array_equal(got, ref)
    sim.close()


def test_noalloc_rejects_large_grids_and_other_fields(pk):
    case = W.noisy_drop(1100, 1000, precision=W.PREC_FP32)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    rc, _ = _noalloc(pk, sim, pk.LBM_F_POP, (9, 1000, 1100))
    assert rc == pk.LBM_EINVAL
    assert "at most" in pk.lbm_last_error(sim.handle)
    sim.close()
    small = W.noisy_drop(64, 48, precision=W.PREC_FP32)
    sim = pk.Simulation(small.params)
    sim.init_fields(small.phi)
    rc, _ = _noalloc(pk, sim, pk.LBM_PHI, (48, 64))
    assert rc == pk.LBM_EINVAL
    sim.close()


def test_noalloc_refuses_a_call_from_another_device(pk):
    """The staging array's address is per device; a call made while a device
    other than the handle's is current is refused, not run against the other
    device's array."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second CUDA device")
    small = W.noisy_drop(64, 48, precision=W.PREC_FP32)
    with torch.cuda.device(0):
        sim = pk.Simulation(small.params)
        sim.init_fields(small.phi)
    with torch.cuda.device(1):
        rc, _ = _noalloc(pk, sim, pk.LBM_F_POP, (9, 48, 64))
    assert rc == pk.LBM_EINVAL
    assert "handle lives on device" in pk.lbm_last_error(sim.handle)
    with torch.cuda.device(0):
        rc, _ = _noalloc(pk, sim, pk.LBM_F_POP, (9, 48, 64))
        assert rc == pk.LBM_OK
        sim.close()
