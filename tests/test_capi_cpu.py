"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point its header declares, and rejects bad parameters
with an error code and a message instead of aborting."""
import ctypes as C
import math
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pk():
    from paper_2111_00847_gb300 import build

    build.build()
    import paper_2111_00847_gb300 as pk

    pk.load()
    return pk


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "pflbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_fields", "lbm_destroy",
                     "lbm_last_error", "lbm_set_fields", "lbm_fields_region"):
        assert required in names


def test_library_exports_every_declared_symbol(pk):
    lib = pk.load()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding exposes the same names
    for n in _declared_functions():
        assert hasattr(pk, n), n


def test_params_struct_layout(pk):
    """The ctypes image matches the C layout (int32 block, then doubles)."""
    s = pk.LbmParams
    assert s.phiA.offset == 14 * 4
    assert C.sizeof(s) == 14 * 4 + 36 * 8
    assert s.n_delta.offset == 14 * 4 + 35 * 8


def _bad(prm_kw):
    prm = W.Params(nx=16, ny=16)
    for k, v in prm_kw.items():
        setattr(prm, k, v)
    return prm


@pytest.mark.parametrize("kw,code", [
    (dict(nx=2), -1), (dict(ny=0), -1), (dict(phiA=0.0), -1), (dict(rhoA=-1.0), -1),
    (dict(bc=(1, 0, 0, 0)), -1), (dict(theta_deg=(90, 90, 200, 90)), -1),
    (dict(s_f=(1.0, 1.0, 1.0, 2.5, 1, 1, 1, 1, 1)), -1), (dict(width=0.5), -1),
    (dict(precision=7), -1), (dict(flux_model=W.FLUX_CORRECTED), -5),
    (dict(phase_model=7), -1), (dict(nx=70000, ny=70000), -1), (dict(flags=8), -1),
    (dict(n_delta=-1e-3), -1),
    (dict(precision=W.PREC_FP16_DEV, rhoA=3e8), -1), (dict(precision=W.PREC_FP16_DEV, phiA=1e-4, phiB=0.0), -1),
])
def test_create_rejects_bad_parameters(pk, kw, code):
    with pytest.raises(pk.LbmError) as ei:
        pk.lbm_create(pk.params_struct(_bad(kw)))
    assert ei.value.code == code
    assert pk.lbm_last_error()


def test_null_handle_calls_fail_cleanly(pk):
    lib = pk.load()
    assert lib.lbm_step(None, 1) == pk.LBM_EINVAL
    assert lib.lbm_init_fields(None, None, None, None, None) == pk.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    lib.lbm_destroy(None)


def test_create_without_device_reports_ecuda(pk):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(pk.LbmError) as ei:
        pk.lbm_create(pk.params_struct(W.Params(nx=16, ny=16)))
    assert ei.value.code == pk.LBM_ECUDA


def test_allocator_hook_validation(pk):
    a = pk.LbmAllocator()
    with pytest.raises(pk.LbmError) as ei:
        pk.lbm_create(pk.params_struct(W.Params(nx=16, ny=16)), 0, a)
    assert ei.value.code == pk.LBM_EINVAL


def test_nan_rates_mean_default_rule():
    prm = W.Params(nx=8, ny=8)
    assert all(math.isnan(v) for v in prm.s_f)
