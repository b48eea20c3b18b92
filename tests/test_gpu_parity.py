"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Grids span several x-strips and y-segments of the marching kernel and end in
ragged tails; cases cover periodic, wall and wetting boundaries, both phase
models, every gravity mode and both viscosity laws.  Tolerances (from the
method's specification): FP64 max |delta f|, |delta g| <= 1e-12 after 100
steps; FP32 max |delta| / max |ref| <= 1e-5 per population array; total phi
conserved to 1e-12 relative in FP64.
"""
import math

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


def _cmp_pops(pk, oracle_mod, sim, o, fp64):
    out = {}
    for which_g, which_o, name in ((pk.LBM_F_POP, oracle_mod.F_POP, "f"),
                                   (pk.LBM_G_POP, oracle_mod.G_POP, "g")):
        a = sim.fields(which_g)
        b = o.fields(which_o)
        assert np.isfinite(a).all()
        if fp64:
            err = np.abs(a - b).max()
            assert err <= 1e-12, (name, err)
        else:
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err <= 1e-5, (name, err)
        out[name] = err
    return out


CASES = {
    "periodic_ac": dict(walls="none"),
    "ywalls_wet_ac": dict(walls="y", theta=(90, 90, 50, 130), gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -2e-5)),
    "xwalls_wet_ac": dict(walls="x", theta=(40, 140, 90, 90), gravity=(W.GRAV_RHO, 1e-5, 0.0)),
    "allwalls_ac_inverse_nu": dict(walls="all", theta=(60, 120, 75, 105), gravity=(W.GRAV_RHO, 0.0, -1e-5),
                                   visc_law=W.VISC_INVERSE_NU),
    "periodic_ch": dict(walls="none", model=W.MODEL_CH),
    "allwalls_ch": dict(walls="all", model=W.MODEL_CH, theta=(70, 110, 80, 100), gravity=(W.GRAV_CONST, 1e-6, -1e-6)),
    "original_flux": dict(walls="y", flux=W.FLUX_ORIGINAL),
    "mrt_rates": dict(walls="none", s_f=(1.0, 1.2, 0.8, 0.9, 1.1, 0.9, 1.3, 1.0, 1.0),
                      s_g=(1.0, 1.1, 0.9, 1.0, 1.7, 1.0, 1.7, math.nan, math.nan)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_population_parity(pk, oracle_mod, name, prec):
    case = W.noisy_drop(300, 150, precision=prec, **CASES[name])
    sim, o = _both(pk, oracle_mod, case, 100)
    _cmp_pops(pk, oracle_mod, sim, o, prec == W.PREC_FP64)


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
    case = W.noisy_drop(200, 140, precision=prec, walls="y", theta=(90, 90, 45, 135),
                        gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -1e-5))
    sim, o = _both(pk, oracle_mod, case, 0)
    tol = 1e-13 if prec == W.PREC_FP64 else 2e-6
    for step in (0, 37):
        if step:
            sim.step(step)
            o.step(step)
        for wg, wo in ((pk.LBM_PHI, oracle_mod.PHI), (pk.LBM_UX, oracle_mod.UX),
                       (pk.LBM_UY, oracle_mod.UY), (pk.LBM_P, oracle_mod.P),
                       (pk.LBM_RHO, oracle_mod.RHO), (pk.LBM_MU, oracle_mod.MU),
                       (pk.LBM_MCX, oracle_mod.MCX), (pk.LBM_MCY, oracle_mod.MCY),
                       (pk.LBM_HIST, oracle_mod.HIST)):
            a, b = sim.fields(wg), o.fields(wo)
            scale = max(np.abs(b).max(), 1e-30)
            assert np.abs(a - b).max() <= tol * scale + 1e-300, (step, wg, np.abs(a - b).max() / scale)


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
    reproduces the window's interior exactly (up to rounding)."""
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        pytest.skip("needs ~50 GB of device memory")
    case = W.rti_multimode(n, precision=W.PREC_FP32)
    k = 8
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
        fo = o.fields(oracle_mod.F_POP)[sl]
        go = o.fields(oracle_mod.G_POP)[sl]
        for a, b in ((got[y0][0], fo), (got[y0][1], go)):
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err <= 1e-5, (y0, err)
