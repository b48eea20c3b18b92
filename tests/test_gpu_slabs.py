"""y-slab decomposition (lbm_create_slab, lbm_slab_pack / unpack) on one GPU:
slabs of one grid, exchanging their halos by device-to-device copies after
every step, reproduce the undivided grid's own rows bit for bit.

The update of a node reads only neighbours (the streaming of Eqs. (17) and
(40) and the stencils of Eqs. (C.9)-(C.10)), so with the neighbours'
boundary rows in the ghost rows each own row performs exactly the
arithmetic of the undivided grid.  Cases: wetting walls at the outer faces
(contact angles other than 90 degrees, where the wall ghost of Eq. (50)
enters), periodic y with three slabs, Cahn-Hilliard, FP64 and FP32.
"""
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


CASES = {
    "ywalls_wet_ac": dict(walls="y", theta=(90, 90, 50, 130), gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -2e-5)),
    "allwalls_ac": dict(walls="all", theta=(60, 120, 75, 105), gravity=(W.GRAV_RHO, 0.0, -1e-5),
                        visc_law=W.VISC_INVERSE_NU),
    "periodic_ac": dict(walls="none"),
    "ywalls_ch": dict(walls="y", model=W.MODEL_CH, theta=(90, 90, 70, 110), gravity=(W.GRAV_CONST, 1e-6, -1e-6)),
    "periodic_ch": dict(walls="none", model=W.MODEL_CH),
}


def _run(pk, case, parts, steps):
    from paper_2111_00847_gb300 import slabs

    prm = case.params
    periodic = prm.bc[2] == W.BC_PERIODIC
    sims = []
    for y_lo, own in slabs.partition(prm.ny, parts):
        s = pk.Simulation(prm, slab=(y_lo, own))
        s.init_fields(*(slabs.local_field(a, s) for a in (case.phi, case.ux, case.uy, case.p)))
        sims.append(s)
    bufs = slabs.exchange_local(sims, periodic)
    for _ in range(steps):
        for s in sims:
            s.step(1)
        slabs.exchange_local(sims, periodic, bufs)
    return sims


def _own(sim, which):
    y_lo, own, glo, ghi = sim.slab
    return sim.fields(which)[..., glo:glo + own, :]


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,parts", [("ywalls_wet_ac", 2), ("allwalls_ac", 3), ("periodic_ac", 3),
                                        ("ywalls_ch", 2), ("periodic_ch", 2)])
def test_slabs_reproduce_the_undivided_grid(pk, name, parts, prec):
    case = W.noisy_drop(300, 150, precision=prec, noise=0.005, u_amp=0.002, **CASES[name])
    steps = 60
    case.params.diag_every = steps  # both record phi(t-1) at the last step, for S_m
    ref = pk.Simulation(case.params)
    ref.init_fields(case.phi, case.ux, case.uy, case.p)
    ref.step(steps)
    sims = _run(pk, case, parts, steps)
    worst = 0.0
    for which in (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST):
        full = ref.fields(which)
        got = np.concatenate([_own(s, which) for s in sims], axis=-2)
        d = np.abs(got - full).max()
        worst = max(worst, d)
        assert np.array_equal(got, full), (which, d)
    print(f"\n[slabs] {name} x{parts} {'fp64' if prec == W.PREC_FP64 else 'fp32'}: {steps} steps, "
          f"max |slabs - undivided| = {worst:.1e} (bit for bit)")
    # diagnostics: the slabs' records combine to the undivided grid's
    from paper_2111_00847_gb300 import slabs

    d_ref = ref.diag()
    d = slabs.combine_diag([s.diag() for s in sims])
    assert d["n_avg"] == d_ref["n_avg"]
    for k in ("sum_phi", "Du_rms", "Sm_rms", "umax"):
        assert d[k] == pytest.approx(d_ref[k], rel=1e-12, abs=1e-300), k
    for s in sims:
        s.close()
    ref.close()


def test_slab_rules(pk):
    case = W.noisy_drop(64, 48, precision=W.PREC_FP32, walls="y")
    s = pk.Simulation(case.params, slab=(0, 24))
    assert s.slab == (0, 24, 0, pk.LBM_SLAB_GHOST)  # the bottom side is the global wall
    assert s.ny == 24 + pk.LBM_SLAB_GHOST
    with pytest.raises(pk.LbmError) as ei:
        s.step(2)
    assert ei.value.code == pk.LBM_EINVAL
    with pytest.raises(pk.LbmError) as ei:
        s.set_solid(np.ones((s.ny, 64), dtype=np.uint8))
    assert ei.value.code == pk.LBM_EUNSUPPORTED
    import torch

    buf = torch.empty(s.halo_bytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(pk.LbmError) as ei:
        s.pack(pk.LBM_BOTTOM, buf)  # a wall: nothing to exchange
    assert ei.value.code == pk.LBM_EINVAL
    s.pack(pk.LBM_TOP, buf)
    s.close()
    with pytest.raises(pk.LbmError):
        pk.Simulation(case.params, slab=(0, 2))  # fewer own rows than ghost rows
