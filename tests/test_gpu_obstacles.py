"""Solid obstacles on the GPU (lbm_set_solid) against the FP64 CPU oracle.

The obstacle path runs as separate passes (phi, neutral-wetting fill, mu_phi
for Cahn-Hilliard, node update), so it is checked like the fused step:
populations, history and fields after 100 steps of seeded cases spanning
several 128-column blocks with ragged tails, at the tolerances of the fused
path (FP64 1e-12 absolute on populations, FP32 1e-5 relative per array,
16-bit storage in units of its roundoff).  Two checks need no oracle: a
frame of solid nodes reproduces the walled box computed by the fused TMA
kernels, and total phi is conserved.  The dam break over the obstacle at the
size the benchmark times is checked on sampled windows."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

U16 = {W.PREC_FP16_DEV: 2.0 ** -11, W.PREC_BF16_DEV: 2.0 ** -8}


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


def obstacles(nx, ny):
    """A trapezoid on the bottom, a disc, a single solid node, a block on the
    left side and a thin plate across a 128-column block boundary."""
    m = W.trapezoid_mask(nx, ny, 0.5 * nx, 0.2 * ny, 0.1 * nx)
    m |= W.disc_mask(nx, ny, 0.3 * nx, 0.7 * ny, 0.08 * ny)
    m[ny // 2, (3 * nx) // 4] = True
    m[ny // 3: ny // 3 + 6, 0:5] = True
    m[(4 * ny) // 5, 120:140] = True
    return m


def _pair(pk, oracle_mod, case, solid, steps, oracle_prec=W.PREC_FP64):
    # diagnostics due at the last step, so that both sides hold phi(t-1) for S_m
    prm = case.params.with_(diag_every=steps)
    sim = pk.Simulation(prm)
    sim.set_solid(solid)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    o = oracle_mod.Oracle(prm.with_(precision=oracle_prec))
    o.set_solid(solid)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    sim.step(steps)
    o.step(steps)
    return sim, o


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


FIELDS = (("LBM_PHI", "PHI"), ("LBM_UX", "UX"), ("LBM_UY", "UY"), ("LBM_P", "P"), ("LBM_MU", "MU"),
          ("LBM_MCX", "MCX"), ("LBM_MCY", "MCY"))


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("walls", ["none", "y", "all"])
def test_obstacle_parity(pk, oracle_mod, model, prec, walls):
    nx, ny = 300, 150
    case = W.noisy_drop(nx, ny, precision=prec, model=model, walls=walls, theta=(60, 120, 45, 135),
                        gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    solid = obstacles(nx, ny)
    sim, o = _pair(pk, oracle_mod, case, solid, 100)
    fp64 = prec == W.PREC_FP64
    for wg, wo, name in ((pk.LBM_F_POP, oracle_mod.F_POP, "f"), (pk.LBM_G_POP, oracle_mod.G_POP, "g"),
                         (pk.LBM_HIST, oracle_mod.HIST, "hist")):
        a, b = sim.fields(wg), o.fields(wo)
        assert np.isfinite(a).all()
        assert not a[:, solid].any(), name  # nothing at solid nodes
        if fp64:
            assert np.abs(a - b).max() <= 1e-12, (name, np.abs(a - b).max())
        else:
            assert rel(a, b) <= 1e-5, (name, rel(a, b))
    for gname, oname in FIELDS:
        a, b = sim.fields(getattr(pk, gname)), o.fields(getattr(oracle_mod, oname))
        assert not a[solid].any(), gname
        if fp64:
            assert np.abs(a - b).max() <= 1e-11 * max(1.0, np.abs(b).max()), (gname, np.abs(a - b).max())
        elif gname == "LBM_PHI":
            assert rel(a, b) <= 1e-5, (gname, rel(a, b))
    da, db = sim.diag(), o.diag()
    assert da["n_avg"] == db["n_avg"]
    # FP32: the drift bar of the fused FP32 path, 1e-5 of the phi mass scale
    scale = np.abs(o.fields(oracle_mod.PHI)).sum()
    assert abs(da["sum_phi"] - db["sum_phi"]) <= (1e-12 if fp64 else 1e-5) * scale
    if fp64:
        for k in ("Du_rms", "Sm_rms", "umax"):
            assert da[k] == pytest.approx(db[k], rel=1e-9), k


@pytest.mark.parametrize("prec", [W.PREC_FP16_DEV, W.PREC_BF16_DEV], ids=["fp16dev", "bf16dev"])
@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
def test_obstacle_parity_16bit(pk, oracle_mod, prec, model):
    """16-bit deviation storage with obstacles, at the bounds of the fused
    16-bit path: f <= 0.2 u, g <= 8 u (dynamic part 16 u), u the unit roundoff."""
    nx, ny = 300, 150
    case = W.noisy_drop(nx, ny, precision=prec, model=model, walls="all", theta=(60, 120, 45, 135),
                        gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    solid = obstacles(nx, ny)
    sim, o = _pair(pk, oracle_mod, case, solid, 100)
    u = U16[prec]
    f, F = sim.fields(pk.LBM_F_POP), o.fields(oracle_mod.F_POP)
    g, G = sim.fields(pk.LBM_G_POP), o.fields(oracle_mod.G_POP)
    assert not f[:, solid].any() and not g[:, solid].any()
    assert rel(f, F) <= 0.2 * u, rel(f, F) / u
    assert rel(g, G) <= 8 * u, rel(g, G) / u
    gd, Gd = g.copy(), G.copy()
    gd[0][~solid] -= case.params.rho0
    Gd[0][~solid] -= case.params.rho0
    assert rel(gd, Gd) <= 16 * u, rel(gd, Gd) / u


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32], ids=["fp64", "fp32"])
def test_dam_break_over_obstacle(pk, oracle_mod, prec):
    """The paper's last case at 400 x 200 (a = 100): water column, trapezoid of
    height a/2 at Lx/2, walls on all sides, rho ratio 1000, 100 steps."""
    case = W.dam_break_obstacle(nx=400, ny=200, precision=prec)
    sim, o = _pair(pk, oracle_mod, case, case.solid, 100)
    for wg, wo in ((pk.LBM_F_POP, oracle_mod.F_POP), (pk.LBM_G_POP, oracle_mod.G_POP)):
        a, b = sim.fields(wg), o.fields(wo)
        if prec == W.PREC_FP64:
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
        else:
            assert rel(a, b) <= 1e-5
    s0 = o.diag()["sum_phi"]
    scale = np.abs(o.fields(oracle_mod.PHI)).sum()
    assert abs(sim.diag()["sum_phi"] - s0) <= (1e-12 if prec == W.PREC_FP64 else 1e-5) * scale


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
@pytest.mark.parametrize("walls", ["y", "x", "all"])
def test_solid_frame_matches_fused_walls(pk, model, walls):
    """A one-node solid frame on a periodic grid (obstacle passes) and the
    walled box at 90 degrees (fused TMA kernels): same populations at every
    fluid node after 60 steps, FP64, 300 x 150 fluid nodes."""
    nx, ny = 300, 150
    case = W.noisy_drop(nx, ny, precision=W.PREC_FP64, model=model, walls=walls,
                        gravity=(W.GRAV_RHO, 1e-6 if walls == "x" else 0.0, 0.0 if walls == "x" else -1e-5))
    ox = 1 if walls in ("x", "all") else 0
    oy = 1 if walls in ("y", "all") else 0
    NX, NY = nx + 2 * ox, ny + 2 * oy
    sl = (slice(oy, oy + ny), slice(ox, ox + nx))
    solid = np.ones((NY, NX), dtype=bool)
    solid[sl] = False

    def emb(a):
        out = np.zeros((NY, NX))
        out[sl] = a
        return out

    a = pk.Simulation(case.params)
    a.init_fields(case.phi, case.ux, case.uy, case.p)
    b = pk.Simulation(case.params.with_(nx=NX, ny=NY, bc=(0, 0, 0, 0)))
    b.set_solid(solid)
    b.init_fields(emb(case.phi), emb(case.ux), emb(case.uy), emb(case.p))
    a.step(60)
    b.step(60)
    for which in (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST):
        fa, fb = a.fields(which), b.fields(which)[(slice(None),) + sl]
        assert np.abs(fa - fb).max() <= 1e-12 * max(1.0, np.abs(fa).max()), which


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32, W.PREC_FP16_DEV], ids=["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("walls", ["none", "y", "x", "all"])
@pytest.mark.parametrize("nx,ny", [(300, 150), (16, 70), (257, 129), (129, 200)])
def test_tma_obstacle_step_matches_passes(pk, prec, walls, nx, ny, model):
    """The step with obstacles on the TMA kernels (phi, and mu_phi for
    Cahn-Hilliard, from the filled planes; link words in the staged pulls)
    and on the one-thread-per-node passes (LBM_FLAG_NO_TMA): rounding-level
    agreement after one step, the parity bar after 20.  129 columns leave a one-column last strip, 200 rows
    several segments and a ragged one; the obstacles touch strip and segment
    boundaries and the walls."""
    case = W.noisy_drop(nx, ny, precision=prec, walls=walls, noise=0.005, u_amp=0.002, model=model,
                        theta=(60, 120, 45, 135), gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    solid = obstacles(nx, ny)
    solid[:, min(nx - 1, 128)] |= np.arange(ny) % 7 == 0  # dots on a strip boundary
    solid[min(ny - 1, 64), :] |= np.arange(nx) % 5 == 0   # and on a segment boundary
    sims = []
    for flags in (0, pk.LBM_FLAG_NO_TMA):
        sim = pk.Simulation(case.params.with_(flags=flags))
        sim.set_solid(solid)
        sim.init_fields(case.phi, case.ux, case.uy, case.p)
        sims.append(sim)
    # 16-bit storage: the bars of the fused kernels' A/B test, 0.05 u and 0.2 u
    # on the populations (a rounding difference can move a deviation by one
    # 16-bit step)
    lowp = prec == W.PREC_FP16_DEV
    u = U16[W.PREC_FP16_DEV]
    tol1 = {W.PREC_FP64: 1e-14, W.PREC_FP32: 1e-6, W.PREC_FP16_DEV: 0.05 * u}[prec]
    tol20 = {W.PREC_FP64: 1e-12, W.PREC_FP32: 1e-5, W.PREC_FP16_DEV: 0.2 * u}[prec]
    for steps, tol in ((1, tol1), (19, tol20)):
        for sim in sims:
            sim.step(steps)
        for which in ((pk.LBM_F_POP, pk.LBM_G_POP) if lowp else (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST)):
            a, b = sims[0].fields(which), sims[1].fields(which)
            d = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
            assert d <= tol, (steps, which, d)


def test_obstacles_can_be_removed_and_adjoint_refuses(pk):
    nx, ny = 64, 48
    case = W.noisy_drop(nx, ny, precision=W.PREC_FP64, walls="y")
    sim = pk.Simulation(case.params)
    sim.set_solid(obstacles(nx, ny))
    sim.init_fields(case.phi)
    with pytest.raises(pk.LbmError) as ei:
        sim.adjoint_seed(np.ones((ny, nx)))
    assert ei.value.code == pk.LBM_EUNSUPPORTED
    sim.set_solid(None)  # back to the fused kernels
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    ref = pk.Simulation(case.params)
    ref.init_fields(case.phi, case.ux, case.uy, case.p)
    sim.step(10)
    ref.step(10)
    assert np.array_equal(sim.fields(pk.LBM_F_POP), ref.fields(pk.LBM_F_POP))
    sim.set_solid(np.zeros((ny, nx), dtype=np.uint8))  # all fluid: no obstacles
    sim.step(1)


def test_full_size_dam_break_obstacle_windows(pk, oracle_mod):
    """The obstacle workload at the benchmark's size and launch configuration
    (4096 x 2048, FP32), checked on sampled windows after k steps: a node
    depends only on nodes within 2k (3k for the fill), so the oracle on the
    window plus a margin reproduces the window (walls at the real sides,
    artificial walls beyond the margin elsewhere)."""
    case = W.dam_break_obstacle(nx=4096, ny=2048, precision=W.PREC_FP32)
    nx, ny = case.params.nx, case.params.ny
    a = nx // 4
    k = 8
    m = 3 * k + 6
    wsz = 48
    # left foot of the trapezoid, its top-left corner, the water column's corner
    windows = ((nx // 2 - (3 * a) // 4 - wsz // 2, 0), (nx // 2 - a // 4 - wsz // 2, a // 2 - wsz // 2),
               (a - wsz // 2, a - wsz // 2))
    sim = pk.Simulation(case.params)
    sim.set_solid(case.solid)
    sim.init_fields(case.phi)
    sim.step(k)
    got = {w: sim.fields(pk.LBM_F_POP, region=(w[0], w[1], wsz, wsz)) for w in windows}
    gotg = {w: sim.fields(pk.LBM_G_POP, region=(w[0], w[1], wsz, wsz)) for w in windows}
    sim.close()
    for (x0, y0) in windows:
        xlo, xhi = max(0, x0 - m), min(nx, x0 + wsz + m)
        ylo, yhi = max(0, y0 - m), min(ny, y0 + wsz + m)
        sub = case.params.with_(nx=xhi - xlo, ny=yhi - ylo, precision=W.PREC_FP64)
        o = oracle_mod.Oracle(sub)
        o.set_solid(case.solid[ylo:yhi, xlo:xhi])
        o.init_fields(np.ascontiguousarray(case.phi[ylo:yhi, xlo:xhi]))
        o.step(k)
        sl = (slice(None), slice(y0 - ylo, y0 - ylo + wsz), slice(x0 - xlo, x0 - xlo + wsz))
        fo, go = o.fields(oracle_mod.F_POP)[sl], o.fields(oracle_mod.G_POP)[sl]
        assert rel(got[(x0, y0)], fo) <= 1e-5, ((x0, y0), rel(got[(x0, y0)], fo))
        assert rel(gotg[(x0, y0)], go) <= 1e-5, ((x0, y0), rel(gotg[(x0, y0)], go))


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP16_DEV], ids=["fp64", "fp16dev"])
def test_set_fields_round_trip_with_obstacles(pk, oracle_mod, prec):
    """Populations written with lbm_set_fields (the inverse pull, with the
    reflecting links of the mask) come back from lbm_fields and
    lbm_fields_noalloc: exactly for FP64 storage, within the 16-bit rounding
    of the deviations otherwise; zero at solid nodes."""
    nx, ny = 200, 150
    case = W.noisy_drop(nx, ny, precision=W.PREC_FP64, walls="all", theta=(60, 120, 45, 135))
    solid = obstacles(nx, ny)
    o = oracle_mod.Oracle(case.params)
    o.set_solid(solid)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    o.step(10)
    sim = pk.Simulation(case.params.with_(precision=prec))
    sim.set_solid(solid)
    sim.init_fields(case.phi)
    for which, ow in ((pk.LBM_F_POP, oracle_mod.F_POP), (pk.LBM_G_POP, oracle_mod.G_POP)):
        a = o.fields(ow)
        sim.set_fields(which, a)
        b = sim.fields(which)
        c = np.empty_like(b)
        pk.lbm_fields_noalloc(sim.handle, which, c)
        assert np.array_equal(b, c)
        assert not b[:, solid].any()
        if prec == W.PREC_FP64:
            assert np.array_equal(b[:, ~solid], a[:, ~solid])
        else:
            assert rel(b, a) <= 0.05 * U16[prec], rel(b, a)
