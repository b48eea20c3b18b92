"""Pins of the oracle's solid obstacles (half-way bounce-back at solid links,
neutral-wetting values of phi and mu_phi at solid nodes).

The paper states the wall treatment for plane walls only (Sec. 4, Eqs.
(49)-(50)); the obstacle rule is a reading.  It is pinned to the paper by
reduction: a frame of solid nodes around a periodic grid must reproduce the
walled box at theta = 90 degrees (bounce-back links, mirror ghosts, corner
rule, the diagnostics' boundary exclusion) node for node.  Around that:
conservation of phi, invariance of a fluid at rest, mirror symmetry of a
symmetric problem, and exactness of the fill on linear fields."""
import numpy as np
import pytest

import workloads as W

FIELDS_1 = ("PHI", "UX", "UY", "P", "RHO", "MU", "MCX", "MCY")


def _embed(case, walls):
    """The case's fields on a grid one node larger on each walled side, with
    the added nodes solid and every side periodic."""
    nx, ny = case.params.nx, case.params.ny
    ox, oy = (1, 1) if walls in ("x", "all") else (0, 0), (1, 1) if walls in ("y", "all") else (0, 0)
    NX, NY = nx + sum(ox), ny + sum(oy)
    solid = np.ones((NY, NX), dtype=bool)
    sl = (slice(oy[0], oy[0] + ny), slice(ox[0], ox[0] + nx))
    solid[sl] = False

    def emb(a, fill):
        if a is None:
            return None
        out = np.full((NY, NX), fill)
        out[sl] = a
        return out

    prm = case.params.with_(nx=NX, ny=NY, bc=(0, 0, 0, 0))
    big = W.Case("framed", prm, emb(case.phi, 0.3), emb(case.ux, 0.01), emb(case.uy, -0.02),
                 emb(case.p, 0.005), solid=solid)
    return big, sl


def _run(oracle_mod, case, steps):
    o = oracle_mod.Oracle(case.params)
    if case.solid is not None:
        o.set_solid(case.solid)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    o.step(steps)
    return o


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
@pytest.mark.parametrize("walls", ["y", "x", "all"])
def test_solid_frame_reproduces_neutral_walls(oracle_mod, model, walls):
    """Walls at theta = 90 degrees and a one-node solid frame on a periodic grid
    give the same populations, history and fields at every fluid node, and
    the same diagnostics (40 steps, noisy drop, gravity, rho ratio 10)."""
    g = (W.GRAV_RHO, 1e-5 if walls == "x" else 0.0, -1e-5 if walls != "x" else 0.0)
    case = W.noisy_drop(20, 16, model=model, walls=walls, gravity=g)
    big, sl = _embed(case, walls)
    steps = 40
    a = _run(oracle_mod, case, steps)
    b = _run(oracle_mod, big, steps)
    om = oracle_mod
    for which, name in ((om.F_POP, "f"), (om.G_POP, "g"), (om.HIST, "hist")):
        fa, fb = a.fields(which), b.fields(which)[(slice(None),) + sl]
        err = np.abs(fa - fb).max() / max(1.0, np.abs(fa).max())
        assert err <= 1e-12, (name, err)
    for name in FIELDS_1:
        fa, fb = a.fields(getattr(om, name)), b.fields(getattr(om, name))[sl]
        err = np.abs(fa - fb).max() / max(1.0, np.abs(fa).max())
        assert err <= 1e-12, (name, err)
        # solid nodes carry nothing
        frame = b.fields(getattr(om, name)).copy()
        frame[sl] = 0.0
        assert not frame.any(), name
    da, db = a.diag(), b.diag()
    assert db["n_avg"] == da["n_avg"] > 0
    for k in ("sum_phi", "Du_rms", "Sm_rms", "umax"):
        assert db[k] == pytest.approx(da[k], rel=1e-11, abs=1e-300), k


def _obstacles(nx, ny):
    m = W.trapezoid_mask(nx, ny, 0.5 * nx, 6.0, 4.0)
    m |= W.disc_mask(nx, ny, 0.25 * nx, 0.7 * ny, 3.0)
    m[ny // 2, (3 * nx) // 4] = True  # a single solid node
    return m


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
def test_fluid_at_rest_stays_at_rest(oracle_mod, model):
    """One phase at rest (phi = phi_A, u = 0, p = 0, no gravity) around
    obstacles: every bounced population meets its equal, so nothing moves."""
    nx, ny = 40, 30
    case = W.noisy_drop(nx, ny, model=model, walls="y", noise=0.0, u_amp=0.0)
    phiA = case.params.phiA
    rest = W.Case("rest", case.params, np.full((ny, nx), phiA), solid=_obstacles(nx, ny))
    o = oracle_mod.Oracle(rest.params)
    o.set_solid(rest.solid)
    o.init_fields(rest.phi)
    f0 = o.fields(oracle_mod.F_POP)
    o.step(60)
    assert np.abs(o.fields(oracle_mod.UX)).max() <= 1e-15
    assert np.abs(o.fields(oracle_mod.UY)).max() <= 1e-15
    assert np.abs(o.fields(oracle_mod.F_POP) - f0).max() <= 1e-15


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
def test_phi_conserved_with_obstacles(oracle_mod, model):
    """Sum of phi over the fluid nodes: bounce-back returns every population
    to the grid and the collision keeps each node's phi (Eq. (C.4))."""
    nx, ny = 40, 30
    case = W.noisy_drop(nx, ny, model=model, walls="all", theta=(60, 120, 45, 135),
                        gravity=(W.GRAV_RHO, 0.0, -2e-5))
    solid = _obstacles(nx, ny)
    o = oracle_mod.Oracle(case.params)
    o.set_solid(solid)
    o.init_fields(np.where(solid, 0.0, case.phi), case.ux, case.uy, case.p)
    s0 = o.diag()["sum_phi"]
    phi0 = o.fields(oracle_mod.PHI)
    assert s0 == pytest.approx(phi0[~solid].sum(), rel=1e-14)
    o.step(200)
    s1 = o.diag()["sum_phi"]
    assert abs(s1 - s0) <= 1e-13 * abs(s0)
    assert np.isfinite(o.fields(oracle_mod.PHI)).all()


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
def test_mirror_symmetric_problem_stays_symmetric(oracle_mod, model):
    """A problem symmetric under x -> nx - 1 - x (obstacles, drop, walls at
    equal angles, vertical gravity) keeps phi even and u odd in x: catches a
    swapped direction or an asymmetric fill."""
    nx, ny = 40, 32
    case = W.noisy_drop(nx, ny, model=model, walls="all", theta=(70, 70, 50, 130),
                        gravity=(W.GRAV_RHO, 0.0, -2e-5), noise=0.0, u_amp=0.0)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    prm = case.params
    r = np.sqrt((X - 0.5 * nx) ** 2 + (Y - 0.55 * ny) ** 2)
    phi = W.tanh_profile(8.0 - r, prm.width, prm.phiA, prm.phiB)
    solid = W.trapezoid_mask(nx, ny, 0.5 * nx, 7.0, 6.0)
    solid |= W.disc_mask(nx, ny, 8.5, 0.7 * ny, 2.5) | W.disc_mask(nx, ny, nx - 8.5, 0.7 * ny, 2.5)
    assert (solid == solid[:, ::-1]).all()
    o = oracle_mod.Oracle(prm)
    o.set_solid(solid)
    o.init_fields(phi)
    o.step(120)
    ph, ux, uy = (o.fields(w) for w in (oracle_mod.PHI, oracle_mod.UX, oracle_mod.UY))
    assert np.abs(ux).max() > 1e-7  # the flow is not trivial
    assert np.abs(ph - ph[:, ::-1]).max() <= 1e-13
    assert np.abs(ux + ux[:, ::-1]).max() <= 1e-15
    assert np.abs(uy - uy[:, ::-1]).max() <= 1e-15


def test_fill_is_exact_on_linear_fields(oracle_mod):
    """The padded phi seen by the stencils after lbm_init_fields: an isolated
    solid node inside a linear field shows the field's own value (the mean of
    opposite neighbours); on a 3 x 3 solid block an edge node shows its one
    fluid axis neighbour, a corner node the mean of its two, and the enclosed
    centre 0.  (A solid node with diagonal fluid neighbours only occurs at the
    corners of the solid frame in test_solid_frame_reproduces_neutral_walls.)"""
    nx, ny = 16, 12
    case = W.noisy_drop(nx, ny, walls="none")
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    lin = 0.3 + 0.02 * X - 0.015 * Y
    solid = np.zeros((ny, nx), dtype=bool)
    solid[5, 4] = True                   # isolated node
    solid[2:5, 9:12] = True              # 3 x 3 block: centre sees no fluid
    o = oracle_mod.Oracle(case.params)
    o.set_solid(solid)
    o.init_fields(np.where(solid, 7.0, lin))
    # the pad of the init's phase pass is overwritten by the history pass,
    # which sees phi = sum f (zero at solid nodes); both fill from fluid nodes
    pad = o.padded(0)
    phi = o.fields(oracle_mod.PHI)
    assert pad[5 + 1, 4 + 1] == pytest.approx(0.25 * (phi[5, 3] + phi[5, 5] + phi[4, 4] + phi[6, 4]), rel=1e-15)
    assert pad[5 + 1, 4 + 1] == pytest.approx(lin[5, 4], rel=1e-12)
    # block edge node (2, 10): one fluid axis neighbour (1, 10) below it
    assert pad[2 + 1, 10 + 1] == phi[1, 10]
    # block corner node (2, 9): fluid axis neighbours (1, 9) and (2, 8)
    assert pad[2 + 1, 9 + 1] == pytest.approx(0.5 * (phi[2, 8] + phi[1, 9]), rel=1e-15)
    # block centre (3, 10): no fluid neighbour at all -> 0
    assert pad[3 + 1, 10 + 1] == 0.0


def test_dam_break_obstacle_geometry():
    """The trapezoid of the last dam break (reading of Sec. 4.5's figure): on
    the bottom wall, centred at Lx/2, a/2 tall, a/2 wide at the top and 3a/2
    at the bottom (45-degree flanks), a = Lx/4; the water column a x a at the
    left, clear of it."""
    nx, ny = 400, 200
    case = W.dam_break_obstacle(nx=nx, ny=ny)
    a = nx // 4
    s = case.solid
    rows = np.nonzero(s.any(axis=1))[0]
    assert rows.min() == 0 and rows.max() == a // 2 - 1
    for j in (0, a // 4, a // 2 - 1):
        cols = np.nonzero(s[j])[0]
        y = j + 0.5
        half = 0.25 * a + (0.5 * a - y)  # top half-width a/4, slope 1
        assert cols.min() == int(np.ceil(0.5 * nx - half - 0.5))
        assert cols.max() == int(np.floor(0.5 * nx + half - 0.5))
        assert abs((cols.min() + cols.max() + 1) / 2 - 0.5 * nx) < 1e-9  # centred
    assert not (s & (case.phi > 0.5)).any()
    assert case.phi[: a - 8, : a - 8].min() > 0.99  # column interior is water
