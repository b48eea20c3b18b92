"""Pins of the oracle's whole time step against what the paper and the
mathematics fix: conservation (Eq. (16a) under periodic / no-flux
boundaries), consistency of reduction (Sec. 2), symmetry of the lattice
scheme, the analytic layered-Poiseuille profile (Sec. 4.2, Eq. (46)), the
contact angle of a spreading drop (Sec. 4.3, Eq. (52), Table 3), the Laplace
law implied by the surface force mu_phi grad phi with Eq. (3), and the
direction of Table 1 (S_m^rms of the present model below the original)."""
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _run(o_mod, case, steps):
    o = o_mod.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    if steps:
        o.step(steps)
    return o


@pytest.mark.parametrize("walls,model", [("none", W.MODEL_AC), ("y", W.MODEL_AC),
                                         ("all", W.MODEL_AC), ("none", W.MODEL_CH),
                                         ("all", W.MODEL_CH)])
def test_total_phi_conserved(oracle_mod, walls, model):
    c = W.noisy_drop(24, 20, walls=walls, model=model, theta=(60, 120, 45, 135),
                     gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    o = _run(oracle_mod, c, 0)
    s0 = o.fields(oracle_mod.PHI).sum()
    o.step(300)
    phi = o.fields(oracle_mod.PHI)
    assert np.isfinite(phi).all()
    assert abs(phi.sum() - s0) <= 1e-12 * np.abs(c.phi).sum()


def test_first_step_has_zero_time_derivatives(oracle_mod):
    """The history is initialised to the values the scheme computes at t = 0."""
    c = W.noisy_drop(16, 12)
    o = _run(oracle_mod, c, 0)
    h = o.fields(oracle_mod.HIST)
    u = o.fields(oracle_mod.UX)
    v = o.fields(oracle_mod.UY)
    phi = o.fields(oracle_mod.PHI)
    mx = o.fields(oracle_mod.MCX)
    my = o.fields(oracle_mod.MCY)
    assert np.allclose(h[0], phi * u, atol=1e-16, rtol=1e-14)
    assert np.allclose(h[1], phi * v, atol=1e-16, rtol=1e-14)
    assert np.allclose(h[2], u * mx + v * my, atol=1e-18, rtol=1e-12)
    assert np.allclose(h[3], u * mx - v * my, atol=1e-18, rtol=1e-12)
    assert np.allclose(h[4], u * my + v * mx, atol=1e-18, rtol=1e-12)


def test_consistency_of_reduction(oracle_mod):
    """rho_A = rho_B: m^{phi C} vanishes, so the present and original models
    are the same computation (bit for bit), Sec. 2."""
    c = W.noisy_drop(20, 16, rho_ratio=1.0)
    a = _run(oracle_mod, c, 40)
    c2 = W.noisy_drop(20, 16, rho_ratio=1.0, flux=W.FLUX_ORIGINAL)
    b = _run(oracle_mod, c2, 40)
    assert np.array_equal(a.fields(oracle_mod.F_POP), b.fields(oracle_mod.F_POP))
    assert np.array_equal(a.fields(oracle_mod.G_POP), b.fields(oracle_mod.G_POP))
    # but with a density contrast they differ
    c3 = W.noisy_drop(20, 16, rho_ratio=5.0)
    c4 = W.noisy_drop(20, 16, rho_ratio=5.0, flux=W.FLUX_ORIGINAL)
    assert not np.array_equal(_run(oracle_mod, c3, 5).fields(oracle_mod.G_POP),
                              _run(oracle_mod, c4, 5).fields(oracle_mod.G_POP))


def _transpose_case(c):
    """Swap x and y: fields transposed, u <-> v, gravity and sides swapped."""
    p = c.params
    bc = (p.bc[2], p.bc[3], p.bc[0], p.bc[1])
    th = (p.theta_deg[2], p.theta_deg[3], p.theta_deg[0], p.theta_deg[1])
    q = p.with_(nx=p.ny, ny=p.nx, bc=bc, theta_deg=th, gx=p.gy, gy=p.gx)
    return W.Case(c.name + "_T", q, c.phi.T.copy(), c.uy.T.copy(), c.ux.T.copy(), c.p.T.copy())


@pytest.mark.parametrize("walls,model", [("y", W.MODEL_AC), ("none", W.MODEL_CH)])
def test_transpose_symmetry(oracle_mod, walls, model):
    """With s^3 = s^5, s^4 = s^6 and s^7 = s^8 the scheme commutes with the
    exchange of x and y; catches any transposed index or swapped component."""
    c = W.noisy_drop(18, 14, walls=walls, model=model, theta=(70, 80, 50, 130),
                     gravity=(W.GRAV_RHO_MINUS_MEAN, 2e-6, -3e-6))
    a = _run(oracle_mod, c, 30)
    b = _run(oracle_mod, _transpose_case(c), 30)
    for fa, fb in ((oracle_mod.PHI, oracle_mod.PHI), (oracle_mod.P, oracle_mod.P),
                   (oracle_mod.UX, oracle_mod.UY), (oracle_mod.UY, oracle_mod.UX)):
        A = a.fields(fa)
        B = b.fields(fb).T
        assert np.allclose(A, B, atol=1e-13 * max(1.0, np.abs(A).max()), rtol=0), (fa, fb)


def test_mirror_symmetry(oracle_mod):
    """x -> nx-1-x with u -> -u maps solutions to solutions (catches a sign
    slip in any c_x term)."""
    c = W.noisy_drop(18, 14, walls="x", theta=(60, 110, 90, 90), gravity=(W.GRAV_RHO, 1e-6, -2e-6))
    a = _run(oracle_mod, c, 30)
    p = c.params
    q = p.with_(theta_deg=(p.theta_deg[1], p.theta_deg[0], p.theta_deg[2], p.theta_deg[3]), gx=-p.gx)
    m = W.Case("mirror", q, c.phi[:, ::-1].copy(), -c.ux[:, ::-1].copy(), c.uy[:, ::-1].copy(),
               c.p[:, ::-1].copy())
    b = _run(oracle_mod, m, 30)
    assert np.allclose(a.fields(oracle_mod.PHI), b.fields(oracle_mod.PHI)[:, ::-1], atol=1e-13)
    assert np.allclose(a.fields(oracle_mod.UX), -b.fields(oracle_mod.UX)[:, ::-1], atol=1e-15)
    assert np.allclose(a.fields(oracle_mod.UY), b.fields(oracle_mod.UY)[:, ::-1], atol=1e-15)


def test_single_phase_poiseuille(oracle_mod):
    """Uniform fluid in a channel with half-way bounce-back walls: the
    parabola u = G y (H - y) / (2 mu)."""
    ny, G, mu = 32, 1e-6, 0.1
    prm = W.Params(nx=3, ny=ny, bc=(0, 0, 1, 1), rhoA=1, rhoB=1, muA=mu, muB=mu,
                   gravity_mode=W.GRAV_CONST, gx=G, sigma=0.0)
    o = oracle_mod.Oracle(prm)
    o.init_fields(np.ones((ny, 3)))
    o.step(20000)
    u = o.fields(oracle_mod.UX)[:, 1]
    y = np.arange(ny) + 0.5
    ue = G / (2 * mu) * y * (ny - y)
    assert np.abs(u - ue).max() <= 1e-3 * ue.max()


def test_shear_wave_decays_at_the_viscous_rate_with_zero_divergence(oracle_mod):
    """A single-phase shear wave u = A sin(k y) x (periodic, nu = 0.1): its
    amplitude decays as exp(-nu k^2 t) (the unsteady momentum balance and the
    viscous rate s_g^{7,8} = 1/(nu/c_s^2 + 1/2) of Sec. 4; measured rate
    within 0.1 % of nu k^2), and D_u^rms of Eq. (42), the rms of tr S from
    Eq. (35), stays at the second-order level of a divergence-free flow
    (measured 4e-9 against A k = 1e-4): the trace of the local strain rate
    takes no part of the shear stress."""
    nx, ny, A, nu = 8, 64, 1e-3, 0.1
    prm = W.Params(nx=nx, ny=ny, rhoA=1.0, rhoB=1.0, muA=nu, muB=nu, sigma=0.0)
    k = 2.0 * np.pi / ny
    y = np.arange(ny) + 0.5
    ux = np.tile((A * np.sin(k * y))[:, None], (1, nx))
    o = oracle_mod.Oracle(prm)
    o.init_fields(np.ones((ny, nx)), ux, None, None)
    o.step(5)
    a5 = np.abs(o.fields(oracle_mod.UX)).max()
    o.step(45)
    a50 = np.abs(o.fields(oracle_mod.UX)).max()
    rate = np.log(a5 / a50) / 45.0
    assert rate == pytest.approx(nu * k * k, rel=1e-3), (rate, nu * k * k)
    assert o.diag()["Du_rms"] < 1e-3 * A * k


def _poiseuille_err(oracle_mod, ny, W_, rhoA, muA, muB, steps):
    c = W.layered_poiseuille(nx=3, ny=ny, rhoA=rhoA, muA=muA, muB=muB, Gx=1e-6, W=W_)
    o = _run(oracle_mod, c, steps)
    u = o.fields(oracle_mod.UX)[:, 1]
    ue = W.layered_poiseuille_exact(ny, W_, muA, muB, 1e-6)
    return np.abs(u - ue).sum() / np.abs(ue).sum()


@pytest.mark.slow
def test_layered_poiseuille_converges_to_analytic(oracle_mod):
    """Err_u (Eq. (47)) against Eq. (46) at the paper's grid (ny = 100, W = 4,
    nu_A = nu_B = 0.1, density ratio 10) is of the order of Table 2, and it
    falls at second order when the interface is resolved by twice as many
    nodes (W = 8): by a factor above 3.3 (order > 1.7; measured 1.06e-2 ->
    2.77e-3, order 1.94)."""
    table = {int(r[0]): float(r[1]) for r in _golden("table2_layered_poiseuille.txt")}
    e4 = _poiseuille_err(oracle_mod, 100, 4.0, 10.0, 1.0, 0.1, 170000)
    e8 = _poiseuille_err(oracle_mod, 100, 8.0, 10.0, 1.0, 0.1, 170000)
    assert e4 < 10 * table[10], e4
    assert e8 < 0.3 * e4, (e4, e8)


@pytest.mark.slow
@pytest.mark.parametrize("ratio", [100, 150, 1000])
def test_layered_poiseuille_table2_density_ratios(oracle_mod, ratio):
    """The high density ratios of Table 2 (nu_A = nu_B = 0.1, so the dynamic
    viscosity ratio equals the density ratio): Err_u within 2.5 x the
    table's value (measured 1.27e-2, 8.99e-3, 1.03e-2 against 6.57e-3,
    7.16e-3, 8.37e-3).  The error does not grow with the ratio: a mistake
    that leaves O(grad rho) terms in the recovered stress, or a sharpening
    flux that widens the interface tails (a tail of 1e-3 in phi doubles the
    light phase's viscosity at ratio 1000), fails at ratio 1000."""
    table = {int(r[0]): float(r[1]) for r in _golden("table2_layered_poiseuille.txt")}
    e = _poiseuille_err(oracle_mod, 100, 4.0, float(ratio), 0.1 * ratio, 0.1, 170000)
    assert e < 2.5 * table[ratio], (ratio, e, e / table[ratio])


def _crossings(row, x):
    s = row - 0.5
    idx = np.where(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    return [x[i] + (0.5 - row[i]) / (row[i + 1] - row[i]) * (x[i + 1] - x[i]) for i in idx]


def contact_angle(phi):
    """theta = 2 arctan(2H/L) (Sec. 4.3): H on the centre column, L from the
    phi = 1/2 crossings of the two rows next to the wall, extrapolated to it."""
    ny, nx = phi.shape
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    c0, c1 = _crossings(phi[0], x), _crossings(phi[1], x)
    L0, L1 = c0[-1] - c0[0], c1[-1] - c1[0]
    L = L0 + 0.5 * (L0 - L1)
    H = _crossings(phi[:, nx // 2], y)[0]
    return H, L, math.degrees(2 * math.atan(2 * H / L))


# Drop radius, grid and steps per angle: the 30 degree drop spreads to a chord
# of 67 nodes and takes longer to settle; at 150 degrees the chord is short,
# and half a node of error in L moves theta by about 2.5 degrees at R0 = 16,
# so the drop is twice as large.
CONTACT_CASES = {30.0: (16, 160, 48, 30000), 45.0: (16, 96, 48, 12000), 60.0: (16, 96, 48, 12000),
                 90.0: (16, 96, 48, 12000), 120.0: (16, 96, 48, 12000), 150.0: (32, 128, 96, 20000)}


@pytest.mark.slow
@pytest.mark.parametrize("theta", sorted(CONTACT_CASES))
def test_contact_angle(oracle_mod, theta):
    """Every angle of Table 3: the angle from theta = 2 arctan(2H/L) within
    1.5 degrees (or twice the paper's own deviation), and H, L within 5 % of
    the circular-cap values of Eq. (52)."""
    table = {float(r[0]): float(r[1]) for r in _golden("table3_contact_angle.txt")}
    paper_dev = abs(table[theta] - theta)
    R0, nx, ny, steps = CONTACT_CASES[theta]
    c = W.droplet_spreading(nx=nx, ny=ny, R0=R0, theta=theta, rhoA=10, muA=1.0, muB=0.1,
                            W=4.0, mobility=0.1, sigma=0.05, precision=W.PREC_FP64)
    o = _run(oracle_mod, c, steps)
    H, L, th = contact_angle(o.fields(oracle_mod.PHI))
    assert abs(th - theta) <= max(1.5, 2 * paper_dev), (th, H, L)
    He, Le, _ = W.spreading_exact(R0, theta)
    assert abs(H - He) < 0.05 * He and abs(L - Le) < 0.05 * Le


@pytest.mark.slow
@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
def test_laplace_law(oracle_mod, model):
    """p_in - p_out = sigma / R for a 2-D drop (surface force mu grad phi with
    beta, k of Eq. (3)), with either phase field; W = 4 resolves it to better
    than 10 % (Cahn-Hilliard measured 0.992 and 0.984 at R = 12, 16)."""
    res = []
    for R in (12.0, 16.0):
        c = W.static_drop(64, R, rho_ratio=10.0, model=model)
        o = _run(oracle_mod, c, 8000)
        p = o.fields(oracle_mod.P)
        dp = p[30:34, 30:34].mean() - p[:3, :3].mean()
        res.append(dp * R / c.params.sigma)
        assert o.diag()["umax"] < 1e-4
    for r in res:
        assert 0.85 < r < 1.1, res
    assert abs(res[0] - res[1]) < 0.1, res


def test_square_droplet_statistics(oracle_mod):
    """Table 1's direction, on the model Table 1 uses (Cahn-Hilliard,
    phi in [-1, 1]): once the drop has relaxed, the consistent flux gives a
    smaller S_m^rms than the original model (m = rho u), while D_u^rms is the
    same for both (the velocity fields agree to leading order)."""
    rows = {r[0]: [float(x) for x in r[1:]] for r in _golden("table1_square_droplet.txt")}
    assert rows["Sm_rms"][2] < rows["Sm_rms"][0]
    out = {}
    for flux in (W.FLUX_PRESENT, W.FLUX_ORIGINAL):
        c = W.square_droplet(n=48, D=24, steps=3000)
        c.params.flux_model = flux
        c.params.phase_model = W.MODEL_CH
        c.params.phiA, c.params.phiB = 1.0, -1.0
        c.phi = 2.0 * c.phi - 1.0
        o = _run(oracle_mod, c, 3000)
        out[flux] = o.diag()
    assert out[W.FLUX_PRESENT]["Sm_rms"] < 0.8 * out[W.FLUX_ORIGINAL]["Sm_rms"], out
    assert out[W.FLUX_PRESENT]["Du_rms"] == pytest.approx(out[W.FLUX_ORIGINAL]["Du_rms"], rel=0.2)
    assert out[W.FLUX_PRESENT]["Du_rms"] < 1e-5


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
def test_flat_interface_is_stationary(oracle_mod, model):
    """A flat tanh interface is the equilibrium of both phase-field models
    (for CH, mu_phi = 0 exactly on it; for AC, grad phi = lambda n): it stays
    within O(dx^2) of its start and drives only round-off-level flow."""
    c = W.flat_interface(4, 48, model=model)
    o = _run(oracle_mod, c, 2000)
    phi = o.fields(oracle_mod.PHI)
    dphi = c.params.phiA - c.params.phiB
    assert np.abs(phi - c.phi).max() < 0.02 * dphi
    assert np.abs(o.fields(oracle_mod.UX)).max() < 1e-10
    assert np.abs(o.fields(oracle_mod.UY)).max() < 1e-5


def test_diagnostics_vanish_for_fluid_at_rest(oracle_mod):
    """Eqs. (42)-(43): a uniform fluid at rest has div u = 0 and
    d rho/dt + div m^CC = 0, so D_u^rms and S_m^rms are zero; Sum phi is the
    node count times phi."""
    for walls in ("none", "all"):
        bc = (0, 0, 0, 0) if walls == "none" else (1, 1, 1, 1)
        prm = W.Params(nx=20, ny=16, bc=bc, rhoA=5.0, rhoB=1.0, muA=0.5, muB=0.1, diag_every=5)
        o = oracle_mod.Oracle(prm)
        o.init_fields(np.full((16, 20), 0.3))
        o.step(10)
        d = o.diag()
        assert d["Du_rms"] < 1e-15 and d["Sm_rms"] < 1e-15, d
        assert d["umax"] < 1e-15
        assert d["sum_phi"] == pytest.approx(0.3 * 320, rel=1e-14)
        assert d["n_avg"] == (320 if walls == "none" else 18 * 14)
