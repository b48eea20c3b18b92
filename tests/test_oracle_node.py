"""Pins of the oracle's node-level pieces against what the paper fixes.

The oracle forms its equilibria and forcing directly as the moment vectors of
App. C (Eqs. (C.2)-(C.4)).  These tests rebuild the same quantities in
velocity space from the *other* printed forms (Eqs. (19)-(21) with M_2F of
Eq. (34) in the second way of Remark 1) and from the moment conditions of
Eq. (28), then project them with the oracle's M; a dropped term, a wrong sign
or a transposed index in either form breaks the agreement.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat(oracle_mod):
    cx, cy, w = oracle_mod.lattice()
    M, Mi = oracle_mod.moment_matrix()
    return cx, cy, w, M, Mi


def test_lattice_isotropy(lat):
    cx, cy, w, M, Mi = lat
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs((w * cx).sum()) < 1e-15 and abs((w * cy).sum()) < 1e-15
    assert abs((w * cx * cx).sum() - CS2) < 1e-15
    assert abs((w * cy * cy).sum() - CS2) < 1e-15
    assert abs((w * cx * cy).sum()) < 1e-15
    # fourth-order isotropy: sum w c_a c_b c_c c_d = cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    assert abs((w * cx**4).sum() - 3 * CS2**2) < 1e-15
    assert abs((w * cx**2 * cy**2).sum() - CS2**2) < 1e-15
    # opposite directions pair up
    for i in range(9):
        j = [k for k in range(9) if cx[k] == -cx[i] and cy[k] == -cy[i]]
        assert len(j) == 1


def test_moment_matrix_structure_and_inverse(lat):
    cx, cy, w, M, Mi = lat
    assert np.allclose(M @ Mi, np.eye(9), atol=1e-15, rtol=0)
    assert np.allclose(Mi @ M, np.eye(9), atol=1e-15, rtol=0)
    # rows are the D2Q9 moment basis in the order of Eq. (C.1):
    # density, energy, energy square, j_x, q_x, j_y, q_y, p_xx, p_xy
    c2 = cx**2 + cy**2
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[1], 3 * c2 - 4)
    assert np.array_equal(M[2], (9 * c2**2 - 21 * c2 + 8) // 2)
    assert np.array_equal(M[3], cx)
    assert np.array_equal(M[4], (3 * c2 - 5) * cx)
    assert np.array_equal(M[5], cy)
    assert np.array_equal(M[6], (3 * c2 - 5) * cy)
    assert np.array_equal(M[7], cx**2 - cy**2)
    assert np.array_equal(M[8], cx * cy)
    # mutually orthogonal rows
    G = M @ M.T
    assert np.allclose(G - np.diag(np.diag(G)), 0)


def _random_node(rng, model):
    v = dict(phi=rng.uniform(0.05, 0.95), mu=rng.normal(0, 1e-3), u=rng.normal(0, 0.05),
             v=rng.normal(0, 0.05), p=rng.normal(0, 1e-3), rho=rng.uniform(1, 50),
             mcx=rng.normal(0, 0.01), mcy=rng.normal(0, 0.01), Fx=rng.normal(0, 1e-4),
             Fy=rng.normal(0, 1e-4), drx=rng.normal(0, 0.5), dry=rng.normal(0, 0.5),
             lam=rng.uniform(0, 0.25), dphiu=rng.normal(0, 1e-4), dphiv=rng.normal(0, 1e-4),
             dum=rng.normal(0, 1e-5), dA=rng.normal(0, 1e-5), dB=rng.normal(0, 1e-5))
    ang = rng.uniform(0, 2 * math.pi)
    v["nx"], v["ny"] = math.cos(ang), math.sin(ang)
    return v


def _velocity_space_g(v, prm, cx, cy, w):
    """g^eq (Eqs. (19)-(20)) and F_i (Eq. (21)) with M_2F of Eq. (34), way 2."""
    u = np.array([v["u"], v["v"]])
    m = np.array([v["mcx"], v["mcy"]])
    rho, p = v["rho"], v["p"]
    # rho u u + m u  (the tensor (m u)_ab = m_a u_b)
    T = rho * np.outer(u, u) + np.outer(m, u)
    gr = np.array([v["drx"], v["dry"]])
    F = np.array([v["Fx"], v["Fy"]])
    ugr = u @ gr
    # d/dt (m u) from the three histories: d(u.m), d(u mx - v my), d(u my + v mx)
    dxx = 0.5 * (v["dum"] + v["dA"])  # d(mx u)
    dyy = 0.5 * (v["dum"] - v["dA"])  # d(my v)
    dsym = 0.5 * v["dB"]  # symmetric part of d(mx v), d(my u)
    dTm = np.array([[dxx, dsym], [dsym, dyy]])
    M2F = (np.outer(u, F) + np.outer(F, u) + dTm
           + CS2 * (np.outer(u, gr) + np.outer(u, gr).T) + CS2 * ugr * np.eye(2))
    geq = np.empty(9)
    Fi = np.empty(9)
    for i in range(9):
        c = np.array([cx[i], cy[i]], dtype=float)
        Q = np.outer(c, c) - CS2 * np.eye(2)
        alpha = ((w[0] - 1.0) * p / CS2 + prm.rho0) if i == 0 else w[i] * p / CS2
        s = w[i] * (c @ (rho * u) / CS2 + np.sum(T * Q) / (2 * CS2**2))
        geq[i] = alpha + s
        Fi[i] = w[i] * (ugr + c @ F / CS2 + np.sum((M2F - CS2 * ugr * np.eye(2)) * Q) / (2 * CS2**2))
    return geq, Fi, M2F


@pytest.mark.parametrize("seed", range(6))
def test_hydrodynamic_moments_match_velocity_space(oracle_mod, lat, seed):
    cx, cy, w, M, Mi = lat
    rng = np.random.default_rng(seed)
    prm = W.Params(nx=8, ny=8, rho0=rng.uniform(0.5, 2.0))
    v = _random_node(rng, W.MODEL_AC)
    mfeq, mR, mgeq, mF = oracle_mod.node_moments(prm, **v)
    geq, Fi, M2F = _velocity_space_g(v, prm, cx, cy, w)
    assert np.allclose(M @ geq, mgeq, atol=1e-14, rtol=1e-13)
    assert np.allclose(M @ Fi, mF, atol=1e-14, rtol=1e-13)
    # moment conditions of Eq. (28b)-(28c)
    u = np.array([v["u"], v["v"]])
    m = np.array([v["mcx"], v["mcy"]])
    g = Mi @ mgeq
    Fv = Mi @ mF
    C = np.stack([cx, cy]).astype(float)
    assert abs(g.sum() - prm.rho0) < 1e-14
    assert np.allclose(C @ g, v["rho"] * u, atol=1e-14)
    Pi = np.einsum("ai,bi,i->ab", C, C, g)
    T = v["rho"] * np.outer(u, u) + np.outer(m, u)
    assert np.allclose(Pi, 0.5 * (T + T.T) + v["p"] * np.eye(2), atol=1e-14)
    assert abs(Fv.sum() - u @ np.array([v["drx"], v["dry"]])) < 1e-14
    assert np.allclose(C @ Fv, [v["Fx"], v["Fy"]], atol=1e-15)
    assert np.allclose(np.einsum("ai,bi,i->ab", C, C, Fv), M2F, atol=1e-14)


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH])
@pytest.mark.parametrize("seed", range(4))
def test_phase_field_moments(oracle_mod, lat, model, seed):
    """f^eq carries phi, phi u and c_s^2 eta chi I (chi = phi for AC, mu for CH),
    and the source R_i has zero mass and first moment lambda c_s^2 n + d(phi u)/dt
    (AC) or d(phi u)/dt (CH), as Eqs. (C.3)-(C.4) imply with c = 1."""
    cx, cy, w, M, Mi = lat
    rng = np.random.default_rng(100 + seed)
    eta = rng.uniform(0.5, 2.0)
    prm = W.Params(nx=8, ny=8, phase_model=model, eta=eta)
    v = _random_node(rng, model)
    mfeq, mR, mgeq, mF = oracle_mod.node_moments(prm, **v)
    f = Mi @ mfeq
    R = Mi @ mR
    C = np.stack([cx, cy]).astype(float)
    chi = v["phi"] if model == W.MODEL_AC else v["mu"]
    assert abs(f.sum() - v["phi"]) < 1e-15
    assert np.allclose(C @ f, [v["phi"] * v["u"], v["phi"] * v["v"]], atol=1e-15)
    assert np.allclose(np.einsum("ai,bi,i->ab", C, C, f), CS2 * eta * chi * np.eye(2), atol=1e-15)
    X = np.array([v["dphiu"], v["dphiv"]])
    if model == W.MODEL_AC:
        X = X + CS2 * v["lam"] * np.array([v["nx"], v["ny"]])
    assert abs(R.sum()) < 1e-16
    assert np.allclose(C @ R, X, atol=1e-16)
    # the source is first-order only: it equals w_i c_i . X / c_s^2
    Rv = np.array([w[i] * (cx[i] * X[0] + cy[i] * X[1]) / CS2 for i in range(9)])
    assert np.allclose(R, Rv, atol=1e-16)


def test_stencils_exact_on_quadratics(oracle_mod):
    """Eqs. (C.9)-(C.10) are exact for quadratic fields (interior nodes)."""
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a, b, c, d, e, f0 = 0.3, -0.7, 0.11, -0.05, 0.08, 1.3
    q = f0 + a * x + b * y + c * x * x + d * y * y + e * x * y
    gx, gy, lap = oracle_mod.grad_lap(q)
    s = (slice(1, -1), slice(1, -1))
    assert np.allclose(gx[s], (a + 2 * c * x + e * y)[s], atol=1e-12)
    assert np.allclose(gy[s], (b + 2 * d * y + e * x)[s], atol=1e-12)
    assert np.allclose(lap[s], 2 * c + 2 * d, atol=1e-12)
    # a periodic Fourier mode: symbols of the isotropic stencils
    k = 2 * math.pi / nx
    fm = np.sin(k * x) * np.ones((ny, nx))
    gx, gy, lap = oracle_mod.grad_lap(fm)
    # grad symbol: (2/3 + 1/3 cos 0) sin k  along x; lap symbol: 2 * (2/3)(cos k - 1) + (1/3)*2*(cos k - 1)
    assert np.allclose(gx, np.sin(k) * np.cos(k * x), atol=1e-13)
    assert np.allclose(gy, 0, atol=1e-13)
    assert np.allclose(lap, 2 * (np.cos(k) - 1) * np.sin(k * x), atol=1e-13)


@pytest.mark.parametrize("theta", [15.0, 30.0, 60.0, 90.0, 120.0, 150.0, 170.0])
def test_wetting_boundary(oracle_mod, theta):
    """phi_w solves Eq. (50); the quadratic through the wall and the first two
    fluid nodes has the wall slope of Eq. (49); 90 degrees mirrors."""
    prm = W.Params(nx=8, ny=8, width=4.0, sigma=0.01)
    rng = np.random.default_rng(int(theta))
    for _ in range(20):
        phi1 = rng.uniform(0.0, 1.0)
        phi2 = np.clip(phi1 + rng.uniform(-0.2, 0.2), 0, 1)
        pw, ghost = oracle_mod.wall_phi(prm, phi1, phi2, theta)
        ct = 0.0 if theta == 90.0 else math.cos(math.radians(theta))
        a = 4 * ct / prm.width
        b = 8 / 3 - a
        c = phi2 / 3 - 3 * phi1
        assert abs(a * pw * pw + b * pw + c) < 1e-14
        # quadratic q(s) through (0, pw), (1/2, phi1), (3/2, phi2)
        A = np.array([[1, 0, 0], [1, 0.5, 0.25], [1, 1.5, 2.25]])
        q0, q1, q2 = np.linalg.solve(A, [pw, phi1, phi2])
        slope = q1  # d q / d s at the wall, s pointing into the fluid
        beta = 12 * prm.sigma / prm.width
        k = 1.5 * prm.sigma * prm.width
        assert abs(slope + math.sqrt(2 * beta / k) * (1 - pw) * pw * ct) < 1e-12
        assert abs(ghost - (q0 - 0.5 * q1 + 0.25 * q2)) < 1e-12
        if theta == 90.0:
            assert ghost == pytest.approx(phi1, abs=1e-15)
