"""Pins of the oracle's pressure scheme and its diagnostics against closed
forms, and tests that the pins catch plausible mistakes.

Pressure, Eq. (39) in the second way of Remark 1:
    p = c_s^2/(1 - w_0) [ sum_{i!=0} g_i + (1/2 + H) u.grad rho + s_0
                          + K (2 F.u + d_t(m.u)) ],
    s_0 = -w_0 (rho |u|^2 + m.u) / (2 c_s^2),  H = (s_g^2 - s_g^0)/(9 s_g^0 s_g^2),  K = 1/3.

* Equilibrium identity.  The weights satisfy sum_i s_i = 0 (Eq. (20)), so
  for g = g^eq(p0, u) of Eqs. (19)-(20) the bracket's first and third terms
  give exactly (1 - w_0) p0 / c_s^2, whatever rho, u and m^{phi C} are.  On a
  state built as g^eq with F = 0 (sigma = 0, no gravity) and a varying phi
  (so grad rho != 0 and m^{phi C} != 0), the recovered pressure is then
  p0 + c_s^2/(1 - w_0) (1/2 + H) u.grad_h rho exactly, grad_h being the
  stencil of Eq. (C.9), whose symbol on a Fourier mode e^{ikx} is i sin k.
* Uniformly accelerated fluid.  A periodic single-phase fluid under a
  constant body force G stays uniform.  With the rates the paper leaves at 1
  (s_g^{0,1,2,3,5} = 1), u(t) = u0 + (t + 1/2) G / rho (the half step from
  Eq. (22b)), and the pressure the scheme recovers is constant in time,
  p(t) = p0 + |G|^2 / (10 rho).  Derivation: the energy and energy-square
  moments relax to their equilibria (Eq. (C.2)) plus half their forcing
  moments, +6 u.F and -6 u.F, and sum_{i!=0} g = (8 m_0 + m_1 - m_2)/9, so
  after one step sum_{i!=0} g = (5/3) p + (2/3)(rho |u|^2 + u.G); with
  u' = u + G/rho the next recovery adds s_0 = -(2/3) rho |u'|^2 and
  K 2 G.u', and the bracket is (5/3) p again exactly when K = 1/3.  At t = 0
  the populations are g^eq(p0, u0) while the recovered velocity is
  u0 + G/(2 rho), which gives the constant offset |G|^2 / (10 rho).

Diagnostics, Eqs. (42)-(43) with Eq. (35):
* S_m = d_t rho + div_h(rho u + m^{phi C}), d_t rho = rho(t) - rho(t-1).  With
  the original flux (m^{phi C} = 0), u = (A, 0) uniform and
  rho(t) = rho_c + rho_1 cos kx, rho(t) - rho(t-1) = rho' eps sin kx:
  S_m = (rho' eps - A rho_1 sin k) sin kx, so S_m^rms = |...| / sqrt(2).
* tr S = -s_2/(2 rho c_s^2) [tr sum c c (g - g^eq) + tr M_2F / 2].  Adding
  a w_i (|c_i|^2 - 2 c_s^2) to a uniform equilibrium at rest in phi (F = 0,
  m = 0, u uniform) raises tr sum c c g by 4a/9 and the recovered pressure
  by (8/45) a, hence tr sum c c g^eq by (16/45) a:  tr S = -2 s_2 a / (15 rho).
  Adding b to g_0 changes m_0 and m_1 but not the trace (a check of the
  factor 4 on m_0 - m_0^eq).
"""
import math

import numpy as np
import pytest

import workloads as W

CS2 = 1.0 / 3.0


def _lib(oracle_mod, lib_):
    return lib_ if lib_ is not None else oracle_mod.lib()


def _grid(nx, ny):
    x = np.arange(nx, dtype=np.float64)[None, :] * np.ones((ny, 1))
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    return x, y


# ---------------------------------------------------------------- pins
def identity_error(oracle_mod, lib_=None, rates=False):
    """max |p - p_expected| after building g = g^eq(p0, u0) on a varying phi
    (equilibrium identity plus the (1/2 + H) u.grad rho term)."""
    nx, ny = 64, 48
    kx, ky = 2 * math.pi * 2 / nx, 2 * math.pi * 3 / ny
    x, y = _grid(nx, ny)
    phi = 0.5 + 0.2 * np.cos(kx * x) + 0.15 * np.sin(ky * y)
    u0 = 0.02 + 0.01 * np.sin(ky * y + 0.3)
    v0 = -0.015 + 0.01 * np.cos(kx * x - 0.2)
    p0 = 1e-3 * np.cos(kx * x + ky * y)
    sg = [math.nan] * 9
    if rates:
        sg[0], sg[2] = 1.0, 1.4
    prm = W.Params(nx=nx, ny=ny, rhoA=3.0, rhoB=1.0, muA=0.3, muB=0.1, sigma=0.0, mobility=0.05,
                   s_g=tuple(sg))
    o = oracle_mod.Oracle(prm, _lib(oracle_mod, lib_))
    o.init_fields(phi, u0, v0, p0)
    p = o.fields(oracle_mod.P)
    drho = prm.rhoA - prm.rhoB
    gx = drho * (-0.2 * math.sin(kx) * np.sin(kx * x))
    gy = drho * (0.15 * math.sin(ky) * np.cos(ky * y))
    s0, s2 = (1.0, 1.4) if rates else (1.0, 1.0)
    H = (s2 - s0) / (9 * s0 * s2)
    expect = p0 + CS2 / (1 - 4.0 / 9.0) * (0.5 + H) * (u0 * gx + v0 * gy)
    # the recovered velocity is u0 (F = 0); the flux m^{phi C} is not zero
    assert np.abs(o.fields(oracle_mod.UX) - u0).max() < 1e-15
    assert np.abs(o.fields(oracle_mod.MCX)).max() > 1e-3
    return float(np.abs(p - expect).max())


def accelerated_error(oracle_mod, lib_=None, steps=(0, 1, 10, 200)):
    """max deviation of u(t), p(t) from the uniformly accelerated closed form."""
    nx, ny = 32, 24
    G = np.array([3e-5, -2e-5])
    rho = 2.0
    prm = W.Params(nx=nx, ny=ny, rhoA=rho, rhoB=rho, muA=0.2, muB=0.2, sigma=0.01,
                   gravity_mode=W.GRAV_CONST, gx=G[0], gy=G[1])
    u0, v0, p0 = 0.01, 0.02, 2e-3
    o = oracle_mod.Oracle(prm, _lib(oracle_mod, lib_))
    full = np.ones((ny, nx))
    o.init_fields(0.7 * full, u0 * full, v0 * full, p0 * full)
    worst = 0.0
    t = 0
    for s in steps:
        o.step(s - t)
        t = s
        ue = u0 + (t + 0.5) * G[0] / rho
        ve = v0 + (t + 0.5) * G[1] / rho
        pe = p0 + (G @ G) / (10 * rho)
        du = max(np.abs(o.fields(oracle_mod.UX) - ue).max(), np.abs(o.fields(oracle_mod.UY) - ve).max())
        dp = np.abs(o.fields(oracle_mod.P) - pe).max()
        worst = max(worst, du, dp)
    return worst


def sm_error(oracle_mod, lib_=None):
    """|S_m^rms - closed form| / closed form on the prescribed state."""
    nx, ny = 60, 8
    k = 2 * math.pi * 3 / nx
    x, _ = _grid(nx, ny)
    b, eps, A = 0.2, 0.01, 0.03
    prm = W.Params(nx=nx, ny=ny, rhoA=3.0, rhoB=1.0, muA=0.3, muB=0.1, sigma=0.0,
                   flux_model=W.FLUX_ORIGINAL)
    drho = prm.rhoA - prm.rhoB
    phi_b = 0.5 + b * np.cos(k * x)
    phi_a = phi_b - eps * np.sin(k * x)
    o = oracle_mod.Oracle(prm, _lib(oracle_mod, lib_))
    o.init_fields(phi_a, A * np.ones((ny, nx)), None, None)
    f = np.zeros((9, ny, nx))
    f[0] = phi_b
    o.set_fields(oracle_mod.F_POP, f)
    rho_b = drho * (phi_b - prm.phiB) + prm.rhoB
    g = np.zeros((9, ny, nx))
    g[0] = prm.rho0
    g[1] = rho_b * A
    o.set_fields(oracle_mod.G_POP, g)
    assert np.abs(o.fields(oracle_mod.UX) - A).max() < 1e-15
    d = o.diag()
    expect = abs(drho * eps - A * drho * b * math.sin(k)) / math.sqrt(2.0)
    assert d["n_avg"] == nx * ny
    return abs(d["Sm_rms"] - expect) / expect


def du_error(oracle_mod, lib_=None):
    """|D_u^rms - closed form| / closed form on a uniform state with a
    prescribed non-equilibrium part."""
    nx, ny = 48, 6
    k = 2 * math.pi * 2 / nx
    x, _ = _grid(nx, ny)
    prm = W.Params(nx=nx, ny=ny, rhoA=3.0, rhoB=1.0, muA=0.3, muB=0.1, sigma=0.01)
    phi = 0.6
    rho = (prm.rhoA - prm.rhoB) * phi + prm.rhoB
    mu = phi * (prm.muA - prm.muB) + prm.muB
    s2 = 1.0 / (mu / rho / CS2 + 0.5)
    full = np.ones((ny, nx))
    o = oracle_mod.Oracle(prm, _lib(oracle_mod, lib_))
    o.init_fields(phi * full, 0.02 * full, -0.01 * full, 1e-3 * full)
    cx, cy, w = oracle_mod.lattice()
    a0, b0 = 1e-3, 4e-3
    a = a0 * np.cos(k * x)
    g = o.fields(oracle_mod.G_POP)
    for i in range(9):
        g[i] += a * w[i] * (cx[i] ** 2 + cy[i] ** 2 - 2 * CS2)
    g[0] += b0 * np.sin(k * x)
    o.set_fields(oracle_mod.G_POP, g)
    d = o.diag()
    expect = 2 * s2 * a0 / (15 * rho) / math.sqrt(2.0)
    return abs(d["Du_rms"] - expect) / expect


# ---------------------------------------------------------------- tests
def test_pressure_equilibrium_identity(oracle_mod):
    """Eq. (39) returns p0 from g^eq(p0, u) (Eqs. (19)-(20)) plus the
    (1/2 + H) u.grad rho term, with u != 0, m^{phi C} != 0, grad rho != 0."""
    assert identity_error(oracle_mod) < 1e-14


def test_pressure_identity_with_nonzero_H(oracle_mod):
    """The same with s_g^0 != s_g^2, so that H of App. C is not zero."""
    assert identity_error(oracle_mod, rates=True) < 1e-14


def test_uniformly_accelerated_fluid(oracle_mod):
    """u(t) = u0 + (t + 1/2) G / rho and a pressure constant in time, the K
    and s_0 terms of Eq. (39) cancelling the forcing's change of the
    energy moments (K = 1/3)."""
    assert accelerated_error(oracle_mod) < 1e-14


def test_mass_source_statistic_closed_form(oracle_mod):
    """S_m^rms (Eq. (43)) equals its closed form on a prescribed state."""
    assert sm_error(oracle_mod) < 1e-13


def test_velocity_divergence_statistic_closed_form(oracle_mod):
    """D_u^rms (Eq. (42) through tr S of Eq. (35)) equals its closed form."""
    assert du_error(oracle_mod) < 1e-10


# ---- each pin fails on a planted mistake in a copy of the oracle
SRC_S0 = "const double s0 = -WI[0] * (rho * (u * u + v * v) + c2) / (2.0 * CS2);"
PLANTS = {
    "s0_sign": ([(SRC_S0, SRC_S0.replace("= -WI[0]", "= WI[0]"))], ("identity", "accelerated")),
    "s0_without_m_dot_u": ([(SRC_S0, SRC_S0.replace(" + c2)", ")"))], ("identity",)),
    "K_one_sixth": ([("st->Kc = 1.0 / 3.0;", "st->Kc = 1.0 / 6.0;")], ("accelerated",)),
    "half_dropped": ([("(0.5 + st->Hc) * (u * rx + v * ry)", "st->Hc * (u * rx + v * ry)")], ("identity",)),
    "H_sign": ([("st->Hc = (s2 - s0) / (9.0 * s0 * s2);", "st->Hc = (s0 - s2) / (9.0 * s0 * s2);")],
               ("identity_rates",)),
    "dt_rho_sign": ([("st->drho_dphi * (st->phi[n] - st->phi_prev[n])",
                      "st->drho_dphi * (st->phi_prev[n] - st->phi[n])")], ("sm",)),
    "div_weights_swapped": ([("div += WI[k] * (CX[k] * Jx + CY[k] * Jy) / CS2;",
                              "div += WI[k < 5 ? k + 4 : k - 4] * (CX[k] * Jx + CY[k] * Jy) / CS2;")], ("sm",)),
    "trace_factor_m0": ([("4.0 * (m[0] - mgeq[0])", "2.0 * (m[0] - mgeq[0])")], ("du",)),
    "strain_without_cs2": ([("-s2 / (2.0 * st->rho[n] * CS2)", "-s2 / (2.0 * st->rho[n])")], ("du",)),
}
PINS = {
    "identity": (lambda om, L: identity_error(om, L), 1e-14),
    "identity_rates": (lambda om, L: identity_error(om, L, rates=True), 1e-14),
    "accelerated": (lambda om, L: accelerated_error(om, L), 1e-14),
    "sm": (lambda om, L: sm_error(om, L), 1e-13),
    "du": (lambda om, L: du_error(om, L), 1e-10),
}


@pytest.mark.parametrize("plant", list(PLANTS))
def test_pins_catch_planted_mistake(oracle_mod, tmp_path, plant):
    edits, pins = PLANTS[plant]
    L = oracle_mod.build_variant(edits, str(tmp_path), tag=plant)
    for name in pins:
        fn, tol = PINS[name]
        err = fn(oracle_mod, L)
        assert err > 1e3 * tol, (plant, name, err)
