"""The oracle's pins catch plausible mistakes: each case plants one mistake
in a copy of the oracle (oracle.build_variant: a flipped sign, a dropped
term, a wrong weight or coefficient, a wrong reflection) and shows that a
pin of the function it sits in fails on the copy while the oracle passes.

Pins used (each written from the paper or the mathematics, not from the
oracle's code):
  stencil   Eqs. (C.9)-(C.10) are exact on quadratic fields.
  ghost     the 90-degree wetting ghost is the mirror value, and phi_w
            solves Eq. (50) at other angles.
  geq       the moments of g^eq built in velocity space from Eqs. (19)-(20)
            equal the oracle's equilibrium moments (App. C).
  accel     uniformly accelerated fluid: u = u0 + (t + 1/2) G / rho, p
            constant (Eq. (22b) with the half force; Eq. (39)).
  shear     a shear wave decays at nu k^2 with s_g^{7,8} = 1/(nu/c_s^2 + 1/2).
  poiseuille  single-phase channel flow with half-way bounce-back walls is
            the parabola.
  flat      a flat tanh interface is the Allen-Cahn equilibrium
            (grad phi = lambda n, Eqs. (7)-(8)).
The pressure and statistics pins have their own planted cases in
test_oracle_pressure_diag.py.
"""
import math

import numpy as np
import pytest

import workloads as W

CS2 = 1.0 / 3.0


def pin_stencil(om, L):
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a, b, c, d, e, f0 = 0.3, -0.7, 0.11, -0.05, 0.08, 1.3
    q = f0 + a * x + b * y + c * x * x + d * y * y + e * x * y
    gx, gy, lap = om.grad_lap(q, L)
    s = (slice(1, -1), slice(1, -1))
    return max(np.abs(gx - (a + 2 * c * x + e * y))[s].max(), np.abs(gy - (b + 2 * d * y + e * x))[s].max(),
               np.abs(lap - (2 * c + 2 * d))[s].max())


def pin_ghost(om, L):
    prm = W.Params(nx=8, ny=8, width=4.0, sigma=0.01)
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(20):
        phi1 = rng.uniform(0.0, 1.0)
        phi2 = float(np.clip(phi1 + rng.uniform(-0.2, 0.2), 0, 1))
        _, ghost = om.wall_phi(prm, phi1, phi2, 90.0, L)
        worst = max(worst, abs(ghost - phi1))
        pw, _ = om.wall_phi(prm, phi1, phi2, 60.0, L)
        a = 4 * math.cos(math.radians(60.0)) / prm.width
        worst = max(worst, abs(a * pw * pw + (8 / 3 - a) * pw + phi2 / 3 - 3 * phi1))
    return worst


def pin_geq(om, L):
    from test_oracle_node import _random_node, _velocity_space_g

    cx, cy, w = om.lattice()
    M, _ = om.moment_matrix()
    prm = W.Params(nx=8, ny=8)
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(5):
        v = _random_node(rng, W.MODEL_AC)
        geq, _, _ = _velocity_space_g(v, prm, cx, cy, w)
        _, _, mgeq, _ = om.node_moments(prm, lib_=L, **v)
        worst = max(worst, np.abs(M @ geq - mgeq).max())
    return worst


def pin_accel(om, L):
    from test_oracle_pressure_diag import accelerated_error

    return accelerated_error(om, L)


def pin_shear(om, L):
    nx, ny, A, nu = 8, 64, 1e-3, 0.1
    prm = W.Params(nx=nx, ny=ny, rhoA=1.0, rhoB=1.0, muA=nu, muB=nu, sigma=0.0)
    k = 2.0 * np.pi / ny
    y = np.arange(ny) + 0.5
    o = om.Oracle(prm, L)
    o.init_fields(np.ones((ny, nx)), np.tile((A * np.sin(k * y))[:, None], (1, nx)), None, None)
    o.step(5)
    a5 = np.abs(o.fields(om.UX)).max()
    o.step(45)
    a50 = np.abs(o.fields(om.UX)).max()
    return abs(np.log(a5 / a50) / 45.0 / (nu * k * k) - 1.0)


def pin_poiseuille(om, L):
    ny, G, mu = 32, 1e-6, 0.1
    prm = W.Params(nx=3, ny=ny, bc=(0, 0, 1, 1), rhoA=1, rhoB=1, muA=mu, muB=mu,
                   gravity_mode=W.GRAV_CONST, gx=G, sigma=0.0)
    o = om.Oracle(prm, L)
    o.init_fields(np.ones((ny, 3)))
    o.step(20000)
    u = o.fields(om.UX)[:, 1]
    y = np.arange(ny) + 0.5
    ue = G / (2 * mu) * y * (ny - y)
    return np.abs(u - ue).max() / ue.max()


def pin_flat(om, L):
    c = W.flat_interface(4, 48, model=W.MODEL_AC)
    o = om.Oracle(c.params, L)
    o.init_fields(c.phi, c.ux, c.uy, c.p)
    o.step(2000)
    return np.abs(o.fields(om.PHI) - c.phi).max()


# pin: (function, bar the oracle meets)
PINS = {"stencil": (pin_stencil, 1e-12), "ghost": (pin_ghost, 1e-13), "geq": (pin_geq, 1e-13),
        "accel": (pin_accel, 1e-14), "shear": (pin_shear, 1e-3), "poiseuille": (pin_poiseuille, 1e-3),
        "flat": (pin_flat, 0.02)}

# planted mistake: ([(text in the oracle, replacement)], pin that must fail)
PLANTS = {
    "gradient_uniform_weight": ([("sx += WI[k] * CX[k] * v;", "sx += WI[1] * CX[k] * v;")], "stencil"),
    "laplacian_half": ([("sl += 2.0 * WI[k] * (v - c0);", "sl += WI[k] * (v - c0);")], "stencil"),
    "ghost_linear_extrapolation": ([("return 8.0 / 3.0 * phiw - 2.0 * phi1 + phi2 / 3.0;",
                                     "return 2.0 * phiw - phi1;")], "ghost"),
    "geq_energy_without_m_dot_u": ([("mgeq[1] = -4.0 * rho0 + 6.0 * p + 3.0 * rho * uu + 3.0 * um;",
                                     "mgeq[1] = -4.0 * rho0 + 6.0 * p + 3.0 * rho * uu;")], "geq"),
    "velocity_full_force": ([("const double u = (jx + 0.5 * Fx) / rho;", "const double u = (jx + Fx) / rho;")],
                            "accel"),
    "viscous_rate_without_cs2": ([("st->s78[n] = 1.0 / (nu / CS2 + 0.5);", "st->s78[n] = 1.0 / (nu + 0.5);")],
                                 "shear"),
    "wall_reflects_same_direction": ([("dst[i][n] = wall ? src[OPP[i]][n] :", "dst[i][n] = wall ? src[i][n] :")],
                                     "poiseuille"),
    "lambda_coefficient_halved": ([("sqrt(2.0 * st->beta / st->kappa)", "sqrt(0.5 * st->beta / st->kappa)")],
                                  "flat"),
}


@pytest.mark.parametrize("pin", list(PINS))
def test_oracle_meets_its_pin(oracle_mod, pin):
    fn, bar = PINS[pin]
    assert fn(oracle_mod, None) <= bar


@pytest.mark.parametrize("plant", list(PLANTS))
def test_planted_mistake_fails_its_pin(oracle_mod, tmp_path, plant):
    edits, pin = PLANTS[plant]
    L = oracle_mod.build_variant(edits, str(tmp_path), tag=plant)
    fn, bar = PINS[pin]
    err = fn(oracle_mod, L)
    assert err > 2 * bar, (plant, pin, err)  # the pin fails, with a margin
