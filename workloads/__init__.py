"""Seeded synthetic inputs for the phase-field lattice Boltzmann cases.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds only problem set-up -- parameter sets in the paper's
physical terms and initial fields -- and no arithmetic of the lattice
Boltzmann method itself (no equilibria, stencils, relaxation rules or
free-energy constants).  Every random number comes from SplitMix64 followed by
Box-Muller, both written out below from their published definitions, so the
fields are bit-identical on every machine and need no numpy RNG.

Grid convention: arrays are row-major ``[ny][nx]`` (x fastest); node (i, j)
sits at (i + 1/2, j + 1/2) in a box whose walls, where present, are at 0 and
N (half-way bounce-back puts the wall midway between a node and its image).

The cases follow Sec. 4 of Zhan, Chai & Shi, "Consistent and conservative
phase-field based lattice Boltzmann method for incompressible two-phase
flows" (arXiv:2111.00847): square droplet (Sec. 4.1, Eq. (41)), layered
Poiseuille flow (Sec. 4.2, Eq. (44)), droplet spreading (Sec. 4.3, Eq. (48)),
Rayleigh-Taylor instability (Sec. 4.4, Eqs. (53)-(54)) and dam break
(Sec. 4.5, Eq. (55)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

DEFAULT_SEED = 2111008470

# Integer codes of the C-ABI parameter block (both the CUDA library and the
# oracle use the same numbering).
PREC_FP64, PREC_FP32, PREC_FP16_DEV, PREC_BF16_DEV = 0, 1, 2, 3
MODEL_AC, MODEL_CH = 0, 1
FLUX_PRESENT, FLUX_ORIGINAL, FLUX_CORRECTED = 0, 1, 2
VISC_LINEAR_MU, VISC_INVERSE_NU = 0, 1
GRAV_CONST, GRAV_RHO, GRAV_RHO_MINUS_MEAN = 0, 1, 2
BC_PERIODIC, BC_WALL = 0, 1
SIDE_LEFT, SIDE_RIGHT, SIDE_BOTTOM, SIDE_TOP = 0, 1, 2, 3

NAN = float("nan")


# --------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014; Box-Muller
# 1958).  Pure Python integers, masked to 64 bits.
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator: state advances by the golden-ratio constant and
    the output is the state passed through the two xor-shift-multiply mixes."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal_pair(self) -> tuple[float, float]:
        """Two independent standard normals by the Box-Muller transform."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)

    def normals(self, n: int) -> list[float]:
        out: list[float] = []
        while len(out) < n:
            out.extend(self.normal_pair())
        return out[:n]


def uniform_array(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) from SplitMix64 (vectorised with uint64 numpy ops,
    identical bit for bit to repeated ``SplitMix64.uniform``)."""
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# Parameter block (mirrors the C struct field by field; each side converts it
# to its own ctypes structure).
# --------------------------------------------------------------------------
@dataclass
class Params:
    nx: int
    ny: int
    precision: int = PREC_FP64
    phase_model: int = MODEL_AC
    flux_model: int = FLUX_PRESENT
    visc_law: int = VISC_LINEAR_MU
    gravity_mode: int = GRAV_CONST
    bc: tuple = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    diag_every: int = 0
    flags: int = 0  # library option bits (not part of the method)
    phiA: float = 1.0
    phiB: float = 0.0
    rhoA: float = 1.0
    rhoB: float = 1.0
    muA: float = 0.1  # dynamic viscosities; nu = mu / rho
    muB: float = 0.1
    mobility: float = 0.02
    width: float = 4.0
    sigma: float = 0.01
    eta: float = 1.0
    gx: float = 0.0
    gy: float = 0.0
    rho0: float = 1.0
    theta_deg: tuple = (90.0, 90.0, 90.0, 90.0)
    s_f: tuple = (NAN,) * 9  # NaN = the paper's default rule
    s_g: tuple = (NAN,) * 9
    n_delta: float = 0.0  # regularisation of n (units of dphi / W); 0 = the default 5e-3

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


@dataclass
class Case:
    """A named workload: parameters plus initial fields (row-major [ny][nx])."""

    name: str
    params: Params
    phi: np.ndarray
    ux: np.ndarray | None = None
    uy: np.ndarray | None = None
    p: np.ndarray | None = None
    steps: int = 100
    notes: dict = field(default_factory=dict)
    solid: np.ndarray | None = None  # [ny][nx] bool, solid obstacle nodes


def _coords(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y, indexing="xy")  # shapes [ny][nx]


def tanh_profile(dist: np.ndarray, width: float, phiA: float, phiB: float) -> np.ndarray:
    """Equilibrium interface profile used by every initial condition of Sec. 4:
    (phiA+phiB)/2 + (phiA-phiB)/2 tanh(2 d / W), d > 0 inside phase A."""
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * dist / width)


# --------------------------------------------------------------------------
# Sec. 4.1: square droplet (Eq. (41)); periodic box, phase A inside.
# --------------------------------------------------------------------------
def square_droplet_phi(n: int, D: float, W: float, phiA: float, phiB: float) -> np.ndarray:
    X, Y = _coords(n, n)
    x = X - 0.5 * n
    y = Y - 0.5 * n
    lo, hi = 0.5 * (W - D), 0.5 * (D - W)
    phi = np.full((n, n), phiA)
    prof = lambda d: tanh_profile(d, W, phiA, phiB)  # noqa: E731
    for cx_, xs in ((lo, x <= lo), (hi, x >= hi)):
        for cy_, ys in ((lo, y <= lo), (hi, y >= hi)):
            m = xs & ys
            r = np.sqrt((x - cx_) ** 2 + (y - cy_) ** 2)
            phi[m] = prof(0.5 * W - r)[m]
    midx = (x > lo) & (x < hi)
    midy = (y > lo) & (y < hi)
    m = midx & (y <= lo)
    phi[m] = prof(0.5 * D + y)[m]
    m = midx & (y >= hi)
    phi[m] = prof(0.5 * D - y)[m]
    m = (x <= lo) & midy
    phi[m] = prof(0.5 * D + x)[m]
    m = (x >= hi) & midy
    phi[m] = prof(0.5 * D - x)[m]
    return phi


def square_droplet(n: int = 128, D: float = 64.0, precision: int = PREC_FP64,
                   density_ratio: float = 10.0, steps: int = 1000) -> Case:
    """Square droplet, plain method: 128^2 periodic, AC, density ratio 10,
    nu = 0.1 in both phases, W = 4, M = 0.02, sigma = 0.01, u = 0."""
    prm = Params(nx=n, ny=n, precision=precision, phase_model=MODEL_AC,
                 rhoA=density_ratio, rhoB=1.0, muA=0.1 * density_ratio, muB=0.1,
                 mobility=0.02, width=4.0, sigma=0.01, diag_every=10)
    phi = square_droplet_phi(n, D, 4.0, prm.phiA, prm.phiB)
    return Case("square_droplet", prm, phi, steps=steps)


# --------------------------------------------------------------------------
# Sec. 4.2: layered Poiseuille flow (Eqs. (44)-(47)); fluid A below y = 0.
# --------------------------------------------------------------------------
def layered_poiseuille(nx: int = 4, ny: int = 256, rhoA: float = 100.0, rhoB: float = 1.0,
                       muA: float = 10.0, muB: float = 1.0, Gx: float = 1e-6,
                       W: float = 4.0, sigma: float = 1e-3, mobility: float = 0.1,
                       precision: int = PREC_FP64, steps: int = 300000) -> Case:
    # n regularised at 1e-5 dphi / W: the viscosity follows phi into the far
    # interface tails, which the default regularisation widens (Table 2)
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=MODEL_AC,
                 bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL),
                 rhoA=rhoA, rhoB=rhoB, muA=muA, muB=muB, mobility=mobility,
                 width=W, sigma=sigma, gravity_mode=GRAV_CONST, gx=Gx, gy=0.0, n_delta=1e-5)
    _, Y = _coords(nx, ny)
    y = Y - 0.5 * ny
    phi = tanh_profile(-y, W, prm.phiA, prm.phiB)
    return Case("layered_poiseuille", prm, phi, steps=steps,
                notes={"h": 0.5 * ny, "Gx": Gx})


def layered_poiseuille_exact(ny: int, W: float, muA: float, muB: float, Gx: float,
                             npts: int = 20001) -> np.ndarray:
    """Steady velocity of the layered channel at the node centres, from
    d/dy(mu du/dy) = -Gx with u(-h) = u(h) = 0 and the tanh viscosity of
    Eq. (45); the integrals of Eq. (46) are evaluated by composite Simpson
    quadrature on a fine grid.  (Eq. (46) is this solution with Gx eliminated
    in favour of the centre-line speed U_c.)"""
    h = 0.5 * ny
    ys = np.linspace(-h, h, npts)
    mu = 0.5 * (muA + muB) + 0.5 * (muA - muB) * np.tanh(-2.0 * ys / W)

    def cumint(v):
        # cumulative trapezoid on the fine grid (error O(dy^2) ~ 1e-8 relative)
        c = np.zeros_like(v)
        c[1:] = np.cumsum(0.5 * (v[1:] + v[:-1]) * np.diff(ys))
        return c

    I1 = cumint(1.0 / mu)
    Iy = cumint(ys / mu)
    A, B = Iy[-1], I1[-1]
    u_fine = Gx * (-Iy + (A / B) * I1)
    yn = np.arange(ny) + 0.5 - h
    return np.interp(yn, ys, u_fine)


# --------------------------------------------------------------------------
# Sec. 4.3: droplet spreading on an ideal wall (Eqs. (48)-(52)).
# --------------------------------------------------------------------------
def droplet_spreading(nx: int = 2048, ny: int = 1024, R0: float = 256.0, theta: float = 60.0,
                      rhoA: float = 1000.0, rhoB: float = 1.0, muA: float = 10.0,
                      muB: float = 0.1, W: float = 5.0, mobility: float = 0.1,
                      sigma: float = 0.01, precision: int = PREC_FP32,
                      steps: int = 2000) -> Case:
    """Semicircular drop of radius R0 on the bottom wall (contact angle theta),
    neutral (90 degree) top wall, periodic in x."""
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=MODEL_AC,
                 bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL),
                 theta_deg=(90.0, 90.0, float(theta), 90.0),
                 rhoA=rhoA, rhoB=rhoB, muA=muA, muB=muB, mobility=mobility,
                 width=W, sigma=sigma)
    X, Y = _coords(nx, ny)
    r = np.sqrt((X - 0.5 * nx) ** 2 + Y ** 2)  # wall at y = 0
    phi = tanh_profile(R0 - r, W, prm.phiA, prm.phiB)
    return Case("droplet_spreading", prm, phi, steps=steps, notes={"R0": R0, "theta": theta})


def spreading_exact(R0: float, theta_deg: float) -> tuple[float, float, float]:
    """Eq. (52): equilibrium height H, base length L and radius R of a 2-D
    drop of initial radius R0 at contact angle theta."""
    th = math.radians(theta_deg)
    R = R0 * math.sqrt((math.pi / 2.0) / (th - math.sin(th) * math.cos(th)))
    return R - R * math.cos(th), 2.0 * R * math.sin(th), R


# --------------------------------------------------------------------------
# Sec. 4.4: Rayleigh-Taylor instability (Eqs. (53)-(54)).
# --------------------------------------------------------------------------
def rti_parameters(d: float, atwood: float = 0.5, Re: float = 3000.0, sqrt_gd: float = 0.04,
                   rhoB: float = 1.0):
    """Lattice parameters of the RTI case: heavy fluid A of density
    rhoB (1+At)/(1-At), gravity g from the velocity scale sqrt(g d), equal
    kinematic viscosity nu = sqrt(g d) d / Re in both fluids."""
    rhoA = rhoB * (1.0 + atwood) / (1.0 - atwood)
    g = sqrt_gd ** 2 / d
    nu = sqrt_gd * d / Re
    return rhoA, rhoB, g, nu


def rti(nx: int, ny: int, d: float | None = None, atwood: float = 0.5, Re: float = 3000.0,
        modes=None, amp0: float | None = None, precision: int = PREC_FP32, W: float = 4.0,
        sigma: float = 5e-5, seed: int = DEFAULT_SEED, steps: int = 2000,
        mode_sigma: float = 4.0, n_modes: int = 32) -> Case:
    """RTI: heavy fluid A above y = ny/2 + h(x), periodic in x, no-flux walls
    at the bottom and top, body force G = -(rho - (rhoA+rhoB)/2) g e_y.

    h(x) is either the single mode  amp0 cos(2 pi x / nx)  (amp0 given) or a
    sum of n_modes seeded modes a_k cos(2 pi k x / nx + psi_k) with
    a_k ~ N(0, mode_sigma^2), psi_k ~ U[0, 2 pi) (modes == "random"), or an
    explicit list of cosine amplitudes (modes = [a_1, a_2, ...]).

    The relaxation rates follow Sec. 4.4 (s_f^{3,5} = 0.9 realised through
    the mobility M = c_s^2 (1/0.9 - 1/2), s_g^{4,6} = 1.7)."""
    d = float(nx) if d is None else d
    rhoA, rhoB, g, nu = rti_parameters(d, atwood, Re)
    mob = (1.0 / 0.9 - 0.5) / 3.0
    sg = [NAN] * 9
    sg[4] = sg[6] = 1.7
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=MODEL_AC,
                 bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL),
                 rhoA=rhoA, rhoB=rhoB, muA=rhoA * nu, muB=rhoB * nu,
                 mobility=mob, width=W, sigma=sigma,
                 gravity_mode=GRAV_RHO_MINUS_MEAN, gx=0.0, gy=-g, s_g=tuple(sg))
    x = np.arange(nx, dtype=np.float64) + 0.5
    notes = {"d": d, "g": g, "nu": nu}
    if amp0 is not None:
        h = amp0 * np.cos(2.0 * math.pi * x / nx)
    elif isinstance(modes, str) and modes == "random":
        rng = SplitMix64(seed)
        a = np.array(rng.normals(n_modes)) * mode_sigma
        psi = np.array([2.0 * math.pi * rng.uniform() for _ in range(n_modes)])
        k = np.arange(1, n_modes + 1)
        h = (a[:, None] * np.cos(2.0 * math.pi * k[:, None] * x[None, :] / nx + psi[:, None])).sum(0)
        notes.update(a=a.tolist(), psi=psi.tolist())
    else:
        a = np.asarray(modes, dtype=np.float64)
        k = np.arange(1, len(a) + 1)
        h = (a[:, None] * np.cos(2.0 * math.pi * k[:, None] * x[None, :] / nx)).sum(0)
        notes.update(a=a.tolist())
    y = np.arange(ny, dtype=np.float64) + 0.5
    dist = y[:, None] - (0.5 * ny + h[None, :])
    phi = tanh_profile(dist, W, prm.phiA, prm.phiB)
    return Case("rti", prm, phi, steps=steps, notes=notes)


def rti_single_mode(nx: int = 1024, ny: int = 4096, precision: int = PREC_FP32,
                    steps: int = 20000) -> Case:
    """RTI, 1024 x 4096, Atwood 0.5, Re = 3000, interface
    y = 2048 + 0.1 * 1024 cos(2 pi x / 1024)."""
    return rti(nx, ny, d=float(nx), amp0=0.1 * nx, precision=precision, steps=steps)


def rti_multimode(n: int = 16384, precision: int = PREC_FP32, seed: int = DEFAULT_SEED,
                  steps: int = 2000) -> Case:
    """Throughput workload: square n x n RTI, Atwood 0.5, Re = 3000, d = n,
    32 seeded random modes of standard deviation 4 cells."""
    return rti(n, n, d=float(n), modes="random", precision=precision, seed=seed, steps=steps)


def rti_adjoint(nx: int = 512, ny: int = 2048, seed: int = DEFAULT_SEED,
                precision: int = PREC_FP32, steps: int = 2000) -> Case:
    """Adjoint workload: 512 x 2048 RTI, Atwood 0.5, Re = 1000, 8 cosine
    modes with amplitudes a_k ~ N(0, 2^2) by seed."""
    a = np.array(SplitMix64(seed).normals(8)) * 2.0
    return rti(nx, ny, d=float(nx), Re=1000.0, modes=a.tolist(), precision=precision, steps=steps)


# --------------------------------------------------------------------------
# Sec. 4.5: dam break (Eq. (55)); walls on all sides.
# --------------------------------------------------------------------------
def dam_break(nx: int = 4096, ny: int = 2048, col_w: int = 1024, col_h: int | None = None,
              rhoA: float = 1000.0, rhoB: float = 1.0, nuB: float = 0.1, mu_ratio: float = 100.0,
              g: float = 1e-5, W: float = 4.0, sigma: float = 0.01, mobility: float = 0.05,
              theta: float = 90.0, precision: int = PREC_FP32, steps: int = 2000) -> Case:
    """Water column (phase A) of col_w x col_h cells against the left wall
    (col_h = None: the full height), inverse-linear kinematic viscosity,
    G = (0, -rho g)."""
    muB = rhoB * nuB
    muA = mu_ratio * muB
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=MODEL_AC,
                 visc_law=VISC_INVERSE_NU, bc=(BC_WALL,) * 4,
                 theta_deg=(float(theta),) * 4, rhoA=rhoA, rhoB=rhoB, muA=muA, muB=muB,
                 mobility=mobility, width=W, sigma=sigma,
                 gravity_mode=GRAV_RHO, gx=0.0, gy=-g)
    X, Y = _coords(nx, ny)
    if col_h is None or col_h >= ny:
        phi = tanh_profile(col_w - X, W, prm.phiA, prm.phiB)
    else:
        a_x, a_y = float(col_w), float(col_h)
        dx = a_x - X
        dy = a_y - Y
        # signed distance to the column's top-right corner region (rounded
        # corner of radius W as in Eq. (55))
        phi = np.where((X <= a_x - W) & (Y >= a_y - W), tanh_profile(dy, W, 1.0, 0.0),
              np.where((X >= a_x - W) & (Y <= a_y - W), tanh_profile(dx, W, 1.0, 0.0),
              np.where((X >= a_x - W) & (Y >= a_y - W),
                       tanh_profile(W - np.sqrt((X - a_x + W) ** 2 + (Y - a_y + W) ** 2), W, 1.0, 0.0),
                       1.0)))
    return Case("dam_break", prm, phi, steps=steps)


# --------------------------------------------------------------------------
# Sec. 4.5, last case: dam break over a trapezoidal obstacle on the bottom wall.
# The paper gives the obstacle's height (a/2) and position (centred at Lx/2)
# and shows its shape only in a figure; reading: an isosceles trapezoid with
# 45-degree flanks and a top of width a/2 (base 3a/2).  Solid nodes are those
# whose centre (i + 1/2, j + 1/2) lies inside it.
# --------------------------------------------------------------------------
def trapezoid_mask(nx: int, ny: int, xc: float, height: float, top: float,
                   slope: float = 1.0) -> np.ndarray:
    """Solid nodes of a trapezoid standing on the bottom wall: centred at
    x = xc, `height` tall, `top` wide at the top, flanks of dx/dy = slope."""
    X, Y = _coords(nx, ny)
    half = 0.5 * top + slope * (height - Y)
    return (Y <= height) & (np.abs(X - xc) <= half)


def disc_mask(nx: int, ny: int, xc: float, yc: float, r: float) -> np.ndarray:
    X, Y = _coords(nx, ny)
    return (X - xc) ** 2 + (Y - yc) ** 2 <= r * r


def dam_break_obstacle(nx: int = 4096, ny: int = 2048, precision: int = PREC_FP32,
                       steps: int = 2000, **kw) -> Case:
    """Dam break in a 4a x 2a chamber (a = nx/4): a x a water column at the
    left, trapezoidal obstacle of height a/2 at x = Lx/2 (the reading above)."""
    a = nx // 4
    case = dam_break(nx=nx, ny=ny, col_w=a, col_h=a, precision=precision, steps=steps, **kw)
    solid = trapezoid_mask(nx, ny, 0.5 * nx, 0.5 * a, 0.5 * a)
    phi = np.where(solid, case.params.phiB, case.phi)
    return Case("dam_break_obstacle", case.params, phi, steps=steps, solid=solid,
                notes={"a": a, "obstacle": "trapezoid h=a/2 top=a/2 45deg at Lx/2"})


# --------------------------------------------------------------------------
# Small seeded cases for parity tests: smooth droplets plus random noise in
# phi, u and p so that every term of the scheme is exercised.
# --------------------------------------------------------------------------
def noisy_drop(nx: int, ny: int, seed: int = DEFAULT_SEED, precision: int = PREC_FP64,
               model: int = MODEL_AC, walls: str = "none", rho_ratio: float = 10.0,
               noise: float = 0.02, u_amp: float = 0.01, theta=(90.0, 90.0, 90.0, 90.0),
               gravity=(GRAV_CONST, 0.0, 0.0), visc_law: int = VISC_LINEAR_MU,
               flux: int = FLUX_PRESENT, s_f=None, s_g=None) -> Case:
    """A drop of radius min(nx, ny)/4 off-centre, with seeded uniform noise of
    amplitude `noise` on phi and seeded velocity and pressure perturbations.

    walls: "none" (periodic), "y" (walls bottom/top), "x" (walls left/right)
    or "all"."""
    if model == MODEL_CH:
        phiA, phiB = 1.0, -1.0
    else:
        phiA, phiB = 1.0, 0.0
    bc = {"none": (0, 0, 0, 0), "y": (0, 0, 1, 1), "x": (1, 1, 0, 0), "all": (1, 1, 1, 1)}[walls]
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=model, flux_model=flux,
                 visc_law=visc_law, bc=bc, theta_deg=tuple(float(t) for t in theta),
                 phiA=phiA, phiB=phiB, rhoA=rho_ratio, rhoB=1.0, muA=0.1 * rho_ratio * 0.5,
                 muB=0.1, mobility=0.05, width=4.0, sigma=0.01,
                 gravity_mode=gravity[0], gx=gravity[1], gy=gravity[2])
    if s_f is not None:
        prm.s_f = tuple(s_f)
    if s_g is not None:
        prm.s_g = tuple(s_g)
    X, Y = _coords(nx, ny)
    R = 0.25 * min(nx, ny)
    r = np.sqrt((X - 0.45 * nx) ** 2 + (Y - 0.55 * ny) ** 2)
    phi = tanh_profile(R - r, prm.width, phiA, phiB)
    n = nx * ny
    u = uniform_array(seed, 4 * n).reshape(4, ny, nx) - 0.5
    phi = phi + noise * (phiA - phiB) * u[0]
    ux = 2.0 * u_amp * u[1]
    uy = 2.0 * u_amp * u[2]
    p = 1e-3 * u[3]
    return Case("noisy_drop", prm, phi, ux, uy, p, steps=100)


def static_drop(n: int, R: float, rho_ratio: float = 10.0, W: float = 4.0, sigma: float = 0.01,
                mobility: float = 0.05, model: int = MODEL_AC, nu: float = 0.1,
                precision: int = PREC_FP64) -> Case:
    """Circular drop of radius R centred in a periodic n x n box (Laplace law)."""
    phiA, phiB = (1.0, -1.0) if model == MODEL_CH else (1.0, 0.0)
    prm = Params(nx=n, ny=n, precision=precision, phase_model=model, phiA=phiA, phiB=phiB,
                 rhoA=rho_ratio, rhoB=1.0, muA=nu * rho_ratio, muB=nu, mobility=mobility,
                 width=W, sigma=sigma)
    X, Y = _coords(n, n)
    r = np.sqrt((X - 0.5 * n) ** 2 + (Y - 0.5 * n) ** 2)
    return Case("static_drop", prm, tanh_profile(R - r, W, phiA, phiB), notes={"R": R})


def flat_interface(nx: int, ny: int, model: int = MODEL_AC, W: float = 4.0,
                   rho_ratio: float = 10.0, precision: int = PREC_FP64) -> Case:
    """Flat interface at y = ny/2 (phase A above), periodic in x, walls in y."""
    phiA, phiB = (1.0, -1.0) if model == MODEL_CH else (1.0, 0.0)
    prm = Params(nx=nx, ny=ny, precision=precision, phase_model=model, phiA=phiA, phiB=phiB,
                 bc=(0, 0, 1, 1), rhoA=rho_ratio, rhoB=1.0, muA=0.1 * rho_ratio, muB=0.1,
                 mobility=0.05, width=W, sigma=0.01)
    _, Y = _coords(nx, ny)
    return Case("flat_interface", prm, tanh_profile(Y - 0.5 * ny, W, phiA, phiB))


# --------------------------------------------------------------------------
# The paper's six workloads at sizes the oracle runs in seconds, several
# strips and segments of the step kernels wide with ragged tails (the parity
# cases of the CUDA path and of the oracle's sensitivity record).
# --------------------------------------------------------------------------
PAPER_PARITY_CASES = ("square_droplet_ac", "square_droplet_ch", "rti", "droplet_spreading", "dam_break",
                      "layered_poiseuille")


def paper_parity_case(name: str, precision: int = PREC_FP64, n_delta: float | None = None) -> Case:
    """One of PAPER_PARITY_CASES; n_delta (None: the case's own value)
    sets the regularisation of the interface normal."""
    if name == "square_droplet_ac":
        c = square_droplet(n=256, D=128, precision=precision)
    elif name == "square_droplet_ch":
        c = square_droplet(n=260, D=128, precision=precision)
        c.params.phase_model = MODEL_CH
        c.params.phiA, c.params.phiB = 1.0, -1.0
        c.phi = 2.0 * c.phi - 1.0
    elif name == "rti":
        c = rti(260, 300, d=260.0, amp0=26.0, precision=precision)
    elif name == "droplet_spreading":
        c = droplet_spreading(nx=300, ny=150, R0=60.0, theta=60.0, precision=precision)
    elif name == "dam_break":
        # the less viscous air of the first dam-break recipe (nu_B = 0.1,
        # nu_A = 0.01): the harder case for the normal's conditioning
        c = dam_break(nx=300, ny=150, col_w=100, col_h=100, nuB=0.1, precision=precision)
    elif name == "layered_poiseuille":
        c = layered_poiseuille(nx=4, ny=256, precision=precision)
    else:
        raise ValueError(name)
    c.name = name
    if n_delta is not None:
        c.params = c.params.with_(n_delta=n_delta)
    return c


# Rough seeded inputs that exercise every boundary, model, gravity mode,
# viscosity law, flux model and rate path (noise on phi, u and p excites
# grid-scale dynamics), 300 x 150.
STRESS_CASES = {
    "periodic_ac": dict(walls="none"),
    "ywalls_wet_ac": dict(walls="y", theta=(90, 90, 50, 130), gravity=(GRAV_RHO_MINUS_MEAN, 0.0, -2e-5)),
    "xwalls_wet_ac": dict(walls="x", theta=(40, 140, 90, 90), gravity=(GRAV_RHO, 1e-5, 0.0)),
    "allwalls_ac_inverse_nu": dict(walls="all", theta=(60, 120, 75, 105), gravity=(GRAV_RHO, 0.0, -1e-5),
                                   visc_law=VISC_INVERSE_NU),
    "periodic_ch": dict(walls="none", model=MODEL_CH),
    "allwalls_ch": dict(walls="all", model=MODEL_CH, theta=(70, 110, 80, 100), gravity=(GRAV_CONST, 1e-6, -1e-6)),
    "original_flux": dict(walls="y", flux=FLUX_ORIGINAL),
    "mrt_rates": dict(walls="none", s_f=(1.0, 1.2, 0.8, 0.9, 1.1, 0.9, 1.3, 1.0, 1.0),
                      s_g=(1.0, 1.1, 0.9, 1.0, 1.7, 1.0, 1.7, NAN, NAN)),
}


def stress_case(name: str, precision: int = PREC_FP64) -> Case:
    c = noisy_drop(300, 150, precision=precision, noise=0.005, u_amp=0.002, **STRESS_CASES[name])
    c.name = name
    return c
