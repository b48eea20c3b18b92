"""Differentiable FP64 re-expression of the scheme in PyTorch tensor ops.

TEST INFRASTRUCTURE ONLY: the adjoint tests use it as the autograd reference
on tiny grids (reverse mode through the whole time loop by PyTorch's own
autograd).  It is written again from the paper -- it shares no code with the
C oracle beside it or with the CUDA path -- and is pinned to the C oracle by
brute-force comparison of whole steps on small grids (tests/test_torch_ref.py).

One time step t -> t+1 (Sec. 3, App. C), on pulled populations f, g
[9, ny, nx] and the history chi(t-1) [5, ny, nx] of the explicit-Euler time
derivatives:
  phi = sum f (Eq. (22a)); ghost ring of phi (x sides first, then y sides
  over the extended x range; wetting ghosts from Eqs. (49)-(50)); isotropic
  grad and Laplacian (Eqs. (C.9)-(C.10)); mu_phi (Eq. (5)); Allen-Cahn
  lambda, n, D (Eqs. (7)-(8), n = grad phi / (|grad phi|^4 + delta_n^4)^(1/4));
  rho, nu (Eqs. (10)-(12)); m^{phi C} (Eq. (15)); F = mu grad phi + G;
  u (Eq. (22b)); p (Eq. (39), second way of Remark 1); MRT collisions
  (Eqs. (17), (40) with the moment vectors of Eqs. (C.2)-(C.4)); pull
  streaming with half-way bounce-back.
Only the Allen-Cahn phase field is expressed (the adjoint covers it).
"""
from __future__ import annotations

import math

import torch

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
CS2 = 1.0 / 3.0


def moment_matrix(dtype=torch.float64):
    """The orthogonal D2Q9 transformation of Eq. (C.1): rows are the basis
    vectors 1, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy evaluated on c_i."""
    rows = []
    for fn in (lambda x, y: 1.0,
               lambda x, y: -4.0 + 3.0 * (x * x + y * y),
               lambda x, y: 4.0 - 10.5 * (x * x + y * y) + 4.5 * (x * x + y * y) ** 2,
               lambda x, y: float(x),
               lambda x, y: (-5.0 + 3.0 * (x * x + y * y)) * x,
               lambda x, y: float(y),
               lambda x, y: (-5.0 + 3.0 * (x * x + y * y)) * y,
               lambda x, y: float(x * x - y * y),
               lambda x, y: float(x * y)):
        rows.append([fn(CX[i], CY[i]) for i in range(9)])
    return torch.tensor(rows, dtype=dtype)


class TorchScheme:
    """The scheme for one parameter set (a workloads.Params); AC only."""

    def __init__(self, prm):
        if prm.phase_model != 0:
            raise ValueError("the tensor re-expression covers the Allen-Cahn phase field only")
        if prm.flux_model not in (0, 1):
            raise ValueError("flux model")
        self.p = prm
        self.nx, self.ny = prm.nx, prm.ny
        self.M = moment_matrix()
        # M^{-1} = M^T diag(1 / |row|^2) (orthogonal rows)
        self.Minv = self.M.t() / (self.M * self.M).sum(1)
        dphi = prm.phiA - prm.phiB
        self.beta = 12.0 * prm.sigma / (prm.width * dphi ** 4)          # Eq. (3)
        self.kappa = 1.5 * prm.sigma * prm.width / dphi ** 2
        self.lam_coef = (math.sqrt(2.0 * self.beta / self.kappa) if prm.sigma > 0
                         else 4.0 / (prm.width * dphi))                   # Eq. (8)
        self.drho = (prm.rhoA - prm.rhoB) / dphi                          # Eq. (10)
        nd = getattr(prm, "n_delta", 0.0)
        self.delta_n = (nd if nd > 0 else 5e-3) * dphi / prm.width
        sfm = 1.0 / (prm.mobility / (prm.eta * CS2) + 0.5)
        self.Sf = [(sfm if k in (3, 5) else 1.0) if math.isnan(prm.s_f[k]) else prm.s_f[k] for k in range(9)]
        self.Sg = [1.0 if math.isnan(prm.s_g[k]) else prm.s_g[k] for k in range(9)]
        self.sg_node = [math.isnan(prm.s_g[k]) and k in (7, 8) for k in range(9)]
        self.wall_x = prm.bc[0] == 1
        self.wall_y = prm.bc[2] == 1
        self.cos_t = [0.0 if t == 90.0 else math.cos(math.radians(t)) for t in prm.theta_deg]
        # H = (s_g^2 - s_g^0) / (9 s_g^0 s_g^2), K = 1/3 (App. C, Eq. (39))
        self.H = (self.Sg[2] - self.Sg[0]) / (9.0 * self.Sg[0] * self.Sg[2])
        self.K = 1.0 / 3.0
        yy = torch.arange(self.ny, dtype=torch.float64).view(-1, 1).expand(self.ny, self.nx)
        self.ycentre = yy + 0.5

    # -- wetting ghost, Eqs. (49)-(50): quadratic through (0, phi_w), (1/2, phi_1),
    #    (3/2, phi_2) evaluated at -1/2; phi_w the root the paper selects
    def wall_ghost(self, phi1, phi2, side):
        p = self.p
        a = 4.0 * self.cos_t[side] / (p.width * (p.phiA - p.phiB))
        b = 8.0 / 3.0 - a * (p.phiA + p.phiB)
        c = a * p.phiA * p.phiB + phi2 / 3.0 - 3.0 * phi1
        disc = torch.clamp(b * b - 4.0 * a * c, min=0.0)
        phiw = 2.0 * c / (-b - torch.sqrt(disc))
        return 8.0 / 3.0 * phiw - 2.0 * phi1 + phi2 / 3.0

    def pad(self, phi):
        """[ny + 2, nx + 2] with the ghost ring."""
        if self.wall_x:
            left = self.wall_ghost(phi[:, 0], phi[:, 1], 0)
            right = self.wall_ghost(phi[:, -1], phi[:, -2], 1)
        else:
            left, right = phi[:, -1], phi[:, 0]
        ext = torch.cat([left.unsqueeze(1), phi, right.unsqueeze(1)], dim=1)
        if self.wall_y:
            bot = self.wall_ghost(ext[0], ext[1], 2)
            top = self.wall_ghost(ext[-1], ext[-2], 3)
        else:
            bot, top = ext[-1], ext[0]
        return torch.cat([bot.unsqueeze(0), ext, top.unsqueeze(0)], dim=0)

    def stencils(self, phi):
        """grad = sum w_i c_i phi(x + c_i) / c_s^2, lap = sum 2 w_i (phi(x + c_i) - phi) / c_s^2."""
        P = self.pad(phi)
        ny, nx = self.ny, self.nx
        gx = torch.zeros_like(phi)
        gy = torch.zeros_like(phi)
        lap = torch.zeros_like(phi)
        for k in range(1, 9):
            v = P[1 + CY[k]:1 + CY[k] + ny, 1 + CX[k]:1 + CX[k] + nx]
            gx = gx + W[k] * CX[k] * v / CS2
            gy = gy + W[k] * CY[k] * v / CS2
            lap = lap + 2.0 * W[k] * (v - phi) / CS2
        return gx, gy, lap

    def macro(self, f, g, hist, G):
        """Everything the collisions need at time t (dictionary of fields)."""
        p = self.p
        phi = f.sum(0)
        gx, gy, lap = self.stencils(phi)
        mu = 4.0 * self.beta * (phi - p.phiA) * (phi - p.phiB) * (phi - 0.5 * (p.phiA + p.phiB)) - self.kappa * lap
        lam = self.lam_coef * (p.phiA - phi) * (phi - p.phiB)
        g2 = gx * gx + gy * gy
        gm = torch.sqrt(torch.sqrt(g2 * g2 + self.delta_n ** 4))
        nxv, nyv = gx / gm, gy / gm
        Dx, Dy = gx - lam * nxv, gy - lam * nyv
        rho = self.drho * (phi - p.phiB) + p.rhoB
        rx, ry = self.drho * gx, self.drho * gy
        frac = (phi - p.phiB) / (p.phiA - p.phiB)
        if p.visc_law == 0:
            nu = (frac * (p.muA - p.muB) + p.muB) / rho
        else:
            nu = 1.0 / (frac * (p.rhoA / p.muA - p.rhoB / p.muB) + p.rhoB / p.muB)
        s78 = 1.0 / (nu / CS2 + 0.5)
        if p.flux_model == 0:
            mx, my = -self.drho * p.mobility * Dx, -self.drho * p.mobility * Dy
        else:
            mx, my = torch.zeros_like(phi), torch.zeros_like(phi)
        if p.gravity_mode == 0:
            Gs = torch.ones_like(phi)
        elif p.gravity_mode == 1:
            Gs = rho
        else:
            Gs = rho - 0.5 * (p.rhoA + p.rhoB)
        Fx = mu * gx + Gs * G[0]
        Fy = mu * gy + Gs * G[1]
        jx = sum(CX[i] * g[i] for i in range(9) if CX[i])
        jy = sum(CY[i] * g[i] for i in range(9) if CY[i])
        u = (jx + 0.5 * Fx) / rho
        v = (jy + 0.5 * Fy) / rho
        cur = torch.stack([phi * u, phi * v, u * mx + v * my, u * mx - v * my, u * my + v * mx])
        dt = cur - hist
        s0 = -W[0] * (rho * (u * u + v * v) + cur[2]) / (2.0 * CS2)
        gsum = g[1:].sum(0)
        pr = CS2 / (1.0 - W[0]) * (gsum + (0.5 + self.H) * (u * rx + v * ry) + s0
                                   + self.K * (2.0 * (Fx * u + Fy * v) + dt[2]))
        return dict(phi=phi, mu=mu, lam=lam, nx=nxv, ny=nyv, rho=rho, rx=rx, ry=ry, s78=s78,
                    mx=mx, my=my, Fx=Fx, Fy=Fy, u=u, v=v, cur=cur, dt=dt, p=pr)

    def collide(self, f, g, d):
        p = self.p
        phi, u, v, rho = d["phi"], d["u"], d["v"], d["rho"]
        mx, my, Fx, Fy, rx, ry = d["mx"], d["my"], d["Fx"], d["Fy"], d["rx"], d["ry"]
        dt = d["dt"]
        z = torch.zeros_like(phi)
        # Eq. (C.4) with eta, and its source (lambda c_s^2 n + d_t(phi u)) projected
        mfeq = torch.stack([phi, -4.0 * phi + 2.0 * p.eta * phi, 4.0 * phi - 3.0 * p.eta * phi,
                            phi * u, -phi * u, phi * v, -phi * v, z, z])
        Xx = dt[0] + d["lam"] * d["nx"] / 3.0
        Xy = dt[1] + d["lam"] * d["ny"] / 3.0
        mR = torch.stack([z, z, z, Xx, -Xx, Xy, -Xy, z, z])
        uu = u * u + v * v
        um = u * mx + v * my
        mgeq = torch.stack([z + p.rho0, -4.0 * p.rho0 + 6.0 * d["p"] + 3.0 * rho * uu + 3.0 * um,
                            4.0 * p.rho0 - 9.0 * d["p"] - 3.0 * rho * uu - 3.0 * um,
                            rho * u, -rho * u, rho * v, -rho * v,
                            u * mx - v * my + rho * (u * u - v * v),
                            (u * my + v * mx + 2.0 * rho * u * v) / 2.0])
        ugr = u * rx + v * ry
        uF = u * Fx + v * Fy
        mF = torch.stack([ugr, 3.0 * dt[2] + 6.0 * uF, -ugr - 3.0 * dt[2] - 6.0 * uF, Fx, -Fx, Fy, -Fy,
                          2.0 / 3.0 * (u * rx - v * ry) + 2.0 * (u * Fx - v * Fy) + dt[3],
                          1.0 / 3.0 * (u * ry + v * rx) + (2.0 * (u * Fy + v * Fx) + dt[4]) / 2.0])
        Sf = torch.tensor(self.Sf, dtype=torch.float64).view(9, 1, 1).expand(9, self.ny, self.nx)
        Sg = torch.tensor(self.Sg, dtype=torch.float64).view(9, 1, 1).expand(9, self.ny, self.nx).clone()
        for k in (7, 8):
            if self.sg_node[k]:
                Sg = torch.cat([Sg[:k], d["s78"].unsqueeze(0), Sg[k + 1:]])
        mf = torch.einsum("kj,jyx->kyx", self.M, f)
        mg = torch.einsum("kj,jyx->kyx", self.M, g)
        msf = (1.0 - Sf) * mf + Sf * mfeq + (1.0 - 0.5 * Sf) * mR
        msg = (1.0 - Sg) * mg + Sg * mgeq + (1.0 - 0.5 * Sg) * mF
        return torch.einsum("ik,kyx->iyx", self.Minv, msf), torch.einsum("ik,kyx->iyx", self.Minv, msg)

    def stream(self, s):
        """Pull with half-way bounce-back: x_i(x) = x_i*(x - c_i), or x_opp(i)*(x)
        where x - c_i lies beyond a wall."""
        out = []
        X = torch.arange(self.nx).view(1, -1)
        Y = torch.arange(self.ny).view(-1, 1)
        for i in range(9):
            moved = torch.roll(s[i], shifts=(CY[i], CX[i]), dims=(0, 1))
            beyond = torch.zeros(self.ny, self.nx, dtype=torch.bool)
            if self.wall_x:
                beyond = beyond | ((X - CX[i]) < 0) | ((X - CX[i]) >= self.nx)
            if self.wall_y:
                beyond = beyond | ((Y - CY[i]) < 0) | ((Y - CY[i]) >= self.ny)
            out.append(torch.where(beyond, s[OPP[i]], moved))
        return torch.stack(out)

    # -- the initial state (reading: f = f^eq(phi0, 0), g = g^eq(0, 0) with
    #    m^{phi C}(phi0), then chi(-1) := chi(0) so the first derivatives vanish)
    def init(self, phi0, G):
        p = self.p
        z = torch.zeros_like(phi0)
        mfeq = torch.stack([phi0, -4.0 * phi0 + 2.0 * p.eta * phi0, 4.0 * phi0 - 3.0 * p.eta * phi0,
                            z, z, z, z, z, z])
        mgeq = torch.stack([z + p.rho0, z - 4.0 * p.rho0, z + 4.0 * p.rho0, z, z, z, z, z, z])
        f = torch.einsum("ik,kyx->iyx", self.Minv, mfeq)
        g = torch.einsum("ik,kyx->iyx", self.Minv, mgeq)
        hist0 = torch.zeros(5, self.ny, self.nx, dtype=torch.float64)
        d = self.macro(f, g, hist0, G)
        return f, g, d["cur"]

    def step(self, f, g, hist, G):
        d = self.macro(f, g, hist, G)
        fs, gs = self.collide(f, g, d)
        return self.stream(fs), self.stream(gs), d["cur"]

    def run(self, phi0, G, steps):
        """phi after `steps` steps from phi0 (u = p = 0) under gravity G = (gx, gy)."""
        f, g, h = self.init(phi0, G)
        for _ in range(steps):
            f, g, h = self.step(f, g, h, G)
        return f.sum(0), (f, g, h)

    def centroid_y(self, phi):
        """The phi-weighted vertical centroid (node centres at j + 1/2)."""
        return (phi * self.ycentre).sum() / phi.sum()
