"""Pins of the differentiable tensor re-expression (oracle/torch_ref.py), the
autograd reference of the adjoint tests: whole steps against the C oracle by
brute force on tiny grids, and its reverse-mode gradients against central
differences of the C oracle."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")

CASES = {
    "periodic": dict(walls="none"),
    "ywalls_wet_rho_minus_mean": dict(walls="y", theta=(90, 90, 50, 130),
                                      gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -2e-5)),
    "xwalls_wet_rho": dict(walls="x", theta=(40, 140, 90, 90), gravity=(W.GRAV_RHO, 1e-5, 0.0)),
    "allwalls_inverse_nu": dict(walls="all", theta=(60, 120, 75, 105), gravity=(W.GRAV_RHO, 0.0, -1e-5),
                                visc_law=W.VISC_INVERSE_NU),
    "original_flux": dict(walls="y", flux=W.FLUX_ORIGINAL, gravity=(W.GRAV_CONST, 1e-6, -1e-6)),
    "mrt_rates": dict(walls="none", s_f=(1.0, 1.2, 0.8, 0.9, 1.1, 0.9, 1.3, 1.0, 1.0),
                      s_g=(1.0, 1.1, 0.9, 1.0, 1.7, 1.0, 1.7, math.nan, math.nan)),
}


def _ref(prm):
    from oracle.torch_ref import TorchScheme

    return TorchScheme(prm)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nx,ny", [(8, 8), (32, 64)])
def test_tensor_steps_match_oracle(oracle_mod, name, nx, ny):
    """Populations and history after 12 steps from a rough seeded state agree
    with the C oracle to rounding."""
    case = W.noisy_drop(nx, ny, precision=W.PREC_FP64, **CASES[name])
    o = oracle_mod.Oracle(case.params)
    o.init_fields(case.phi)
    ts = _ref(case.params)
    G = torch.tensor([case.params.gx, case.params.gy], dtype=torch.float64)
    f, g, h = ts.init(torch.tensor(case.phi), G)
    for step in (0, 12):
        if step:
            o.step(step)
            for _ in range(step):
                f, g, h = ts.step(f, g, h, G)
        for a, b in ((f, oracle_mod.F_POP), (g, oracle_mod.G_POP), (h, oracle_mod.HIST)):
            ref = o.fields(b)
            err = np.abs(a.detach().numpy() - ref).max()
            assert err <= 1e-13 * max(1.0, np.abs(ref).max()), (name, step, b, err)


def test_tensor_gradients_match_oracle_differences(oracle_mod):
    """d J / d gy and d J / d phi0 at three nodes by autograd through 20 steps,
    against central differences of the C oracle (J = phi-weighted vertical
    centroid)."""
    case = W.noisy_drop(16, 24, precision=W.PREC_FP64, walls="y", theta=(90, 90, 70, 110),
                        gravity=(W.GRAV_RHO, 0.0, -2e-4), noise=0.01, u_amp=0.0)
    prm = case.params
    steps = 20
    ts = _ref(prm)
    phi0 = torch.tensor(case.phi, requires_grad=True)
    G = torch.tensor([prm.gx, prm.gy], dtype=torch.float64, requires_grad=True)
    phiN, _ = ts.run(phi0, G, steps)
    J = ts.centroid_y(phiN)
    J.backward()
    yc = np.arange(prm.ny).reshape(-1, 1) + 0.5

    def J_oracle(prm_, phi_):
        o = oracle_mod.Oracle(prm_)
        o.init_fields(phi_)
        o.step(steps)
        ph = o.fields(oracle_mod.PHI)
        return float((ph * yc).sum() / ph.sum())

    h = 1e-4 * abs(prm.gy)
    fd = (J_oracle(prm.with_(gy=prm.gy + h), case.phi) - J_oracle(prm.with_(gy=prm.gy - h), case.phi)) / (2 * h)
    assert G.grad[1].item() == pytest.approx(fd, rel=1e-5)
    for (j, i) in ((12, 8), (5, 3), (0, 15)):
        hp = 1e-5
        pp = case.phi.copy()
        pm = case.phi.copy()
        pp[j, i] += hp
        pm[j, i] -= hp
        fd = (J_oracle(prm, pp) - J_oracle(prm, pm)) / (2 * hp)
        assert phi0.grad[j, i].item() == pytest.approx(fd, rel=1e-5, abs=1e-9), (j, i)
