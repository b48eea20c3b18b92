"""The hand-written discrete adjoint (lbm_adjoint_*, behind the autograd
function of paper_2111_00847_gb300.adjoint) against
  * PyTorch autograd through the tensor re-expression of the scheme
    (oracle/torch_ref.py) on tiny grids, every boundary and model path the
    adjoint covers, several checkpoint segments with a ragged last one:
    dJ/dphi0 and dJ/dG to 1e-9 relative (FP64 against FP64, different
    operation order);
  * central differences of the FP64 GPU forward on the adjoint workload
    (512 x 2048 RTI, Atwood 0.5, Re 1000, 8 seeded cosine modes, 2000 steps,
    checkpoints every 100): dJ/da_k and dJ/dg to 1e-4 relative, J the
    phi-weighted vertical centroid.
"""
import math
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


CASES = {
    "periodic": dict(walls="none", gravity=(W.GRAV_CONST, 1e-5, -2e-5)),
    "ywalls_wet_rho_minus_mean": dict(walls="y", theta=(90, 90, 50, 130),
                                      gravity=(W.GRAV_RHO_MINUS_MEAN, 0.0, -2e-5)),
    "xwalls_wet_rho": dict(walls="x", theta=(40, 140, 90, 90), gravity=(W.GRAV_RHO, 1e-5, -1e-5)),
    "allwalls_inverse_nu": dict(walls="all", theta=(60, 120, 75, 105), gravity=(W.GRAV_RHO, 2e-6, -1e-5),
                                visc_law=W.VISC_INVERSE_NU),
    "original_flux": dict(walls="y", flux=W.FLUX_ORIGINAL, gravity=(W.GRAV_CONST, 1e-6, -1e-6)),
    "mrt_rates": dict(walls="none", s_f=(1.0, 1.2, 0.8, 0.9, 1.1, 0.9, 1.3, 1.0, 1.0),
                      s_g=(1.0, 1.1, 0.9, 1.0, 1.7, 1.0, 1.7, math.nan, math.nan),
                      gravity=(W.GRAV_RHO, 1e-6, -1e-5)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [W.PREC_FP64])
def test_adjoint_matches_autograd(pk, name, prec):
    from oracle.torch_ref import TorchScheme
    from paper_2111_00847_gb300.adjoint import rollout

    case = W.noisy_drop(32, 64, precision=prec, noise=0.01, **CASES[name])
    prm = case.params
    steps, every = 60, 16  # three full segments and a ragged one of 12 steps
    wts = torch.from_numpy(W.uniform_array(7, prm.nx * prm.ny).reshape(prm.ny, prm.nx) - 0.5)

    phi0 = torch.tensor(case.phi, requires_grad=True)
    G = torch.tensor([prm.gx, prm.gy], dtype=torch.float64, requires_grad=True)
    ts = TorchScheme(prm)
    phiN_ref, _ = ts.run(phi0, G, steps)
    (phiN_ref * wts).sum().backward()
    g_phi_ref, g_G_ref = phi0.grad.clone(), G.grad.clone()

    phi0b = torch.tensor(case.phi, requires_grad=True)
    Gb = torch.tensor([prm.gx, prm.gy], dtype=torch.float64, requires_grad=True)
    phiN = rollout(phi0b, Gb, prm, steps, every)
    assert torch.abs(phiN - phiN_ref.detach()).max() <= 1e-12
    (phiN * wts).sum().backward()
    e_phi = (phi0b.grad - g_phi_ref).abs().max() / g_phi_ref.abs().max()
    assert e_phi <= 1e-9, float(e_phi)
    for k in range(2):
        assert Gb.grad[k].item() == pytest.approx(g_G_ref[k].item(), rel=1e-9, abs=1e-12 * abs(g_G_ref).max().item())


def test_adjoint_one_segment_equals_many(pk):
    """The gradient does not depend on the checkpoint spacing."""
    from paper_2111_00847_gb300.adjoint import centroid_y, rollout

    case = W.noisy_drop(48, 40, precision=W.PREC_FP64, walls="y", theta=(90, 90, 60, 120),
                        gravity=(W.GRAV_RHO, 0.0, -1e-5))
    out = []
    for every in (1, 7, 50):
        phi0 = torch.tensor(case.phi, requires_grad=True)
        G = torch.tensor([case.params.gx, case.params.gy], dtype=torch.float64, requires_grad=True)
        centroid_y(rollout(phi0, G, case.params, 50, every)).backward()
        out.append((phi0.grad.clone(), G.grad.clone()))
    for a, b in out[1:]:
        assert torch.equal(a, out[0][0]) and torch.equal(b, out[0][1])


def test_adjoint_rti_workload_central_differences(pk, capsys):
    """The adjoint workload: gradient of the final phi-weighted centroid with
    respect to the 8 seeded amplitudes and g, against central differences
    of the FP64 forward (Richardson-extrapolated from steps h and h/2)."""
    from paper_2111_00847_gb300 import LBM_PHI, Simulation
    from paper_2111_00847_gb300.adjoint import centroid_y, interface_phi0, rollout

    if torch.cuda.mem_get_info()[0] < 40e9:
        pytest.skip("needs ~30 GB of device memory")
    case = W.rti_adjoint(precision=W.PREC_FP64)
    prm = case.params
    a0 = torch.tensor(case.notes["a"], dtype=torch.float64)
    g0 = -prm.gy
    steps, every = 2000, 100

    def phi0_of(a):
        return interface_phi0(a, prm.nx, prm.ny, prm.width, prm.phiA, prm.phiB)

    assert np.abs(phi0_of(a0).numpy() - case.phi).max() < 1e-12

    a = a0.clone().requires_grad_(True)
    gv = torch.tensor([0.0, -g0], dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phiN = rollout(phi0_of(a), gv, prm, steps, every)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    J = centroid_y(phiN)
    t0 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    grad_a = a.grad.numpy().copy()
    grad_g = -gv.grad[1].item()

    yc = np.arange(prm.ny).reshape(-1, 1) + 0.5

    def J_of(av, g):
        sim = Simulation(prm.with_(gy=-g))
        sim.init_fields(phi0_of(torch.tensor(av)).numpy())
        sim.step(steps)
        ph = sim.fields(LBM_PHI)
        sim.close()
        return float((ph * yc).sum() / ph.sum())

    def richardson(fun, x, h):
        d1 = (fun(x + h) - fun(x - h)) / (2 * h)
        d2 = (fun(x + h / 2) - fun(x - h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_a = []
    for k in range(8):
        def fk(v, k=k):
            av = a0.numpy().copy()
            av[k] = v
            return J_of(av, g0)
        fd_a.append(richardson(fk, float(a0[k]), 0.05))
    fd_g = richardson(lambda g: J_of(a0.numpy(), g), g0, 0.02 * g0)
    with capsys.disabled():
        print(f"\n[adjoint 512x2048 RTI, {steps} steps, checkpoints every {every}] J = {J.item():.9f}")
        for k in range(8):
            print(f"  dJ/da_{k + 1}: adjoint {grad_a[k]: .9e}  central difference {fd_a[k]: .9e}")
        print(f"  dJ/dg:    adjoint {grad_g: .9e}  central difference {fd_g: .9e}")
        print(f"  forward {t_fwd:.2f} s, backward (recompute + adjoint) {t_bwd:.2f} s, "
              f"ratio {t_bwd / t_fwd:.2f}")
    scale = max(np.abs(grad_a).max(), 1e-300)
    for k in range(8):
        assert abs(grad_a[k] - fd_a[k]) <= 1e-4 * max(abs(fd_a[k]), 1e-3 * scale), k
    assert grad_g == pytest.approx(fd_g, rel=1e-4)


def test_fp32_adjoint_tracks_fp64(pk, capsys):
    """The same workload run and differentiated in FP32 (forward state and
    adjoint arithmetic): the gradient stays within 5e-3 of the FP64 one
    relative to its largest component (measured 1.4e-3), dJ/dg within 1e-3
    (measured 9e-5) -- a 7x cheaper path where that accuracy suffices."""
    from paper_2111_00847_gb300.adjoint import centroid_y, interface_phi0, rollout

    if torch.cuda.mem_get_info()[0] < 40e9:
        pytest.skip("needs ~30 GB of device memory")
    out = {}
    for prec in (W.PREC_FP64, W.PREC_FP32):
        case = W.rti_adjoint(precision=prec)
        prm = case.params
        a = torch.tensor(case.notes["a"], dtype=torch.float64, requires_grad=True)
        G = torch.tensor([prm.gx, prm.gy], dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phiN = rollout(interface_phi0(a, prm.nx, prm.ny, prm.width, prm.phiA, prm.phiB), G, prm, 2000, 100)
        centroid_y(phiN).backward()
        torch.cuda.synchronize()
        out[prec] = (a.grad.numpy().copy(), G.grad[1].item(), time.perf_counter() - t0)
    g64, gy64, t64 = out[W.PREC_FP64]
    g32, gy32, t32 = out[W.PREC_FP32]
    e = np.abs(g32 - g64).max() / np.abs(g64).max()
    with capsys.disabled():
        print(f"\n[adjoint FP32 vs FP64] amplitudes {e:.2e}, g {abs(gy32 - gy64) / abs(gy64):.2e}; "
              f"forward + backward {t64:.2f} s (FP64), {t32:.2f} s (FP32)")
    assert e <= 5e-3
    assert gy32 == pytest.approx(gy64, rel=1e-3)


def test_snapshot_restore_continues_bit_exactly(pk):
    """A state restored from a snapshot steps on exactly as the run it was
    taken from."""
    case = W.noisy_drop(96, 80, precision=W.PREC_FP32, walls="all", theta=(60, 120, 75, 105),
                        gravity=(W.GRAV_RHO, 0.0, -1e-5))
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    sim.step(10)
    buf = sim.snapshot(sim.new_state_buffer())
    sim.step(20)
    ref = [sim.fields(w) for w in (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST)]
    sim.step(5)
    sim.restore(buf, 10)
    assert sim.t == 10
    sim.step(20)
    for a, w in zip(ref, (pk.LBM_F_POP, pk.LBM_G_POP, pk.LBM_HIST)):
        assert np.array_equal(a, sim.fields(w))


def test_adjoint_rejects_what_it_does_not_cover(pk):
    """Cahn-Hilliard, 16-bit storage and an initial velocity are refused with
    LBM_EUNSUPPORTED; an adjoint step before the seed with LBM_EINVAL."""
    dj = np.zeros((40, 48))
    for prm in (W.noisy_drop(48, 40, precision=W.PREC_FP64, model=W.MODEL_CH).params,
                W.noisy_drop(48, 40, precision=W.PREC_FP16_DEV).params):
        sim = pk.Simulation(prm)
        sim.init_fields(np.full((40, 48), 0.5))
        with pytest.raises(pk.LbmError) as ei:
            sim.adjoint_seed(dj)
        assert ei.value.code == pk.LBM_EUNSUPPORTED
    case = W.noisy_drop(48, 40, precision=W.PREC_FP64)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy)
    s0 = sim.snapshot(sim.new_state_buffer())
    with pytest.raises(pk.LbmError) as ei:
        sim.adjoint_step(s0)
    assert ei.value.code == pk.LBM_EINVAL
    sim.adjoint_seed(dj)
    with pytest.raises(pk.LbmError) as ei:
        sim.adjoint_init(s0)
    assert ei.value.code == pk.LBM_EUNSUPPORTED
