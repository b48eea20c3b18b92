"""16-bit deviation storage (FP16 / BF16 populations, FP32 arithmetic and
history) against the FP64 oracle, the FP32 / FP64 GPU paths and the
storage codec's own guarantees.

Error bounds are stated in units of the 16-bit unit roundoff u (2^-11 for
FP16, 2^-8 for BF16), the relative error of one stored deviation:
  * populations after 100 steps of the paper's workloads:
      max |df| / max |f| <= 0.2 u, max |dg| / max |g| <= 8 u, and the dynamic
      part of g (rho0 removed) <= 16 u
    (a deviation is at most a few per cent of the population it encodes,
    and each step re-rounds it: measured 0.05-0.09 u for f, 0.3-5 u for g);
  * one encode/decode round trip: max |df| / max |f| <= 0.05 u and the sum
    of all f unchanged to 1e-7 (phi conserved by the codec);
  * total phi drift <= 1e-5 relative after 500 steps, the bar of the FP32
    path (the codec conserves phi exactly; what remains is FP32 rounding).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

U16 = {W.PREC_FP16_DEV: 2.0 ** -11, W.PREC_BF16_DEV: 2.0 ** -8}
LOWP = [W.PREC_FP16_DEV, W.PREC_BF16_DEV]
LOWP_IDS = ["fp16dev", "bf16dev"]


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2111_00847_gb300 as pk

    return pk


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def paper_cases(prec):
    sq = W.square_droplet(n=256, D=128, precision=prec)
    ch = W.square_droplet(n=260, D=128, precision=prec)
    ch.params.phase_model = W.MODEL_CH
    ch.params.phiA, ch.params.phiB = 1.0, -1.0
    ch.phi = 2.0 * ch.phi - 1.0
    return {
        "square_droplet_ac": sq,
        "square_droplet_ch": ch,
        "rti": W.rti(260, 300, d=260.0, amp0=26.0, precision=prec),
        "droplet_spreading": W.droplet_spreading(nx=300, ny=150, R0=60.0, theta=60.0, precision=prec),
        "dam_break": W.dam_break(nx=300, ny=150, col_w=100, col_h=100, precision=prec),
        "noisy_walls": W.noisy_drop(200, 150, precision=prec, walls="all", theta=(60, 120, 45, 135),
                                    gravity=(W.GRAV_RHO, 1e-6, -1e-5)),
    }


@pytest.mark.parametrize("name", ["square_droplet_ac", "square_droplet_ch", "rti", "droplet_spreading",
                                  "dam_break", "noisy_walls"])
@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
def test_lowp_parity_paper_workloads(pk, oracle_mod, name, prec):
    case = paper_cases(prec)[name]
    u = U16[prec]
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    o = oracle_mod.Oracle(case.params.with_(precision=W.PREC_FP64))
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    sim.step(100)
    o.step(100)
    f, F = sim.fields(pk.LBM_F_POP), o.fields(oracle_mod.F_POP)
    g, G = sim.fields(pk.LBM_G_POP), o.fields(oracle_mod.G_POP)
    assert np.isfinite(f).all() and np.isfinite(g).all()
    ef = rel(f, F)
    eg = rel(g, G)
    gd, Gd = g.copy(), G.copy()
    gd[0] -= case.params.rho0
    Gd[0] -= case.params.rho0
    egd = rel(gd, Gd)
    assert ef <= 0.2 * u, (name, ef / u)
    assert eg <= 8 * u, (name, eg / u)
    assert egd <= 16 * u, (name, egd / u)
    ephi = float(np.abs(sim.fields(pk.LBM_PHI) - o.fields(oracle_mod.PHI)).max())
    assert ephi <= 0.2 * u * (case.params.phiA - case.params.phiB), (name, ephi)


@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
@pytest.mark.parametrize("walls", ["none", "y", "all"])
def test_lowp_codec_roundtrip_conserves_phi(pk, oracle_mod, prec, walls):
    """Populations written with lbm_set_fields come back within the 16-bit
    rounding of their deviations, and the sum of all f (total phi) is kept."""
    case = W.noisy_drop(200, 150, precision=W.PREC_FP64, walls=walls)
    o = oracle_mod.Oracle(case.params)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    o.step(10)
    sim = pk.Simulation(case.params.with_(precision=prec))
    sim.init_fields(case.phi)
    u = U16[prec]
    for which, ow in ((pk.LBM_F_POP, oracle_mod.F_POP), (pk.LBM_G_POP, oracle_mod.G_POP)):
        a = o.fields(ow)
        sim.set_fields(which, a)
        b = sim.fields(which)
        assert rel(b, a) <= 0.05 * u, (which, rel(b, a) / u)
        if which == pk.LBM_F_POP:
            assert abs(b.sum() - a.sum()) <= 1e-7 * np.abs(a).sum()


@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
@pytest.mark.parametrize("walls", ["y", "all"])
def test_lowp_total_phi_drift(pk, prec, walls):
    case = W.noisy_drop(256, 192, precision=prec, walls=walls, theta=(50, 130, 60, 120),
                        gravity=(W.GRAV_RHO, 0.0, -1e-5))
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi, case.ux, case.uy, case.p)
    s0 = sim.diag()["sum_phi"]
    sim.step(500)
    s1 = sim.diag()["sum_phi"]
    assert abs(s1 - s0) <= 1e-5 * abs(s0)


@pytest.mark.parametrize("model", [W.MODEL_AC, W.MODEL_CH], ids=["ac", "ch"])
@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
@pytest.mark.parametrize("walls", ["none", "y", "x", "all"])
@pytest.mark.parametrize("nx,ny", [(300, 150), (16, 70), (257, 129)])
def test_lowp_tma_kernel_matches_register_kernel(pk, prec, walls, nx, ny, model):
    """Both step kernels decode, update and encode the same way; they differ
    only in FP32 rounding (operation order), which can move a deviation to
    the neighbouring 16-bit value.  After one step they agree to a fraction
    of u, after 20 steps to the parity bar."""
    case = W.noisy_drop(nx, ny, precision=prec, walls=walls, noise=0.005, u_amp=0.002, model=model,
                        theta=(60, 120, 45, 135), gravity=(W.GRAV_RHO, 1e-6, -1e-5))
    u = U16[prec]
    sims = []
    for flags in (0, pk.LBM_FLAG_NO_TMA):
        sim = pk.Simulation(case.params.with_(flags=flags))
        sim.init_fields(case.phi, case.ux, case.uy, case.p)
        sims.append(sim)
    for steps, tf in ((1, 0.05 * u), (19, 0.2 * u)):
        for sim in sims:
            sim.step(steps)
        for which in (pk.LBM_F_POP, pk.LBM_G_POP):
            d = rel(sims[0].fields(which), sims[1].fields(which))
            assert d <= tf, (steps, which, d / u)


def _front(phi_row, level=0.5):
    """x of the last crossing of phi = level along a row (linear interpolation)."""
    idx = np.nonzero(phi_row >= level)[0]
    if len(idx) == 0:
        return 0.0
    i = int(idx.max())
    if i + 1 >= len(phi_row):
        return float(i)
    a, b = phi_row[i], phi_row[i + 1]
    return i + (a - level) / (a - b)


@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
def test_lowp_dam_break_full_size(pk, prec, capsys):
    """The reduced-precision configuration: dam break at 4096 x 2048, density
    ratio 1000, viscosity ratio 100, a full-height water column 1024 wide at
    the left wall, gravity 1e-5, walls with 90-degree wetting.  After 4000
    steps (the surge has run about 180 cells; these parameters stay stable
    to about 5500 steps in every precision) the front on the bottom row and
    the total phi drift are compared with the FP32 and FP64 GPU paths.
    Bounds: FP32 within 0.1 cell of FP64, FP16 deviations within 1 cell,
    BF16 deviations within 10 % of the distance the front has run (its
    8-bit significand carries the heavy fluid's momentum at ~0.4 %)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.mem_get_info()[0] < 8e9:
        pytest.skip("needs ~5 GB of device memory")
    steps = 4000
    res = {}
    for p in (W.PREC_FP64, W.PREC_FP32, prec):
        case = W.dam_break(precision=p)
        sim = pk.Simulation(case.params)
        sim.init_fields(case.phi)
        s0 = sim.diag()["sum_phi"]
        sim.step(steps)
        phi = sim.fields(pk.LBM_PHI)
        s1 = sim.diag()["sum_phi"]
        assert np.isfinite(phi).all(), p
        res[p] = (_front(phi[0]), (s1 - s0) / s0, phi)
        sim.close()
    x64, d64, phi64 = res[W.PREC_FP64]
    x32, d32, phi32 = res[W.PREC_FP32]
    xl, dl, phil = res[prec]
    with capsys.disabled():
        print(f"\n[dam break 4096x2048, {steps} steps] front x: fp64 {x64:.3f} fp32 {x32:.3f} "
              f"{LOWP_IDS[LOWP.index(prec)]} {xl:.3f} (start 1024); phi drift: fp64 {d64:.2e} "
              f"fp32 {d32:.2e} lowp {dl:.2e}; max|dphi| vs fp64: fp32 {np.abs(phi32 - phi64).max():.2e} "
              f"lowp {np.abs(phil - phi64).max():.2e}")
    assert x64 > 1024 + 100  # the column has collapsed
    assert abs(x32 - x64) <= 0.1
    if prec == W.PREC_FP16_DEV:
        assert abs(xl - x64) <= 1.0
    else:
        assert abs(xl - x64) <= 0.1 * (x64 - 1024)
    assert abs(d64) <= 1e-12
    assert abs(dl) <= 1e-4 and abs(d32) <= 1e-4


@pytest.mark.parametrize("prec", LOWP, ids=LOWP_IDS)
def test_lowp_full_size_sampled_windows(pk, oracle_mod, prec):
    """The throughput workload at 16384^2 in 16-bit storage, in the launch
    configuration the benchmark times, checked on sampled windows against
    the oracle run on the windows with a 2k margin (k = 100 steps, the
    horizon of the paper-workload bars of this file)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.mem_get_info()[0] < 60e9:
        pytest.skip("needs ~50 GB of device memory")
    n, k, wy = 16384, 100, 48
    m = 2 * k + 6
    case = W.rti_multimode(n, precision=prec)
    x0 = n // 3
    windows = (0, n // 2 - wy // 2, n - wy)
    sim = pk.Simulation(case.params)
    sim.init_fields(case.phi)
    sim.step(k)
    got = {y0: (sim.fields(pk.LBM_F_POP, region=(x0, y0, wy, wy)),
                sim.fields(pk.LBM_G_POP, region=(x0, y0, wy, wy))) for y0 in windows}
    sim.close()
    u = U16[prec]
    rho0 = case.params.rho0
    ref = {}
    for y0 in windows:
        ylo, yhi = max(0, y0 - m), min(n, y0 + wy + m)
        sub = case.params.with_(nx=wy + 2 * m, ny=yhi - ylo, bc=(0, 0, 1, 1), precision=W.PREC_FP64)
        o = oracle_mod.Oracle(sub)
        o.init_fields(np.ascontiguousarray(case.phi[ylo:yhi, x0 - m:x0 + wy + m]))
        o.step(k)
        sl = (slice(None), slice(y0 - ylo, y0 - ylo + wy), slice(m, m + wy))
        go = o.fields(oracle_mod.G_POP)[sl]
        go[0] -= rho0
        ref[y0] = (o.fields(oracle_mod.F_POP)[sl], go)
    # relative to the array maximum over the sampled windows (g without rho0)
    fmax = max(np.abs(ref[y][0]).max() for y in windows)
    gmax = max(np.abs(ref[y][1]).max() for y in windows)
    for y0 in windows:
        fa, ga = got[y0]
        fo, go = ref[y0]
        ga = ga.copy()
        ga[0] -= rho0
        ef, eg = np.abs(fa - fo).max() / fmax / u, np.abs(ga - go).max() / gmax / u
        print(f"\n[16-bit full size, {k} steps] window y0={y0}: f {ef:.3f} u (bar 0.2 u), g {eg:.2f} u (bar 16 u)",
              end="")
        assert ef <= 0.2, (y0, ef)
        assert eg <= 16, (y0, eg)
