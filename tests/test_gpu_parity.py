"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (FP32 mesh/FFT/particle arithmetic against FP64):
  single-step PM force rel-L2 <= 1e-5; 2LPT fields rel-L2 <= 1e-5;
  FFT rel-L2 <= 1e-6; step table rel <= 1e-9 (both FP64);
  P(k) per bin rel <= 1e-5 on identical positions, mode counts exact;
  after a full 40-step run: P(k) within 1e-3 for k <= k_Ny/2 and rms
  displacement difference <= 1e-3 of the mean inter-particle spacing.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cola as ocola
from oracle import cosmology as cm
from oracle import lpt, pm, power
from synth import random_displacements, random_mesh

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev, f32, host, rel_l2  # noqa: E402

COSMO = cm.Cosmology()


def config(nq, ng, L, n_steps=40, a_init=0.05, **kw):
    return C.make_config(nq, ng, L, a_init, 1.0, n_steps, **kw)


@pytest.fixture(scope="module")
def growth():
    return cm.Growth(COSMO)


@pytest.fixture(scope="module")
def plin():
    return cm.LinearPower(COSMO)


# ---------------------------------------------------------------- FFT ------
def _check_fft3d(n):
    x = random_mesh(n, (n, n, n)).astype(np.float64)
    P = C.cola_fft_pitch(n)
    buf = torch.zeros((n, n, 2 * P), dtype=torch.float32, device="cuda")
    buf[:, :, :n] = dev(x)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    C.cola_fft3d_r2c(n, buf, ws)
    got = host(buf).reshape(n, n, P, 2)
    got = got[..., 0] + 1j * got[..., 1]
    ref = np.fft.rfftn(f32(x))
    assert rel_l2(got[:, :, : n // 2 + 1], ref) < 1e-6
    C.cola_fft3d_c2r(n, buf, ws)
    back = host(buf)[:, :, :n] / n**3
    assert rel_l2(back, f32(x)) < 1e-6


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12, 18, 20, 30, 48, 96, 128, 160, 192, 250, 256, 384])
def test_fft3d_r2c_c2r_vs_numpy(n):
    _check_fft3d(n)


# (n, B): every specialised strided-pass tile (compile-time n and width) and
# runtime-engine widths next to them; cola_fft_set_tile forces the width
TILE_CASES = [(96, 16), (128, 16), (160, 16), (192, 16), (256, 8), (256, 16), (288, 16), (288, 8), (320, 16),
              (320, 4), (384, 8), (384, 16), (480, 8), (480, 16), (250, 2)]


@pytest.mark.parametrize("n,B", TILE_CASES)
def test_fft3d_tile_widths_vs_numpy(n, B):
    C.cola_fft_set_tile(n, B)
    try:
        _check_fft3d(n)
    finally:
        C.cola_fft_set_tile(n, 0)


def test_fft_set_tile_rejects_bad_widths():
    for n, B in ((96, 3), (96, 32), (1, 4), (8192, 4), (4096, 16)):
        with pytest.raises(C.ColaError):
            C.cola_fft_set_tile(n, B)


def test_fft_rejects_bad_sizes():
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    buf = torch.zeros(4096, dtype=torch.float32, device="cuda")
    for n in (14, 7, 0, 8192):
        with pytest.raises(C.ColaError):
            C.cola_fft3d_r2c(n, buf, ws)


# ---------------------------------------------------------------- tables ---
@pytest.mark.parametrize("sampling,p,flags", [(C.SAMPLING_LINEAR, 1.0, 0), (C.SAMPLING_LOG, 1.0, 0),
                                               (C.SAMPLING_POW, 0.8, 0), (C.SAMPLING_LINEAR, 1.0, C.FLAG_MODIFIED_KDK),
                                               (C.SAMPLING_LOG, 1.0, C.FLAG_MODIFIED_KDK)])
def test_step_table_vs_oracle(growth, sampling, p, flags):
    cfg = config(8, 16, 64.0, n_steps=12, a_init=1 / 40, sampling=sampling, sampling_p=p, flags=flags)
    sim = C.Simulation(cfg)
    sim.init_tables()
    got = host(sim.table())
    name = {C.SAMPLING_LINEAR: "linear", C.SAMPLING_LOG: "log", C.SAMPLING_POW: "pow"}[sampling]
    a = cm.time_nodes(1 / 40, 1.0, 12, name, p)
    t = cm.step_table(COSMO, a, growth, modified=bool(flags & C.FLAG_MODIFIED_KDK))
    for col, name in enumerate(C.TABLE_COLUMNS):
        ref = getattr(t, name)
        np.testing.assert_allclose(got[:, col], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max(), err_msg=name)


# ---------------------------------------------------------------- deposit --
@pytest.mark.parametrize("nq,ng,L", [(32, 96, 128.0), (6, 18, 30.0), (10, 30, 50.0), (8, 12, 40.0), (16, 16, 64.0)])
def test_density_vs_oracle(nq, ng, L):
    d = random_displacements(nq * 7 + ng, nq, 0.6 * L / nq)
    cfg = config(nq, ng, L)
    sim = C.Simulation(cfg)
    sim.init_tables()
    sim.d.copy_(dev(d))
    got = host(sim.density())
    ref = pm.density_contrast(f32(d), nq, ng, L)
    m3 = (ng / nq) ** 3
    assert np.abs(got - ref).max() < 3e-6 * m3 * (1 + np.abs(ref).max() / m3)
    assert abs(got.mean()) < 1e-6 * m3
    again = host(sim.density())
    np.testing.assert_array_equal(got, again)  # fixed-point deposit is deterministic


# (nq, ng): whole tiles, ragged bricks (nq not a multiple of 8) and ragged tiles
TRAVERSAL_CASES = [(32, 96), (20, 60), (36, 72), (90, 180)]


@pytest.mark.parametrize("nq,ng", TRAVERSAL_CASES)
def test_particle_traversal_tiles_give_identical_results(nq, ng):
    # the tile order of the particle kernels visits every particle once, so the
    # deposit (integer adds), forces and a fused kick + drift are bit-identical
    L = float(ng)
    d = f32(random_displacements(5 * nq + 1, nq, 2.0 * L / nq))
    rng = np.random.default_rng(nq)
    v, psi1, psi2 = (f32(rng.standard_normal((3, nq**3)) * 0.3) for _ in range(3))
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    out = {}
    try:
        for edge, bk in ((0, 0), (32, 8), (32, 16), (64, 8), (64, 32), (128, 64), (256, 256), (4096, 16)):
            C.cola_particle_set_traversal(edge, bk)
            sim.load_state(dev(d), dev(v), dev(psi1), dev(psi2))
            rho = host(sim.density())
            F = host(sim.force(0.5))
            sim.step(7)
            out[edge, bk] = (rho, F, host(sim.d), host(sim.v))
    finally:
        C.cola_particle_set_traversal(0, 0)
    for key, res in out.items():
        for a, b in zip(res, out[0, 0]):
            np.testing.assert_array_equal(a, b, err_msg=f"edge, brick {key}")
    ref = pm.density_contrast(d, nq, ng, L)
    m3 = (ng / nq) ** 3
    assert np.abs(out[0, 0][0] - ref).max() < 3e-6 * m3 * (1 + np.abs(ref).max() / m3)
    assert sim.status() == 0


def test_density_with_every_particle_on_one_point():
    # the degenerate deposit: 32^3 particles on one point fill the eight cells around
    # it with fixed-point sums of up to 2^40 x 2^15 each (no uint64 overflow)
    nq, ng, L = 32, 96, 128.0
    p = np.arange(nq**3)
    q = np.stack([p // (nq * nq), (p // nq) % nq, p % nq]).astype(np.float64) * (L / nq) + L / (2 * ng)
    target = np.array([[37.3], [5.9], [101.7]])
    d = f32(target - q)
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.d.copy_(dev(d))
    got = host(sim.density())
    ref = pm.density_contrast(d, nq, ng, L)
    m3 = (ng / nq) ** 3
    hot = ref > 0
    assert hot.sum() == 8
    # FP32 positions round the CIC fractions at ~1e-5 of a cell for every particle alike
    np.testing.assert_allclose(got[hot], ref[hot], rtol=1e-4)
    np.testing.assert_array_equal(got[~hot], -1.0)
    assert (got + 1).sum() == pytest.approx(nq**3 * m3, rel=1e-6)


# ---------------------------------------------------------------- force ----
def _oracle_state(seed, nq, L, plin, growth, a=0.05):
    D1, _, D2, _ = growth(np.array([a]))
    return lpt.initial_conditions(seed, nq, L, plin, D1[0], D2[0])


@pytest.mark.parametrize("nq,ng,L", [(32, 96, 128.0), (16, 48, 64.0), (10, 30, 40.0), (12, 18, 48.0)])
def test_pm_force_vs_oracle_initial_field(nq, ng, L, plin, growth):
    st = _oracle_state(3, nq, L, plin, growth)
    d = f32(st["d"])
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.d.copy_(dev(d))
    got = host(sim.force(0.05))
    ref = pm.pm_force(d, nq, ng, L, 1.5 * COSMO.omega_m / 0.05)
    assert rel_l2(got, ref) < 1e-5


# (nq, ng, B): the fused Green pass and the y passes at every specialised
# tile, on seeded Gaussian displacements of 0.7 particle spacings rms
FORCE_TILE_CASES = [(48, 96, 16), (64, 128, 16), (80, 160, 16), (64, 192, 16), (128, 256, 8), (128, 256, 16),
                    (96, 288, 16), (160, 320, 16), (128, 384, 8), (128, 384, 16), (160, 480, 8), (160, 480, 16),
                    (64, 192, 4)]


@pytest.mark.parametrize("nq,ng,B", FORCE_TILE_CASES)
def test_pm_force_tile_widths_vs_oracle(nq, ng, B):
    L = float(ng)
    d = f32(random_displacements(11, nq, 0.7 * L / nq))
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.d.copy_(dev(d))
    C.cola_fft_set_tile(ng, B)
    try:
        got = host(sim.force(0.5))
    finally:
        C.cola_fft_set_tile(ng, 0)
    ref = pm.pm_force(d, nq, ng, L, 1.5 * COSMO.omega_m / 0.5)
    assert rel_l2(got, ref) < 1e-5


def test_pm_force_vs_oracle_clustered(plin, growth):
    # a strongly displaced state: 2LPT field scaled to a ~ 1 amplitude
    nq, ng, L = 32, 96, 128.0
    st = _oracle_state(5, nq, L, plin, growth, a=1.0)
    d = f32(st["d"])
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.d.copy_(dev(d))
    got = host(sim.force(1.0))
    ref = pm.pm_force(d, nq, ng, L, 1.5 * COSMO.omega_m)
    assert rel_l2(got, ref) < 1e-5
    assert np.abs(got.sum(axis=1)).max() < 1e-5 * np.abs(got).sum() / got.shape[1] * 10


# ---------------------------------------------------------------- 2LPT -----
@pytest.mark.parametrize("nq,L", [(32, 128.0), (18, 60.0), (20, 100.0)])
def test_ic_2lpt_vs_oracle(nq, L, plin, growth):
    sim = C.Simulation(config(nq, 3 * nq, L))
    sim.ic(seed=42)
    ref = _oracle_state(42, nq, L, plin, growth)
    assert rel_l2(host(sim.psi1), ref["psi1"]) < 1e-5
    assert rel_l2(host(sim.psi2), ref["psi2"]) < 1e-5
    assert rel_l2(host(sim.d), ref["d"]) < 1e-5
    assert np.all(host(sim.v) == 0)
    assert sim.status() == 0


# ---------------------------------------------------------------- step -----
def test_single_cola_step_vs_oracle(plin, growth):
    nq, ng, L = 32, 96, 128.0
    tab = cm.step_table(COSMO, cm.time_nodes(0.05, 1.0, 40), growth)
    ref = _oracle_state(9, nq, L, plin, growth)
    rng = np.random.default_rng(0)
    ref["v"] = rng.standard_normal(ref["d"].shape) * 0.05
    for key in ref:
        ref[key] = f32(ref[key])
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.load_state(*(dev(ref[k]) for k in ("d", "v", "psi1", "psi2")))
    for j in (0, 17):
        sim.load_state(*(dev(ref[k]) for k in ("d", "v", "psi1", "psi2")))
        sim.step(j)
        o = {k: v.copy() for k, v in ref.items()}
        ocola.cola_step(o, j, tab, nq, ng, L)
        dq = L / nq
        assert np.sqrt(np.mean((host(sim.d) - o["d"]) ** 2)) < 1e-5 * dq
        assert rel_l2(host(sim.v) - ref["v"], o["v"] - ref["v"]) < 1e-5


# (nq, ng, L): 3x, 1.5x (fractional lattice-to-mesh ratio) and 1x meshes
@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("nq,ng,L", [(32, 96, 128.0), (32, 48, 128.0), (24, 24, 96.0)])
def test_both_pm_paths_vs_oracle(path, nq, ng, L, plin, growth):
    # fused passes (1) and separate kernels (2): force and one node against the oracle
    tab = cm.step_table(COSMO, cm.time_nodes(0.05, 1.0, 40), growth)
    ref = _oracle_state(9, nq, L, plin, growth, a=0.5)
    ref["v"] = np.random.default_rng(2).standard_normal(ref["d"].shape) * 0.05
    for key in ref:
        ref[key] = f32(ref[key])
    assert C.LIB.cola_pm_set_path(path) == 0
    try:
        sim = C.Simulation(config(nq, ng, L))
        sim.init_tables()
        sim.load_state(*(dev(ref[k]) for k in ("d", "v", "psi1", "psi2")))
        got = host(sim.force(0.5))
        j = 23
        sim.step(j)
        assert sim.status() == 0
    finally:
        C.LIB.cola_pm_set_path(0)
    assert rel_l2(got, pm.pm_force(ref["d"], nq, ng, L, 1.5 * COSMO.omega_m / 0.5)) < 1e-5
    o = {k: v.copy() for k, v in ref.items()}
    ocola.cola_step(o, j, tab, nq, ng, L)
    assert np.sqrt(np.mean((host(sim.d) - o["d"]) ** 2)) < 1e-5 * L / nq
    assert rel_l2(host(sim.v) - ref["v"], o["v"] - ref["v"]) < 1e-5


def test_separate_path_survives_other_users_of_its_mesh_region():
    # the separate path keeps its fixed-point counts zero between steps and
    # clears them only after another call wrote the region (the fused path's
    # bins, P(k), density): interleaving those calls changes no result
    nq, ng, L = 16, 48, 64.0

    def run(interleave):
        sim = C.Simulation(config(nq, ng, L))
        sim.ic(seed=4)
        for j in range(4):
            assert C.LIB.cola_pm_set_path(2) == 0
            sim.step(j)
            if interleave:
                sim.density()
                sim.power(48)
                assert C.LIB.cola_pm_set_path(1) == 0
                sim.force(0.3)
        C.LIB.cola_pm_set_path(0)
        assert sim.status() == 0
        return host(sim.d), host(sim.v)

    try:
        plain, mixed = run(False), run(True)
    finally:
        C.LIB.cola_pm_set_path(0)
    np.testing.assert_array_equal(mixed[0], plain[0])
    np.testing.assert_array_equal(mixed[1], plain[1])


def test_pm_path_setter_validates():
    assert C.LIB.cola_pm_set_path(3) == -1
    assert C.LIB.cola_pm_set_path(-1) == -1
    assert C.LIB.cola_pm_set_path(0) == 0


@pytest.mark.parametrize("node", [11, 39])
def test_step_host_matches_device_step(node, plin, growth):
    # the host-buffer entry point copies in, runs the same node and copies back
    nq, ng, L = 32, 96, 128.0
    ref = _oracle_state(9, nq, L, plin, growth, a=0.3)
    ref["v"] = np.random.default_rng(1).standard_normal(ref["d"].shape) * 0.05
    st = {k: f32(ref[k]) for k in ("d", "v", "psi1", "psi2")}
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.load_state(*(dev(st[k]) for k in ("d", "v", "psi1", "psi2")))
    sim.step(node)
    want_d, want_v = host(sim.d), host(sim.v)
    hst = [torch.as_tensor(st[k], dtype=torch.float32).pin_memory() for k in ("d", "v", "psi1", "psi2")]
    sim.load_state(*(torch.zeros_like(x, device="cuda") for x in hst))  # the call must bring the state in
    sim.step_host(C.make_state(*hst), node)
    np.testing.assert_array_equal(hst[0].numpy(), want_d)
    np.testing.assert_array_equal(hst[1].numpy(), want_v)
    np.testing.assert_array_equal(hst[2].numpy(), st["psi1"])  # inputs only
    np.testing.assert_array_equal(host(sim.d), want_d)
    assert sim.status() == 0


# ---------------------------------------------------------------- P(k) -----
@pytest.mark.parametrize("flags", [0, C.PK_DECONV_CIC, C.PK_ALIAS_JING])
def test_power_spectrum_vs_oracle(flags, plin, growth):
    nq, ng, L = 32, 96, 128.0
    st = _oracle_state(11, nq, L, plin, growth, a=0.5)
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.load_state(*(dev(f32(st[k])) for k in ("d", "v", "psi1", "psi2")))
    for ng_pk in (64, 96):
        k, p, n = (host(x) for x in sim.power(ng_pk, a_out=None, flags=flags, node=0))
        kr, pr, nr = power.power_spectrum(f32(st["d"]), nq, ng_pk, L, flags)
        np.testing.assert_array_equal(n, nr)
        np.testing.assert_allclose(k, kr, rtol=1e-6)
        np.testing.assert_allclose(p, pr, rtol=2e-5)


@pytest.mark.parametrize("ng_pk", [64, 96])
def test_power_spectrum_iterated_jing_vs_oracle(ng_pk, plin, growth):
    # the iterated Jing (2005) correction: three passes of per-mode image sums with
    # slopes from the previous estimate (FP32 sums on the GPU, FP64 in the oracle)
    nq, ng, L = 32, 96, 128.0
    st = _oracle_state(11, nq, L, plin, growth, a=1.0)
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.load_state(*(dev(f32(st[k])) for k in ("d", "v", "psi1", "psi2")))
    k, p, n = (host(x) for x in sim.power(ng_pk, a_out=None, flags=C.PK_ALIAS_ITER, node=0))
    kr, pr, nr = power.power_jing_iterative(pm.density_contrast(f32(st["d"]), nq, ng_pk, L), L)
    np.testing.assert_array_equal(n, nr)
    np.testing.assert_allclose(k, kr, rtol=1e-6)
    # the slope from the neighbouring bins amplifies the closed-form pass's 2e-5 by
    # about b (ln((b+1)/(b-1)) ~ 2/b), to ~1e-3 in n_eff at b = 48; it enters C through
    # the alias fraction (~0.3 at Nyquist) times ln(ratio)/2: ~1.5e-4 in P
    np.testing.assert_allclose(p, pr, rtol=5e-4)
    _, pc, _ = (host(x) for x in sim.power(ng_pk, a_out=None, flags=C.PK_DECONV_CIC | C.PK_ALIAS_JING, node=0))
    assert np.abs(p[-1] / pc[-1] - 1) > 1e-3  # the iteration does change the Nyquist bins


def test_power_spectrum_snapshot_drift(plin, growth):
    nq, ng, L = 16, 48, 64.0
    st = _oracle_state(12, nq, L, plin, growth)
    st["v"] = np.random.default_rng(1).standard_normal(st["d"].shape) * 0.1
    for key in st:
        st[key] = f32(st[key])
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    sim.load_state(*(dev(st[k]) for k in ("d", "v", "psi1", "psi2")))
    node = 5
    a_node = cm.time_nodes(0.05, 1.0, 40)[node]
    a_out = a_node + 0.01
    k, p, n = (host(x) for x in sim.power(48, a_out=a_out, node=node))
    dout = ocola.snapshot_displacement(st, a_node, a_out, growth, COSMO, cm.drift_integral)
    kr, pr, nr = power.power_spectrum(dout, nq, 48, L)
    np.testing.assert_allclose(p, pr, rtol=5e-5)


@pytest.mark.parametrize("pm_only,da", [(False, 0.0), (False, 0.01), (True, 0.0)])
def test_redshift_space_multipoles_vs_oracle(pm_only, da, plin, growth):
    # a 2LPT field at a = 0.4 with a random residual momentum: positions moved
    # along z by p_z / (a^2 E), multipoles about z (at the node or after a snapshot drift)
    nq, ng, L = 16, 48, 64.0
    st = _oracle_state(14, nq, L, plin, growth, a=0.4)
    st["v"] = np.random.default_rng(2).standard_normal(st["d"].shape) * 0.3
    for key in st:
        st[key] = f32(st[key])
    sim = C.Simulation(config(nq, ng, L, flags=C.FLAG_PM_ONLY if pm_only else 0))
    sim.init_tables()
    sim.load_state(*(dev(st[k]) for k in ("d", "v", "psi1", "psi2")))
    node = 15
    a_node = cm.time_nodes(0.05, 1.0, 40)[node]
    a_out = a_node + da
    k, p0, p2, p4, n = (host(x) for x in sim.multipoles(48, a_out=a_out, node=node))
    ref = dict(st)
    if da:
        ref["d"] = ocola.snapshot_displacement(st, a_node, a_out, growth, COSMO, cm.drift_integral)
    _, D1p, _, D2p = (x[0] for x in growth(np.array([a_out])))
    ds = power.redshift_space_displacement(ref, a_out, D1p, D2p, COSMO, pm_only=pm_only)
    kr, r0, r2, r4, nr = power.power_multipoles(ds, nq, 48, L)
    np.testing.assert_array_equal(n, nr)
    np.testing.assert_allclose(k, kr, rtol=1e-6)
    np.testing.assert_allclose(p0, r0, rtol=5e-5)
    np.testing.assert_allclose(p2, r2, rtol=0, atol=1e-4 * np.abs(r0).max())
    np.testing.assert_allclose(p4, r4, rtol=0, atol=1e-4 * np.abs(r0).max())
    assert np.abs(r2).max() > 0.05 * np.abs(r0).max()  # the shift makes a real quadrupole


# ---------------------------------------------------------------- run ------
SAMPLINGS = {C.SAMPLING_LINEAR: "linear", C.SAMPLING_LOG: "log", C.SAMPLING_POW: "pow"}


@pytest.mark.parametrize("sampling,p,a_init,flags", [
    (C.SAMPLING_LINEAR, 1.0, 0.05, 0),      # the paper's optimal setup: 40 linear steps from z = 19
    (C.SAMPLING_LOG, 1.0, 0.05, 0),         # Sec. 4.2, Eq. 3 with f = ln a
    (C.SAMPLING_POW, 0.5, 0.05, 0),         # Sec. 4.2, f = a^p
    (C.SAMPLING_POW, 0.8, 0.05, 0),
    (C.SAMPLING_LINEAR, 1.0, 0.1, 0),       # Sec. 4.3: z_i = 9
    (C.SAMPLING_LINEAR, 1.0, 1.0 / 40, 0),  # z_i = 39
    (C.SAMPLING_LINEAR, 1.0, 1.0 / 101, 0), # z_i = 100
    (C.SAMPLING_LINEAR, 1.0, 0.05, C.FLAG_MODIFIED_KDK),  # Tassev et al. (2013) kick and drift
])
def test_full_run_small_config_vs_oracle(sampling, p, a_init, flags, plin, growth):
    """32^3 particles on a 96^3 mesh, L = 128 Mpc/h, 40 steps to z = 0 with the
    paper's time samplings and initial redshifts."""
    nq, ng, L = 32, 96, 128.0
    cfg = config(nq, ng, L, a_init=a_init, sampling=sampling, sampling_p=p, flags=flags)
    sim = C.Simulation(cfg)
    sim.ic(seed=1)
    sim.run()
    assert sim.status() == 0
    tab = cm.step_table(COSMO, cm.time_nodes(a_init, 1.0, 40, SAMPLINGS[sampling], p), growth,
                        modified=bool(flags & C.FLAG_MODIFIED_KDK))
    ref = _oracle_state(1, nq, L, plin, growth, a=a_init)
    ocola.run(ref, tab, nq, ng, L)
    dq = L / nq
    rms = np.sqrt(np.mean(np.sum((host(sim.d) - ref["d"]) ** 2, axis=0)))
    assert rms <= 1e-3 * dq
    k, p, n = (host(x) for x in sim.power(ng, node=39))
    kr, pr, nr = power.power_spectrum(ref["d"], nq, ng, L)
    kny = np.pi * ng / L
    sel = kr <= kny / 2
    assert np.max(np.abs(p[sel] / pr[sel] - 1)) <= 1e-3


def test_pm_only_run_vs_oracle(plin, growth):
    """App. B's PM-only mode (the same loop without the LPT frame): the state
    starts at the 2LPT displacement and momentum; 32^3 on 96^3, 40 steps."""
    nq, ng, L = 32, 96, 128.0
    sim = C.Simulation(config(nq, ng, L, flags=C.FLAG_PM_ONLY))
    sim.ic(seed=1)
    ref = _oracle_state(1, nq, L, plin, growth)
    c1, c2 = cm.lpt_momentum_coeffs(0.05, COSMO, growth)
    ref["v"] = c1 * ref["psi1"] + c2 * ref["psi2"]
    assert rel_l2(host(sim.v), ref["v"]) < 1e-5
    sim.run()
    assert sim.status() == 0
    tab = cm.step_table(COSMO, cm.time_nodes(0.05, 1.0, 40), growth)
    ocola.run(ref, tab, nq, ng, L, pm_only=True)
    dq = L / nq
    rms = np.sqrt(np.mean(np.sum((host(sim.d) - ref["d"]) ** 2, axis=0)))
    assert rms <= 1e-3 * dq
    k, p, n = (host(x) for x in sim.power(ng, node=39))
    kr, pr, nr = power.power_spectrum(ref["d"], nq, ng, L)
    sel = kr <= np.pi * ng / L / 2
    assert np.max(np.abs(p[sel] / pr[sel] - 1)) <= 1e-3


@pytest.mark.parametrize("path", [1, 2])
def test_nonfinite_position_in_a_step(path, plin, growth):
    # one particle with a NaN position: the step latches COLA_ENONFINITE, leaves
    # that particle's state as it was and moves every other particle to finite values
    nq, ng, L = 16, 48, 64.0
    st = _oracle_state(2, nq, L, plin, growth, a=0.3)
    d = f32(st["d"])
    d[0, 123] = np.nan
    v = f32(np.random.default_rng(5).standard_normal(d.shape) * 0.05)
    assert C.LIB.cola_pm_set_path(path) == 0
    try:
        sim = C.Simulation(config(nq, ng, L))
        sim.init_tables()
        sim.load_state(dev(d), dev(v), dev(f32(st["psi1"])), dev(f32(st["psi2"])))
        sim.step(12)
        status = sim.status()
    finally:
        C.LIB.cola_pm_set_path(0)
    assert status == -6
    dn, vn = host(sim.d), host(sim.v)
    assert np.isnan(dn[0, 123])
    np.testing.assert_array_equal(vn[:, 123], v[:, 123])
    others = np.ones(nq**3, bool)
    others[123] = False
    assert np.isfinite(dn[:, others]).all() and np.isfinite(vn[:, others]).all()
    assert np.abs(vn[:, others] - v[:, others]).max() > 0


def test_nonfinite_input_sets_status():
    nq, ng, L = 8, 24, 32.0
    sim = C.Simulation(config(nq, ng, L))
    sim.init_tables()
    d = np.zeros((3, nq**3), np.float32)
    d[1, 17] = np.nan
    sim.d.copy_(dev(d))
    sim.density()
    assert sim.status() == -6
    assert sim.status() == 0  # cleared after reading
