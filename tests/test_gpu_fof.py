"""Friends-of-friends halos on the GPU against the oracle: group labels,
halo catalogue and mass function compared exactly (integer results; the
friendship test is the same FP32 formula on both sides), degenerate inputs,
and properties of the groups at the benchmarked size (512^3 particles after a
40-step run)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cosmology as cm
from oracle import fof, lpt
from synth import clumpy_displacements

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev  # noqa: E402

COSMO = cm.Cosmology()


def _sim(nq, L):
    return C.Simulation(C.make_config(nq, 3 * nq, L, 0.05))


def _gpu_fof(nq, L, d, b=0.2, nmin=100):
    s = _sim(nq, L)
    s.d.copy_(dev(d))
    g, roots, sizes = s.fof(b, nmin)
    return s, g.cpu().numpy(), roots.cpu().numpy(), sizes.cpu().numpy()


def _check(nq, L, d, b=0.2, nmin=100):
    s, g, roots, sizes = _gpu_fof(nq, L, d, b, nmin)
    want = fof.fof_groups(d, nq, L, b)
    np.testing.assert_array_equal(g, want)
    r_want, s_want = fof.halo_catalog(want, nmin)
    np.testing.assert_array_equal(roots, r_want)
    np.testing.assert_array_equal(sizes, s_want)
    return s, g, roots, sizes


@pytest.mark.parametrize("nq,L,nclump,spread", [(32, 64.0, 40, 0.6), (20, 40.0, 12, 0.4), (48, 96.0, 80, 0.8),
                                                (30, 30.0, 30, 0.5)])
def test_fof_groups_match_oracle_on_clumps(nq, L, nclump, spread):
    d = clumpy_displacements(nq + nclump, nq, L, nclump, spread)
    s, g, roots, sizes = _check(nq, L, d)
    assert len(roots) > 0 and len(np.unique(g)) < nq**3


@pytest.mark.parametrize("b", [0.1, 0.2, 0.3])
def test_fof_groups_match_oracle_on_a_2lpt_state(b):
    # the oracle's 2LPT field at a = 1: shell crossing, sheets and knots
    nq, L = 32, 128.0
    D1, _, D2, _ = cm.Growth(COSMO)(np.array([1.0]))
    st = lpt.initial_conditions(4, nq, L, cm.LinearPower(COSMO), D1[0], D2[0])
    d = st["d"].astype(np.float32)
    _check(nq, L, d, b=b, nmin=20)


def test_mass_function_matches_oracle():
    nq, L = 48, 96.0
    d = clumpy_displacements(7, nq, L, 120, 0.7)
    s, g, roots, sizes = _check(nq, L, d, nmin=30)
    mp = fof.particle_mass(COSMO.omega_m, L, nq)
    lo, dlog, nb = 13.0, 0.1, 30
    lm = np.log10(fof.warren_mass(sizes, mp))
    edge = np.abs((lm - lo) / dlog - np.round((lm - lo) / dlog)).min()
    assert edge > 1e-9  # no halo sits on a bin edge, where log10 rounding could flip a bin
    got = s.mass_function(torch.as_tensor(sizes, device="cuda"), lo, dlog, nb).cpu().numpy()
    np.testing.assert_array_equal(got, fof.mass_function(sizes, mp, lo, dlog, nb))
    assert got.sum() > 0


def test_fof_degenerate_inputs():
    nq, L = 16, 16.0
    # the unperturbed lattice: neighbours are a full spacing apart, every particle alone
    s, g, roots, sizes = _gpu_fof(nq, L, np.zeros((3, nq**3), np.float32))
    np.testing.assert_array_equal(g, np.arange(nq**3))
    assert len(roots) == 0
    # every particle on one point: one group (the union-find under full contention)
    q = fof.lattice_sites(nq).astype(np.float64)
    d = ((np.array([[3.3], [7.7], [0.1]]) - q) * (L / nq)).astype(np.float32)
    s, g, roots, sizes = _gpu_fof(nq, L, d, nmin=1)
    assert np.all(g == 0) and list(sizes) == [nq**3]
    # a chain across the periodic boundary, just inside the linking length
    d = np.zeros((3, nq**3), np.float32)
    chain = np.arange(0, 12) * 37 + 5
    for m, p in enumerate(chain):
        d[:, p] = (np.array([(nq - 0.6 + 0.19 * m) % nq, 0.5, 0.5]) - q[:, p]) * (L / nq)
    _check(nq, L, d, nmin=12)


def test_fof_rejects_bad_arguments_and_reports_nonfinite_input():
    nq, L = 16, 16.0
    s = _sim(nq, L)
    g = torch.empty(nq**3, dtype=torch.int32, device="cuda")
    fws = torch.empty(C.cola_fof_workspace_size(s.cfg), dtype=torch.uint8, device="cuda")
    for b in (0.0, 0.5, -0.1, float("nan")):
        with pytest.raises(C.ColaError) as e:
            C.cola_fof(s.cfg, s.state, b, g, fws)
        assert e.value.code == -1
    with pytest.raises(C.ColaError) as e:
        C.cola_fof(s.cfg, s.state, 0.2, g, fws[:-1])
    assert e.value.code == -2
    d = np.zeros((3, nq**3), np.float32)
    d[1, 77] = np.nan
    s.d.copy_(dev(d))
    with pytest.raises(C.ColaError) as e:
        C.cola_fof(s.cfg, s.state, 0.2, g, fws)
    assert e.value.code == -6
    gg = g.cpu().numpy()
    assert gg[77] == 77  # the bad particle is left alone, the others still get their (single) groups
    np.testing.assert_array_equal(np.delete(gg, 77), np.delete(np.arange(nq**3), 77))


def test_fof_at_the_benchmarked_size():
    # 512^3 particles after the 40-step run at L = 1536 Mpc/h: every sampled
    # particle's friends (found by brute force with the same FP32 rule) carry its
    # label, labels are the smallest members, and the halos hold the particles
    nq, ng, L = 512, 1536, 1536.0
    s = C.Simulation(C.make_config(nq, ng, L, 0.05))
    s.ic(seed=1)
    s.run()
    g, roots, sizes = s.fof(0.2, 101)
    assert s.status() == 0
    n = nq**3
    assert len(roots) > 1000
    idx = torch.arange(n, device="cuda", dtype=torch.int32)
    assert bool((g <= idx).all()) and bool((g[g.long()] == g).all())
    assert bool((g[roots.long()] == roots).all())
    counts = torch.bincount(g.long(), minlength=n)
    assert bool((counts[roots.long()] == sizes).all())
    assert int((counts >= 101).sum()) == len(roots)
    # FP32 positions as the kernels form them
    inv = torch.tensor(nq / L, dtype=torch.float32, device="cuda")
    nqf = torch.tensor(float(nq), dtype=torch.float32, device="cuda")
    p = torch.arange(n, device="cuda", dtype=torch.int64)
    q = torch.stack([p // (nq * nq), (p // nq) % nq, p % nq]).float()
    u = q + s.d * inv
    u = u - nqf * torch.floor(u / nqf)
    u = torch.where(u < 0, u + nqf, u)
    u = torch.where(u >= nqf, u - nqf, u)
    del q
    rng = np.random.default_rng(0)
    sample = torch.as_tensor(np.concatenate([rng.choice(n, 200, replace=False),
                                             roots[:100].long().cpu().numpy()]), device="cuda")
    b2 = torch.tensor(np.float32(0.2 * 0.2), device="cuda")
    half = torch.tensor(np.float32(nq / 2), device="cuda")
    for sp in sample.tolist():
        dl = u[:, sp:sp + 1] - u
        dl = torch.where(dl > half, dl - nqf, dl)
        dl = torch.where(dl < -half, dl + nqf, dl)
        r2 = (dl[0] * dl[0] + dl[1] * dl[1]) + dl[2] * dl[2]
        friends = torch.nonzero(r2 <= b2).flatten()
        assert bool((g[friends] == g[sp]).all())


def test_fof_retry_cap_reports_timeout_and_resets():
    # every particle on one point: the union-find's chains are deepest there.
    # With the retry bound at 1 the loops give up at once: COLA_ETIMEOUT, no hang;
    # with the default bound restored the same call labels one group again.
    nq, L = 16, 16.0
    q = fof.lattice_sites(nq).astype(np.float64)
    d = ((np.array([[3.3], [7.7], [0.1]]) - q) * (L / nq)).astype(np.float32)
    s = _sim(nq, L)
    s.d.copy_(dev(d))
    g = torch.empty(nq**3, dtype=torch.int32, device="cuda")
    fws = torch.empty(C.cola_fof_workspace_size(s.cfg), dtype=torch.uint8, device="cuda")
    C.cola_fof_set_retry_cap(1)
    try:
        with pytest.raises(C.ColaError) as e:
            C.cola_fof(s.cfg, s.state, 0.2, g, fws)
        assert e.value.code == -5
    finally:
        C.cola_fof_set_retry_cap(0)
    C.cola_fof(s.cfg, s.state, 0.2, g, fws)
    assert bool((g == 0).all())
    with pytest.raises(C.ColaError):
        C.cola_fof_set_retry_cap(-1)
