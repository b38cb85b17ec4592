"""Learned coarse-mesh correction: CUDA (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 oracle on the same BF16-rounded weights.
Tolerances: filter-only force rel-L2 <= 1e-5 (FP32 path); net residual force
and every gradient tensor rel-L2 <= 2e-2 and cosine >= 0.999 (BF16 weights and
activations, FP32 accumulation)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cosmology as cm
from oracle import learned as ol
from oracle import lpt, pm

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev, f32, host, rel_l2  # noqa: E402

COSMO = cm.Cosmology()
GRAD_REL, GRAD_COS = 2e-2, 0.999


def _cos(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b))


def _params(seed, scale=1.0):
    p = ol.init_params(seed, scale=scale)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.05
    vec = np.zeros(C.NET_NPARAMS)
    for k, (off, shape) in C.NET_OFFSETS.items():
        vec[off: off + int(np.prod(shape))] = p[k].reshape(-1) if k.startswith("b") else p[k].reshape(shape).reshape(-1)
    t = torch.tensor(vec, dtype=torch.float32, device="cuda")
    # the oracle sees the BF16-rounded weights the kernels use (biases stay FP32)
    pr = {}
    for k, (off, shape) in C.NET_OFFSETS.items():
        vals = t[off: off + int(np.prod(shape))]
        if k.startswith("W"):
            vals = vals.to(torch.bfloat16).to(torch.float64)
        arr = vals.cpu().numpy().astype(np.float64)
        pr[k] = arr.reshape(shape[0], shape[1], 3, 3, 3) if k.startswith("W") else arr
    return t, pr


def _setup(nq=32, L=64.0, a=0.5, seed=3, nfilt=8):
    plin = cm.LinearPower(COSMO)
    g = cm.Growth(COSMO)
    D1, _, D2, _ = g(np.array([a]))
    st = lpt.initial_conditions(seed, nq, L, plin, D1[0], D2[0])
    d = f32(st["d"])
    T = 1.0 + 0.3 * np.sin(np.arange(nfilt))
    return d, T


def _sim(nq, L, params, T, learned=True):
    wpack = torch.zeros(C.NET_NPACK, dtype=torch.bfloat16, device="cuda")
    filt = torch.tensor(T, dtype=torch.float32, device="cuda")
    net = C.make_net(params, wpack, filt)
    C.cola_net_pack(net)
    cfg = C.make_config(nq, nq, L, 0.05, flags=C.FLAG_LEARNED if learned else 0, net=net)
    sim = C.Simulation(cfg)
    sim.init_tables()
    sim._keep = (wpack, filt, net)
    return sim


def _oracle_fields(d, nq, L, a, T):
    green = 1.5 * COSMO.omega_m / a
    u = pm.mesh_coords(d, nq, nq, L)
    delta = pm.cic_deposit(u, nq) - 1.0
    F = pm.force_mesh_from_delta(delta, L, green, filt=T)
    x = np.concatenate([delta[None], F / green])
    return u, F, x, green


def test_filtered_force_and_net_residual_vs_oracle():
    nq, L, a = 32, 64.0, 0.5
    d, T = _setup(nq, L, a)
    params, pr = _params(7)
    zero = torch.zeros_like(params)
    sim0 = _sim(nq, L, zero, T)  # net of zeros: the filtered coarse force alone
    sim0.d.copy_(dev(d))
    f0 = host(sim0.force(a))
    u, F, x, green = _oracle_fields(d, nq, L, a, T)
    ref0 = np.stack([pm.cic_gather(F[j], u) for j in range(3)])
    assert rel_l2(f0, ref0) < 1e-5
    sim = _sim(nq, L, params, T)
    sim.d.copy_(dev(d))
    f1 = host(sim.force(a))
    out, _ = ol.net_forward(x, pr)
    ref_res = np.stack([pm.cic_gather(green * out[j], u) for j in range(3)])
    e, c = rel_l2(f1 - f0, ref_res), _cos(f1 - f0, ref_res)
    print("net residual force rel-L2, cosine:", e, c)
    assert e < GRAD_REL and c > GRAD_COS, (e, c)


def test_scale_factor_filter_rows_vs_oracle():
    # a table of three filter rows (a = 0.05, 0.525, 1): each force uses the
    # row nearest its scale factor
    nq, L = 32, 64.0
    d, _ = _setup(nq, L, 0.5)
    rows = np.stack([1.0 + 0.3 * np.sin(np.arange(8) + r) for r in range(3)])
    wpack = torch.zeros(C.NET_NPACK, dtype=torch.bfloat16, device="cuda")
    filt = torch.tensor(rows, dtype=torch.float32, device="cuda")
    params = torch.zeros(C.NET_NPARAMS, dtype=torch.float32, device="cuda")  # referenced by net until the end
    net = C.make_net(params, wpack, filt)
    C.cola_net_pack(net)
    sim = C.Simulation(C.make_config(nq, nq, L, 0.05, flags=C.FLAG_LEARNED, net=net))
    sim.init_tables()
    sim.d.copy_(dev(d))
    for a in (0.1, 0.3, 0.7, 0.95):
        got = host(sim.force(a))
        r = ol.filter_row(a, 3, 0.05, 1.0)
        u, F, _, _ = _oracle_fields(d, nq, L, a, rows[r])
        ref = np.stack([pm.cic_gather(F[j], u) for j in range(3)])
        assert rel_l2(got, ref) < 1e-5, a


def test_filter_only_correction_on_a_1p5x_mesh_vs_oracle():
    # the correction without a net (params = wpack = NULL) on a 1.5x mesh whose
    # size is not a multiple of 16 (the net's bricks would need one)
    nq, ng, L, a = 20, 30, 60.0, 0.5
    plin = cm.LinearPower(COSMO)
    D1, _, D2, _ = cm.Growth(COSMO)(np.array([a]))
    d = f32(lpt.initial_conditions(8, nq, L, plin, D1[0], D2[0])["d"])
    rows = np.stack([1.0 + 0.25 * np.cos(np.arange(8) + r) for r in range(2)])
    filt = torch.tensor(rows, dtype=torch.float32, device="cuda")
    net = C.make_net(None, None, filt)
    sim = C.Simulation(C.make_config(nq, ng, L, 0.05, flags=C.FLAG_LEARNED, net=net))
    sim.init_tables()
    sim.d.copy_(dev(d))
    green = 1.5 * COSMO.omega_m / a
    u = pm.mesh_coords(d, nq, ng, L)
    delta = pm.cic_deposit(u, ng) * (ng / nq) ** 3 - 1.0
    F = pm.force_mesh_from_delta(delta, L, green, filt=rows[ol.filter_row(a, 2, 0.05, 1.0)])
    ref = np.stack([pm.cic_gather(F[j], u) for j in range(3)])
    assert rel_l2(host(sim.force(a)), ref) < 1e-5
    # no net: its gradient call is refused
    grad = torch.zeros(C.NET_NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(C.ColaError):
        C.cola_net_grad(sim.cfg, sim.state, a, dev(ref), grad, loss, sim.ws)


def test_net_gradients_vs_oracle():
    nq, L, a = 32, 64.0, 0.5
    d, T = _setup(nq, L, a, seed=4)
    params, pr = _params(11)
    sim = _sim(nq, L, params, T)
    sim.d.copy_(dev(d))
    rng = np.random.default_rng(2)
    u, F, x, green = _oracle_fields(d, nq, L, a, T)
    target = np.stack([pm.cic_gather(F[j], u) for j in range(3)]) * (1 + 0.2 * rng.standard_normal((3, nq**3)))
    target = f32(target)
    grad = torch.zeros(C.NET_NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    C.cola_net_grad(sim.cfg, sim.state, a, dev(target), grad, loss, sim.ws)
    out, cache = ol.net_forward(x, pr)
    lo, dmesh = ol.particle_loss(F + green * out, u, target)
    g = ol.net_backward(green * dmesh, cache, pr)
    assert host(loss)[0] == pytest.approx(lo, rel=2e-3)
    gh = host(grad)
    errs = {}
    for k, (off, shape) in C.NET_OFFSETS.items():
        got = gh[off: off + int(np.prod(shape))]
        ref = g[k].reshape(-1)
        errs[k] = (rel_l2(got, ref), _cos(got, ref))
    print("net gradient rel-L2, cosine per tensor:", errs)
    for k, (e, c) in errs.items():
        assert e < GRAD_REL and c > GRAD_COS, errs


def test_filter_least_squares_recovers_a_known_filter():
    nq, L, a = 32, 64.0, 0.5
    d, T = _setup(nq, L, a, seed=5, nfilt=10)
    zero = torch.zeros(C.NET_NPARAMS, dtype=torch.float32, device="cuda")
    truth = _sim(nq, L, zero, T)  # target = the coarse force filtered with T
    truth.d.copy_(dev(d))
    target = truth.force(a)
    plain = _sim(nq, L, zero, np.ones(10), learned=False)
    plain.d.copy_(dev(d))
    nb = 10
    basis = torch.empty((nb, 3 * nq**3), dtype=torch.float32, device="cuda")
    ATA = torch.zeros((nb, nb), dtype=torch.float64, device="cuda")
    ATy = torch.zeros(nb, dtype=torch.float64, device="cuda")
    C.cola_filter_accumulate(plain.cfg, plain.state, a, target, nb, basis, ATA, ATy, plain.ws)
    Tfit = torch.zeros(nb, dtype=torch.float32, device="cuda")
    C.cola_filter_solve(ATA, ATy, nb, 0.0, Tfit)
    got = host(Tfit)
    # nodes below the corner of the k-cube carry modes; the last node sits at sqrt(3) k_Ny
    np.testing.assert_allclose(got[:8], T[:8], rtol=2e-3, atol=2e-3)


def test_adam_step():
    n = 1000
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal(n)
    g0 = rng.standard_normal(n)
    p = dev(p0)
    gr = dev(g0)
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    C.cola_adam(p, gr, m, v, n, 1, 0.01)
    # first step of Adam: update = lr * g / (|g| + eps) = lr * sign(g)
    np.testing.assert_allclose(host(p), f32(p0) - 0.01 * np.sign(f32(g0)), rtol=1e-5, atol=1e-6)
