"""GPU transport-data surrogate (BF16 tensor-core network, FP32 accumulate)
against the FP64 CPU oracle, through the C ABI.

Tolerances: the 128 x 128 layer rounds its operands to BF16 (relative
2^-9 each) and tanh is the hardware approximation (~5e-4), so outputs and
gradients are compared norm-wise per parameter block at 2e-2 relative; Adam's
first step, lr g / (|g| + eps), is compared where the oracle's gradient is
well above that error."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _problem(n, seed=1):
    r = np.random.default_rng(seed)
    th = W.mlp_init(30 + seed)
    th[M.OFF["b1"]:M.OFF["b1"] + 128] = r.normal(0, 0.3, 128)
    th[M.OFF["b2"]:M.OFF["b2"] + 128] = r.normal(0, 0.3, 128)
    th[M.OFF["b3"]:M.OFF["b3"] + 6] = r.normal(0, 0.3, 6)
    th = th.astype(np.float32).astype(np.float64)  # the values the GPU holds
    x = r.normal(0, 1, (n, 2)).astype(np.float32).astype(np.float64)
    t = r.normal(0, 1, (n, 6)).astype(np.float32).astype(np.float64)
    return th, x, t


def _dev(a):
    return torch.as_tensor(np.asarray(a, np.float32)).cuda()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n", [1, 37, 4096 + 5])
def test_forward_matches_oracle(n, variant):
    """variant 0: tcgen05 (TMEM accumulators, h1 and h2 in BF16); 1: mma.sync."""
    from paper_2110_14494_gb300 import mlp_forward
    th, x, _ = _problem(n)
    y = mlp_forward(_dev(th), _dev(x), variant=variant).cpu().numpy()
    ref = M.forward(th, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 2e-2
    assert np.abs(y - ref).max() < 5e-2 * np.abs(ref).max()


def test_gradient_matches_oracle():
    """The backward kernels (two BF16 tensor-core products per batch plus the
    FP32 output and input layers) against backpropagation in FP64."""
    from paper_2110_14494_gb300 import mlp_loss_grad
    th, x, t = _problem(512, seed=2)
    loss, g = mlp_loss_grad(_dev(th), _dev(x), _dev(t))
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = M.loss_grad(th, x, t)
    assert abs(loss.item() - lref) <= 1e-2 * lref
    for name in M.SHAPES:
        a, b = M.unpack(g)[name], M.unpack(gref)[name]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), name


def test_adam_steps_match_oracle():
    """Three full-batch Adam steps on the GPU against the oracle's updates."""
    from paper_2110_14494_gb300 import mlp_train
    th, x, t = _problem(256, seed=3)
    p, m, v = _dev(th), torch.zeros(M.N_PARAMS, device="cuda"), torch.zeros(M.N_PARAMS, device="cuda")
    mlp_train(p, m, v, 0, _dev(x), _dev(t), 1, lr=1e-3)
    ref = th.copy()
    mr, vr = np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    _, g = M.loss_grad(th, x, t)
    M.adam(ref, mr, vr, g, 1, lr=1e-3)
    d_gpu = p.cpu().numpy().astype(np.float64) - th
    d_ref = ref - th
    strong = np.abs(g) > 0.1 * np.abs(g).max()
    # first step: every parameter with a clear gradient moves by lr against it
    assert np.allclose(d_gpu[strong], d_ref[strong], rtol=2e-2, atol=2e-6)
    assert np.mean(np.sign(d_gpu) == np.sign(d_ref)) > 0.97


def test_training_follows_oracle():
    """200 full-batch steps from the same start: both reduce the loss of a
    smooth target by the same factor within 25 %."""
    from paper_2110_14494_gb300 import mlp_loss_grad, mlp_train
    r = np.random.default_rng(6)
    x = r.uniform(-1, 1, (256, 2))
    t = np.stack([np.sin(2 * x[:, 0]), x[:, 1] ** 2, x[:, 0] * x[:, 1], np.cos(x[:, 1]), x[:, 0], -x[:, 1]], 1)
    th = W.mlp_init(21).astype(np.float32).astype(np.float64)
    p, m, v = _dev(th), torch.zeros(M.N_PARAMS, device="cuda"), torch.zeros(M.N_PARAMS, device="cuda")
    xd, td = _dev(x), _dev(t)
    l0 = mlp_loss_grad(p, xd, td)[0].item()
    mlp_train(p, m, v, 0, xd, td, 200, lr=3e-3)
    l_gpu = mlp_loss_grad(p, xd, td)[0].item()
    ref, mr, vr = th.copy(), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    M.train(ref, mr, vr, 0, x, t, 200, lr=3e-3)
    l_ref = M.loss_grad(ref, x, t)[0]
    assert l_gpu < 0.05 * l0 and l_ref < 0.05 * l0
    assert abs(np.log(l_gpu / l_ref)) < np.log(1.25) + 0.3, (l0, l_gpu, l_ref)


@pytest.mark.parametrize("variant", [0, 1])
def test_inference_on_many_points_sampled(variant):
    """2^20 + 77 query points (several blocks' worth of tiles and a ragged
    tail); a random sample checked against the oracle."""
    from paper_2110_14494_gb300 import mlp_forward
    th, _, _ = _problem(1, seed=4)
    r = np.random.default_rng(7)
    n = (1 << 20) + 77
    x = r.normal(0, 1, (n, 2)).astype(np.float32)
    y = mlp_forward(_dev(th), _dev(x), variant=variant).cpu().numpy()
    idx = np.concatenate([r.choice(n, 2000, replace=False), np.arange(n - 77, n)])
    ref = M.forward(th, x[idx].astype(np.float64))
    assert np.linalg.norm(y[idx] - ref) / np.linalg.norm(ref) < 2e-2
    assert np.isfinite(y).all()


def test_surrogate_gain_over_swarms():
    """The trained surrogate against the method without it.  Training table:
    batched swarms at 64 E/N values (20-800 Td) x 4 O2 fractions; held out: 12
    fresh swarms at random (E/N, f) from another seed.  The surrogate must
    (i) predict the well-determined log targets (mu N, D_L N, D_T N, mean
    energy, and alpha / N above 300 Td) of the held-out swarms within their
    scatter, no worse than bilinear interpolation in the same table, and
    (ii) answer queries at least 1e4 times faster than running a swarm."""
    import time
    from paper_2110_14494_gb300 import surrogate as S
    from paper_2110_14494_gb300 import swarm_run
    kw = dict(precision=32, n0=2000, n_steps=400, dt=1e-12, n_lo=500, n_hi=20000, seed=11)
    EN = 20.0 * 40.0 ** (np.arange(64) / 63)
    fr = np.array([0.1, 0.1667, 0.2333, 0.3])
    X, Y, _ = S.swarm_points(lambda f: W.synthetic_air(o2_frac=f), EN, fr, W.N_GAS, **kw)
    sur = S.Surrogate(W.mlp_init(40), X, Y)
    trace, secs = sur.fit(4000, lr=2e-3)
    assert trace[-1][1] < 0.05, trace[-4:]
    q = W.mlp_query_points(12, 41, en_lo=25.0, en_hi=700.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    held = []
    for k in range(len(q)):
        res, _, _ = swarm_run(W.synthetic_air(o2_frac=q[k, 1]), q[k:k + 1, 0], batched=True, **dict(kw, seed=500 + k))
        held.append(S.targets(res, q[k:k + 1, 0], W.N_GAS)[0])
    torch.cuda.synchronize()
    swarm_qps = len(q) / (time.perf_counter() - t0)
    held = np.array(held)
    pred = sur.predict(q[:, 0], q[:, 1])
    table = Y.reshape(len(fr), len(EN), 6)
    lin = S.table_interp(EN, fr, table, q[:, 0], q[:, 1])
    cols = [0, 1, 2, 5]
    err_s = np.sqrt(np.mean((pred[:, cols] - held[:, cols]) ** 2))
    err_t = np.sqrt(np.mean((lin[:, cols] - held[:, cols]) ** 2))
    hi = q[:, 0] > 300
    err_a = np.sqrt(np.mean((pred[hi, 3] - held[hi, 3]) ** 2)) if hi.any() else 0.0
    print("surrogate", err_s, "table", err_t, "alpha", err_a, "loss", trace[-1])
    assert err_s < 0.08 and err_a < 0.15, (err_s, err_a)
    assert err_s < 1.5 * err_t + 0.02, (err_s, err_t)
    # query throughput: 2^20 standardized points on the device
    xs = torch.as_tensor(sur.sx.fwd(S.features(W.mlp_query_points(1 << 20, 42)[:, 0], 0.2)).astype(np.float32)).cuda()
    sur.predict_std(xs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        sur.predict_std(xs)
    torch.cuda.synchronize()
    mlp_qps = 5 * (1 << 20) / (time.perf_counter() - t0)
    assert mlp_qps > 1e4 * swarm_qps, (mlp_qps, swarm_qps)
