"""The surrogate's kernels against the FP64 network oracle (forward, bfloat16
forward, backward, Adam), a training run, and the ensemble's TT fallback."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = (15, 48, 40, 1)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, surrogate, ttprice

    build.build()
    return torch, surrogate, ttprice


def _oracle_params(net):
    return [(w.double().cpu().numpy(), b.double().cpu().numpy()) for w, b in zip(net.w, net.b)]


def test_forward_and_backward_match_the_oracle(env):
    torch, sg, _ = env
    net = sg.Net(seed=3, sizes=SIZES)
    rng = np.random.default_rng(4)
    for b in net.b:
        b.copy_(torch.tensor(rng.standard_normal(b.shape[0]) * 0.1, dtype=torch.float32))
    x = rng.standard_normal((70, 15))  # 70 rows: a ragged 64-row tile
    t = rng.standard_normal((70, 1))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = net.forward(xd).cpu().numpy()
    params = _oracle_params(net)
    yo, cache = omlp.forward(params, xd.double().cpu().numpy())
    assert np.allclose(y, yo, rtol=1e-5, atol=1e-5)
    _, dyo = omlp.mse(yo, t)
    grads = omlp.backward(params, cache, dyo)
    dy = torch.tensor(dyo, dtype=torch.float32, device="cuda")
    net.backward(xd, dy)
    for l, (gw, gb) in enumerate(grads):
        scale = np.abs(gw).max()
        assert np.abs(net.grads[2 * l].cpu().numpy() - gw).max() < 1e-4 * scale, l
        assert np.abs(net.grads[2 * l + 1].cpu().numpy() - gb).max() < 1e-4 * max(np.abs(gb).max(), 1e-12), l


def test_bf16_forward_and_adam(env):
    torch, sg, _ = env
    net = sg.Net(seed=5, sizes=SIZES)
    net.to_bf16()
    x = np.random.default_rng(6).standard_normal((33, 15))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = net.forward(xd, bf16=True).cpu().numpy()
    # the oracle with the weights rounded to bfloat16 (to nearest even)
    params = []
    for w, b in zip(net.w, net.b):
        wb = w.cpu().to(torch.bfloat16).to(torch.float64).numpy()
        params.append((wb, b.double().cpu().numpy()))
    yo, _ = omlp.forward(params, xd.double().cpu().numpy())
    assert np.allclose(y, yo, rtol=1e-5, atol=1e-5)
    # Adam: two steps against the oracle's
    p0 = net.w[0].double().cpu().numpy().copy()
    g = np.random.default_rng(7).standard_normal(p0.shape)
    for gr in net.grads:
        gr.zero_()
    net.grads[0].copy_(torch.tensor(g, dtype=torch.float32))
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    po = p0
    for step in (1, 2):
        net.adam(1e-3)
        po, m, v = omlp.adam(po, g, m, v, step, lr=1e-3)
    assert np.abs(net.w[0].double().cpu().numpy() - po).max() < 1e-6


def test_training_reduces_the_loss(env):
    torch, sg, _ = env
    rng = np.random.default_rng(8)
    x = rng.standard_normal((8192, 15))
    y = (np.sin(x[:, :5]).sum(1) + 0.3 * x[:, 5] * x[:, 6])[:, None]
    y = (y - y.mean()) / y.std()
    net = sg.Net(seed=9, sizes=(15, 64, 64, 1))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    losses = sg.train(net, xd, yd, epochs=12, batch=256, lr=3e-3, seed=1, lr_final=3e-4)
    assert losses[-1] < 0.25 * losses[0] and losses[-1] < losses[len(losses) // 2]


def test_ensemble_quotes_fall_back_to_the_tt_pricer(env):
    torch, sg, tp = env
    train_ps = inputs.surrogate_batch(256, n_grid=32, max_rank=8)
    pr = tp.Pricer(max_d=5, max_n=32, max_rank=8, max_batch=256, precision="mixed")
    _, prices, _ = pr.evaluate(train_ps)
    s = sg.Surrogate(members=2, sizes=(15, 32, 32, 1))
    s.fit(train_ps, prices, epochs=3, batch=64)
    qs = train_ps[:12]
    _, ref, _ = pr.evaluate(qs)
    p_all, back_all, _ = s.quote(qs, pricer=pr, tol=0.0)
    assert back_all.all() and np.array_equal(p_all, ref)
    p_none, back_none, spread = s.quote(qs, pricer=pr, tol=np.inf)
    assert not back_none.any() and np.all(np.isfinite(p_none)) and np.all(spread >= 0)
    pr.close()


@pytest.mark.parametrize("batch,k,n,act", [(300, 256, 256, 1), (300, 16, 256, 1), (129, 256, 64, 0),
                                           (128, 32, 16, 1), (1000, 256, 256, 0)])
def test_tensor_core_layer_against_fp64(env, batch, k, n, act):
    """tt_mlp_forward_tc (tcgen05.mma kind::f16) against the FP64 product of the same
    bfloat16 operands: several 128-row tiles with a ragged last one, K = 16 .. 256,
    N = 16 .. 256, both activations.  Products of bfloat16 values are exact in FP32,
    so the FP32 accumulation leaves ~K 2^-24 of the output's scale; the bfloat16
    output is the FP32 output rounded to nearest."""
    torch, sg, _ = env
    lib = sg._bind(sg.ttprice.load_library())
    rng = np.random.default_rng(batch + k + n + act)
    x = torch.tensor(rng.standard_normal((batch, k)), dtype=torch.float32).to(torch.bfloat16)
    w = torch.tensor(rng.standard_normal((n, k)) * np.sqrt(2.0 / k), dtype=torch.float32).to(torch.bfloat16)
    b = torch.tensor(rng.standard_normal(n) * 0.1, dtype=torch.float32)
    ref = x.double().numpy() @ w.double().numpy().T + b.double().numpy()
    if act:
        ref = omlp.silu(ref)
    xd, wd, bd = x.cuda().contiguous(), w.cuda().contiguous(), b.cuda()
    af = torch.empty((batch, n), dtype=torch.float32, device="cuda")
    ab = torch.empty((batch, n), dtype=torch.bfloat16, device="cuda")
    rc = lib.tt_mlp_forward_tc(xd.data_ptr(), batch, k, wd.data_ptr(), bd.data_ptr(), n, act, af.data_ptr(),
                               ab.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    got = af.cpu().double().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-6
    assert torch.equal(ab.cpu(), af.cpu().to(torch.bfloat16))


def test_tensor_core_inference_matches_the_bf16_weight_path(env):
    """The surrogate at its real width (15 -> 256 x 4 -> 1) on 700 quotes: the
    tensor-core layers (bfloat16 activations) against the bfloat16-weight path (FP32
    activations) to bfloat16 rounding of the activations."""
    torch, sg, _ = env
    s = sg.Surrogate(members=2, seed=9)
    ps = inputs.surrogate_batch(700, index=9)
    f = sg.features(ps)
    s.fx = (f.mean(0), f.std(0) + 1e-12)
    s.fy = (0.0, 1.0)
    for net in s.nets:
        net.to_bf16()
    m_tc, sp_tc = s.predict_device(s.standardise_tc(ps))
    m_32, sp_32 = s.predict_device(s.standardise(ps))
    a, c = m_tc.cpu().numpy(), m_32.cpu().numpy()
    assert np.abs(a - c).max() < 2e-2 * max(1.0, np.abs(c).max())
