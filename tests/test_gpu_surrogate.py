"""Tensor-core surrogate network on the GPU against references.

* ems_gemm_bf16 (tcgen05, FP32 accumulate) against a PyTorch FP32 matmul of
  the same BF16 operands, within the FP32 accumulation bound K * 2^-23 *
  (|A| |B|^T).
* The fused inference kernel against (a) a plain PyTorch CPU forward that
  rounds weights and activations to BF16 where the kernel does, and (b) the
  FP64 oracle, within the BF16 rounding budget (unit roundoff 2^-8 per
  rounding, ~10 roundings along a path: rms error <= 3 %).
* Gradients of the BF16 training kernels against the FP64 oracle's backward,
  one Adam step against the oracle's Adam applied to the same gradients, and
  a loss that falls when trained on a learnable map.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def sg():
    _need_gpu()
    from paper_2604_10743_gb300 import surrogate
    return surrogate


def _bf(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K,bias,relu", [
    (1, 16, 64, False, False), (130, 256, 64, True, True), (300, 144, 192, True, False),
    (257, 256, 256, False, True), (64, 32, 512, True, True), (1000, 16, 256, True, False)])
def test_gemm_bf16_matches_fp32_reference(sg, M, N, K, bias, relu):
    g = torch.Generator().manual_seed(M * 7 + N + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bi = torch.randn(N, generator=g) if bias else None
    d, d16 = sg.gemm_bf16(a.cuda(), b.cuda(), None if bi is None else bi.cuda(), relu=relu, scale=0.5,
                          out_bf16=True)
    torch.cuda.synchronize()
    ref = 0.5 * (a.float() @ b.float().T)
    if bi is not None:
        ref = ref + bi
    if relu:
        ref = torch.relu(ref)
    bound = K * 2.0 ** -23 * (0.5 * a.float().abs() @ b.float().abs().T) + 1e-6
    err = (d.cpu() - ref).abs()
    assert torch.all(err <= bound), float((err / bound).max())
    # BF16 output = FP32 result rounded once (one BF16 ulp of slack for ties)
    e16 = (d16.cpu().float() - ref).abs()
    assert torch.all(e16 <= 2.0 ** -8 * ref.abs() + bound)


def _ref_forward_bf16(layers, xs):
    """Plain PyTorch CPU forward with BF16 weights, BF16 activations between
    layers and FP32 accumulation / bias, as the kernels compute."""
    h = xs.to(torch.bfloat16).float()
    for li, (W, b) in enumerate(layers):
        z = h @ _bf(W).float().T + torch.as_tensor(b, dtype=torch.float32)
        if li + 1 < len(layers):
            h = torch.relu(z).to(torch.bfloat16).float()
        else:
            h = z
    return h


def _net(sg, seed, n_hidden=4):
    m = sg.Mlp(n_hidden=n_hidden, seed=seed)
    rng = np.random.default_rng(seed)
    flat = m.params()
    layers = sg.Mlp.unflatten(flat.copy(), n_hidden)
    layers = [(W, rng.normal(0, 0.1, size=b.shape).astype(np.float32)) for W, b in layers]
    m.set_params(sg.Mlp.flatten(layers))
    return m, layers


def test_predict_matches_bf16_reference_and_oracle(sg):
    from oracle import mlp as om
    m, layers = _net(sg, 3)
    rng = np.random.default_rng(4)
    rows = 1000                                        # 4 CTAs' worth, ragged last pair of tiles
    xm = rng.normal(size=24).astype(np.float32)
    xsd = rng.uniform(0.5, 2.0, size=24).astype(np.float32)
    tm = np.array([7.5, 0.4], np.float32); tsd = np.array([1.3, 0.3], np.float32)
    m.set_norm(xm, xsd, tm, tsd)
    x = (rng.normal(size=(rows, 24)) * xsd + xm).astype(np.float32)
    y = m.predict(torch.from_numpy(x).cuda()).cpu()
    xs = (torch.from_numpy(x) - torch.from_numpy(xm)) / torch.from_numpy(xsd)
    ref = _ref_forward_bf16(layers, xs) * torch.from_numpy(tsd) + torch.from_numpy(tm)
    scale = ref.std(0)
    assert torch.all((y - ref).abs() <= 1e-2 * scale + 1e-3 * ref.abs()), float((y - ref).abs().max())
    # FP64 oracle without any BF16 rounding
    yo, _ = om.forward([(W.astype(np.float64), b.astype(np.float64)) for W, b in layers],
                       xs.numpy().astype(np.float64))
    yo = yo * tsd + tm
    rms = np.sqrt(np.mean((y.numpy() - yo) ** 2, axis=0))
    assert np.all(rms <= 3e-2 * yo.std(0)), (rms, yo.std(0))


def test_predict_large_sampled(sg):
    m, layers = _net(sg, 5)
    rows = 1_000_003
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(rows, 24, device="cuda", generator=g)
    y = m.predict(x)
    idx = torch.randint(0, rows, (512,), generator=torch.Generator().manual_seed(1))
    idx[0] = rows - 1
    ref = _ref_forward_bf16(layers, x[idx.cuda()].cpu())
    yy = y[idx.cuda()].cpu()
    assert torch.all((yy - ref).abs() <= 1e-2 * ref.std(0) + 1e-3 * ref.abs())


def _ref_grads_bf16(layers, xs, ts):
    """Plain PyTorch CPU backward with the kernels' roundings: BF16 weights,
    activations and dZ operands, FP32 accumulation, FP32 dZ for the bias sums
    and the ReLU' mask taken from the BF16 activation."""
    acts, h = [xs.to(torch.bfloat16).float()], xs.to(torch.bfloat16).float()
    for li, (W, b) in enumerate(layers):
        z = h @ _bf(W).float().T + torch.as_tensor(b)
        if li + 1 < len(layers):
            h = torch.relu(z).to(torch.bfloat16).float()
            acts.append(h)
        else:
            y = z
    d = (y - ts) / xs.shape[0]
    out = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        db = d.to(torch.bfloat16).float()
        out[li] = ((db.T @ acts[li]).numpy(), d.sum(0).numpy())
        if li > 0:
            d = (db @ _bf(layers[li][0]).float()) * (acts[li] > 0).float()
    return out


def _cmp(a, b):
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
    return rel, cos


def test_gradients_match_oracle(sg):
    from oracle import mlp as om
    m, layers = _net(sg, 7)
    rng = np.random.default_rng(8)
    rows = 300                                        # not a multiple of the 64-row padding
    x = rng.normal(size=(rows, 24)).astype(np.float32)
    t = rng.normal(size=(rows, 2)).astype(np.float32)
    g, loss = m.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    gl = sg.Mlp.unflatten(g, 4)
    # same roundings as the kernels: agreement up to FP32 summation order and
    # the odd BF16 tie
    ref = _ref_grads_bf16(layers, torch.from_numpy(x), torch.from_numpy(t))
    for (gW, gb), (rW, rb) in zip(gl, ref):
        for a, b in ((gW, rW), (gb, rb)):
            rel, cos = _cmp(a, b)
            assert rel <= 1e-2 and cos >= 0.9999, (rel, cos)
    # FP64 oracle: the BF16 roundings (2^-8 each, amplified by the
    # cancellation in batch sums of random-target gradients) stay far below
    # the O(1) error of a dropped term, wrong sign or transposed operand
    p64 = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    y, cache = om.forward(p64, x.astype(np.float64))
    go = om.backward(p64, cache, y, t.astype(np.float64))
    assert abs(loss - om.loss(y, t)) <= 2e-2 * om.loss(y, t)
    for (gW, gb), (oW, ob) in zip(gl, go):
        for a, b in ((gW, oW), (gb, ob)):
            rel, cos = _cmp(a, b)
            assert rel <= 0.15 and cos >= 0.99, (rel, cos)


def test_adam_step_matches_oracle(sg):
    from oracle import mlp as om
    m, layers = _net(sg, 9)
    rng = np.random.default_rng(10)
    x = torch.from_numpy(rng.normal(size=(256, 24)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(256, 2)).astype(np.float32)).cuda()
    g, _ = m.gradients(x, t)
    p0 = m.params().astype(np.float64)
    m.train_step(x, t, lr=1e-3)
    p1 = m.params().astype(np.float64)
    P = sg.Mlp.unflatten(p0, 4)
    G = sg.Mlp.unflatten(g.astype(np.float64), 4)
    opt = om.Adam(P, lr=1e-3)
    ref = sg.Mlp.flatten(opt.step(P, G))
    assert np.allclose(p1 - p0, ref - p0, rtol=1e-4, atol=1e-9)


def test_training_reduces_loss(sg):
    m = sg.Mlp(n_hidden=4, seed=1)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(8192, 24)).astype(np.float32)
    t = np.stack([np.sin(x[:, 0]) + x[:, 1] ** 2, x[:, 2] * x[:, 3]], axis=1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, l0 = m.gradients(xd, td)
    losses = m.train(xd, td, batch=512, epochs=15, lr=1e-3, seed=3)
    _, l1 = m.gradients(xd, td)
    assert np.all(np.isfinite(losses))
    assert l1 < 0.1 * l0, (l0, l1, losses)


def test_fit_norm_matches_column_statistics(sg):
    """ems_mlp_fit_norm: column means and standard deviations (FP64 sums on
    the device) against numpy's, a constant column gets std 1, and the
    installed standardisation is the one the network then uses."""
    rng = np.random.default_rng(3)
    x = rng.normal(2.0, 3.0, size=(50_001, 24)).astype(np.float32)
    x[:, 5] = 7.25                                       # constant column
    t = np.stack([rng.normal(8.0, 1.5, 50_001), rng.uniform(0, 1, 50_001)], 1).astype(np.float32)
    m = sg.Mlp(n_hidden=2, seed=0)
    xm, xs, tm, ts = m.fit_norm(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    xd, td = x.astype(np.float64), t.astype(np.float64)
    assert np.allclose(xm, xd.mean(0), rtol=1e-12, atol=1e-12)
    ref_s = xd.std(0); ref_s[5] = 1.0
    assert np.allclose(xs, ref_s, rtol=1e-10, atol=0)
    assert np.allclose(tm, td.mean(0), rtol=1e-12) and np.allclose(ts, td.std(0), rtol=1e-10)
    # the same statistics through the host call give the same predictions
    xt = torch.from_numpy(x[:4096]).cuda()
    y1 = m.predict(xt).cpu().numpy()
    m.set_norm(xm, xs, tm, ts)
    y2 = m.predict(xt).cpu().numpy()
    assert np.array_equal(y1, y2)
    m.close()
