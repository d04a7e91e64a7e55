"""The U-Net surrogate's GPU forward / backward / Adam kernels against the
FP64 CPU reference.

The GPU network stores bf16 weights and activations and accumulates in FP32.
The reference gets the same bf16-rounded 3x3 weights and input, rounds each
activation it keeps to bf16 as the network does (so that both take every
ReLU mask decision on the same stored values: a unit whose pre-activation
sits within rounding of zero passes or blocks its whole gradient), and
computes everything else in FP64.  What remains is FP32 summation order and
the bf16 rounding of the activation gradients, about 2^-9 relative per layer.
The bars (relative Frobenius error 2e-2 on outputs, 4e-2 on each gradient
tensor, cosine 0.999) sit well above that and far below what a wrong tap, a
transposed weight or a missing mask gives (relative errors of order one).
"""
import numpy as np
import pytest
import torch

from oracle.unet_ref import UNetRef

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import paper_2206_02145_gb300
    return paper_2206_02145_gb300


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _cos(a, b):
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 and nb == 0:
        return 1.0
    return float((a.ravel() @ b.ravel()) / (na * nb))


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("levels,batch,h,w", [(1, 2, 8, 64), (2, 2, 16, 128), (3, 1, 8, 256)])
def test_forward_and_gradients_match_fp64_reference(lib, levels, batch, h, w, tc):
    in_ch, out_ch = 4, 3
    net = lib.UNet(in_ch=in_ch, out_ch=out_ch, base_ch=32, levels=levels, batch=batch, height=h,
                   width=w, seed=7, stream=lib.current_stream())
    net.set_tensor_path(tc)
    ref = UNetRef(levels, 32, in_ch, out_ch, store=_bf16)
    flat = net.weights().astype(np.float64)
    assert flat.size == sum(int(np.prod(s)) for s in ref.shapes) == net.param_count
    params = ref.unflatten(flat)
    # the GPU convolves with bf16 copies of the 3x3 weights; biases and head are FP32
    params = [_bf16(p) if p.ndim == 3 else p for p in params]
    rng = np.random.default_rng(levels)
    x = rng.normal(size=(batch, h, w, in_ch)).astype(np.float32)
    t = rng.normal(size=(batch, h, w, out_ch)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    yd = torch.empty(batch, h, w, out_ch, device="cuda")
    net.forward(xd, yd)
    torch.cuda.synchronize()
    loss = net.grad(xd, td)
    g_gpu = ref.unflatten(net.grads().astype(np.float64))
    loss_ref, y_ref, g_ref = ref.loss_and_grads(_bf16(x), t.astype(np.float64), params)
    assert _rel(yd.cpu().double().numpy(), y_ref) < 2e-2
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    errs = [(_rel(a, b), _cos(a, b)) for a, b in zip(g_gpu, g_ref)]
    print("gradient rel / cos per tensor:", [(f"{r:.2e}", f"{c:.6f}") for r, c in errs])
    for i, (a, b) in enumerate(zip(g_gpu, g_ref)):
        assert a.shape == b.shape
        assert errs[i][0] < 4e-2, (i, ref.shapes[i], errs[i])
        assert errs[i][1] > 0.999, (i, ref.shapes[i], errs[i])
    net.close()


def test_tensor_core_paths_agree_at_full_size(lib):
    # the 512 x 512 four-level network: tcgen05 and mma.sync kernels differ
    # only in FP32 summation order (and the bf16 rounding that follows)
    net = lib.UNet(in_ch=4, out_ch=4, levels=4, batch=1, height=512, width=512, seed=9,
                   stream=lib.current_stream())
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn(1, 512, 512, 4, generator=g).cuda()
    t = torch.randn(1, 512, 512, 4, generator=g).cuda()
    out = {}
    for tc in (True, False):
        net.set_tensor_path(tc)
        y = torch.empty_like(x)
        net.forward(x, y)
        loss = net.grad(x, t)
        out[tc] = (y.cpu().double().numpy(), loss, net.grads().astype(np.float64))
    net.status()
    assert _rel(out[True][0], out[False][0]) < 1e-2
    assert out[True][1] == pytest.approx(out[False][1], rel=1e-3)
    assert _rel(out[True][2], out[False][2]) < 3e-2
    assert _cos(out[True][2], out[False][2]) > 0.9995
    net.close()


def test_set_weights_round_trip_and_forward_follows(lib):
    net = lib.UNet(in_ch=2, out_ch=1, levels=2, batch=1, height=8, width=128, seed=3,
                   stream=lib.current_stream())
    w0 = net.weights()
    x = torch.randn(1, 8, 128, 2, device="cuda")
    y0 = torch.empty(1, 8, 128, 1, device="cuda")
    y1 = torch.empty_like(y0)
    net.forward(x, y0)
    net.set_weights(w0 * 0.5)
    np.testing.assert_array_equal(net.weights(), (w0 * 0.5).astype(np.float32))
    net.forward(x, y1)
    torch.cuda.synchronize()
    assert not torch.equal(y0, y1)
    net.set_weights(w0)
    net.forward(x, y1)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    with pytest.raises(ValueError):
        net.set_weights(w0[:-1])
    net.close()


def test_adam_training_reduces_the_loss(lib):
    # fit a fixed smooth map of the input: loss must fall by a factor of 5
    net = lib.UNet(in_ch=4, out_ch=4, levels=3, batch=2, height=32, width=256, seed=11,
                   stream=lib.current_stream())
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(2, 32, 256, 4, generator=g).cuda()
    t = (0.5 * torch.roll(x, 1, dims=2) - 0.25 * x).contiguous()
    l0 = net.grad(x, t)
    loss = torch.zeros(1, device="cuda")
    for _ in range(300):
        net.train_step(x, t, 2e-3, loss)
    torch.cuda.synchronize()
    l1 = net.grad(x, t)
    assert np.isfinite(l1) and l1 < l0 / 5, (l0, l1)
    net.close()


def test_training_is_bit_reproducible(lib):
    # the same schedule from the same initialisation twice, on the configured
    # depth with a 16-channel first layer (the per-tap weight gradient), the
    # nine-tap kernel's layers and the 1x1 head: identical weights
    from paper_2206_02145_gb300 import surrogate as S
    kw = dict(in_ch=4, out_ch=4, levels=4, batch=2, height=32, width=512, seed=5,
              stream=lib.current_stream())
    g = torch.Generator(device="cpu").manual_seed(9)
    X = torch.randn(5, 32, 512, 4, generator=g).cuda()
    T = (0.2 * torch.roll(X, 1, dims=1) - 0.1 * X).contiguous()
    runs = []
    for _ in range(2):
        net = lib.UNet(**kw)
        S.train(net, X, T, 12, lr=1e-3, seed=2, log_every=6)
        net.status()
        runs.append(net.weights())
        net.close()
    assert np.linalg.norm(runs[0]) > 0
    assert np.array_equal(runs[0], runs[1])


def test_library_training_loop_follows_the_explicit_loop(lib):
    # lbpf_surrogate_train against the same minibatches gathered, mirrored and
    # stepped one call at a time.  Every gradient is summed in a fixed order
    # (only the reported loss uses an atomic addition), so the two loops end
    # with the same weights bit for bit.  At learning rate 0 every step's loss
    # is that of the fixed network on its minibatch: equal losses step by step
    # pin the gather and the mirrors, and the weights stay as they were
    from paper_2206_02145_gb300 import surrogate as S
    kw = dict(in_ch=4, out_ch=4, levels=2, batch=2, height=16, width=128, seed=3,
              stream=lib.current_stream())
    g = torch.Generator(device="cpu").manual_seed(8)
    X = torch.randn(7, 16, 128, 4, generator=g).cuda()
    T = (0.3 * torch.roll(X, 1, dims=2) - 0.2 * X).contiguous()
    steps = 23
    idx, flip, rates = S.train_schedule(7, 2, steps, lr=1e-3, seed=4)
    assert set(flip.tolist()) == {0, 1, 2}
    sign = {1: torch.tensor([1.0, 1.0, 1.0, -1.0], device="cuda"),
            2: torch.tensor([1.0, 1.0, -1.0, 1.0], device="cuda")}

    def explicit(net, lrs, every):
        loss = torch.zeros(1, device="cuda")
        out = []
        for s in range(steps):
            k = torch.from_numpy(idx[s].astype(np.int64)).cuda()
            xb, tb = X.index_select(0, k), T.index_select(0, k)
            if flip[s]:
                d = int(flip[s])  # 1 mirrors rows (dim 1), 2 columns (dim 2)
                xb = (xb.flip(d) * sign[d]).contiguous()
                tb = (tb.flip(d) * sign[d]).contiguous()
            net.train_step(xb, tb, float(lrs[s]), loss)
            if (s + 1) % every == 0 or s == steps - 1:
                out.append(float(loss.item()))
        return np.array(out)

    zero = np.zeros(steps, np.float32)
    a, b = lib.UNet(**kw), lib.UNet(**kw)
    w0 = a.weights()
    got = lib.lbpf_surrogate_train(a, X, T, idx, flip, zero, 1)
    want = explicit(b, zero, 1)
    assert got.shape == (steps,) and np.all(got > 0)
    np.testing.assert_allclose(got, want, rtol=1e-5)
    assert np.array_equal(a.weights(), w0)
    # the mirrors matter: the same steps unmirrored give other losses (by
    # 6e-4 to 1e-2 relative for a network of this size at He scale)
    plain = lib.lbpf_surrogate_train(a, X, T, idx, np.zeros(steps, np.int32), zero, 1)
    assert np.median(np.abs(plain / got - 1)[flip != 0]) > 1e-3
    assert np.array_equal(plain[flip == 0], got[flip == 0]) or \
        np.allclose(plain[flip == 0], got[flip == 0], rtol=1e-5)
    a.close()
    b.close()

    a, b = lib.UNet(**kw), lib.UNet(**kw)
    hist = S.train(a, X, T, steps, lr=1e-3, seed=4, log_every=5)
    want = explicit(b, rates, 5)
    wa, wb = a.weights(), b.weights()
    assert [h[0] for h in hist] == [5, 10, 15, 20, 23]
    assert np.linalg.norm(wb - w0) > 0  # the schedule moved the weights
    assert np.array_equal(wa, wb)
    np.testing.assert_allclose([h[1] for h in hist], want, rtol=2e-2)
    # rejections: a pair index out of range, a flip code, a rate; nothing queued
    bad_idx = idx.copy()
    bad_idx[3, 1] = 7
    for args in ((bad_idx, flip, rates), (idx, np.full(steps, 3), rates),
                 (idx, flip, np.full(steps, np.nan, np.float32))):
        with pytest.raises(lib.LbpfError) as e:
            lib.lbpf_surrogate_train(a, X, T, *args)
        assert e.value.code == lib.EINVAL
    a.close()
    b.close()


def test_rejects_unsupported_shapes(lib):
    with pytest.raises(lib.LbpfError):
        lib.UNet(levels=2, height=16, width=96)  # width / 2 not a multiple of 64
    with pytest.raises(lib.LbpfError):
        lib.UNet(base_ch=48, height=64, width=64, levels=1)
    with pytest.raises(lib.LbpfError):
        lib.UNet(in_ch=17, height=64, width=64, levels=1)


def _maxrel(a, b):
    """Largest element-wise difference, relative to the tensor's largest
    reference magnitude."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_configured_network_elementwise_at_full_size(lib):
    # the propagator's network as configured (4 levels, 32/64/128/256
    # channels, 4 -> 4, 512 x 512, batch 1) on the tcgen05 path: the same
    # layer shapes, hence the same kernel variants (halo and row tiles, every
    # channel chunk and tile width), as the propagator and the benchmark run
    levels, h, w = 4, 512, 512
    net = lib.UNet(in_ch=4, out_ch=4, base_ch=32, levels=levels, batch=1, height=h, width=w,
                   seed=11, stream=lib.current_stream())
    net.set_tensor_path(True)
    ref = UNetRef(levels, 32, 4, 4, store=_bf16)
    params = ref.unflatten(net.weights().astype(np.float64))
    params = [_bf16(p) if p.ndim == 3 else p for p in params]
    rng = np.random.default_rng(21)
    x = rng.normal(size=(1, h, w, 4)).astype(np.float32)
    t = rng.normal(size=(1, h, w, 4)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    yd = torch.empty(1, h, w, 4, device="cuda")
    net.forward(xd, yd)
    torch.cuda.synchronize()
    loss = net.grad(xd, td)
    g_gpu = ref.unflatten(net.grads().astype(np.float64))
    net.status()
    net.close()
    loss_ref, y_ref, g_ref = ref.loss_and_grads(_bf16(x), t.astype(np.float64), params)
    y = yd.cpu().double().numpy()
    # Both sides round every stored activation to bf16 (unit roundoff
    # u = 2^-9); they differ by FP32 summation order, which flips the
    # rounding of a few elements by one bf16 ulp per layer, and by the GPU's
    # bf16 activation gradients.  The output passes 17 stored layers: bound
    # 17 u on its largest element; a gradient passes at most 2 x 17 roundings
    # on the way back: bound 34 u.  A wrong tap, channel or mask gives O(1).
    u = 2.0 ** -9
    e_y = _maxrel(y, y_ref)
    e_g = [_maxrel(a, b) for a, b in zip(g_gpu, g_ref)]
    print(f"output max-rel {e_y:.3e}; gradients max-rel "
          + " ".join(f"{e:.2e}" for e in e_g))
    assert e_y < 17 * u, e_y
    assert loss == pytest.approx(loss_ref, rel=17 * u)
    for i, e in enumerate(e_g):
        assert e < 34 * u, (i, ref.shapes[i], e)
