"""Pins of the FP64 U-Net reference that the GPU surrogate is checked against.

Forward pieces are checked against independent library routines (torch's
FP64 CPU convolution, average pooling and nearest upsampling); the
hand-written backward pass against central finite differences of the loss.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle.unet_ref import UNetRef, conv3x3, conv3x3_bwd, pool, up


def _nchw(a):
    return torch.from_numpy(np.ascontiguousarray(a.transpose(0, 3, 1, 2)))


def test_conv3x3_matches_library_convolution():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7, 3))
    w = rng.normal(size=(9, 4, 3))
    b = rng.normal(size=4)
    # torch weight [Co][Ci][ky][kx] with tap = 3 ky + kx; cross-correlation
    wt = torch.from_numpy(w.reshape(3, 3, 4, 3).transpose(2, 3, 0, 1).copy())
    ref = F.conv2d(_nchw(x), wt, torch.from_numpy(b), padding=1).numpy().transpose(0, 2, 3, 1)
    np.testing.assert_allclose(conv3x3(x, w, b), ref, rtol=1e-12, atol=1e-12)


def test_conv3x3_backward_is_the_adjoint():
    # <conv(x) - b, y> = <x, gx(y)> and d<conv(x), y>/dw = gw(y)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 6, 8, 3))
    w = rng.normal(size=(9, 5, 3))
    gy = rng.normal(size=(1, 6, 8, 5))
    gx, gw, gb = conv3x3_bwd(x, w, gy)
    lhs = float(((conv3x3(x, w, np.zeros(5))) * gy).sum())
    assert lhs == pytest.approx(float((x * gx).sum()), rel=1e-12)
    assert lhs == pytest.approx(float((w * gw).sum()), rel=1e-12)
    np.testing.assert_allclose(gb, gy.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_match_library():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 6, 8, 3))
    np.testing.assert_allclose(pool(x), F.avg_pool2d(_nchw(x), 2).numpy().transpose(0, 2, 3, 1),
                               rtol=1e-13)
    np.testing.assert_allclose(up(x), F.interpolate(_nchw(x), scale_factor=2, mode="nearest")
                               .numpy().transpose(0, 2, 3, 1))


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_network_gradients_match_finite_differences(levels):
    net = UNetRef(levels, 32, 3, 2)
    rng = np.random.default_rng(10 + levels)
    # He-scaled weights keep activations O(1) through every level
    params = [rng.normal(size=s) * (np.sqrt(2.0 / (s[0] * s[-1] if len(s) == 3 else s[-1]))
                                    if len(s) > 1 else 0.05) for s in net.shapes]
    side = 4 << levels
    x = rng.normal(size=(2, side, side, 3))
    t = rng.normal(size=(2, side, side, 2))
    loss, _, grads = net.loss_and_grads(x, t, params)
    assert len(grads) == len(params)
    for pi, p in enumerate(params):
        assert grads[pi].shape == p.shape
        # the three largest-gradient entries of every tensor and one random one
        flat = np.argsort(np.abs(grads[pi]).ravel())[-3:].tolist()
        flat.append(int(rng.integers(0, p.size)))
        for fi in flat:
            idx = np.unravel_index(fi, p.shape)
            h = 1e-7
            q = [a.copy() for a in params]
            q[pi][idx] += h
            lp = net.loss_and_grads(x, t, q)[0]
            q[pi][idx] -= 2 * h
            lm = net.loss_and_grads(x, t, q)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi][idx]) <= 1e-4 * max(1e-3, abs(fd)), (pi, idx, fd,
                                                                           grads[pi][idx])


def test_parameter_count_of_the_four_level_network():
    # 32/64/128/256 channels, 16 padded inputs, 4 outputs
    net = UNetRef(4, 32, 4, 4)
    n = sum(int(np.prod(s)) for s in net.shapes)
    C = [32, 64, 128, 256]
    expect = sum(9 * c * ci + c for c, ci in zip(C, [16] + C[:-1]))
    expect += sum(9 * c * c + c for c in C)
    expect += sum(9 * C[l] * C[l + 1] + C[l] for l in range(3))
    expect += sum(9 * C[l] * 2 * C[l] + C[l] for l in range(3))
    expect += sum(9 * C[l] * C[l] + C[l] for l in range(3))
    expect += 4 * 32 + 4
    assert n == expect
