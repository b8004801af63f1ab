"""Pins of the FP64 training reference (oracle/train_ref.py) against library
routines and closed forms, on the CPU."""

import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import train_ref as T
from paper_2603_25260_b300 import synth

DT = torch.float64


def _frame(L=6, n=300, seed=11):
    xyz = synth.random_cloud(n, L, seed)
    return T.Frame(xyz, L), xyz


def _coords(fr, d):
    return T._decode(fr.keys[d], d)


def _dense(x, coords, side):
    g = torch.zeros(1, x.shape[1], side, side, side, dtype=DT)
    g[0, :, coords[:, 0], coords[:, 1], coords[:, 2]] = x.T
    return g


def test_neighbours_brute_force():
    fr, _ = _frame(L=5, n=200, seed=3)
    d = 5
    keys = fr.keys[d]
    c = _coords(fr, d)
    where = {tuple(p): i for i, p in enumerate(c.tolist())}
    nbr = T.neighbours(keys, d)
    for i, p in enumerate(c.tolist()):
        for o in range(27):
            q = (p[0] + o // 9 - 1, p[1] + (o // 3) % 3 - 1, p[2] + o % 3 - 1)
            assert nbr[i, o] == where.get(q, -1)


def test_conv333_vs_dense_conv3d():
    """Sparse 3x3x3 conv (Eq. 5) equals torch's dense conv3d (padding 1) read
    at the occupied voxels."""
    fr, _ = _frame(L=6, n=400, seed=5)
    d = fr.t
    c = _coords(fr, d)
    g = torch.Generator().manual_seed(0)
    cin, cout = 3, 4
    x = torch.randn(len(c), cin, generator=g, dtype=DT)
    W = torch.randn(27, cout, cin, generator=g, dtype=DT)
    b = torch.randn(cout, generator=g, dtype=DT)
    y = T.conv333(x, fr.nbr[d], W, b)
    w5 = W.reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2)
    yd = F.conv3d(_dense(x, c, 1 << d), w5, b, padding=1)[0]
    ref = yd[:, c[:, 0], c[:, 1], c[:, 2]].T
    torch.testing.assert_close(y, ref, rtol=1e-12, atol=1e-12)


def test_up_vs_conv_transpose3d():
    """Upsampling + Pruning (Eq. 6): the kernel-2 stride-2 transposed conv,
    kept at the occupied children; the child slot c = 4 bx + 2 by + bz."""
    fr, _ = _frame(L=6, n=400, seed=6)
    d = fr.t
    cp, cc = _coords(fr, d - 1), _coords(fr, d)
    g = torch.Generator().manual_seed(1)
    cin, cout = 3, 5
    x = torch.randn(len(cp), cin, generator=g, dtype=DT)
    W = torch.randn(8, cout, cin, generator=g, dtype=DT)
    b = torch.randn(8, cout, generator=g, dtype=DT)
    y = T.up(x, fr.par[d], fr.slot[d], W, torch.zeros_like(b))
    w5 = W.reshape(2, 2, 2, cout, cin).permute(4, 3, 0, 1, 2)
    yd = F.conv_transpose3d(_dense(x, cp, 1 << (d - 1)), w5, stride=2)[0]
    ref = yd[:, cc[:, 0], cc[:, 1], cc[:, 2]].T
    torch.testing.assert_close(y, ref, rtol=1e-12, atol=1e-12)
    slot = torch.from_numpy((cc[:, 0] & 1) * 4 + (cc[:, 1] & 1) * 2 + (cc[:, 2] & 1))
    torch.testing.assert_close(T.up(x, fr.par[d], fr.slot[d], W, b) - y, b[slot])


def test_down_vs_strided_conv3d():
    """Stride-2 down conv (Eq. 4): torch's kernel-2 stride-2 conv3d read at
    the occupied parents."""
    fr, _ = _frame(L=6, n=400, seed=7)
    d = fr.t
    cp, cc = _coords(fr, d - 1), _coords(fr, d)
    g = torch.Generator().manual_seed(2)
    cin, cout = 4, 3
    x = torch.randn(len(cc), cin, generator=g, dtype=DT)
    W = torch.randn(8, cout, cin, generator=g, dtype=DT)
    b = torch.randn(cout, generator=g, dtype=DT)
    y = T.down(x, fr.par[d], fr.slot[d], len(cp), W, b)
    w5 = W.reshape(2, 2, 2, cout, cin).permute(3, 4, 0, 1, 2)
    yd = F.conv3d(_dense(x, cc, 1 << d), w5, b, stride=2)[0]
    ref = yd[:, cp[:, 0], cp[:, 1], cp[:, 2]].T
    torch.testing.assert_close(y, ref, rtol=1e-12, atol=1e-12)


def test_structure_parents_and_slots():
    fr, _ = _frame(L=7, n=500, seed=8)
    for d in range(1, fr.L + 1):
        cp, cc = _coords(fr, d - 1), _coords(fr, d)
        np.testing.assert_array_equal(cp[fr.par[d].numpy()], cc >> 1)
        s = (cc[:, 0] & 1) * 4 + (cc[:, 1] & 1) * 2 + (cc[:, 2] & 1)
        np.testing.assert_array_equal(fr.slot[d].numpy(), s)
        occ = np.zeros(len(cp), dtype=np.int64)
        np.bitwise_or.at(occ, fr.par[d].numpy(), 1 << fr.slot[d].numpy())
        np.testing.assert_array_equal(occ, fr.codes[d - 1])


def test_fake_quant_vs_torch():
    """Eq. 12 with a straight-through gradient equals torch's per-tensor fake
    quantiser on the int8 range, values and gradients."""
    g = torch.Generator().manual_seed(3)
    x = (torch.randn(4000, generator=g, dtype=torch.float32) * 3).requires_grad_()
    for s, z in ((1 / 32, 0), (0.05, -7), (0.011, 20)):
        y = T.fq(x, s, z)
        x2 = x.detach().clone().requires_grad_()
        ref = torch.fake_quantize_per_tensor_affine(x2, s, z, -128, 127)
        torch.testing.assert_close(y, ref, rtol=0, atol=1e-6)
        gy = torch.randn(4000, generator=g)
        (gx,) = torch.autograd.grad(y, x, gy)
        (gr,) = torch.autograd.grad(ref, x2, gy)
        assert torch.equal(gx, gr)


def test_prelu_vs_torch():
    g = torch.Generator().manual_seed(4)
    x = torch.randn(100, 6, generator=g, dtype=DT)
    a = torch.rand(6, generator=g, dtype=DT)
    torch.testing.assert_close(T.prelu(x, a), F.prelu(x, a))


@pytest.fixture(scope="module")
def gframe():
    return T.Frame(synth.make_frame(synth.GRADCHECK), synth.GRADCHECK.L)


def test_uniform_predictor_closed_form(gframe):
    """With the last predictor layer zeroed every code has probability 1/255,
    so the loss is exactly (N_b + ... + N_{b+4}) log2 255 bits: pins which
    five levels the network codes."""
    P = T.to_torch(T.init_params(0))
    with torch.no_grad():
        for j in range(5):
            P[f"P2_{j}.W"].zero_()
            P[f"P2_{j}.b"].zero_()
    bits = float(T.level_bits(P, gframe).detach())
    n = sum(len(gframe.keys[d]) for d in range(gframe.b, gframe.b + 5))
    assert bits == pytest.approx(n * math.log2(255), rel=1e-12)


def test_perfect_predictor_bits_vanish(gframe):
    """Cross-entropy in bits of a near-one-hot predictor tends to zero: scaling
    logits of the true code pins the target index (code - 1)."""
    Y = gframe.Y[gframe.b]
    logits = torch.full((len(Y), 255), -40.0, dtype=DT)
    logits[torch.arange(len(Y)), Y - 1] = 40.0
    bits = F.cross_entropy(logits, Y - 1, reduction="sum") / math.log(2)
    assert float(bits) < 1e-20


def test_level_bits_directional_derivative(gframe):
    P = T.to_torch(T.init_params(1))
    bits = T.level_bits(P, gframe)
    grads = torch.autograd.grad(bits, list(P.values()))
    g = torch.Generator().manual_seed(9)
    V = {k: torch.randn(v.shape, generator=g, dtype=DT) for k, v in P.items()}
    ana = sum(float((gr * V[k]).sum()) for gr, k in zip(grads, P))
    eps = 1e-8  # small enough that few PReLU kinks lie within the step
    with torch.no_grad():
        fp = T.level_bits({k: v + eps * V[k] for k, v in P.items()}, gframe)
        fm = T.level_bits({k: v - eps * V[k] for k, v in P.items()}, gframe)
    num = float(fp - fm) / (2 * eps)
    assert num == pytest.approx(ana, rel=1e-5)


def test_every_parameter_gets_gradient(gframe):
    P = T.to_torch(T.init_params(2))
    bits = T.level_bits(P, gframe, qat=True)
    grads = torch.autograd.grad(bits, list(P.values()))
    for k, g in zip(P, grads):
        assert torch.isfinite(g).all(), k
        assert float(g.abs().sum()) > 0, k
