"""FP64 CPU reference of the differentiable (quantisation-aware) network twin.

TEST INFRASTRUCTURE ONLY (tests/ and the benchmark's CPU leg).  Plain PyTorch
CPU ops in float64 with autograd: every sparse op is written from its
definition with index gathers and index_add, on index structures computed
here from the oracle's octree (binary search on Morton keys).  Shares no code
with the CUDA path.

Network (Sec. 3.1-3.2, Eq. 4-11, with the readings of the integer oracle):
  j = 0: F_b = prelu(Up_0(E_0[Y_{b-1}]));             logits_b = Pred_0(F_b)
  j = 1: y1 = prelu(Conv_a(F_b)); y2 = Conv_b(y1); S_b = prelu(ma y1 + mb y2)
         F_t = prelu(Up_1([S_b | E_1[Y_b]]));          logits_t = Pred_1(F_t)
  j = 1 + m: G = E'_j[Y_{d-1}], m-1 x prelu(Down(G)) to V_t; H = ResBlock([F_t | G]);
         H = prelu(Up_{j,k}([H | E_{j,k}[Y_k]])), k = t..d-1;  logits_d = Pred_j(H)
with t = L - 4 (or L - 3: levels b+1..t then repeat the j = 1 form).  The
ablations of Sec. 4.3 drop the propagated features: every level d > b takes
G = E'_j[Y_{d-1}] brought down to V_k, H = ResBlock(G), m = d - k plain
up-samplings H = prelu(Up_{j,k}(H)); k = t for GRED's levels below t, k = d - 1
for the others and for the baseline.
Loss (supplement, training section): cross-entropy of the true codes, in bits
(divided by ln 2), summed over the network-coded levels.  With qat=True every
activation that is int8 in the integer network, and every weight, passes a
fake quantiser (Eq. 12) with a straight-through gradient.
"""

from __future__ import annotations

import math

import numpy as np
import torch

import oracle as O
from paper_2603_25260_b300 import synth

DT = torch.float64


# --------------------------------------------------------------- structure --

def _decode(keys: np.ndarray, depth: int):
    k = keys.astype(np.uint64)
    out = np.zeros((k.shape[0], 3), dtype=np.int64)
    for i in range(depth):
        out[:, 0] |= ((k >> np.uint64(3 * i + 2)) & np.uint64(1)).astype(np.int64) << i
        out[:, 1] |= ((k >> np.uint64(3 * i + 1)) & np.uint64(1)).astype(np.int64) << i
        out[:, 2] |= ((k >> np.uint64(3 * i)) & np.uint64(1)).astype(np.int64) << i
    return out


def _encode(xyz: np.ndarray, depth: int):
    k = np.zeros(xyz.shape[0], dtype=np.uint64)
    for i in range(depth):
        k |= ((xyz[:, 0] >> i) & 1).astype(np.uint64) << np.uint64(3 * i + 2)
        k |= ((xyz[:, 1] >> i) & 1).astype(np.uint64) << np.uint64(3 * i + 1)
        k |= ((xyz[:, 2] >> i) & 1).astype(np.uint64) << np.uint64(3 * i)
    return k


def _lookup(keys: np.ndarray, q: np.ndarray):
    pos = np.searchsorted(keys, q)
    pos_c = np.minimum(pos, len(keys) - 1)
    return np.where((pos < len(keys)) & (keys[pos_c] == q), pos_c, -1)


def neighbours(keys: np.ndarray, depth: int) -> np.ndarray:
    """[N, 27] rows of the 3x3x3 neighbours, o = 9(dx+1)+3(dy+1)+(dz+1), -1 absent."""
    c = _decode(keys, depth)
    side = 1 << depth
    out = np.full((keys.shape[0], 27), -1, dtype=np.int64)
    for o in range(27):
        d = np.array([o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1])
        q = c + d
        ok = np.all((q >= 0) & (q < side), axis=1)
        r = np.full(keys.shape[0], -1, dtype=np.int64)
        if ok.any():
            r[ok] = _lookup(keys, _encode(q[ok], depth))
        out[:, o] = r
    return out


class _Neighbours(dict):
    """Kernel maps by depth, computed on first use."""

    def __init__(self, keys):
        super().__init__()
        self._keys = keys

    def __missing__(self, d):
        v = self[d] = torch.from_numpy(neighbours(self._keys[d], d))
        return v


class Frame:
    """Levels, codes and index structures of one frame."""

    def __init__(self, xyz: np.ndarray, L: int):
        self.L, self.b, self.t = L, L - 5, L - 4
        self.n = xyz.shape[0]
        self.keys, self.codes = O.build_levels(xyz, L)
        self.par, self.slot = {}, {}
        for d in range(1, L + 1):
            pk = self.keys[d - 1]
            ck = self.keys[d]
            self.par[d] = torch.from_numpy(np.searchsorted(pk, ck >> np.uint64(3)).astype(np.int64))
            self.slot[d] = torch.from_numpy((ck & np.uint64(7)).astype(np.int64))
        self.nbr = _Neighbours(self.keys)
        self.Y = {d: torch.from_numpy(self.codes[d].astype(np.int64)) for d in range(L)}


# ------------------------------------------------------------------- ops --

class _FakeQuant(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, s, z):
        r = torch.round(x / s) + z
        ctx.save_for_backward((r >= -128) & (r <= 127))
        return (torch.clamp(r, -128, 127) - z) * s

    @staticmethod
    def backward(ctx, g):
        (m,) = ctx.saved_tensors
        return g * m, None, None


class _RoundBF16(torch.autograd.Function):
    """Forward: the value a bf16 operand holds (via float32, as the device
    rounds its float32 values); backward: identity."""

    @staticmethod
    def forward(ctx, x):
        return x.float().bfloat16().to(x.dtype)

    @staticmethod
    def backward(ctx, g):
        return g


class _GradRoundBF16(torch.autograd.Function):
    """Forward: identity; backward: the incoming gradient rounded to bf16 (the
    device's bf16 backward multiplies rounded output gradients)."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return g.float().bfloat16().to(g.dtype)


def rb(x):
    return _RoundBF16.apply(x)


def grb(x):
    return _GradRoundBF16.apply(x)


def fq(x, s, z=0):
    return _FakeQuant.apply(x, s, z)


def fq_w(w):
    s = w.detach().abs().max().clamp_min(1e-12) / 127.0
    return _FakeQuant.apply(w, s, 0)


def prelu(x, a):
    return torch.where(x >= 0, x, a * x)


def conv333(x, nbr, W, b):
    xp = torch.cat([x, x.new_zeros(1, x.shape[1])])
    idx = torch.where(nbr >= 0, nbr, torch.full_like(nbr, x.shape[0]))
    return torch.einsum("noc,odc->nd", xp[idx], W) + b


def up(x, par, slot, W, b):
    return torch.einsum("rdc,rc->rd", W[slot], x[par]) + b[slot]


def down(x, par, slot, n_par, W, b):
    contrib = torch.einsum("rdc,rc->rd", W[slot], x)
    return torch.zeros(n_par, W.shape[1], dtype=x.dtype).index_add(0, par, contrib) + b


def linear(x, W, b):
    return x @ W.T + b


# ------------------------------------------------------------------ model --

# Parameter names, shapes and seeded initial values are input generation and
# live in the shared generator module.
param_shapes = synth.twin_param_shapes
init_params = synth.twin_params


ACT_SCALE = 1.0 / 32.0  # fixed activation scale of the fake quantisers


ARCH_XFP, ARCH_GRED, ARCH_BASE = 0, 1, 2  # GRED + XFP; GRED only; baseline (Sec. 4.3)


def level_bits(P: dict, fr: Frame, qat: bool = False, bf16: bool = False, arch: int = ARCH_XFP,
               t_off: int = 4) -> torch.Tensor:
    """Total bits (cross-entropy / ln 2) of the network-coded levels of a frame.

    bf16=True rounds what the device's bf16 mode rounds: both operands of
    every product, and in the sparse ops' backward the output gradient too;
    biases and accumulations stay exact."""
    def ce(logits, d):
        return torch.nn.functional.cross_entropy(logits, fr.Y[d] - 1, reduction="sum") / math.log(2.0)
    return sum(_levels(P, fr, ce, qat, bf16, arch, t_off))


def level_logits(P: dict, fr: Frame, qat: bool = False, arch: int = ARCH_XFP,
                 t_off: int = 4) -> dict:
    """Logits [N_d, 255] of every network-coded level d (in nats)."""
    out = {}

    def keep(logits, d):
        out[d] = logits
        return 0.0
    _levels(P, fr, keep, qat, False, arch, t_off)
    return out


def _levels(P, fr, head, qat, bf16, arch, t_off):
    b, L = fr.b, fr.L
    t = L - t_off
    q = (lambda x: fq(x, ACT_SCALE)) if qat else (lambda x: x)
    w = (lambda n: fq_w(P[n])) if qat else (lambda n: P[n])
    r = rb if bf16 else (lambda x: x)
    g = grb if bf16 else (lambda x: x)

    def pred(j, F):
        h = prelu(linear(r(q(F)), r(w(f"P1_{j}.W")), P[f"P1_{j}.b"]), P[f"P1_{j}.a"])
        return linear(r(q(h)), r(w(f"P2_{j}.W")), P[f"P2_{j}.b"])

    def upl(name, d, x):  # V_{d-1} -> V_d
        y = g(up(r(q(x)), fr.par[d], fr.slot[d], r(w(name + ".W")),
                     torch.zeros_like(P[name + ".b"])))
        return prelu(y + P[name + ".b"][fr.slot[d]], P[name + ".a"])

    def conv(x, d, name):
        return g(conv333(r(q(x)), fr.nbr[d], r(w(name + ".W")), 0.0)) + P[name + ".b"]

    def resblock(j, d, x):
        y1 = prelu(conv(x, d, f"RA_{j}"), P[f"RA_{j}.a"])
        y2 = conv(y1, d, f"RB_{j}")
        return prelu(P[f"RM_{j}.ma"] * y1 + P[f"RM_{j}.mb"] * y2, P[f"RM_{j}.a"])

    F = {b: upl("UP_0", b, P["E_0"][fr.Y[b - 1]])}
    terms = [head(pred(0, F[b]), b)]
    for j in range(1, 5):
        d = b + j
        if arch == ARCH_XFP and d <= t:
            S = resblock(j, d - 1, F[d - 1])
            F[d] = upl(f"UP_{j}", d, torch.cat([S, P[f"E_{j}"][fr.Y[d - 1]]], 1))
            terms.append(head(pred(j, F[d]), d))
            continue
        if arch == ARCH_XFP or (arch == ARCH_GRED and d > t):
            k0 = t
        else:
            k0 = d - 1
        G = P[f"G_{j}"][fr.Y[d - 1]]
        for i in range(1, d - k0):
            k = d - 1 - i  # V_{k+1} -> V_k
            name = f"D_{j}_{i}"
            y = g(down(r(q(G)), fr.par[k + 1], fr.slot[k + 1], len(fr.keys[k]),
                       r(w(name + ".W")), 0.0))
            G = prelu(y + P[name + ".b"], P[name + ".a"])
        H = resblock(j, k0, torch.cat([F[t], G], 1) if arch == ARCH_XFP else G)
        for k in range(d - k0):
            x = torch.cat([H, P[f"E_{j}_{k}"][fr.Y[k0 + k]]], 1) if arch == ARCH_XFP else H
            H = upl(f"UP_{j}_{k}", k0 + k + 1, x)
        terms.append(head(pred(j, H), d))
    return terms


def to_torch(params: dict, requires_grad: bool = True) -> dict:
    return {k: torch.tensor(v, dtype=DT, requires_grad=requires_grad) for k, v in params.items()}
