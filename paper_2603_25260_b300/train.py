"""Differentiable (quantisation-aware) twin of the codec's network on B300.

The sparse ops -- 3x3x3 conv, Upsampling + Pruning (densify), stride-2 down
conv (sparsify), occupancy-code embedding, PReLU and the fake quantiser --
run forward and backward in the hand-written kernels of ``csrc/train.cu``
(C ABI in ``include/lpc_train.h``), exposed as ``torch.autograd.Function``s.
The predictor's two dense linear layers and the cross-entropy are plain
PyTorch.  The loss is the occupancy cross-entropy in bits (supplement,
training section) over the five network-coded levels; training follows the
paper's settings: AdamW, lr 1e-4, weight decay 1e-4, gradient clipping at 1.0.

Index structures (levels, parent rows, child offsets, kernel maps) come from
the codec's own octree and kernel-map kernels.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

from . import lpc

P_, I64, I32 = C.c_void_p, C.c_int64, C.c_int
_done = False


def _lib():
    global _done
    L = lpc.lib()
    if not _done:
        sig = {
            "lpc_t_conv_fwd": [P_, I64, I32, P_, P_, P_, I32, P_, I32, C.c_uint64],
            "lpc_t_conv_bwd": [P_, P_, I64, I32, P_, P_, I32, P_, P_, P_, I32, C.c_uint64],
            "lpc_t_up_fwd": [P_, I64, I32, P_, P_, P_, I64, P_, P_, I32, P_, I32, C.c_uint64],
            "lpc_t_up_bwd": [P_, P_, I64, I32, P_, P_, P_, I64, P_, I32, P_, P_, P_, I32,
                             C.c_uint64],
            "lpc_t_down_fwd": [P_, I64, I32, P_, P_, I64, P_, P_, I32, P_, I32, C.c_uint64],
            "lpc_t_down_bwd": [P_, P_, I64, I32, P_, P_, P_, I64, P_, I32, P_, P_, P_, I32,
                               C.c_uint64],
            "lpc_t_embed_fwd": [P_, I64, P_, I32, P_, C.c_uint64],
            "lpc_t_embed_bwd": [P_, I64, P_, I32, P_, C.c_uint64],
            "lpc_t_prelu_fwd": [P_, I64, I32, P_, P_, C.c_uint64],
            "lpc_t_prelu_bwd": [P_, P_, I64, I32, P_, P_, P_, C.c_uint64],
            "lpc_t_fq_fwd": [P_, I64, C.c_float, I32, P_, P_, C.c_uint64],
            "lpc_t_fq_bwd": [P_, P_, I64, P_, C.c_uint64],
            "lpc_t_fq_w": [P_, I64, P_, P_, C.c_uint64],
            "lpc_t_levels": [P_, I64, I32, P_, P_, P_, P_, P_, I64, C.c_uint64],
            "lpc_t_tc_error": [I32],
            "lpc_t_pred_fwd": [P_, I64, P_, P_, P_, P_, P_, P_, I32, I32, P_, P_, C.c_uint64],
            "lpc_t_pred_bwd": [P_, I64, P_, P_, P_, P_, P_, P_, I32, I32, P_, P_, P_, P_, P_,
                               P_, P_, C.c_uint64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.restype = I32
            f.argtypes = args
        _done = True
    return L


def _p(t):
    return None if t is None else t.data_ptr()


def tc_error(reset: bool = True) -> int:
    """Non-zero if a tensor-core op of the twin gave up on a bounded wait."""
    return int(_lib().lpc_t_tc_error(int(reset)))


def _st():
    return torch.cuda.current_stream().cuda_stream


def _ck(s, what):
    if s != 0:
        raise lpc.LpcError(s, what)


# Per-op device time (profiling passes only): CUDA events on the current
# stream around every kernel call of the twin, by op name.
_PROF = None


def profile(on: bool) -> None:
    """Start (on) or stop timing every op of the twin; profile_read() sums."""
    global _PROF
    _PROF = {} if on else None


def profile_read() -> dict:
    """{op: {"ms": total device ms, "launches": calls, "flops": algorithmic
    floating-point operations}} since profile(True)."""
    torch.cuda.synchronize()
    fl = (_PROF or {}).get("_flops", {})
    return {k: {"ms": sum(a.elapsed_time(b) for a, b in v), "launches": len(v),
                "flops": fl.get(k, 0.0)}
            for k, v in (_PROF or {}).items() if k != "_flops"}


def _flops(what, n):
    """Algorithmic flops of one call (profiling passes only)."""
    if _PROF is not None:
        f = _PROF.setdefault("_flops", {})
        f[what] = f.get(what, 0.0) + float(n)


def _pairs(nbr):
    return float((nbr >= 0).sum()) if _PROF is not None else 0.0


# per predictor row: two linear layers (2 x 32 x 32 + 2 x 255 x 32 flops);
# the backward recomputes them and forms three more products of each size
PRED_FLOPS = 2.0 * 32 * 32 + 2.0 * 255 * 32


def _call(what, fn, *args):
    if _PROF is None:
        return _ck(fn(*args), what)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    st = fn(*args)
    b.record()
    _PROF.setdefault(what, []).append((a, b))
    return _ck(st, what)


# ------------------------------------------------------------- autograd ops --

class ConvFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, nbr, W, b, bf16):
        x, W, b = x.contiguous(), W.contiguous(), b.contiguous()
        N, cin = x.shape
        y = torch.empty(N, W.shape[1], device=x.device, dtype=torch.float32)
        _flops("conv fwd", 2.0 * _pairs(nbr) * cin * W.shape[1])
        _call("conv fwd", _lib().lpc_t_conv_fwd, _p(x), N, cin, _p(nbr), _p(W), _p(b), W.shape[1],
              _p(y), bf16, _st())
        ctx.save_for_backward(x, nbr, W)
        ctx.bf16 = bf16
        return y

    @staticmethod
    def backward(ctx, dy):
        x, nbr, W = ctx.saved_tensors
        dy = dy.contiguous()
        N, cin = x.shape
        dx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dW = torch.zeros_like(W)
        db = torch.zeros(W.shape[1], device=x.device, dtype=torch.float32)
        _flops("conv bwd", 4.0 * _pairs(nbr) * cin * W.shape[1])
        _call("conv bwd", _lib().lpc_t_conv_bwd, _p(x), _p(dy), N, cin, _p(nbr), _p(W), W.shape[1],
              _p(dx), _p(dW), _p(db), ctx.bf16, _st())
        return dx, None, dW, db, None


class UpFn(torch.autograd.Function):
    """y[r] = W[c_r] x[par r] + b[c_r] over the children r of the next level."""

    @staticmethod
    def forward(ctx, x, par, ckey, off, W, b, bf16):
        x, W, b = x.contiguous(), W.contiguous(), b.contiguous()
        Nc = par.shape[0]
        y = torch.empty(Nc, W.shape[1], device=x.device, dtype=torch.float32)
        _flops("up fwd", 2.0 * Nc * x.shape[1] * W.shape[1])
        _call("up fwd", _lib().lpc_t_up_fwd, _p(x), x.shape[0], x.shape[1], _p(off), _p(par),
              _p(ckey), Nc, _p(W), _p(b), W.shape[1], _p(y), bf16, _st())
        ctx.save_for_backward(x, par, ckey, off, W)
        ctx.bf16 = bf16
        return y

    @staticmethod
    def backward(ctx, dy):
        x, par, ckey, off, W = ctx.saved_tensors
        dy = dy.contiguous()
        dx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dW = torch.zeros_like(W)
        db = torch.zeros(8, W.shape[1], device=x.device, dtype=torch.float32)
        _flops("up bwd", 4.0 * par.shape[0] * x.shape[1] * W.shape[1])
        _call("up bwd", _lib().lpc_t_up_bwd, _p(x), _p(dy), x.shape[0], x.shape[1], _p(off),
              _p(par), _p(ckey), par.shape[0], _p(W), W.shape[1], _p(dx), _p(dW), _p(db), ctx.bf16,
              _st())
        return dx, None, None, None, dW, db, None


class DownFn(torch.autograd.Function):
    """y[p] = b + sum over the children r of p of W[c_r] x[r]."""

    @staticmethod
    def forward(ctx, x, par, ckey, off, W, b, bf16):
        x, W, b = x.contiguous(), W.contiguous(), b.contiguous()
        Np = off.shape[0] - 1
        y = torch.empty(Np, W.shape[1], device=x.device, dtype=torch.float32)
        _flops("down fwd", 2.0 * x.shape[0] * x.shape[1] * W.shape[1])
        _call("down fwd", _lib().lpc_t_down_fwd, _p(x), x.shape[0], x.shape[1], _p(off),
              _p(ckey), Np, _p(W), _p(b), W.shape[1], _p(y), bf16, _st())
        ctx.save_for_backward(x, par, ckey, off, W)
        ctx.bf16 = bf16
        return y

    @staticmethod
    def backward(ctx, dy):
        x, par, ckey, off, W = ctx.saved_tensors
        dy = dy.contiguous()
        dx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dW = torch.zeros_like(W)
        db = torch.zeros(W.shape[1], device=x.device, dtype=torch.float32)
        _flops("down bwd", 4.0 * x.shape[0] * x.shape[1] * W.shape[1])
        _call("down bwd", _lib().lpc_t_down_bwd, _p(x), _p(dy), x.shape[0], x.shape[1], _p(off),
              _p(par), _p(ckey), off.shape[0] - 1, _p(W), W.shape[1], _p(dx), _p(dW), _p(db),
              ctx.bf16, _st())
        return dx, None, None, None, dW, db, None


class EmbedFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, codes, E):
        E = E.contiguous()
        y = torch.empty(codes.shape[0], E.shape[1], device=E.device, dtype=torch.float32)
        _call("embed fwd", _lib().lpc_t_embed_fwd, _p(codes), codes.shape[0], _p(E), E.shape[1],
              _p(y), _st())
        ctx.save_for_backward(codes)
        ctx.shape = E.shape
        return y

    @staticmethod
    def backward(ctx, dy):
        (codes,) = ctx.saved_tensors
        dE = torch.zeros(ctx.shape, device=dy.device, dtype=torch.float32)
        _call("embed bwd", _lib().lpc_t_embed_bwd, _p(codes), codes.shape[0], _p(dy.contiguous()),
              ctx.shape[1], _p(dE), _st())
        return None, dE


class PReLUFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, a):
        x, a = x.contiguous(), a.contiguous()
        y = torch.empty_like(x)
        _call("prelu fwd", _lib().lpc_t_prelu_fwd, _p(x), x.shape[0], x.shape[1], _p(a), _p(y),
              _st())
        ctx.save_for_backward(x, a)
        return y

    @staticmethod
    def backward(ctx, dy):
        x, a = ctx.saved_tensors
        dx = torch.empty_like(x)
        da = torch.zeros_like(a)
        _call("prelu bwd", _lib().lpc_t_prelu_bwd, _p(x), _p(dy.contiguous()), x.shape[0],
              x.shape[1], _p(a), _p(dx), _p(da), _st())
        return dx, da


class FakeQuantFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, s, z):
        x = x.contiguous()
        y = torch.empty_like(x)
        mask = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
        _call("fq fwd", _lib().lpc_t_fq_fwd, _p(x), x.numel(), float(s), int(z), _p(y), _p(mask),
              _st())
        ctx.save_for_backward(mask)
        return y

    @staticmethod
    def backward(ctx, dy):
        (mask,) = ctx.saved_tensors
        dx = torch.empty_like(dy)
        _call("fq bwd", _lib().lpc_t_fq_bwd, _p(dy.contiguous()), _p(mask), dy.numel(), _p(dx),
              _st())
        return dx, None, None


class PredBitsFn(torch.autograd.Function):
    """Predictor (Eq. 7) and rate loss (supplement, Training, Eq. 16) in one
    hand-written kernel: bits = sum over rows of -log2 softmax(W2 q(prelu(W1
    q(F) + b1)) + b2)[code - 1]; the backward kernel recomputes the rows and
    returns the gradients of F, both weights, both biases and the slope."""

    @staticmethod
    def forward(ctx, F, W1, b1, a1, W2, b2, codes, qat, bf16):
        F = F.contiguous()
        W1, b1, a1, W2, b2 = (t.contiguous() for t in (W1, b1, a1, W2, b2))
        bits = torch.zeros(1, dtype=torch.float64, device=F.device)
        _flops("pred fwd", PRED_FLOPS * F.shape[0])
        _call("pred fwd", _lib().lpc_t_pred_fwd, _p(F), F.shape[0], _p(W1), _p(b1), _p(a1), _p(W2),
              _p(b2), _p(codes), int(qat), int(bf16), None, _p(bits), _st())
        ctx.save_for_backward(F, W1, b1, a1, W2, b2, codes)
        ctx.flags = (int(qat), int(bf16))
        return bits.float().reshape(())

    @staticmethod
    def backward(ctx, g):
        F, W1, b1, a1, W2, b2, codes = ctx.saved_tensors
        qat, bf16 = ctx.flags
        g = g.reshape(1).float().contiguous()
        dF = torch.empty_like(F)
        dW1, db1, da1 = torch.zeros_like(W1), torch.zeros_like(b1), torch.zeros_like(a1)
        dW2, db2 = torch.zeros_like(W2), torch.zeros_like(b2)
        _flops("pred bwd", 3.0 * PRED_FLOPS * F.shape[0])
        _call("pred bwd", _lib().lpc_t_pred_bwd, _p(F), F.shape[0], _p(W1), _p(b1), _p(a1), _p(W2),
              _p(b2), _p(codes), qat, bf16, _p(g), _p(dF), _p(dW1), _p(db1), _p(da1), _p(dW2),
              _p(db2), _st())
        return dF, dW1, db1, da1, dW2, db2, None, None, None


def pred_logits(F, W1, b1, a1, W2, b2, qat, bf16):
    """The predictor's float logits [N, 255] (no gradient; the float
    inference variant), from the same kernel as PredBitsFn."""
    F = F.detach().contiguous()
    W1, b1, a1, W2, b2 = (t.detach().contiguous() for t in (W1, b1, a1, W2, b2))
    N = F.shape[0]
    out = torch.empty((N, 255), dtype=torch.float32, device=F.device)
    bits = torch.zeros(1, dtype=torch.float64, device=F.device)
    codes = torch.ones(N, dtype=torch.uint8, device=F.device)  # any valid code
    _call("pred logits", _lib().lpc_t_pred_fwd, _p(F), N, _p(W1), _p(b1), _p(a1), _p(W2), _p(b2),
          _p(codes), int(qat), int(bf16), _p(out), _p(bits), _st())
    return out


class FakeQuantWFn(torch.autograd.Function):
    """Per-tensor symmetric weight fake quantisation (scale max|w| / 127 found
    on the device, no host round trip) with a straight-through gradient."""

    @staticmethod
    def forward(ctx, w):
        w = w.contiguous()
        y = torch.empty_like(w)
        mask = torch.empty(w.shape, dtype=torch.uint8, device=w.device)
        _call("fq w", _lib().lpc_t_fq_w, _p(w), w.numel(), _p(y), _p(mask), _st())
        ctx.save_for_backward(mask)
        return y

    @staticmethod
    def backward(ctx, dy):
        (mask,) = ctx.saved_tensors
        dx = torch.empty_like(dy)
        _call("fq bwd", _lib().lpc_t_fq_bwd, _p(dy.contiguous()), _p(mask), dy.numel(), _p(dx),
              _st())
        return dx


def fq_w(w):
    return FakeQuantWFn.apply(w)


# ------------------------------------------------------------ structures --

class Frame:
    """Device index structures of one frame: levels with parent rows, child
    offsets and child slots, kernel maps at V_b and V_t, codes."""

    def __init__(self, xyz: torch.Tensor, L: int):
        _lib()
        self.L, self.b, self.t = L, L - 5, L - 4
        n = xyz.shape[0]
        self.n = n
        cap = max(1, n) * (L + 1)
        keys = torch.empty(cap, dtype=torch.int64, device="cuda")
        codes = torch.empty(cap, dtype=torch.uint8, device="cuda")
        par = torch.empty(cap, dtype=torch.int32, device="cuda")
        off = torch.empty(cap + L + 1, dtype=torch.int32, device="cuda")
        counts = np.zeros(L + 1, dtype=np.int64)
        _call("levels", _lib().lpc_t_levels, _p(xyz), n, L, _p(keys), _p(codes), _p(par), _p(off),
              counts.ctypes.data, cap, _st())
        self.N = counts.tolist()
        self.keys, self.codes, self.par, self.off, self.Y = {}, {}, {}, {}, {}
        kp = cp = op = 0
        for d in range(L + 1):
            N = self.N[d]
            self.keys[d] = keys[kp:kp + N]
            if d > 0:
                self.par[d] = par[kp:kp + N]
            kp += N
            if d < L:
                self.codes[d] = codes[cp:cp + N]
                self.off[d] = off[op:op + N + 1]
                cp += N
                op += N + 1
        for d in range(L):
            self.Y[d] = self.codes[d].long()
        self.nbr = _KernelMaps(self)
        self.nbr[self.b], self.nbr[self.t]  # built now; deeper ones on first use


class _KernelMaps(dict):
    """Kernel maps by depth: hashed at V_b, below it from the parent level's
    map (every node is a child of a node one level up)."""

    def __init__(self, fr):
        super().__init__()
        self._fr = fr

    def __missing__(self, d):
        fr = self._fr
        if d == fr.b:
            v = lpc.kernel_map(fr.keys[d], d)
        else:
            v = lpc.kernel_map_child(fr.keys[d], fr.par[d], self[d - 1], fr.codes[d - 1],
                                     fr.off[d - 1])
        self[d] = v
        return v


class _BatchMaps(dict):
    def __init__(self, frames, R):
        super().__init__()
        self._frames, self._R = frames, R

    def __missing__(self, d):
        v = self[d] = torch.cat([torch.where(f.nbr[d] >= 0, f.nbr[d] + self._R[d][i], f.nbr[d])
                                 for i, f in enumerate(self._frames)])
        return v


class BatchFrame:
    """Frames of one depth L as a single frame: the rows of each level laid
    out frame after frame, with parent rows, child offsets and kernel-map
    entries shifted by the rows of the frames before.  No row of one frame
    refers to a row of another, so every op sees the union of disjoint trees;
    its rate is the sum of the frames' rates and each op runs once per batch
    instead of once per frame."""

    def __init__(self, frames: list):
        L = frames[0].L
        if any(f.L != L for f in frames):
            raise ValueError("a batch holds frames of one depth")
        self.L, self.b, self.t = L, L - 5, L - 4
        self.n = sum(f.n for f in frames)
        self.N = [sum(f.N[d] for f in frames) for d in range(L + 1)]
        # R[d][i]: rows of level d in frames 0..i-1
        R = [np.concatenate([[0], np.cumsum([f.N[d] for f in frames])]).tolist()
             for d in range(L + 1)]
        self.keys, self.codes, self.par, self.off, self.Y = {}, {}, {}, {}, {}
        for d in range(L + 1):
            self.keys[d] = torch.cat([f.keys[d] for f in frames])
            if d > 0:
                self.par[d] = torch.cat([f.par[d] + R[d - 1][i] for i, f in enumerate(frames)])
            if d < L:
                self.codes[d] = torch.cat([f.codes[d] for f in frames])
                tail = torch.full((1,), self.N[d + 1], dtype=torch.int32, device="cuda")
                self.off[d] = torch.cat([f.off[d][:-1] + R[d + 1][i]
                                         for i, f in enumerate(frames)] + [tail])
                self.Y[d] = self.codes[d].long()
        self.nbr = _BatchMaps(frames, R)
        self.nbr[self.b], self.nbr[self.t]


# ------------------------------------------------------------------ model --

ACT_SCALE = 1.0 / 32.0


class QATModel(torch.nn.Module):
    """The float twin of the integer network with optional fake quantisation."""

    def __init__(self, params: dict, qat: bool = False, bf16: bool = False,
                 recompute: bool = False, arch: int = 0, t_off: int = 4):
        """arch, t_off: the architecture (0 GRED + XFP, 1 GRED only,
        2 baseline; Sec. 4.3) and t = L - t_off, as in the weight blob."""
        super().__init__()
        self.recompute = recompute
        self.arch, self.t_off = arch, t_off
        self.names = sorted(params)
        self.p = torch.nn.ParameterDict(
            {k.replace(".", "__"): torch.nn.Parameter(torch.tensor(v, device="cuda"))
             for k, v in params.items()})
        self.qat, self.bf16 = qat, int(bf16)

    def P(self, name):
        return self.p[name.replace(".", "__")]

    def w(self, name):
        return fq_w(self.P(name)) if self.qat else self.P(name)

    def q(self, x):
        return FakeQuantFn.apply(x, ACT_SCALE, 0) if self.qat else x

    def _pred_args(self, j):
        return (self.w(f"P1_{j}.W"), self.P(f"P1_{j}.b"), self.P(f"P1_{j}.a"),
                self.w(f"P2_{j}.W"), self.P(f"P2_{j}.b"))

    def bits(self, fr: Frame) -> torch.Tensor:
        """Rate of the five network levels in bits (cross-entropy / ln 2)."""
        def ce(j, F, d):
            return PredBitsFn.apply(F, *self._pred_args(j), fr.codes[d], self.qat, self.bf16)
        return self._levels(fr, ce, self.recompute)

    def level_logits(self, fr: Frame) -> dict:
        """The float network's logits [N_d, 255] of every network level d (the
        float inference variant)."""
        out = {}

        def keep(j, F, d):
            out[d] = pred_logits(F, *self._pred_args(j), self.qat, self.bf16)
            return F.new_zeros(())
        self._levels(fr, keep, False)
        return out

    def _levels(self, fr: Frame, head, recompute: bool) -> torch.Tensor:
        b, t, P, q, w, bf = fr.b, fr.t, self.P, self.q, self.w, self.bf16

        def prelu(x, name):
            return PReLUFn.apply(x, P(name))

        def upl(name, d, x):  # V_{d-1} -> V_d
            y = UpFn.apply(q(x), fr.par[d], fr.keys[d], fr.off[d - 1], w(name + ".W"),
                           P(name + ".b"), bf)
            return prelu(y, name + ".a")

        def conv(x, d, name):
            return ConvFn.apply(q(x), fr.nbr[d], w(name + ".W"), P(name + ".b"), bf)

        def resblock(j, d, x):
            y1 = prelu(conv(x, d, f"RA_{j}"), f"RA_{j}.a")
            y2 = conv(y1, d, f"RB_{j}")
            return prelu(P(f"RM_{j}.ma") * y1 + P(f"RM_{j}.mb") * y2, f"RM_{j}.a")

        def emb(name, d):
            return EmbedFn.apply(fr.codes[d], P(name))

        L, arch = fr.L, self.arch
        t = L - self.t_off

        def level0():
            Fb = upl("UP_0", b, emb("E_0", b - 1))
            return Fb, head(0, Fb, b)

        def shallow(j, Fp):  # with XFP, b < d <= t (Eq. 8-9)
            d = b + j
            S = resblock(j, d - 1, Fp)
            F = upl(f"UP_{j}", d, torch.cat([S, emb(f"E_{j}", d - 1)], 1))
            return F, head(j, F, d)

        def extracted(j, Ft):
            # features of Y_{d-1} re-densified to V_k; with XFP fused with
            # F^t (Eq. 10-11), otherwise alone (Eq. 4-6)
            d = b + j
            k0 = t if (arch == 0 or (arch == 1 and d > t)) else d - 1
            g = emb(f"G_{j}", d - 1)
            for i in range(1, d - k0):
                k = d - 1 - i
                name = f"D_{j}_{i}"
                g = DownFn.apply(q(g), fr.par[k + 1], fr.keys[k + 1], fr.off[k], w(name + ".W"),
                                 P(name + ".b"), bf)
                g = prelu(g, name + ".a")
            H = resblock(j, k0, torch.cat([Ft, g], 1) if arch == 0 else g)
            for k in range(d - k0):
                x = torch.cat([H, emb(f"E_{j}_{k}", k0 + k)], 1) if arch == 0 else H
                H = upl(f"UP_{j}_{k}", k0 + k + 1, x)
            return head(j, H, d)

        # with recompute, each relative level keeps only its outputs; its
        # activations are recomputed in the backward pass
        run = ((lambda f, *a: checkpoint(f, *a, use_reentrant=False)) if recompute
               else (lambda f, *a: f(*a)))
        F, bits = run(level0)
        for j in range(1, 5):
            if arch == 0 and b + j <= t:
                F, bj = run(lambda Fp, j=j: shallow(j, Fp), F)
            elif arch == 0:
                bj = run(lambda Ft, j=j: extracted(j, Ft), F)
            else:
                bj = run(lambda j=j: extracted(j, None))
            bits = bits + bj
        return bits

    def grads(self) -> dict:
        return {k: self.P(k).grad.detach().cpu().double().numpy() for k in self.names}


def train_step(model: QATModel, opt, frames: list) -> float:
    """One step on a batch of frames: bits per point of the batch, AdamW,
    gradient norm clipped at 1.0 (supplement, training settings).  Each
    element is a Frame or a BatchFrame (one forward and backward pass per
    element)."""
    opt.zero_grad(set_to_none=True)
    npts = sum(f.n for f in frames)
    total = None
    for f in frames:
        loss = model.bits(f) / npts
        loss.backward()
        total = loss.detach() if total is None else total + loss.detach()
    torch.nn.utils.clip_grad_norm_(model.parameters(), 1.0)
    opt.step()
    return float(total)  # the one host round trip of the step


def make_optimizer(model: QATModel):
    return torch.optim.AdamW(model.parameters(), lr=1e-4, weight_decay=1e-4)
