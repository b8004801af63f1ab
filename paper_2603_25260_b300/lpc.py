"""Python binding of the codec's C ABI (include/lpc.h, include/lpc_ops.h).

Argument marshalling only: device tensors are passed as raw pointers
(``tensor.data_ptr()``), every step runs inside ``liblpc.so``.  The binding
refuses to run without the compiled library; there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpc.so")

OK, INVALID_ARG, CAPACITY, HASH_FULL, CORRUPT_STREAM, WEIGHTS_MISMATCH, CUDA_ERROR, TIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "CAPACITY", -3: "HASH_FULL", -4: "CORRUPT_STREAM",
          -5: "WEIGHTS_MISMATCH", -6: "CUDA_ERROR", -7: "TIMEOUT"}


class LpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("L", C.c_int), ("C", C.c_int), ("b_off", C.c_int), ("t_off", C.c_int),
                ("max_points", C.c_int64), ("max_frames", C.c_int), ("chunk", C.c_int),
                ("host_threads", C.c_int), ("cuda_stream", C.c_uint64),
                ("max_batch_points", C.c_int64), ("host_coding", C.c_int)]


_lib = None
P, I64, SZ, I32 = C.c_void_p, C.c_int64, C.c_size_t, C.c_int


def lib():
    """Load liblpc.so (build it first with paper_2603_25260_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2603_25260_b300/build.py")
        L = C.CDLL(LIB_PATH)
        sig = {
            "codec_create": (I32, [C.POINTER(Config), P, SZ, C.POINTER(P)]),
            "codec_destroy": (None, [P]),
            "codec_set_tuning": (I32, [P, P]),
            "codec_tuning": (I32, [P, P, P]),
            "codec_last_error": (C.c_char_p, [P]),
            "encode_frame": (I32, [P, P, I64, P, SZ, C.POINTER(SZ)]),
            "decode_frame": (I32, [P, P, SZ, P, I64, C.POINTER(I64)]),
            "probs_level": (I32, [P, P, I64, I32, P, I64, C.POINTER(I64)]),
            "encode_batch": (I32, [P, I32, P, P, P, P, P, P]),
            "decode_batch": (I32, [P, I32, P, P, P, P, P]),
            "codec_last_stats": (I32, [P, P, P, P]),
            "codec_profile": (I32, [P, C.c_uint]),
            "codec_profile_read": (I32, [P, I32, P, P, P, P]),
            "codec_profile_staged": (I32, [P, I32, P]),
            "codec_profile_name": (C.c_char_p, [I32]),
            "lpc_kernel_launches": (I64, []),
            "codec_last_phases": (I32, [P, P, I32]),
            "lpc_build_levels": (I32, [P, I64, I32, P, P, P, I64, C.c_uint64]),
            "lpc_kernel_map": (I32, [P, I64, I32, P, I32, C.c_uint64]),
            "lpc_kernel_map_noalloc": (I32, [P, I64, I32, P, C.c_uint64]),
            "lpc_rc_encode_rows": (I32, [P, P, I64, P, C.c_size_t, P]),
            "lpc_rc_decode_rows": (I32, [P, I64, P, C.c_size_t, P]),
            "lpc_kernel_map_child": (I32, [P, P, I64, P, P, P, P, C.c_uint64]),
            "lpc_conv333": (I32, [P, I64, I32, P, I32, I32, P, P, P, I32, P, I32, I32, P,
                                  C.c_uint64]),
            "lpc_conv333_variant": (I32, [P, I64, I32, P, I32, I32, P, P, P, I32, P, I32, I32, P,
                                  I32, C.c_uint64]),
            "lpc_down_s2": (I32, [P, I64, P, I64, P, I32, I32, P, P, P, I32, P, I32, I32, P,
                                  C.c_uint64]),
            "lpc_up_prune": (I32, [P, P, I64, P, I64, P, I32, I32, P, P, P, I32, P, I32, I32, P,
                                   C.c_uint64]),
            "lpc_up_prune_variant": (I32, [P, P, I64, P, I64, P, I32, I32, P, P, P, I32, P, I32,
                                           I32, P, I32, C.c_uint64]),
            "lpc_softmax_cdf": (I32, [P, I64, P, P, C.c_uint64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), (t.device, t.dtype)
    return t


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def blob_t_off(blob: bytes) -> int:
    """The threshold offset (t = L - t_off) a weight blob's header names;
    0 there reads as 4."""
    v = int.from_bytes(bytes(blob[24:28]), "little") if len(blob) >= 28 else 0
    return v or 4


class Codec:
    """One codec instance on the current CUDA device and stream."""

    def __init__(self, blob: bytes, L: int, max_points: int, max_frames: int = 1,
                 chunk: int = 256, host_threads: int = 0, stream: int | None = None,
                 max_batch_points: int = 0, host_coding: bool = False):
        """blob: the integer weight blob; its header names the architecture
        (GRED + XFP or an ablation) and t = L - t_off, which the codec takes.
        chunk: nodes per range-coded substream of a network level.  The
        device decoder runs one warp per substream, so a level's decode
        latency is about chunk x ~170 ns, while each substream adds about two
        bytes (its length and the short flush); 256 costs ~0.1 bits per point
        over 1024 on a 64-beam frame.  host_coding: range-code the network levels on
        host threads (tables copied to the host) instead of on the device;
        same bitstream."""
        self._lib = lib()
        self.blob = bytes(blob)
        self.L = L
        self.max_points = max_points
        cfg = Config(L, 32, 5, blob_t_off(self.blob), max_points, max_frames, chunk,
                     host_threads,
                     _stream() if stream is None else stream, max_batch_points,
                     int(bool(host_coding)))
        h = P()
        st = self._lib.codec_create(C.byref(cfg), self.blob, len(self.blob), C.byref(h))
        if st != OK:
            raise LpcError(st, "codec_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.codec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != OK:
            raise LpcError(st, self._lib.codec_last_error(self._h).decode())

    def encode(self, xyz: torch.Tensor, cap: int | None = None) -> bytes:
        xyz = _dev(xyz, torch.int32)
        n = xyz.shape[0]
        cap = cap if cap is not None else 1024 + 8 * n * 8
        out = np.empty(max(cap, 1), dtype=np.uint8)
        ln = C.c_size_t()
        self._check(self._lib.encode_frame(self._h, xyz.data_ptr() if n else None, n,
                                           out.ctypes.data, cap, C.byref(ln)))
        return out[:ln.value].tobytes()

    def encode_into(self, xyz: torch.Tensor, out: np.ndarray) -> int:
        """Encode into a caller-owned host buffer; returns the length."""
        n = xyz.shape[0]
        ln = C.c_size_t()
        self._check(self._lib.encode_frame(self._h, xyz.data_ptr() if n else None, n,
                                           out.ctypes.data, out.nbytes, C.byref(ln)))
        return ln.value

    def decode(self, data, cap: int | None = None, out: torch.Tensor | None = None):
        """Decode one stream (bytes or a contiguous uint8 numpy array, read in
        place) into device voxels [n, 3] int32 (out: optional caller buffer)."""
        cap = cap if cap is not None else self.max_points
        if out is None:
            out = torch.empty((max(cap, 1), 3), dtype=torch.int32, device="cuda")
        nn = C.c_int64()
        buf = np.frombuffer(data, dtype=np.uint8) if len(data) else np.zeros(1, np.uint8)
        self._check(self._lib.decode_frame(self._h, buf.ctypes.data, len(data), out.data_ptr(),
                                           cap, C.byref(nn)))
        return out[:nn.value]

    def probs_level(self, xyz: torch.Tensor, d: int) -> torch.Tensor:
        """CDF table [N_d, 256] of level d as int16 (reinterpret as uint16)."""
        xyz = _dev(xyz, torch.int32)
        n = xyz.shape[0]
        cap = max(n, 1)
        out = torch.empty((cap, 256), dtype=torch.int16, device="cuda")
        nn = C.c_int64()
        self._check(self._lib.probs_level(self._h, xyz.data_ptr() if n else None, n, d,
                                          out.data_ptr(), cap, C.byref(nn)))
        return out[:nn.value]

    def encode_batch(self, frames: list[torch.Tensor], Ls: list[int]) -> list[bytes]:
        nf = len(frames)
        ptrs = (C.c_void_p * nf)(*[f.data_ptr() if f.shape[0] else 0 for f in frames])
        ns = (C.c_int64 * nf)(*[f.shape[0] for f in frames])
        ls = (C.c_int * nf)(*Ls)
        caps = [1024 + 64 * f.shape[0] for f in frames]
        bufs = [np.empty(c, dtype=np.uint8) for c in caps]
        outs = (C.c_void_p * nf)(*[b.ctypes.data for b in bufs])
        capa = (C.c_size_t * nf)(*caps)
        lens = (C.c_size_t * nf)()
        self._check(self._lib.encode_batch(self._h, nf, ptrs, ns, ls, outs, capa, lens))
        return [bufs[i][:lens[i]].tobytes() for i in range(nf)]

    @staticmethod
    def batch_caps(frames: list[torch.Tensor]) -> list[int]:
        """Output bytes reserved per frame by encode_batch_into."""
        return [1024 + 64 * f.shape[0] for f in frames]

    def encode_batch_into(self, frames: list[torch.Tensor], Ls: list[int],
                          out: np.ndarray) -> list[tuple[int, int]]:
        """Encode a batch into one caller-owned uint8 buffer (reusable across
        calls, at least sum(batch_caps(frames)) bytes); frame i goes to its
        own slice.  Returns (offset, length) per frame."""
        nf = len(frames)
        caps = self.batch_caps(frames)
        offs = np.concatenate([[0], np.cumsum(caps)[:-1]]).astype(np.int64)
        assert out.dtype == np.uint8 and out.size >= sum(caps)
        base = out.ctypes.data
        ptrs = (C.c_void_p * nf)(*[f.data_ptr() if f.shape[0] else 0 for f in frames])
        ns = (C.c_int64 * nf)(*[f.shape[0] for f in frames])
        ls = (C.c_int * nf)(*Ls)
        outs = (C.c_void_p * nf)(*[base + int(o) for o in offs])
        capa = (C.c_size_t * nf)(*caps)
        lens = (C.c_size_t * nf)()
        self._check(self._lib.encode_batch(self._h, nf, ptrs, ns, ls, outs, capa, lens))
        return [(int(offs[i]), int(lens[i])) for i in range(nf)]

    def decode_batch_from(self, buf: np.ndarray, spans: list[tuple[int, int]],
                          outs_t: list[torch.Tensor]) -> list[torch.Tensor]:
        """Decode streams lying in one host buffer (as encode_batch_into left
        them) into caller-owned device tensors [cap_i, 3] int32."""
        nf = len(spans)
        base = buf.ctypes.data
        ins = (C.c_void_p * nf)(*[base + o for o, _ in spans])
        lens = (C.c_size_t * nf)(*[n for _, n in spans])
        outs = (C.c_void_p * nf)(*[t.data_ptr() for t in outs_t])
        capa = (C.c_int64 * nf)(*[t.shape[0] for t in outs_t])
        nout = (C.c_int64 * nf)()
        self._check(self._lib.decode_batch(self._h, nf, ins, lens, outs, capa, nout))
        return [outs_t[i][:nout[i]] for i in range(nf)]

    def decode_batch(self, streams: list[bytes], caps: list[int]) -> list[torch.Tensor]:
        nf = len(streams)
        bufs = [np.frombuffer(s, dtype=np.uint8) for s in streams]
        ins = (C.c_void_p * nf)(*[b.ctypes.data for b in bufs])
        lens = (C.c_size_t * nf)(*[len(s) for s in streams])
        outs_t = [torch.empty((max(c, 1), 3), dtype=torch.int32, device="cuda") for c in caps]
        outs = (C.c_void_p * nf)(*[t.data_ptr() for t in outs_t])
        capa = (C.c_int64 * nf)(*caps)
        nout = (C.c_int64 * nf)()
        self._check(self._lib.decode_batch(self._h, nf, ins, lens, outs, capa, nout))
        return [outs_t[i][:nout[i]] for i in range(nf)]

    FAMILIES = ("sort", "levels", "hash_kmap", "embed", "up_prune", "down_s2", "conv333",
                "predictor_cdf", "range_coder")

    def profile(self, mask: int):
        """Time every launch of the kernel families in `mask` (bit i = FAMILIES[i])
        with CUDA events on the codec's stream; resets the counters."""
        self._check(self._lib.codec_profile(self._h, mask))

    def profile_read(self) -> dict:
        out = {}
        for i, name in enumerate(self.FAMILIES):
            ms, b, o = C.c_double(), C.c_double(), C.c_double()
            n = C.c_int64()
            self._check(self._lib.codec_profile_read(self._h, i, C.byref(ms), C.byref(n),
                                                     C.byref(b), C.byref(o)))
            sb = C.c_double()
            self._check(self._lib.codec_profile_staged(self._h, i, C.byref(sb)))
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": b.value, "ops": o.value,
                         "staged_bytes": sb.value}
        return out

    def tuning(self) -> dict:
        """The conv autotuner's choice per input width and the timed variants
        (milliseconds; bit 0 of a variant = alternative ring shape, bit 1 =
        contiguous tile order, bit 2 = TMA gather4 loads of the neighbour rows
        instead of cp.async copies; 8, 9 = 256-row tiles, strided or
        contiguous)."""
        v = (C.c_int * 5)()
        ms = (C.c_float * 26)()
        self._check(self._lib.codec_tuning(self._h, v, ms))
        return {"conv32": v[0], "conv64": v[1], "predictor": v[2], "up32": v[3], "up64": v[4],
                "ms32": [round(x, 4) for x in ms[:10]], "ms64": [round(x, 4) for x in ms[10:20]],
                "ms_pred": [round(x, 4) for x in ms[20:22]],
                "ms_up32": [round(x, 4) for x in ms[22:24]],
                "ms_up64": [round(x, 4) for x in ms[24:26]]}

    def set_tuning(self, conv32: int = -1, conv64: int = -1, predictor: int = -1, up32: int = -1,
                   up64: int = -1):
        """Fix kernel variants instead of autotuning them (-1: tune)."""
        v = (C.c_int * 5)(conv32, conv64, predictor, up32, up64)
        self._check(self._lib.codec_set_tuning(self._h, v))

    def last_phases(self) -> list[float]:
        """Host timeline of the last encode / decode in microseconds (see lpc.h)."""
        us = (C.c_double * 16)()
        self._check(self._lib.codec_last_phases(self._h, us, 16))
        return list(us)

    def last_stats(self):
        counts = (C.c_int64 * 32)()
        g, h = C.c_double(), C.c_double()
        L = self._lib.codec_last_stats(self._h, counts, C.byref(g), C.byref(h))
        return [counts[d] for d in range(L + 1)], g.value, h.value


def kernel_launches() -> int:
    """CUDA kernels launched by liblpc.so in this process so far."""
    return int(lib().lpc_kernel_launches())


# ------------------------------------------------------------------- ops --

def _ops_check(st: int, what: str):
    if st != OK:
        raise LpcError(st, what)


def build_levels(xyz: torch.Tensor, L: int):
    """(keys per depth 0..L, codes per depth 0..L-1) as device tensors."""
    xyz = _dev(xyz, torch.int32)
    n = xyz.shape[0]
    cap = max(1, n) * (L + 1)
    keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    codes = torch.empty(cap, dtype=torch.uint8, device="cuda")
    counts = np.zeros(L + 1, dtype=np.int64)
    _ops_check(lib().lpc_build_levels(xyz.data_ptr() if n else None, n, L, keys.data_ptr(),
                                      codes.data_ptr(), counts.ctypes.data, cap, _stream()),
               "lpc_build_levels")
    ks, cs, kp, cp = [], [], 0, 0
    for d in range(L + 1):
        N = int(counts[d])
        ks.append(keys[kp:kp + N])
        kp += N
        if d < L:
            cs.append(codes[cp:cp + N])
            cp += N
    return ks, cs


def kernel_map(keys: torch.Tensor, depth: int, table_log2: int = 0) -> torch.Tensor:
    keys = _dev(keys, torch.int64)
    N = keys.shape[0]
    nbr = torch.empty((max(N, 1), 27), dtype=torch.int32, device="cuda")
    _ops_check(lib().lpc_kernel_map(keys.data_ptr() if N else None, N, depth, nbr.data_ptr(),
                                    table_log2, _stream()), "lpc_kernel_map")
    return nbr[:N]


def kernel_map_child(ckeys, cpar, pnbr, pcode, poff) -> torch.Tensor:
    """Kernel map of a level from its parent level's map (no hash table)."""
    ckeys, cpar = _dev(ckeys, torch.int64), _dev(cpar, torch.int32)
    pnbr, pcode, poff = _dev(pnbr, torch.int32), _dev(pcode, torch.uint8), _dev(poff, torch.int32)
    N = ckeys.shape[0]
    nbr = torch.empty((max(N, 1), 27), dtype=torch.int32, device="cuda")
    _ops_check(lib().lpc_kernel_map_child(ckeys.data_ptr() if N else None,
                                          cpar.data_ptr() if N else None, N, pnbr.data_ptr(),
                                          pcode.data_ptr(), poff.data_ptr(), nbr.data_ptr(),
                                          _stream()), "lpc_kernel_map_child")
    return nbr[:N]


NOALLOC_MAX_NODES = 1 << 18


def kernel_map_noalloc(keys: torch.Tensor, depth: int, out: torch.Tensor) -> torch.Tensor:
    """Kernel map through the entry point that allocates no device memory.

    For callers that must not allocate at this point (memory fixed at start-up,
    allocator owned by another component).  `out` is the caller's int32
    [N, 27] device buffer; the library's static table limits N to
    NOALLOC_MAX_NODES.  Calls share that table, so do not overlap them on the
    GPU."""
    keys = _dev(keys, torch.int64)
    out = _dev(out, torch.int32)
    N = keys.shape[0]
    assert out.shape[0] >= N and out.shape[1] == 27
    st = lib().lpc_kernel_map_noalloc(keys.data_ptr() if N else None, N, depth,
                                      out.data_ptr() if N else None, _stream())
    if st == CAPACITY:
        raise LpcError(st, f"lpc_kernel_map_noalloc: {N} nodes exceed the static table "
                           f"limit of {NOALLOC_MAX_NODES}")
    _ops_check(st, "lpc_kernel_map_noalloc")
    return out[:N]


def rc_encode_rows(rows: np.ndarray, syms: np.ndarray) -> bytes:
    """Range code symbols 0..254 with host table rows u16 [n, 256] (one
    substream, the codec's host coder)."""
    rows = np.ascontiguousarray(rows, dtype=np.uint16)
    syms = np.ascontiguousarray(syms, dtype=np.uint8)
    n = syms.shape[0]
    assert rows.shape == (n, 256)
    out = np.empty(2 * n + 16, dtype=np.uint8)
    ln = C.c_size_t()
    _ops_check(lib().lpc_rc_encode_rows(rows.ctypes.data, syms.ctypes.data, n, out.ctypes.data,
                                        out.shape[0], C.byref(ln)), "lpc_rc_encode_rows")
    return out[:ln.value].tobytes()


def rc_decode_rows(rows: np.ndarray, data: bytes) -> tuple[int, np.ndarray]:
    """Decode one substream with host table rows u16 [n, 256]: (status, the
    n symbols).  A stream inconsistent with the rows gives CORRUPT_STREAM
    (and whatever symbols the decoder produced), not an exception."""
    rows = np.ascontiguousarray(rows, dtype=np.uint16)
    n = rows.shape[0]
    syms = np.zeros(n, dtype=np.uint8)
    buf = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)
    st = lib().lpc_rc_decode_rows(rows.ctypes.data, n, buf.ctypes.data, len(data),
                                  syms.ctypes.data)
    if st not in (OK, CORRUPT_STREAM):
        _ops_check(st, "lpc_rc_decode_rows")
    return st, syms


def conv333(keys, depth, x, z_in, W, bias, mult, shift, slope, z_out, variant=None):
    keys, x = _dev(keys, torch.int64), _dev(x, torch.int8)
    N, cin = x.shape
    W = _np(W, np.int8)
    cout = W.shape[1]
    out = torch.empty((max(N, 1), cout), dtype=torch.int8, device="cuda")
    b, m = _np(bias, np.int32), _np(mult, np.int32)
    s = None if slope is None else _np(slope, np.int16)
    if variant is None:
        _ops_check(lib().lpc_conv333(keys.data_ptr(), N, depth, x.data_ptr(), cin, z_in, _hp(W),
                                     _hp(b), _hp(m), shift, _hp(s), z_out, cout, out.data_ptr(),
                                     _stream()), "lpc_conv333")
    else:
        _ops_check(lib().lpc_conv333_variant(keys.data_ptr(), N, depth, x.data_ptr(), cin, z_in,
                                             _hp(W), _hp(b), _hp(m), shift, _hp(s), z_out, cout,
                                             out.data_ptr(), variant, _stream()),
                   "lpc_conv333_variant")
    return out[:N]


def down_s2(ckeys, pkeys, x, z_in, W, bias, mult, shift, slope, z_out):
    ckeys, pkeys, x = _dev(ckeys, torch.int64), _dev(pkeys, torch.int64), _dev(x, torch.int8)
    W = _np(W, np.int8)
    cout = W.shape[1]
    Np = pkeys.shape[0]
    out = torch.empty((max(Np, 1), cout), dtype=torch.int8, device="cuda")
    b, m = _np(bias, np.int32), _np(mult, np.int32)
    s = None if slope is None else _np(slope, np.int16)
    _ops_check(lib().lpc_down_s2(ckeys.data_ptr(), ckeys.shape[0], pkeys.data_ptr(), Np,
                                 x.data_ptr(), x.shape[1], z_in, _hp(W), _hp(b), _hp(m), shift,
                                 _hp(s), z_out, cout, out.data_ptr(), _stream()), "lpc_down_s2")
    return out[:Np]


def up_prune(pkeys, codes, ckeys, x, z_in, W, bias, mult, shift, slope, z_out, variant=0):
    pkeys, ckeys = _dev(pkeys, torch.int64), _dev(ckeys, torch.int64)
    codes, x = _dev(codes, torch.uint8), _dev(x, torch.int8)
    W = _np(W, np.int8)
    cout = W.shape[1]
    Nc = ckeys.shape[0]
    out = torch.empty((max(Nc, 1), cout), dtype=torch.int8, device="cuda")
    b, m = _np(bias, np.int32), _np(mult, np.int32)
    s = None if slope is None else _np(slope, np.int16)
    _ops_check(lib().lpc_up_prune_variant(pkeys.data_ptr(), codes.data_ptr(), pkeys.shape[0],
                                          ckeys.data_ptr(), Nc, x.data_ptr(), x.shape[1], z_in,
                                          _hp(W), _hp(b), _hp(m), shift, _hp(s), z_out, cout,
                                          out.data_ptr(), variant, _stream()),
               "lpc_up_prune_variant")
    return out[:Nc]


def softmax_cdf(logits: torch.Tensor, lut: np.ndarray) -> torch.Tensor:
    logits = _dev(logits, torch.int8)
    N = logits.shape[0]
    out = torch.empty((max(N, 1), 256), dtype=torch.int16, device="cuda")
    lut = _np(lut, np.uint32)
    _ops_check(lib().lpc_softmax_cdf(logits.data_ptr(), N, _hp(lut), out.data_ptr(), _stream()),
               "lpc_softmax_cdf")
    return out[:N]


def u16(t: torch.Tensor) -> np.ndarray:
    """int16 device tensor -> uint16 numpy array (bit reinterpretation)."""
    return t.cpu().numpy().view(np.uint16)
