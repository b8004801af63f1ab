"""ctypes wrapper of the C oracle (lpc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports
this package.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpc_oracle.c")
_LIB = os.path.join(_HERE, "liblpc_oracle.so")

STATUS = {0: "OK", -1: "INVALID_ARG", -2: "CAPACITY", -4: "CORRUPT_STREAM", -5: "WEIGHTS_MISMATCH"}


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP for the per-node loops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lpc_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


P = C.c_void_p
I64 = C.c_int64
SZ = C.c_size_t


def _declare(L):
    sig = {
        "or_set_threads": (None, [C.c_int]),
        "or_get_threads": (C.c_int, []),
        "or_last_phase_times": (None, [P, P]),
        "or_requant": (C.c_int, [I64, C.c_int32, C.c_int, C.c_int]),
        "or_prelu": (I64, [I64, C.c_int]),
        "or_morton": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]),
        "or_leaf_keys": (C.c_int, [P, I64, C.c_int, P, P]),
        "or_build_levels": (C.c_int, [P, I64, C.c_int, P, P, P, I64]),
        "or_conv333": (C.c_int, [P, I64, C.c_int, P, C.c_int, C.c_int, P, P, P, C.c_int, P,
                                 C.c_int, C.c_int, P]),
        "or_down_s2": (C.c_int, [P, I64, P, I64, P, C.c_int, C.c_int, P, P, P, C.c_int, P,
                                 C.c_int, C.c_int, P]),
        "or_up_prune": (C.c_int, [P, P, I64, P, I64, P, C.c_int, C.c_int, P, P, P, C.c_int, P,
                                  C.c_int, C.c_int, P]),
        "or_softmax_cdf": (C.c_int, [P, I64, P, P]),
        "or_rc_encode_cdf": (C.c_int, [P, P, I64, P, SZ, P]),
        "or_rc_decode_cdf": (C.c_int, [P, I64, P, SZ, P]),
        "or_rc_encode_adaptive": (C.c_int, [P, I64, P, SZ, P]),
        "or_rc_decode_adaptive": (C.c_int, [I64, P, SZ, P]),
        "or_fnv1a64": (C.c_uint64, [P, SZ]),
        "or_check_blob": (C.c_int, [P, SZ]),
        "or_probs_level": (C.c_int, [P, SZ, P, I64, C.c_int, C.c_int, P, I64, P]),
        "or_logits_level": (C.c_int, [P, SZ, P, I64, C.c_int, C.c_int, P, I64, P]),
        "or_encode": (C.c_int, [P, SZ, P, I64, C.c_int, C.c_int, P, SZ, P]),
        "or_decode": (C.c_int, [P, SZ, P, SZ, P, I64, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(st, what)


def _buf(b: bytes):
    return C.c_char_p(b), len(b)


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def last_phase_times() -> tuple[float, float]:
    """(network + softmax seconds, range-coding seconds) of the calling
    thread's last encode or decode."""
    a, b = C.c_double(), C.c_double()
    lib().or_last_phase_times(C.byref(a), C.byref(b))
    return a.value, b.value


def requant(acc: int, m: int, r: int, z: int) -> int:
    return lib().or_requant(int(acc), int(m), int(r), int(z))


def prelu(acc: int, a: int) -> int:
    return lib().or_prelu(int(acc), int(a))


def morton(x: int, y: int, z: int, bits: int) -> int:
    return lib().or_morton(x, y, z, bits)


def leaf_keys(xyz: np.ndarray, L: int) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    n = xyz.shape[0]
    out = np.zeros(max(n, 1), dtype=np.uint64)
    nn = C.c_int64()
    _check(lib().or_leaf_keys(_p(xyz), n, L, _p(out), C.byref(nn)), "leaf_keys")
    return out[:nn.value].copy()


def build_levels(xyz: np.ndarray, L: int):
    """Returns (keys per depth 0..L, codes per depth 0..L-1)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    n = xyz.shape[0]
    cap = max(1, n) * (L + 1)
    counts = np.zeros(L + 1, dtype=np.int64)
    keys = np.zeros(cap, dtype=np.uint64)
    codes = np.zeros(cap, dtype=np.uint8)
    _check(lib().or_build_levels(_p(xyz), n, L, _p(counts), _p(keys), _p(codes), cap), "levels")
    ks, cs, kp, cp = [], [], 0, 0
    for d in range(L + 1):
        N = int(counts[d])
        ks.append(keys[kp:kp + N].copy())
        kp += N
        if d < L:
            cs.append(codes[cp:cp + N].copy())
            cp += N
    return ks, cs


def conv333(keys, depth, x, z_in, W, bias, mult, shift, slope, z_out):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.int8)
    W = np.ascontiguousarray(W, dtype=np.int8)
    N, cin = x.shape
    cout = W.shape[1]
    out = np.zeros((max(N, 1), cout), dtype=np.int8)
    sl = None if slope is None else np.ascontiguousarray(slope, dtype=np.int16)
    _check(lib().or_conv333(_p(keys), N, depth, _p(x), cin, z_in, _p(W),
                            _p(np.ascontiguousarray(bias, dtype=np.int32)),
                            _p(np.ascontiguousarray(mult, dtype=np.int32)), shift, _p(sl), z_out,
                            cout, _p(out)), "conv333")
    return out[:N]


def down_s2(ckeys, pkeys, x, z_in, W, bias, mult, shift, slope, z_out):
    ckeys = np.ascontiguousarray(ckeys, dtype=np.uint64)
    pkeys = np.ascontiguousarray(pkeys, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.int8)
    W = np.ascontiguousarray(W, dtype=np.int8)
    cin = x.shape[1]
    cout = W.shape[1]
    Np = pkeys.shape[0]
    out = np.zeros((max(Np, 1), cout), dtype=np.int8)
    sl = None if slope is None else np.ascontiguousarray(slope, dtype=np.int16)
    _check(lib().or_down_s2(_p(ckeys), ckeys.shape[0], _p(pkeys), Np, _p(x), cin, z_in, _p(W),
                            _p(np.ascontiguousarray(bias, dtype=np.int32)),
                            _p(np.ascontiguousarray(mult, dtype=np.int32)), shift, _p(sl), z_out,
                            cout, _p(out)), "down_s2")
    return out[:Np]


def up_prune(pkeys, codes, ckeys, x, z_in, W, bias, mult, shift, slope, z_out):
    pkeys = np.ascontiguousarray(pkeys, dtype=np.uint64)
    ckeys = np.ascontiguousarray(ckeys, dtype=np.uint64)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.int8)
    W = np.ascontiguousarray(W, dtype=np.int8)
    cin = x.shape[1]
    cout = W.shape[1]
    Nc = ckeys.shape[0]
    out = np.zeros((max(Nc, 1), cout), dtype=np.int8)
    sl = None if slope is None else np.ascontiguousarray(slope, dtype=np.int16)
    _check(lib().or_up_prune(_p(pkeys), _p(codes), pkeys.shape[0], _p(ckeys), Nc, _p(x), cin,
                             z_in, _p(W), _p(np.ascontiguousarray(bias, dtype=np.int32)),
                             _p(np.ascontiguousarray(mult, dtype=np.int32)), shift, _p(sl), z_out,
                             cout, _p(out)), "up_prune")
    return out[:Nc]


def softmax_cdf(logits: np.ndarray, lut: np.ndarray) -> np.ndarray:
    logits = np.ascontiguousarray(logits, dtype=np.int8)
    N = logits.shape[0]
    out = np.zeros((max(N, 1), 256), dtype=np.uint16)
    _check(lib().or_softmax_cdf(_p(logits), N, _p(np.ascontiguousarray(lut, dtype=np.uint32)),
                                _p(out)), "softmax_cdf")
    return out[:N]


def rc_encode_cdf(cdf: np.ndarray, syms: np.ndarray) -> bytes:
    cdf = np.ascontiguousarray(cdf, dtype=np.uint16)
    syms = np.ascontiguousarray(syms, dtype=np.uint8)
    cap = syms.shape[0] * 4 + 64
    out = np.zeros(cap, dtype=np.uint8)
    ln = C.c_size_t()
    _check(lib().or_rc_encode_cdf(_p(cdf), _p(syms), syms.shape[0], _p(out), cap, C.byref(ln)),
           "rc_encode_cdf")
    return out[:ln.value].tobytes()


def rc_decode_cdf(cdf: np.ndarray, data: bytes) -> np.ndarray:
    cdf = np.ascontiguousarray(cdf, dtype=np.uint16)
    n = cdf.shape[0]
    syms = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib().or_rc_decode_cdf(_p(cdf), n, data, len(data), _p(syms)), "rc_decode_cdf")
    return syms[:n]


def rc_encode_adaptive(syms: np.ndarray) -> bytes:
    syms = np.ascontiguousarray(syms, dtype=np.uint8)
    cap = syms.shape[0] * 4 + 64
    out = np.zeros(cap, dtype=np.uint8)
    ln = C.c_size_t()
    _check(lib().or_rc_encode_adaptive(_p(syms), syms.shape[0], _p(out), cap, C.byref(ln)),
           "rc_encode_adaptive")
    return out[:ln.value].tobytes()


def rc_decode_adaptive(n: int, data: bytes) -> np.ndarray:
    syms = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib().or_rc_decode_adaptive(n, data, len(data), _p(syms)), "rc_decode_adaptive")
    return syms[:n]


def fnv1a64(data: bytes) -> int:
    return lib().or_fnv1a64(data, len(data))


def check_blob(blob: bytes) -> int:
    return lib().or_check_blob(blob, len(blob))


def _level_call(fn, blob, xyz, L, d, width, dtype, what):
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    cap = max(1, xyz.shape[0])
    out = np.zeros((cap, width), dtype=dtype)
    nn = C.c_int64()
    _check(fn(blob, len(blob), _p(xyz), xyz.shape[0], L, d, _p(out), cap, C.byref(nn)), what)
    return out[:nn.value]


def probs_level(blob: bytes, xyz: np.ndarray, L: int, d: int) -> np.ndarray:
    """CDF table [N_d, 256] u16 of level d."""
    return _level_call(lib().or_probs_level, blob, xyz, L, d, 256, np.uint16, "probs_level")


def logits_level(blob: bytes, xyz: np.ndarray, L: int, d: int) -> np.ndarray:
    return _level_call(lib().or_logits_level, blob, xyz, L, d, 255, np.int8, "logits_level")


def encode(blob: bytes, xyz: np.ndarray, L: int, chunk: int = 256) -> bytes:
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    # coded bytes: at most 2 per symbol, plus flush bytes and a length varint
    # per substream (one substream per chunk of every network level and per
    # 4096 nodes of every coarse level) and the coarse levels' sizes
    n = xyz.shape[0]
    cap = 64 + n * 4 * 4 + 4096 + 16 * (5 * (n // chunk + 1) + L) + 16 * L * (n // 4096 + 3)
    out = np.zeros(cap, dtype=np.uint8)
    ln = C.c_size_t()
    _check(lib().or_encode(blob, len(blob), _p(xyz), xyz.shape[0], L, chunk, _p(out), cap,
                           C.byref(ln)), "encode")
    return out[:ln.value].tobytes()


def decode(blob: bytes, data: bytes, cap: int) -> np.ndarray:
    out = np.zeros((max(cap, 1), 3), dtype=np.int32)
    nn = C.c_int64()
    _check(lib().or_decode(blob, len(blob), data, len(data), _p(out), cap, C.byref(nn)), "decode")
    return out[:nn.value]
