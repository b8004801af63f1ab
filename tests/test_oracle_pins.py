"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own code: exact rational
arithmetic for the fixed-point rounding (Eq. 14), set-based octrees and the
kernel-2 stride-2 convolution identity for the level build (supplement,
"Implementation of Octree Operations"), dense integer 3D convolutions for the
sparse layers (Eq. 13 with zero padding), closed forms and error bounds for
the integer softmax (Eq. 15), and round trips plus the ideal code length for
the entropy coder.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2603_25260_b300 import synth

RNG = np.random.Generator(np.random.PCG64(12345))


# --------------------------------------------------------------------------
# Fixed-point requantisation and PReLU (Eq. 14, round half up, clip)
# --------------------------------------------------------------------------

def _round_half_up(fr: Fraction) -> int:
    return math.floor(fr + Fraction(1, 2))


def test_requant_matches_exact_rounding():
    cases = [(0, 1, 1, 0), (1, 1, 1, 0), (-1, 1, 1, 0), (3, 1, 1, 0), (-3, 1, 1, 0),
             (5, 3, 4, 7), (-5, 3, 4, -7), ((1 << 31) - 1, (1 << 31) - 1, 62, 0),
             (-(1 << 31), (1 << 31) - 1, 62, 0), (123456, 9999, 24, -3)]
    for _ in range(4000):
        acc = int(RNG.integers(-(1 << 31), 1 << 31))
        m = int(RNG.integers(0, 1 << 31))
        r = int(RNG.integers(1, 63))
        z = int(RNG.integers(-128, 128))
        cases.append((acc, m, r, z))
    for _ in range(2000):  # unclipped region, where rounding is visible
        r = int(RNG.integers(1, 30))
        m = int(RNG.integers(1, 1 << 12))
        acc = int(RNG.integers(-(1 << 20), 1 << 20))
        cases.append((acc, m, r, int(RNG.integers(-20, 21))))
    for acc, m, r, z in cases:
        q = O.requant(acc, m, r, z)
        exact = Fraction(acc * m, 1 << r)
        want = min(127, max(-128, _round_half_up(exact) + z))
        assert q == want, (acc, m, r, z, q, want)
        if -128 < q < 127:
            assert abs(Fraction(q - z) - exact) <= Fraction(1, 2)


def test_requant_ties_round_up():
    # acc * m / 2^r = k + 1/2 exactly -> k + 1 (towards +inf), for both signs
    for k in range(-40, 40):
        acc = 2 * k + 1
        assert O.requant(acc, 1, 1, 0) == k + 1


def test_prelu_exact():
    for _ in range(3000):
        acc = int(RNG.integers(-(1 << 31), 1 << 31))
        a = int(RNG.integers(-32768, 32768))
        got = O.prelu(acc, a)
        if acc >= 0:
            assert got == acc
        else:
            assert got == _round_half_up(Fraction(acc * a, 1 << 15))


# --------------------------------------------------------------------------
# Morton keys and octree levels
# --------------------------------------------------------------------------

def _interleave_by_string(x, y, z, bits):
    sx, sy, sz = (format(v, f"0{bits}b") for v in (x, y, z))
    return int("".join(a + b + c for a, b, c in zip(sx, sy, sz)), 2) if bits else 0


def test_morton_bit_layout():
    for _ in range(500):
        bits = int(RNG.integers(1, 22))
        x, y, z = (int(v) for v in RNG.integers(0, 1 << bits, size=3))
        k = O.morton(x, y, z, bits)
        assert k == _interleave_by_string(x, y, z, bits)
        # parent = floor-halved coordinates, child index = 4 xbit + 2 ybit + zbit
        if bits > 1:
            assert k >> 3 == O.morton(x >> 1, y >> 1, z >> 1, bits - 1)
        assert k & 7 == 4 * (x & 1) + 2 * (y & 1) + (z & 1)


def _set_octree(xyz, L):
    pts = {tuple(p) for p in xyz.tolist()}
    levels = []
    for d in range(L + 1):
        s = L - d
        levels.append({(x >> s, y >> s, z >> s) for (x, y, z) in pts})
    return levels


@pytest.mark.parametrize("n,L,seed", [(1, 6, 1), (7, 6, 2), (300, 7, 3), (2000, 10, 4),
                                      (500, 21, 5)])
def test_levels_match_set_octree(n, L, seed):
    xyz = synth.random_cloud(n, L, seed)
    xyz = np.concatenate([xyz, xyz[: n // 3]])  # duplicates collapse
    keys, codes = O.build_levels(xyz, L)
    ref = _set_octree(xyz, L)
    for d in range(L + 1):
        want = sorted(_interleave_by_string(x, y, z, d) for (x, y, z) in ref[d])
        assert keys[d].tolist() == want
        if d < L:
            child = ref[d + 1]
            # code bit c set <=> child (2x + cx, 2y + cy, 2z + cz) exists, c = 4cx + 2cy + cz
            for k, code in zip(keys[d].tolist(), codes[d].tolist()):
                x = y = z = 0
                for i in range(d):
                    x |= ((k >> (3 * i + 2)) & 1) << i
                    y |= ((k >> (3 * i + 1)) & 1) << i
                    z |= ((k >> (3 * i)) & 1) << i
                bits = 0
                for c in range(8):
                    if (2 * x + (c >> 2), 2 * y + ((c >> 1) & 1), 2 * z + (c & 1)) in child:
                        bits |= 1 << c
                assert code == bits
                assert 1 <= code <= 255
            assert sum(bin(c).count("1") for c in codes[d].tolist()) == len(keys[d + 1])


def test_code_is_stride2_conv_of_ones():
    """The occupancy code equals a kernel-2 stride-2 convolution with fixed
    weights over an all-ones input (supplement, Occupancy Code Generation)."""
    L = 5
    xyz = synth.random_cloud(3000, L, 9, clustered=False)
    keys, codes = O.build_levels(xyz, L)
    for d in range(L):
        s = L - (d + 1)
        side = 1 << (d + 1)
        occ = np.zeros((side, side, side), dtype=np.int64)
        occ[xyz[:, 0] >> s, xyz[:, 1] >> s, xyz[:, 2] >> s] = 1
        w = np.zeros((2, 2, 2), dtype=np.int64)
        for c in range(8):
            w[c >> 2, (c >> 1) & 1, c & 1] = 1 << c
        blocks = occ.reshape(side // 2, 2, side // 2, 2, side // 2, 2)
        conv = np.einsum("aibjck,ijk->abc", blocks, w)
        parents = np.argwhere(conv > 0)
        want = sorted((_interleave_by_string(int(a), int(b), int(c), d), int(conv[a, b, c]))
                      for a, b, c in parents)
        got = list(zip(keys[d].tolist(), codes[d].tolist()))
        assert got == want


def test_leaf_keys_reject_out_of_range():
    with pytest.raises(O.OracleError):
        O.leaf_keys(np.array([[0, 0, 64]], dtype=np.int32), 6)
    with pytest.raises(O.OracleError):
        O.leaf_keys(np.array([[0, -1, 0]], dtype=np.int32), 6)


# --------------------------------------------------------------------------
# Sparse layers vs dense integer convolutions (Eq. 13 with zero padding)
# --------------------------------------------------------------------------

def _coords(keys, depth):
    out = np.zeros((len(keys), 3), dtype=np.int64)
    for n, k in enumerate(keys.tolist()):
        x = y = z = 0
        for i in range(depth):
            x |= ((k >> (3 * i + 2)) & 1) << i
            y |= ((k >> (3 * i + 1)) & 1) << i
            z |= ((k >> (3 * i)) & 1) << i
        out[n] = (x, y, z)
    return out


def _finish(acc, mult, shift, slope, z_out):
    out = np.zeros(acc.shape, dtype=np.int64)
    for idx, a in np.ndenumerate(acc):
        a = int(a)
        c = idx[-1]
        if slope is not None and a < 0:
            a = _round_half_up(Fraction(a * int(slope[c]), 1 << 15))
        out[idx] = min(127, max(-128, _round_half_up(Fraction(a * int(mult[c]), 1 << shift))
                                + z_out))
    return out


def _layer_params(S, cin, cout, seed, per_slice=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.integers(-127, 128, size=(S, cout, cin)).astype(np.int8)
    shape = (S, cout) if per_slice else (cout,)
    bias = rng.integers(-50000, 50000, size=shape).astype(np.int32)
    mult = rng.integers(1, 1 << 14, size=shape).astype(np.int32)
    slope = rng.integers(-32768, 32768, size=shape).astype(np.int16)
    return W, bias, mult, slope


@pytest.mark.parametrize("depth,n,cin,cout,seed", [(3, 200, 16, 8, 1), (4, 900, 8, 24, 2),
                                                   (5, 2500, 32, 32, 3), (2, 1, 8, 8, 4)])
def test_conv333_matches_dense(depth, n, cin, cout, seed):
    xyz = synth.random_cloud(n, depth, seed)
    keys = O.leaf_keys(xyz, depth)
    N = len(keys)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    x = rng.integers(-128, 128, size=(N, cin)).astype(np.int8)
    W, bias, mult, slope = _layer_params(27, cin, cout, seed)
    z_in, z_out, shift = 5, -3, 20
    for use_slope in (True, False):
        got = O.conv333(keys, depth, x, z_in, W, bias, mult, shift,
                        slope if use_slope else None, z_out)
        side = 1 << depth
        dense = np.zeros((side + 2, side + 2, side + 2, cin), dtype=np.int64)
        P = _coords(keys, depth)
        dense[P[:, 0] + 1, P[:, 1] + 1, P[:, 2] + 1] = x.astype(np.int64) - z_in
        acc = np.tile(bias.astype(np.int64), (N, 1))
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    o = 9 * (dx + 1) + 3 * (dy + 1) + (dz + 1)
                    nb = dense[P[:, 0] + 1 + dx, P[:, 1] + 1 + dy, P[:, 2] + 1 + dz]
                    acc += nb @ W[o].astype(np.int64).T
        want = _finish(acc, mult, shift, slope if use_slope else None, z_out)
        assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("depth,n,cin,cout,seed", [(4, 600, 16, 8, 5), (5, 3000, 32, 32, 6)])
def test_down_s2_matches_dense(depth, n, cin, cout, seed):
    xyz = synth.random_cloud(n, depth, seed)
    ck = O.leaf_keys(xyz, depth)
    pk = np.unique(ck >> np.uint64(3))
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    x = rng.integers(-128, 128, size=(len(ck), cin)).astype(np.int8)
    W, bias, mult, slope = _layer_params(8, cin, cout, seed)
    z_in, z_out, shift = -9, 4, 19
    got = O.down_s2(ck, pk, x, z_in, W, bias, mult, shift, slope, z_out)
    side = 1 << depth
    dense = np.zeros((side, side, side, cin), dtype=np.int64)
    Pc = _coords(ck, depth)
    dense[Pc[:, 0], Pc[:, 1], Pc[:, 2]] = x.astype(np.int64) - z_in
    blocks = dense.reshape(side // 2, 2, side // 2, 2, side // 2, 2, cin)
    Pp = _coords(pk, depth - 1)
    acc = np.tile(bias.astype(np.int64), (len(pk), 1))
    for c in range(8):
        cx, cy, cz = c >> 2, (c >> 1) & 1, c & 1
        v = blocks[Pp[:, 0], cx, Pp[:, 1], cy, Pp[:, 2], cz]
        acc += v @ W[c].astype(np.int64).T
    want = _finish(acc, mult, shift, slope, z_out)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("depth,n,cin,cout,seed", [(4, 500, 16, 8, 8), (6, 3000, 64, 32, 9)])
def test_up_prune_matches_per_child_loop(depth, n, cin, cout, seed):
    xyz = synth.random_cloud(n, depth, seed)
    keys, codes = O.build_levels(xyz, depth)
    d = depth - 1
    pk, cd, ck = keys[d], codes[d], keys[d + 1]
    rng = np.random.Generator(np.random.PCG64(seed + 3))
    x = rng.integers(-128, 128, size=(len(pk), cin)).astype(np.int8)
    W, bias, mult, slope = _layer_params(8, cin, cout, seed, per_slice=True)
    z_in, z_out, shift = 2, -1, 18
    got = O.up_prune(pk, cd, ck, x, z_in, W, bias, mult, shift, slope, z_out)
    Pp = _coords(pk, d)
    want = {}
    for p in range(len(pk)):
        for c in range(8):
            if cd[p] >> c & 1:
                acc = bias[c].astype(np.int64) + W[c].astype(np.int64) @ (x[p].astype(np.int64) - z_in)
                row = _finish(acc[None, :], mult[c], shift, slope[c], z_out)[0]
                cxyz = (2 * Pp[p, 0] + (c >> 2), 2 * Pp[p, 1] + ((c >> 1) & 1), 2 * Pp[p, 2] + (c & 1))
                want[_interleave_by_string(*(int(v) for v in cxyz), d + 1)] = row
    assert len(want) == len(ck)
    for i, k in enumerate(ck.tolist()):
        assert np.array_equal(got[i].astype(np.int64), want[k])


# --------------------------------------------------------------------------
# Integer softmax -> frequencies -> CDF (Eq. 15)
# --------------------------------------------------------------------------

def _freqs_from_row(row):
    C = [0] + [int(v) for v in row[:254]] + [65536]
    return np.diff(np.array(C, dtype=np.int64))


def test_softmax_closed_forms():
    lut = synth.exp_lut()
    # all logits equal: e_i = 2^16, S = 255 * 2^16, f_i = 1 + floor(65281 / 255) = 257,
    # remainder 65536 - 255 * 257 = 1 goes to index 0
    for v in (-128, 0, 127):
        f = _freqs_from_row(O.softmax_cdf(np.full((1, 255), v, np.int8), lut)[0])
        want = np.full(255, 257)
        want[0] += 1
        assert np.array_equal(f, want)
    # one dominant symbol with every other exp entry zero: others get the floor 1
    for s in (0, 100, 254):
        lg = np.full((1, 255), -128, np.int8)
        lg[0, s] = 127
        f = _freqs_from_row(O.softmax_cdf(lg, lut)[0])
        assert f[s] == 65536 - 254 and np.all(np.delete(f, s) == 1)
    # ties for the maximum: the remainder goes to the lowest index
    lg = np.full((1, 255), -128, np.int8)
    lg[0, [7, 30]] = 127
    f = _freqs_from_row(O.softmax_cdf(lg, lut)[0])
    assert f[7] == f[30] + (65536 - 253 - 2 * (1 + (65536 * 65281) // (2 * 65536)))


def test_softmax_properties_and_error_bound():
    lut = synth.exp_lut()
    s = 1.0 / 16.0
    lg = RNG.integers(-128, 128, size=(400, 255)).astype(np.int8)
    lg[:100] = np.clip(RNG.normal(0, 30, size=(100, 255)), -128, 127).astype(np.int8)
    cdf = O.softmax_cdf(lg, lut)
    for n in range(lg.shape[0]):
        f = _freqs_from_row(cdf[n])
        assert f.sum() == 65536 and f.min() >= 1
        assert np.all(np.diff(cdf[n][:254].astype(np.int64)) > 0)
        assert cdf[n][254] == 0xFFFF and cdf[n][255] == 0xFFFF
        l = lg[n].astype(np.int64)
        # monotone: l_i > l_j  =>  f_i >= f_j
        vals = np.unique(l)
        lo = [f[l == v].min() for v in vals]
        hi = [f[l == v].max() for v in vals]
        assert all(lo[k + 1] >= hi[k] for k in range(len(vals) - 1))
        p = np.exp((l - l.max()) * s)
        p /= p.sum()
        # table rounding: |lut_i - 2^16 e^{-i s}| <= 1/2, relative to S >= 2^16;
        # floor + the +1 floor per symbol: <= 256 / 2^16; remainder < 255 on one symbol
        err = np.abs(f / 65536.0 - p)
        assert err.max() <= (256 + 255 + 255 * 0.5) / 65536.0 + 1e-12


# --------------------------------------------------------------------------
# Range coder
# --------------------------------------------------------------------------

def _random_cdf_rows(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lut = synth.exp_lut()
    lg = np.clip(rng.normal(0, 40, size=(n, 255)), -128, 127).astype(np.int8)
    return O.softmax_cdf(lg, lut)


@pytest.mark.parametrize("n,seed", [(0, 1), (1, 2), (5, 3), (5000, 4)])
def test_rc_cdf_round_trip_and_length(n, seed):
    cdf = _random_cdf_rows(max(n, 1), seed)[:n]
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    # draw symbols from the rows themselves so the ideal length is meaningful
    syms = np.zeros(n, dtype=np.uint8)
    ideal = 0.0
    for i in range(n):
        f = _freqs_from_row(cdf[i])
        syms[i] = rng.choice(255, p=f / 65536.0)
        ideal += -math.log2(f[syms[i]] / 65536.0)
    data = O.rc_encode_cdf(cdf, syms)
    assert len(data) <= ideal / 8 + 6
    assert np.array_equal(O.rc_decode_cdf(cdf, data), syms)


@pytest.mark.parametrize("n,seed", [(1, 11), (40, 12), (3000, 13)])
def test_rc_flush_costs_at_most_a_byte(n, seed):
    """Version 3 flush: the coded value is the one with the most trailing
    zero bits inside the final interval, and its trailing zero bytes are left
    out, so a substream costs at most one byte (plus one bit) over the ideal
    length sum -log2(f/2^16), besides the table coder's truncation of
    range / 2^16 (below 2^-8 relative per symbol, so under 0.006 bits); and
    the stream never ends in a zero byte that could have been left out."""
    cdf = _random_cdf_rows(n, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    worst = -1e9
    for rep in range(20):
        syms = np.zeros(n, dtype=np.uint8)
        ideal = 0.0
        for i in range(n):
            f = _freqs_from_row(cdf[i])
            syms[i] = rng.choice(255, p=f / 65536.0)
            ideal += -math.log2(f[syms[i]] / 65536.0)
        data = O.rc_encode_cdf(cdf, syms)
        assert np.array_equal(O.rc_decode_cdf(cdf, data), syms)
        worst = max(worst, 8 * len(data) - ideal - 0.006 * n)
        assert len(data) == 0 or data[-1] != 0
    assert worst <= 9.0, worst


def test_rc_empty_substream_is_empty():
    # no symbols: the value 0 lies in the initial interval and every byte of
    # it is a zero the decoder supplies
    assert O.rc_encode_cdf(np.zeros((0, 256), np.uint16), np.zeros(0, np.uint8)) == b""
    assert O.rc_encode_adaptive(np.zeros(0, np.uint8)) == b""


def test_rc_reads_at_most_four_bytes_past_the_end():
    """The decoder supplies at most four zero bytes after a substream's end;
    a stream that needs more is corrupt (a cut stream is detected)."""
    cdf = _random_cdf_rows(4000, 17)
    syms = RNG.integers(0, 255, size=4000).astype(np.uint8)
    data = O.rc_encode_cdf(cdf, syms)
    for cut in (5, 9, 64):
        with pytest.raises(O.OracleError):
            O.rc_decode_cdf(cdf, data[:-cut])


def test_rc_extreme_symbols():
    lut = synth.exp_lut()
    lg = np.full((3000, 255), -128, np.int8)
    lg[:, 0] = 127  # symbol 254 has the minimum frequency 1 in every row
    cdf = O.softmax_cdf(lg, lut)
    for s in (254, 0):
        syms = np.full(3000, s, np.uint8)
        data = O.rc_encode_cdf(cdf, syms)
        assert np.array_equal(O.rc_decode_cdf(cdf, data), syms)
        ideal = 3000 * -math.log2(_freqs_from_row(cdf[0])[s] / 65536.0)
        assert len(data) <= ideal / 8 + 6


def test_rc_truncated_stream_is_corrupt():
    cdf = _random_cdf_rows(2000, 7)
    syms = RNG.integers(0, 255, size=2000).astype(np.uint8)
    data = O.rc_encode_cdf(cdf, syms)
    with pytest.raises(O.OracleError):
        O.rc_decode_cdf(cdf, data[: len(data) // 2])


@pytest.mark.parametrize("n,seed", [(1, 1), (300, 2), (20000, 3)])
def test_rc_adaptive_round_trip(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    syms = rng.choice(255, size=n, p=np.arange(1, 256) ** 2 / np.sum(np.arange(1, 256) ** 2))
    syms = syms.astype(np.uint8)
    data = O.rc_encode_adaptive(syms)
    assert np.array_equal(O.rc_decode_adaptive(n, data), syms)


def _adaptive_ideal_bits(syms):
    """Ideal code length, in bits, of the coarse-level frequency model
    (supplement, Detailed Model Structure: coarse levels are coded by their
    symbol frequencies; the update rule is this codec's reading): every count
    starts at 1, the coded symbol's count grows by 32, and once the total
    exceeds 2^16 every count is halved, rounding up.  Each symbol costs
    -log2(f_s / total) under the counts seen before it."""
    f = [1] * 255
    total = 255
    bits = 0.0
    for s in syms.tolist():
        bits -= math.log2(f[s] / total)
        f[s] += 32
        total += 32
        if total > 1 << 16:
            f = [(x + 1) >> 1 for x in f]
            total = sum(f)
    return bits


def _drifting_source(n, seed):
    """Piecewise-stationary symbols: every 2,500 symbols a new set of six
    symbols carries 98 % of the mass, so the code length depends on how fast
    the model adapts and forgets (the increment and the halving)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(0, n, 2500):
        hot = rng.choice(255, size=6, replace=False)
        p = np.full(255, 0.02 / 249)
        p[hot] = 0.98 / 6
        out.append(rng.choice(255, size=min(2500, n - k), p=p / p.sum()))
    return np.concatenate(out).astype(np.uint8)


@pytest.mark.parametrize("seed", [1, 2])
def test_rc_adaptive_code_length_matches_model(seed):
    """Two-sided pin of the adaptive model: the coded length must equal the
    model's ideal length up to the coder's fixed per-substream cost (flush
    bytes) and its interval truncation.  On this source a model that never
    adapts, adds 16 instead of 32, or never halves is off by more than
    10^4 bits."""
    syms = _drifting_source(20000, seed)
    data = O.rc_encode_adaptive(syms)
    assert np.array_equal(O.rc_decode_adaptive(syms.shape[0], data), syms)
    excess = 8 * len(data) - _adaptive_ideal_bits(syms)
    assert abs(excess) <= 48, excess


# --------------------------------------------------------------------------
# Whole codec: lossless round trip (the paper's core claim), edge cases
# --------------------------------------------------------------------------

def _voxel_set(xyz):
    return {tuple(p) for p in np.asarray(xyz).tolist()}


@pytest.mark.parametrize("n,L,seed,chunk", [(1, 6, 1, 16384), (50, 6, 2, 7), (2000, 8, 3, 100),
                                            (3000, 11, 4, 16384), (800, 21, 5, 64)])
def test_round_trip_random(blob, n, L, seed, chunk):
    xyz = synth.random_cloud(n, L, seed)
    data = O.encode(blob, xyz, L, chunk)
    dec = O.decode(blob, data, n)
    assert _voxel_set(dec) == _voxel_set(xyz)
    keys = O.leaf_keys(xyz, L)
    assert np.array_equal(O.leaf_keys(dec, L), keys)
    # decoded order is the Morton order of the voxels
    assert [O.morton(int(a), int(b), int(c), L) for a, b, c in dec[:50].tolist()] == \
        keys[:50].tolist()


def test_round_trip_config1(blob):
    xyz = synth.make_frame(synth.C1)
    data = O.encode(blob, xyz, synth.C1.L)
    dec = O.decode(blob, data, xyz.shape[0])
    assert _voxel_set(dec) == _voxel_set(xyz)


def test_empty_frame(blob):
    data = O.encode(blob, np.zeros((0, 3), np.int32), 12)
    assert data[9] & 1
    assert O.decode(blob, data, 10).shape == (0, 3)


def test_weights_mismatch_and_corruption(blob):
    xyz = synth.random_cloud(500, 9, 11)
    data = O.encode(blob, xyz, 9)
    other = synth.make_blob(seed=8)
    with pytest.raises(O.OracleError) as e:
        O.decode(other, data, 500)
    assert e.value.status == -5
    with pytest.raises(O.OracleError) as e:
        O.decode(blob, data[:30], 500)
    assert e.value.status == -4
    bad = bytearray(data)
    bad[0] = ord("X")
    with pytest.raises(O.OracleError):
        O.decode(blob, bytes(bad), 500)
    with pytest.raises(O.OracleError) as e:
        O.decode(blob, data, 3)
    assert e.value.status == -2


def test_blob_validation(blob):
    assert O.check_blob(blob) == 0
    assert O.check_blob(blob[:-16]) != 0
    # a weight of -128 breaks the symmetric-weight assumption (z_w = 0, |w| <= 127)
    recs, lut = synth.make_blob_records()
    recs[1].W[0, 0, 0] = -128
    assert O.check_blob(synth.pack_blob(recs, lut, 32)) != 0
    recs, lut = synth.make_blob_records()
    lut = lut.copy()
    lut[5] = lut[4] + 1  # the exp table must be non-increasing
    assert O.check_blob(synth.pack_blob(recs, lut, 32)) != 0


def test_probs_level_rows_valid(blob):
    xyz = synth.make_frame(synth.C1)
    L = synth.C1.L
    keys, codes = O.build_levels(xyz, L)
    for d in range(L - 5, L):
        cdf = O.probs_level(blob, xyz, L, d)
        assert cdf.shape == (len(keys[d]), 256)
        C = cdf[:, :254].astype(np.int64)
        assert np.all(np.diff(C, axis=1) > 0) and np.all(C[:, 0] >= 1)


def test_fnv1a64_published_vectors():
    """The blob hash carried in every stream header is 64-bit FNV-1a; pinned
    to the test vectors published with the FNV definition."""
    assert O.fnv1a64(b"") == 0xcbf29ce484222325
    assert O.fnv1a64(b"a") == 0xaf63dc4c8601ec8c
    assert O.fnv1a64(b"foobar") == 0x85944171f73967e8


def _varint(data, pos):
    v = s = 0
    while True:
        b = data[pos]
        pos += 1
        v |= (b & 0x7F) << s
        s += 7
        if b < 0x80:
            return v, pos


def test_stream_header_coarse_sizes():
    """Stream version 3: after the chunk lengths the header lists the coarse
    levels' sizes N_1 .. N_{b-1} (those of the octree of the frame), and the
    substream table holds ceil(N_d / 512) substreams per coarse level before
    the network levels' chunks; the lengths (zigzag varints of the difference
    to the previous length) add up to the rest of the stream exactly."""
    blob = synth.make_blob()
    xyz = synth.random_cloud(60000, 17, 71)
    L, chunk = 17, 1000
    data = O.encode(blob, xyz, L, chunk)
    assert data[:4] == b"LPC1" and data[4] == 3
    keys, codes = O.build_levels(xyz, L)
    b = L - 5
    c, pos = _varint(data, 18)
    kc, pos = _varint(data, pos)
    assert (c, kc) == (chunk, 512)
    sizes = []
    for _ in range(1, b):
        v, pos = _varint(data, pos)
        sizes.append(v)
    assert sizes == [len(keys[d]) for d in range(1, b)]
    nsub, pos = _varint(data, pos)
    want = sum(-(-len(keys[d]) // kc) for d in range(b)) + \
        sum(-(-len(keys[d]) // chunk) for d in range(b, L))
    assert nsub == want
    assert max(len(keys[d]) for d in range(b)) > kc  # a level in several chunks
    prev, total = 0, 0
    for _ in range(nsub):
        z, pos = _varint(data, pos)
        prev += z >> 1 if z % 2 == 0 else -((z + 1) >> 1)
        assert prev >= 0
        total += prev
    assert pos + total == len(data)


def test_stream_header_bad_coarse_size_is_corrupt():
    blob = synth.make_blob()
    xyz = synth.random_cloud(3000, 12, 72)
    data = bytearray(O.encode(blob, xyz, 12))
    pos = 18
    _, pos = _varint(data, pos)
    _, pos = _varint(data, pos)
    assert data[pos] < 0x80  # N_1 is a one-byte varint
    for v in (data[pos] + 1, 0):
        bad = bytearray(data)
        bad[pos] = v
        with pytest.raises(O.OracleError) as e:
            O.decode(blob, bytes(bad), 3000)
        assert e.value.status == -4
