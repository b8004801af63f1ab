"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Everything is integer, so every comparison is exact: level arrays, kernel
maps (as sets of present neighbours), every layer's int8 outputs, cumulative
tables, and whole bitstreams byte for byte.  Inputs are seeded synthetic
frames and seeded weight blobs.
"""

import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_25260_b300 import synth

pytestmark = pytest.mark.gpu

O.set_threads(os.cpu_count() or 1)


@pytest.fixture(scope="module")
def lpc():
    from paper_2603_25260_b300 import build, lpc as mod
    build.build()
    mod.lib()
    return mod


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _params(S, cin, cout, seed, per_slice=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.integers(-127, 128, size=(S, cout, cin)).astype(np.int8)
    shape = (S, cout) if per_slice else (cout,)
    bias = rng.integers(-(1 << 20), 1 << 20, size=shape).astype(np.int32)
    mult = rng.integers(1, 1 << 16, size=shape).astype(np.int32)
    slope = rng.integers(-32768, 32768, size=shape).astype(np.int16)
    return W, bias, mult, slope


# ------------------------------------------------------------------ levels --

@pytest.mark.parametrize("n,L,seed", [(1, 6, 1), (5, 6, 2), (4097, 9, 3), (30000, 12, 4),
                                      (20000, 19, 5), (9000, 16, 6)])
def test_levels_match_oracle(lpc, n, L, seed):
    xyz = synth.random_cloud(n, L, seed)
    xyz = np.concatenate([xyz, xyz[: n // 2]])  # duplicates, out of order
    ks, cs = lpc.build_levels(_cuda(xyz), L)
    ok, oc = O.build_levels(xyz, L)
    for d in range(L + 1):
        assert np.array_equal(ks[d].cpu().numpy().view(np.uint64), ok[d])
        if d < L:
            assert np.array_equal(cs[d].cpu().numpy(), oc[d])


def test_levels_config1(lpc):
    xyz = synth.make_frame(synth.C1)
    ks, cs = lpc.build_levels(_cuda(xyz), synth.C1.L)
    ok, oc = O.build_levels(xyz, synth.C1.L)
    for d in range(synth.C1.L):
        assert np.array_equal(ks[d].cpu().numpy().view(np.uint64), ok[d])
        assert np.array_equal(cs[d].cpu().numpy(), oc[d])


def test_out_of_range_coordinate_is_rejected(lpc):
    xyz = np.array([[0, 0, 0], [3, 64, 1]], dtype=np.int32)
    with pytest.raises(lpc.LpcError) as e:
        lpc.build_levels(_cuda(xyz), 6)
    assert e.value.status == lpc.INVALID_ARG


# -------------------------------------------------------------- kernel map --

@pytest.mark.parametrize("n,depth,seed", [(1, 4, 1), (700, 5, 2), (5000, 7, 3), (40000, 12, 4),
                                          (3000, 20, 8), (3000, 21, 9)])
def test_kernel_map(lpc, n, depth, seed):
    xyz = synth.random_cloud(n, depth, seed)
    keys = O.leaf_keys(xyz, depth)
    nbr = lpc.kernel_map(_cuda(keys.view(np.int64)), depth).cpu().numpy()
    pos = {int(k): i for i, k in enumerate(keys.tolist())}
    side = 1 << depth
    coords = np.stack([xyz[:, 0], xyz[:, 1], xyz[:, 2]], 1)
    # brute force on the unique voxels
    uniq = {}
    for x, y, z in coords.tolist():
        uniq[O.morton(x, y, z, depth)] = (x, y, z)
    for i, k in enumerate(keys.tolist()[:3000]):
        x, y, z = uniq[k]
        for o in range(27):
            qx, qy, qz = x + o // 9 - 1, y + (o // 3) % 3 - 1, z + o % 3 - 1
            want = -1
            if 0 <= qx < side and 0 <= qy < side and 0 <= qz < side:
                want = pos.get(O.morton(qx, qy, qz, depth), -1)
            assert nbr[i, o] == want


def _brute_map(keys, depth):
    """27-neighbour rows of Morton keys by coordinates and a dictionary."""
    pos = {int(k): i for i, k in enumerate(keys.tolist())}
    side = 1 << depth
    out = np.full((len(keys), 27), -1, dtype=np.int32)
    for i, k in enumerate(keys.tolist()):
        x = y = z = 0
        for b in range(depth):
            x |= ((k >> (3 * b + 2)) & 1) << b
            y |= ((k >> (3 * b + 1)) & 1) << b
            z |= ((k >> (3 * b)) & 1) << b
        for o in range(27):
            qx, qy, qz = x + o // 9 - 1, y + (o // 3) % 3 - 1, z + o % 3 - 1
            if 0 <= qx < side and 0 <= qy < side and 0 <= qz < side:
                out[i, o] = pos.get(O.morton(qx, qy, qz, depth), -1)
    return out


@pytest.mark.parametrize("n,L,d,seed", [(1, 6, 3, 1), (900, 8, 6, 2), (6000, 12, 9, 3),
                                        (4000, 19, 14, 4)])
def test_kernel_map_child(lpc, n, L, d, seed):
    """The map of depth d derived from the map of depth d - 1 (octree
    neighbour rule) equals the brute-force map; every input is the oracle's."""
    xyz = synth.random_cloud(n, L, seed)
    ok, oc = O.build_levels(xyz, L)
    pk, ck, pcode = ok[d - 1], ok[d], oc[d - 1]
    cpar = np.searchsorted(pk, ck >> np.uint64(3)).astype(np.int32)
    poff = np.concatenate([[0], np.cumsum([bin(int(c)).count("1") for c in pcode])])
    pnbr = _brute_map(pk, d - 1)
    got = lpc.kernel_map_child(_cuda(ck.view(np.int64)), _cuda(cpar), _cuda(pnbr), _cuda(pcode),
                               _cuda(poff.astype(np.int32))).cpu().numpy()
    assert np.array_equal(got, _brute_map(ck, d))


def test_hash_full_is_reported(lpc):
    keys = O.leaf_keys(synth.random_cloud(3000, 10, 7), 10)
    with pytest.raises(lpc.LpcError) as e:
        lpc.kernel_map(_cuda(keys.view(np.int64)), 10, table_log2=8)
    assert e.value.status == lpc.HASH_FULL


# ------------------------------------------------------------------ layers --

@pytest.mark.parametrize("n,depth,cin,seed", [(1, 3, 32, 1), (333, 5, 32, 2), (4100, 8, 64, 3),
                                              (20000, 12, 64, 4), (3000, 6, 64, 5)])
def test_conv333(lpc, n, depth, cin, seed):
    xyz = synth.random_cloud(n, depth, seed)
    keys = O.leaf_keys(xyz, depth)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(-128, 128, size=(len(keys), cin)).astype(np.int8)
    W, bias, mult, slope = _params(27, cin, 32, seed)
    for sl, shift in ((slope, 24), (None, 20)):
        want = O.conv333(keys, depth, x, 7, W, bias, mult, shift, sl, -5)
        got = lpc.conv333(_cuda(keys.view(np.int64)), depth, _cuda(x), 7, W, bias, mult, shift,
                          sl, -5).cpu().numpy()
        assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("cin", [32, 64])
@pytest.mark.parametrize("n", [40000, 40100])
def test_conv333_variants(lpc, cin, variant, n):
    """Every kernel variant the autotuner may pick (ring shape, tile order,
    cp.async or TMA gather4 gather, 128- or 256-row tiles) matches the
    oracle, over several tiles and a ragged tail (for 256-row tiles one that
    ends in the first or the second half of a tile)."""
    depth, seed = 9, 21
    xyz = synth.random_cloud(n, depth, seed)
    keys = O.leaf_keys(xyz, depth)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(-128, 128, size=(len(keys), cin)).astype(np.int8)
    W, bias, mult, slope = _params(27, cin, 32, seed)
    want = O.conv333(keys, depth, x, 7, W, bias, mult, 24, slope, -5)
    got = lpc.conv333(_cuda(keys.view(np.int64)), depth, _cuda(x), 7, W, bias, mult, 24, slope,
                      -5, variant=variant).cpu().numpy()
    assert np.array_equal(got, want)


def test_codec_autotuner_picks_variants(lpc, blob):
    xyz = synth.random_cloud(20000, 14, 4)
    cod = _codec(lpc, blob, 14, 20000)
    data = cod.encode(_cuda(xyz))
    t = cod.tuning()
    assert 0 <= t["conv32"] < 10 and 0 <= t["conv64"] < 10 and 0 <= t["predictor"] < 2
    assert 0 <= t["up32"] < 2 and 0 <= t["up64"] < 2
    assert all(0 < m < 1e3 for m in t["ms32"] + t["ms64"] + t["ms_pred"] + t["ms_up32"] +
               t["ms_up64"])
    assert data == O.encode(blob, xyz, 14)  # and the next call runs the captured graphs
    assert cod.encode(_cuda(xyz)) == data


def test_conv333_extreme_accumulator(lpc):
    """Worst-case magnitudes: every input at -128 with z = 127 and every
    weight at +-127 over 27 present neighbours (|acc| near 27*64*255*127)."""
    depth = 4
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"), -1)
    xyz = g.reshape(-1, 3).astype(np.int32) + 5
    keys = O.leaf_keys(xyz, depth)
    x = np.full((len(keys), 64), -128, np.int8)
    for sign in (1, -1):
        W = np.full((27, 32, 64), 127 * sign, np.int8)
        bias = np.zeros(32, np.int32)
        mult = np.full(32, 1 << 10, np.int32)
        want = O.conv333(keys, depth, x, 127, W, bias, mult, 30, None, 0)
        got = lpc.conv333(_cuda(keys.view(np.int64)), depth, _cuda(x), 127, W, bias, mult, 30,
                          None, 0).cpu().numpy()
        assert np.array_equal(got, want)


@pytest.mark.parametrize("n,depth,seed", [(1, 4, 1), (900, 6, 2), (20000, 11, 3)])
def test_down_s2(lpc, n, depth, seed):
    xyz = synth.random_cloud(n, depth, seed)
    ck = O.leaf_keys(xyz, depth)
    pk = np.unique(ck >> np.uint64(3))
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(-128, 128, size=(len(ck), 32)).astype(np.int8)
    W, bias, mult, slope = _params(8, 32, 32, seed)
    want = O.down_s2(ck, pk, x, -9, W, bias, mult, 22, slope, 4)
    got = lpc.down_s2(_cuda(ck.view(np.int64)), _cuda(pk.view(np.int64)), _cuda(x), -9, W, bias,
                      mult, 22, slope, 4).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n,depth,cin,seed", [(1, 4, 32, 1), (900, 6, 64, 2), (25000, 12, 64, 3),
                                              (5000, 9, 32, 4), (70000, 14, 64, 5)])
def test_up_prune(lpc, n, depth, cin, seed, variant):
    xyz = synth.random_cloud(n, depth, seed)
    keys, codes = O.build_levels(xyz, depth)
    d = depth - 1
    pk, cd, ck = keys[d], codes[d], keys[d + 1]
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(-128, 128, size=(len(pk), cin)).astype(np.int8)
    W, bias, mult, slope = _params(8, cin, 32, seed, per_slice=True)
    want = O.up_prune(pk, cd, ck, x, 3, W, bias, mult, 21, slope, -2)
    got = lpc.up_prune(_cuda(pk.view(np.int64)), _cuda(cd), _cuda(ck.view(np.int64)), _cuda(x), 3,
                       W, bias, mult, 21, slope, -2, variant=variant).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", [0, 1])
def test_up_prune_extreme_accumulator(lpc, variant):
    """Worst-case magnitudes of the up-step: every input at -128 with
    z_in = 127 (q - z = -255) and every weight at +-127 over 64 channels
    (|acc| = 64 * 255 * 127), mixed signs by slot, no PReLU."""
    xyz = synth.random_cloud(3000, 8, 9)
    keys, codes = O.build_levels(xyz, 8)
    pk, cd, ck = keys[7], codes[7], keys[8]
    x = np.full((len(pk), 64), -128, np.int8)
    W = np.full((8, 32, 64), 127, np.int8)
    W[1::2] = -127
    W[2, :, ::3] = -127
    bias = np.arange(8 * 32, dtype=np.int32).reshape(8, 32) * 1001 - 90000
    mult = np.full((8, 32), 3, np.int32)
    want = O.up_prune(pk, cd, ck, x, 127, W, bias, mult, 15, None, 1)
    got = lpc.up_prune(_cuda(pk.view(np.int64)), _cuda(cd), _cuda(ck.view(np.int64)), _cuda(x),
                       127, W, bias, mult, 15, None, 1, variant=variant).cpu().numpy()
    assert np.array_equal(got, want)
    assert len(np.unique(want)) > 3  # the extremes do not all clip to one value


def test_softmax_cdf(lpc):
    rng = np.random.Generator(np.random.PCG64(3))
    lut = synth.exp_lut()
    lg = rng.integers(-128, 128, size=(5000, 255)).astype(np.int8)
    lg[:1000] = np.clip(rng.normal(0, 20, size=(1000, 255)), -128, 127).astype(np.int8)
    lg[1000] = 0
    lg[1001] = -128
    lg[1001, 254] = 127
    lg[1002] = -128
    lg[1002, [3, 200]] = 127
    lg[1003] = 127
    want = O.softmax_cdf(lg, lut)
    got = lpc.u16(lpc.softmax_cdf(_cuda(lg), lut))
    assert np.array_equal(got, want)


# ------------------------------------------------------ whole path parity --

@pytest.fixture(scope="module")
def c1():
    return synth.make_frame(synth.C1)


def _codec(lpc, blob, L, n, **kw):
    return lpc.Codec(blob, L, max(n, 16), **kw)


def test_probs_level_config1(lpc, blob, c1):
    L = synth.C1.L
    cod = _codec(lpc, blob, L, c1.shape[0])
    xyz = _cuda(c1)
    for d in range(L - 5, L):
        want = O.probs_level(blob, c1, L, d)
        got = lpc.u16(cod.probs_level(xyz, d))
        assert np.array_equal(got, want), d


def test_encode_byte_identical_config1(lpc, blob, c1):
    L = synth.C1.L
    cod = _codec(lpc, blob, L, c1.shape[0])
    assert cod.encode(_cuda(c1)) == O.encode(blob, c1, L)


@pytest.mark.parametrize("n,L,seed", [(0, 12, 0), (20000, 16, 8)])
def test_trained_blob_byte_identical(lpc, c1, n, L, seed):
    """The exported blob of the trained twin (other value ranges than the
    seeded blob: larger biases, skewed predictions): same streams as the
    oracle, lossless round trip."""
    from paper_2603_25260_b300 import export
    with open(export.TRAINED_BLOB, "rb") as f:
        tb = f.read()
    xyz = c1 if n == 0 else synth.random_cloud(n, L, seed)
    cod = _codec(lpc, tb, L, xyz.shape[0])
    data = cod.encode(_cuda(xyz))
    assert data == O.encode(tb, xyz, L)
    dec = cod.decode(data).cpu().numpy()
    assert np.array_equal(O.leaf_keys(dec, L), O.leaf_keys(xyz, L))
    got = lpc.u16(cod.probs_level(_cuda(xyz), L - 1))
    assert np.array_equal(got, O.probs_level(tb, xyz, L, L - 1))


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
@pytest.mark.parametrize("n,L,seed,chunk", [(1, 6, 1, 16384), (2, 7, 2, 16384),
                                            (3000, 10, 3, 100), (20000, 14, 4, 4096),
                                            (5000, 19, 5, 16384), (12000, 12, 6, 999),
                                            (7000, 11, 7, 1)])
def test_encode_decode_random(lpc, blob, n, L, seed, chunk, host_coding):
    xyz = synth.random_cloud(n, L, seed)
    cod = _codec(lpc, blob, L, n, chunk=chunk, host_coding=host_coding)
    data = cod.encode(_cuda(xyz))
    assert data == O.encode(blob, xyz, L, chunk)
    dec = cod.decode(data).cpu().numpy()
    assert np.array_equal(O.leaf_keys(dec, L), O.leaf_keys(xyz, L))
    assert np.array_equal(dec, O.decode(blob, data, n))


def test_cross_decode(lpc, blob, c1):
    """Oracle stream decodes on the GPU and GPU stream decodes on the oracle."""
    L = synth.C1.L
    cod = _codec(lpc, blob, L, c1.shape[0])
    so = O.encode(blob, c1, L)
    assert np.array_equal(cod.decode(so).cpu().numpy(), O.decode(blob, so, c1.shape[0]))
    sg = cod.encode(_cuda(c1))
    assert np.array_equal(O.decode(blob, sg, c1.shape[0]), cod.decode(sg).cpu().numpy())


def test_empty_and_failures(lpc, blob):
    L = 12
    cod = _codec(lpc, blob, L, 1000)
    empty = cod.encode(torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    assert empty == O.encode(blob, np.zeros((0, 3), np.int32), L)
    assert cod.decode(empty).shape[0] == 0
    xyz = synth.random_cloud(500, L, 3)
    data = cod.encode(_cuda(xyz))
    other = _codec(lpc, synth.make_blob(seed=8), L, 1000)
    with pytest.raises(lpc.LpcError) as e:
        other.decode(data)
    assert e.value.status == lpc.WEIGHTS_MISMATCH
    with pytest.raises(lpc.LpcError) as e:
        cod.decode(data[:40])
    assert e.value.status == lpc.CORRUPT_STREAM
    with pytest.raises(lpc.LpcError) as e:
        cod.decode(data, cap=10)
    assert e.value.status == lpc.CAPACITY
    bad = xyz.copy()
    bad[7, 1] = 1 << L
    with pytest.raises(lpc.LpcError) as e:
        cod.encode(_cuda(bad))
    assert e.value.status == lpc.INVALID_ARG
    with pytest.raises(lpc.LpcError) as e:
        cod.encode(_cuda(xyz), cap=10)
    assert e.value.status == lpc.CAPACITY
    # the codec stays usable after every failure
    assert cod.encode(_cuda(xyz)) == data


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
@pytest.mark.parametrize("spec", [synth.C2, synth.C3], ids=["kitti64_L16", "dense128_L18"])
def test_full_size_frames_byte_identical(lpc, blob, spec, host_coding):
    xyz = synth.make_frame(spec)
    cod = _codec(lpc, blob, spec.L, xyz.shape[0], host_coding=host_coding)
    data = cod.encode(_cuda(xyz))
    assert data == O.encode(blob, xyz, spec.L)
    dec = cod.decode(data).cpu().numpy()
    assert np.array_equal(O.leaf_keys(dec, spec.L), O.leaf_keys(xyz, spec.L))


def test_batch_matches_per_frame_oracle(lpc, blob):
    specs = synth.batch_specs(6)
    frames = [synth.make_frame(s)[:20000] for s in specs]
    Ls = [s.L for s in specs]
    cod = lpc.Codec(blob, max(Ls), 20000, max_frames=len(frames))
    outs = cod.encode_batch([_cuda(f) for f in frames], Ls)
    for f, L, o in zip(frames, Ls, outs):
        assert o == O.encode(blob, f, L)
    decs = cod.decode_batch(outs, [f.shape[0] for f in frames])
    for f, L, dcd in zip(frames, Ls, decs):
        assert np.array_equal(O.leaf_keys(dcd.cpu().numpy(), L), O.leaf_keys(f, L))


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
def test_batch_mixed_with_empty_frames(lpc, blob, host_coding):
    """A batch mixing depths 6..19, tiny and empty frames: every stream equals
    the oracle's stream of that frame alone, and the batch decodes exactly
    (also the oracle's streams, decoded as one batch)."""
    specs = [(300, 6, 1), (0, 12, 2), (4000, 19, 3), (1, 9, 4), (25000, 16, 5), (0, 7, 6),
             (9000, 13, 7)]
    frames = [synth.random_cloud(n, L, s) for n, L, s in specs]
    Ls = [L for _, L, _ in specs]
    cod = lpc.Codec(blob, 19, 25000, max_frames=len(frames), chunk=1000, host_coding=host_coding)
    outs = cod.encode_batch([_cuda(f) for f in frames], Ls)
    want = [O.encode(blob, f, L, 1000) for f, L in zip(frames, Ls)]
    assert outs == want
    decs = cod.decode_batch(want, [max(f.shape[0], 1) for f in frames])
    for f, L, dcd in zip(frames, Ls, decs):
        assert np.array_equal(dcd.cpu().numpy(), O.decode(blob, O.encode(blob, f, L, 1000),
                                                          max(f.shape[0], 1)))


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
def test_corrupt_payload(lpc, blob, host_coding):
    """Flipped payload bytes: decoding either reports the stream as corrupt
    (or its levels as too large) or returns some other point set, never
    anything else, and the codec stays usable."""
    L = 10
    xyz = synth.random_cloud(3000, L, 9)
    cod = _codec(lpc, blob, L, 3000, chunk=256, host_coding=host_coding)
    data = cod.encode(_cuda(xyz))
    want = O.decode(blob, data, 3000)
    rng = np.random.Generator(np.random.PCG64(5))
    outcomes = set()
    for trial in range(12):
        bad = bytearray(data)
        lo = len(data) // 3 if trial % 2 else 40
        for pos in rng.integers(lo, len(data), size=3):
            bad[pos] ^= int(rng.integers(1, 256))
        try:
            dec = cod.decode(bytes(bad), cap=3000)
            outcomes.add("decoded")
            assert dec.shape[1] == 3
        except lpc.LpcError as e:
            assert e.status in (lpc.CORRUPT_STREAM, lpc.CAPACITY), e
            outcomes.add(e.status)
    assert outcomes
    assert np.array_equal(cod.decode(data).cpu().numpy(), want)


@pytest.mark.parametrize("n,L,seed,chunk", [(20000, 14, 41, 1024), (3000, 10, 42, 1),
                                            (9000, 16, 43, 333)])
def test_repeated_decode_graph_path(lpc, blob, n, L, seed, chunk):
    """From the second decode on, the network levels run as captured graphs
    with the substream tables built on the device (no host round trip per
    level): the same voxels as the oracle on every call, also with one chunk
    per node."""
    xyz = synth.random_cloud(n, L, seed)
    cod = _codec(lpc, blob, L, n, chunk=chunk)
    data = O.encode(blob, xyz, L, chunk)
    want = O.decode(blob, data, n)
    for _ in range(3):
        assert np.array_equal(cod.decode(data).cpu().numpy(), want)
    bad = bytearray(data)
    bad[len(bad) // 2] ^= 0x33
    try:
        cod.decode(bytes(bad), cap=n)
    except lpc.LpcError as e:
        assert e.status in (lpc.CORRUPT_STREAM, lpc.CAPACITY), e
    assert np.array_equal(cod.decode(data).cpu().numpy(), want)


def test_batch_split_decode(lpc, blob):
    """Batches of 8 frames or more decode in two groups (coarse levels of the
    second decoded on the host while the device decodes the first): the
    voxels of every frame equal the oracle's decode of its own stream, in a
    batch with mixed depths, sizes and an empty frame; a corrupt frame in the
    second group is reported and the codec stays usable."""
    specs = [(2000, 9, 21), (15000, 14, 22), (0, 11, 23), (500, 7, 24), (30000, 16, 25),
             (7000, 12, 26), (12000, 18, 27), (100, 8, 28), (22000, 15, 29), (4000, 10, 30),
             (9000, 13, 31), (1, 6, 32)]
    frames = [synth.random_cloud(n, L, sd) for n, L, sd in specs]
    Ls = [L for _, L, _ in specs]
    cod = lpc.Codec(blob, 18, 30000, max_frames=len(frames), chunk=700)
    streams = [O.encode(blob, f, L, 700) for f, L in zip(frames, Ls)]
    caps = [max(f.shape[0], 1) for f in frames]
    for _ in range(2):
        decs = cod.decode_batch(streams, caps)
        for f, L, s, dcd in zip(frames, Ls, streams, decs):
            want = O.decode(blob, s, max(f.shape[0], 1))
            assert np.array_equal(dcd.cpu().numpy(), want)
    assert cod.encode_batch([_cuda(f) for f in frames], Ls) == streams
    # corrupt the coarse data of the largest frame (second group)
    big = int(np.argmax([f.shape[0] for f in frames]))
    bad = list(streams)
    b = bytearray(bad[big])
    for pos in range(40, 60):
        b[pos] ^= 0x5A
    bad[big] = bytes(b)
    try:
        cod.decode_batch(bad, caps)
    except lpc.LpcError as e:
        assert e.status in (lpc.CORRUPT_STREAM, lpc.CAPACITY), e
    decs = cod.decode_batch(streams, caps)
    for f, L, dcd in zip(frames, Ls, decs):
        assert np.array_equal(O.leaf_keys(dcd.cpu().numpy(), L), O.leaf_keys(f, L))


def test_batch_into_reusable_buffer(lpc, blob):
    """The buffer-reusing batch calls give the same streams and voxels."""
    specs = [(3000, 10, 11), (0, 9, 12), (8000, 14, 13)]
    frames = [synth.random_cloud(n, L, s) for n, L, s in specs]
    Ls = [L for _, L, _ in specs]
    cod = lpc.Codec(blob, 14, 8000, max_frames=3)
    xs = [_cuda(f) for f in frames]
    want = cod.encode_batch(xs, Ls)
    buf = np.zeros(sum(lpc.Codec.batch_caps(xs)), dtype=np.uint8)
    outs = [torch.empty((max(f.shape[0], 1), 3), dtype=torch.int32, device="cuda") for f in frames]
    for _ in range(2):
        spans = cod.encode_batch_into(xs, Ls, buf)
        assert [bytes(buf[o:o + n]) for o, n in spans] == want
        decs = cod.decode_batch_from(buf, spans, outs)
        for f, L, d in zip(frames, Ls, decs):
            assert np.array_equal(O.leaf_keys(d.cpu().numpy(), L), O.leaf_keys(f, L))


@pytest.mark.parametrize("variants", [(0, 0, 0, 0, 0), (3, 3, 1, 1, 1), (1, 2, 1, 0, 1),
                                      (2, 1, 0, 1, 0), (4, 4, 1, 1, 1), (7, 5, 1, 0, 0),
                                      (5, 6, 0, 1, 1), (8, 8, 1, 0, 0), (9, 9, 1, 1, 1)])
def test_fixed_variants_byte_identical(lpc, blob, variants):
    """Every fixed combination of conv, predictor and up-step variants gives
    the oracle's stream and decodes it (graphs captured with those
    variants)."""
    xyz = synth.random_cloud(15000, 13, 6)
    cod = _codec(lpc, blob, 13, 15000)
    cod.set_tuning(*variants)
    want = O.encode(blob, xyz, 13)
    for _ in range(2):
        data = cod.encode(_cuda(xyz))
        assert data == want
        dec = cod.decode(data).cpu().numpy()
        assert np.array_equal(O.leaf_keys(dec, 13), O.leaf_keys(xyz, 13))
    t = cod.tuning()
    assert (t["predictor"], t["up32"], t["up64"]) == variants[2:]


@pytest.mark.parametrize("threads", [1, 2, 4])
def test_few_host_threads(lpc, blob, threads):
    """Fewer host threads than coarse levels: the leading levels run in order
    on the calling thread and each deeper level on its own worker, still
    pipelined; one thread decodes the levels in order.  Same voxels."""
    xyz = synth.random_cloud(20000, 16, 61)
    data = O.encode(blob, xyz, 16)
    want = O.decode(blob, data, xyz.shape[0])
    cod = _codec(lpc, blob, 16, xyz.shape[0], host_threads=threads)
    assert cod.encode(_cuda(xyz)) == data
    for _ in range(2):
        assert np.array_equal(cod.decode(data).cpu().numpy(), want)


def test_bad_coarse_size_is_corrupt(lpc, blob):
    """A coarse level size in the header that the codes above it do not
    expand to, or zero: the stream is reported corrupt (and a good stream
    still decodes after it)."""
    xyz = synth.random_cloud(3000, 12, 72)
    data = O.encode(blob, xyz, 12)
    cod = _codec(lpc, blob, 12, 3000)
    pos = 18
    for _ in range(2):  # chunk, coarse chunk
        while data[pos] >= 0x80:
            pos += 1
        pos += 1
    assert data[pos] < 0x80
    for v in (data[pos] + 1, 0):
        bad = bytearray(data)
        bad[pos] = v
        with pytest.raises(lpc.LpcError) as e:
            cod.decode(bytes(bad))
        assert e.value.status == lpc.CORRUPT_STREAM
    assert np.array_equal(cod.decode(data).cpu().numpy(), O.decode(blob, data, 3000))


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
def test_repeated_encode_graph_path(lpc, blob, host_coding):
    """From the second encode on, the five levels run as one captured graph
    with levels 3 and 4 on their own streams and scratch, queued behind the
    octree: the same stream as the oracle on every call."""
    xyz = synth.random_cloud(30000, 16, 81)
    want = O.encode(blob, xyz, 16)
    cod = _codec(lpc, blob, 16, xyz.shape[0], host_coding=host_coding)
    x = _cuda(xyz)
    for _ in range(4):
        assert cod.encode(x) == want


def test_encode_batch_capacity_per_frame(lpc, blob):
    """A batch (more than two frames, so the streams are assembled one frame
    per pool task) where one frame's output buffer is too small: the call
    returns LPC_CAPACITY with that frame's needed length, and every other
    frame still receives the oracle's stream."""
    import ctypes as C
    L = 12
    frames = [synth.random_cloud(n, L, 60 + k) for k, n in enumerate([3000, 500, 4000, 0, 2500])]
    cod = lpc.Codec(blob, L, 4000, max_frames=len(frames))
    xs = [_cuda(f) for f in frames]
    want = [O.encode(blob, f, L) for f in frames]
    nf = len(frames)
    caps = [len(w) + 64 for w in want]
    caps[2] = 10
    bufs = [np.zeros(c, dtype=np.uint8) for c in caps]
    lib = cod._lib
    ptrs = (C.c_void_p * nf)(*[x.data_ptr() if x.shape[0] else 0 for x in xs])
    ns = (C.c_int64 * nf)(*[x.shape[0] for x in xs])
    ls = (C.c_int * nf)(*([L] * nf))
    outs = (C.c_void_p * nf)(*[b.ctypes.data for b in bufs])
    capa = (C.c_size_t * nf)(*caps)
    lens = (C.c_size_t * nf)()
    st = lib.encode_batch(cod._h, nf, ptrs, ns, ls, outs, capa, lens)
    assert st == lpc.CAPACITY
    assert lens[2] == len(want[2])
    for i in (0, 1, 3, 4):
        assert lens[i] == len(want[i])
        assert bytes(bufs[i][:lens[i]]) == want[i]
    # the codec stays usable
    assert cod.encode_batch(xs, [L] * nf) == want
