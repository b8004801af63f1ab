"""GPU parity of the ablation architectures (Sec. 4.3; supplement, choice of
t): GRED + XFP, GRED only and the baseline, each with t = L - 4 or L - 3, run
by the same kernels.  Every stream equals the CPU oracle's byte for byte,
per frame, in batches of mixed depths, with device and host range coding,
and through the captured-graph decode path; the per-level tables equal the
oracle's."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_25260_b300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = [(a, t) for a in (synth.ARCH_XFP, synth.ARCH_GRED, synth.ARCH_BASE) for t in (4, 3)]
IDS = [f"{n}_t{t}" for n in ("gred_xfp", "gred", "baseline") for t in (4, 3)]


@pytest.fixture(scope="module")
def lpc():
    from paper_2603_25260_b300 import lpc as m
    m.lib()
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("arch,t_off", VARIANTS, ids=IDS)
def test_probs_and_stream_byte_identical(lpc, arch, t_off):
    blob = synth.make_blob(arch=arch, t_off=t_off)
    xyz = synth.make_frame(synth.C1)
    L = synth.C1.L
    cod = lpc.Codec(blob, L, xyz.shape[0])
    for d in range(L - 5, L):
        got = lpc.u16(cod.probs_level(_cuda(xyz), d))
        assert np.array_equal(got, O.probs_level(blob, xyz, L, d)), d
    data = cod.encode(_cuda(xyz))
    assert data == O.encode(blob, xyz, L)
    assert data[7] == L - t_off
    want = O.decode(blob, data, xyz.shape[0])
    for _ in range(3):  # the second decode on runs the captured graphs
        assert np.array_equal(cod.decode(data).cpu().numpy(), want)


@pytest.mark.parametrize("host_coding", [False, True], ids=["device_rc", "host_rc"])
@pytest.mark.parametrize("arch,t_off", VARIANTS, ids=IDS)
def test_batch_mixed_depths(lpc, arch, t_off, host_coding):
    """Depths 6..19, a tiny and an empty frame in one batch: each stream is
    the oracle's stream of that frame alone, and the batch decodes exactly."""
    blob = synth.make_blob(arch=arch, t_off=t_off)
    specs = [(300, 6, 1), (0, 12, 2), (4000, 19, 3), (1, 9, 4), (20000, 16, 5), (7000, 13, 7)]
    frames = [synth.random_cloud(n, L, s) for n, L, s in specs]
    Ls = [L for _, L, _ in specs]
    cod = lpc.Codec(blob, 19, 20000, max_frames=len(frames), chunk=1000,
                    host_coding=host_coding)
    for _ in range(2):
        outs = cod.encode_batch([_cuda(f) for f in frames], Ls)
        assert outs == [O.encode(blob, f, L, 1000) for f, L in zip(frames, Ls)]
        decs = cod.decode_batch(outs, [max(f.shape[0], 1) for f in frames])
        for f, L, dcd in zip(frames, Ls, decs):
            assert np.array_equal(O.leaf_keys(dcd.cpu().numpy(), L), O.leaf_keys(f, L))


def test_full_size_frame_baseline(lpc):
    """The 64-beam frame at depth 16 with the baseline (kernel maps and
    ResBlocks at four levels, the deepest at L - 2) and with GRED, t = L - 3."""
    xyz = synth.make_frame(synth.C2)
    L = synth.C2.L
    for arch, t_off in ((synth.ARCH_BASE, 4), (synth.ARCH_GRED, 3)):
        blob = synth.make_blob(arch=arch, t_off=t_off)
        cod = lpc.Codec(blob, L, xyz.shape[0])
        data = cod.encode(_cuda(xyz))
        assert data == O.encode(blob, xyz, L)
        dec = cod.decode(data).cpu().numpy()
        assert np.array_equal(O.leaf_keys(dec, L), O.leaf_keys(xyz, L))


def test_stream_of_another_architecture_is_refused(lpc):
    xyz = synth.random_cloud(3000, 11, 9)
    a = synth.make_blob(arch=synth.ARCH_GRED)
    b = synth.make_blob(arch=synth.ARCH_BASE)
    data = lpc.Codec(a, 11, 3000).encode(_cuda(xyz))
    with pytest.raises(lpc.LpcError) as e:
        lpc.Codec(b, 11, 3000).decode(data)
    assert e.value.status == lpc.WEIGHTS_MISMATCH


def test_batch_two_groups_ablation(lpc):
    """Ten frames (the decoder's two-group path: host coarse decoding of one
    group beside the device's network levels of the other) with GRED only
    and t = L - 3: every stream equals the oracle's, the batch decodes
    exactly."""
    blob = synth.make_blob(arch=synth.ARCH_GRED, t_off=3)
    specs = [(2000 + 700 * i, 9 + i % 8, 90 + i) for i in range(10)]
    frames = [synth.random_cloud(n, L, s) for n, L, s in specs]
    Ls = [L for _, L, _ in specs]
    cod = lpc.Codec(blob, 16, max(f.shape[0] for f in frames), max_frames=len(frames))
    for _ in range(2):
        outs = cod.encode_batch([_cuda(f) for f in frames], Ls)
        assert outs == [O.encode(blob, f, L) for f, L in zip(frames, Ls)]
        decs = cod.decode_batch(outs, [f.shape[0] for f in frames])
        for f, L, dcd in zip(frames, Ls, decs):
            assert np.array_equal(O.leaf_keys(dcd.cpu().numpy(), L), O.leaf_keys(f, L))
