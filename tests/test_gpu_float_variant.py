"""The float inference variant against the integer path (the paper's
motivation, Sec. 1 and Fig. 2): float tables depend on the device that
computes the softmax, integer tables do not."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_25260_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2603_25260_b300 import build, float_variant, lpc, train
    build.build()
    return lpc, train, float_variant


def test_float_tables_device_dependent_integer_tables_not(mods):
    lpc, TR, FV = mods
    spec = synth.C1
    xyz = synth.make_frame(spec)
    L = spec.L
    fr = TR.Frame(torch.from_numpy(xyz).cuda(), L)
    model = TR.QATModel(synth.twin_params(0), qat=False, bf16=False)
    with torch.no_grad():
        logits = model.level_logits(fr)
    assert sorted(logits) == list(range(L - 5, L))
    rows = differ = 0
    for d, lg in logits.items():
        assert lg.shape == (fr.N[d], 255)
        g = FV.float_cdf(lg).cpu()
        c = FV.float_cdf(lg.cpu())
        for t in (g, c):  # valid tables: increasing, last real entry below 2^16
            assert bool((t[:, 1:254] > t[:, :253]).all()) and bool((t[:, 253] < 65536).all())
        differ += int((g != c).any(dim=1).sum())
        rows += lg.shape[0]
    print(f"float tables: {differ} of {rows} rows differ between the GPU and the CPU softmax")
    # the integer tables: the GPU codec and the CPU oracle agree on every row
    blob = synth.make_blob()
    cod = lpc.Codec(blob, L, xyz.shape[0])
    x = torch.from_numpy(xyz).cuda()
    for d in range(L - 5, L):
        assert np.array_equal(lpc.u16(cod.probs_level(x, d)), O.probs_level(blob, xyz, L, d))


def test_float_cdf_closed_forms(mods):
    """Equal logits give 1 + floor((2^16 - 255) / 255) = 257 per symbol and
    the remainder (1) on symbol 0; one dominant logit takes all but the floor
    of 1 per symbol."""
    _, _, FV = mods
    lg = torch.zeros(2, 255, device="cuda")
    lg[1, 17] = 80.0
    t = FV.float_cdf(lg).cpu().numpy().astype(np.int64)
    f0 = np.diff(np.concatenate([[0], t[0, :254], [65536]]))
    assert f0[0] == 258 and (f0[1:] == 257).all()
    f1 = np.diff(np.concatenate([[0], t[1, :254], [65536]]))
    assert f1[17] == 65536 - 254 and (np.delete(f1, 17) == 1).all()


def test_float_stream_fails_across_devices_integer_stream_does_not(mods):
    """The paper's cross-platform failure (Sec. 1, Fig. 1b/c) shown on the
    float variant of the 64-beam frame: a stream range coded with the tables
    of the GPU's float softmax decodes exactly with those tables, but the
    tables the CPU's softmax makes from the very same logits decode it wrong
    (a corrupt stream or other occupancy codes, so another cloud).  The
    integer path's stream of the same frame is the CPU oracle's byte for
    byte, and the oracle decodes it to the GPU decoder's voxels."""
    lpc, TR, FV = mods
    spec = synth.C2
    xyz = synth.make_frame(spec)
    L, n = spec.L, xyz.shape[0]
    fr = TR.Frame(torch.from_numpy(xyz).cuda(), L)
    model = TR.QATModel(synth.twin_params(0), qat=False, bf16=False)
    with torch.no_grad():
        logits = model.level_logits(fr)
    r = FV.cross_device_decode(logits, fr.codes)
    print(r)
    assert r["same_device_round_trip"]
    levels = r["levels"].values()
    assert sum(v["rows_differing"] for v in levels) > 0
    assert r["cloud_differs"]
    assert sum(v["symbols_wrong"] + v["substreams_reported_corrupt"] for v in levels) > 0
    for v in levels:  # where every row agrees, the other device decodes it too
        if v["rows_differing"] == 0:
            assert v["substreams_failing"] == 0
    blob = synth.make_blob()
    cod = lpc.Codec(blob, L, n, chunk=256)
    data = cod.encode(torch.from_numpy(xyz).cuda())
    assert data == O.encode(blob, xyz, L, 256)
    assert np.array_equal(cod.decode(data).cpu().numpy(), O.decode(blob, data, n))
