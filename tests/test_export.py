"""Integer blob export of the quantisation-aware twin (CPU): the exported
blob is valid, and the integer network it defines (run by the oracle) codes
each level at the rate the twin's fake-quantised float network predicts."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import train_ref as T
from paper_2603_25260_b300 import export, synth


@pytest.fixture(scope="module")
def setup():
    spec = synth.GRADCHECK
    xyz = synth.make_frame(spec)
    return xyz, spec.L, T.Frame(xyz, spec.L)


def _ideal_bits(blob, xyz, L, d, codes):
    cdf = O.probs_level(blob, xyz, L, d).astype(np.int64)
    C = np.concatenate([np.zeros((len(cdf), 1), np.int64), cdf[:, :254],
                        np.full((len(cdf), 1), 65536, np.int64)], 1)
    s = codes.astype(np.int64) - 1
    f = C[np.arange(len(s)), s + 1] - C[np.arange(len(s)), s]
    return float(-np.log2(f / 65536.0).sum())


def test_export_blob_is_valid():
    blob = export.quantize_twin(synth.twin_params(3))
    assert O.check_blob(blob) == 0


@pytest.mark.parametrize("seed", [0, 5])
def test_integer_rate_matches_twin(setup, seed):
    """The integer tables' ideal code length over the five network levels
    with the exported blob is within 3 % of the twin's cross-entropy (fake
    quantisers on).  The predictors' last biases are set to the log
    frequencies of the frame's codes, so the predictions are far from
    uniform (about 5 bits per node instead of 8) and a wrong logit scale
    moves the rate by about 50 %."""
    xyz, L, fr = setup
    ok, oc = O.build_levels(xyz, L)
    P = {k: v.copy() for k, v in synth.twin_params(seed).items()}
    allc = np.concatenate([oc[d] for d in range(L - 5, L)]).astype(np.int64)
    freq = np.bincount(allc - 1, minlength=255)[:255] + 0.5
    for j in range(5):
        P[f"P2_{j}.b"] = np.log(freq / freq.sum()).astype(np.float32)
    blob = export.quantize_twin(P)
    Pt = T.to_torch(P, requires_grad=False)
    total_twin = float(T.level_bits(Pt, fr, qat=True))
    total_int = 0.0
    for d in range(L - 5, L):
        total_int += _ideal_bits(blob, xyz, L, d, oc[d])
    assert total_int == pytest.approx(total_twin, rel=0.03)


def test_export_scales():
    """Closed forms of the per-layer constants on a hand-made parameter set."""
    P = synth.twin_params(1)
    P = {k: v.copy() for k, v in P.items()}
    W = P["P1_0.W"]
    W[:] = 0.0
    W[0, 0] = 0.254  # s_w = 0.002
    P["P1_0.b"][:] = 0.001
    P["P1_0.a"][:] = 0.25
    blob = export.quantize_twin(P)
    # parse the blob: header 32 B, LUT 1 KB, then records in network order
    off = 32 + 1024
    C = 32
    for (name, kind, S, cin, cout, prelu, _, _) in synth.network_records(C):
        hdr = np.frombuffer(blob[off:off + 48], dtype="<i4")
        off += 48

        def take(nbytes):
            nonlocal off
            b = blob[off:off + nbytes]
            off += nbytes + (-nbytes) % 16
            return b
        if kind in (synth.KIND_SUM, synth.KIND_SELECT):
            rows = S if kind == synth.KIND_SELECT else 1
            Wq = np.frombuffer(take(S * cout * cin), dtype=np.int8)
            bias = np.frombuffer(take(4 * rows * cout), dtype="<i4")
            mult = np.frombuffer(take(4 * rows * cout), dtype="<i4")
            slope = np.frombuffer(take(2 * rows * cout), dtype="<i2")
            if name == "P1_0":
                assert hdr[7] == 24  # shift
                assert Wq[0] == 127 and np.count_nonzero(Wq) == 1
                # b / (s_w s_a) = 0.001 / (0.002 / 32) = 16
                assert np.all(bias == 16)
                # s_w s_a / s_a 2^24 = 0.002 * 2^24
                assert np.all(mult == round(0.002 * (1 << 24)))
                assert np.all(slope == 8192)
                return
        elif kind == synth.KIND_EMBED:
            take(256 * cout)
        else:
            take(4 * 2 * cout)
            take(2 * cout)
    pytest.fail("P1_0 not found")
