"""The codec's host range coder (the coarse levels' coder, and the network
levels' coder in host-coding mode), called through its C-ABI entry points on
caller tables.  It makes no CUDA calls, so these checks run on the CPU: its
substreams equal the oracle's byte for byte (stream version 3 framing) and
round trip; a cut stream is reported corrupt."""

import numpy as np
import pytest

import oracle as O
from paper_2603_25260_b300 import lpc, synth


def _rows(n, seed, sigma=40):
    rng = np.random.Generator(np.random.PCG64(seed))
    lg = np.clip(rng.normal(0, sigma, size=(n, 255)), -128, 127).astype(np.int8)
    return O.softmax_cdf(lg, synth.exp_lut())


@pytest.mark.parametrize("n,seed,sigma", [(0, 1, 40), (1, 2, 40), (700, 3, 40), (5000, 4, 8),
                                          (3000, 5, 200)])
def test_host_table_coder_matches_oracle(n, seed, sigma):
    rows = _rows(max(n, 1), seed, sigma)[:n]
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    syms = rng.integers(0, 255, size=n).astype(np.uint8)
    data = lpc.rc_encode_rows(rows, syms)
    assert data == O.rc_encode_cdf(rows, syms)
    st, got = lpc.rc_decode_rows(rows, data)
    assert st == lpc.OK and np.array_equal(got, syms)


def test_host_table_coder_cut_stream_is_corrupt():
    rows = _rows(2000, 9)
    syms = np.random.Generator(np.random.PCG64(10)).integers(0, 255, 2000).astype(np.uint8)
    data = lpc.rc_encode_rows(rows, syms)
    for cut in (5, 100, len(data) // 2):
        st, _ = lpc.rc_decode_rows(rows, data[:-cut])
        assert st == lpc.CORRUPT_STREAM


def test_host_table_coder_rejects_bad_symbol():
    rows = _rows(3, 11)
    with pytest.raises(lpc.LpcError):
        lpc.rc_encode_rows(rows, np.array([0, 255, 3], np.uint8))
