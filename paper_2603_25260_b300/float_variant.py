"""The float inference variant (the paper's "Ours (Float)" rows, Sec. 4; the
motivation of Sec. 1 / Fig. 2): the same network in floating point, its
logits turned into 16-bit cumulative tables with a float softmax.

The tables come from `torch.softmax` on whatever device holds the logits, so
two devices (or two kernels) that round one exp or one sum differently give
different tables, and a stream coded with one table set cannot be decoded
with the other.  The integer path has no such dependence: its tables are a
function of the integer logits only, identical on the GPU and in the CPU
oracle.
"""

from __future__ import annotations

import numpy as np
import torch

FREQ_TOTAL = 1 << 16
N_SYMBOLS = 255


def float_cdf(logits: torch.Tensor) -> torch.Tensor:
    """u16 table rows [N, 256] (entry s = C_{s+1} for s < 254, then 0xFFFF)
    from float logits [N, 255]: f_s = 1 + floor(p_s (2^16 - 255)) with the
    remainder on the first maximum, computed on the logits' device."""
    p = torch.softmax(logits.float(), dim=1)
    f = 1 + torch.floor(p * (FREQ_TOTAL - N_SYMBOLS)).to(torch.int64)
    rem = FREQ_TOTAL - f.sum(dim=1)
    first = torch.argmax(logits.float(), dim=1)  # lowest index of the maximum
    f[torch.arange(f.shape[0], device=f.device), first] += rem
    c = torch.cumsum(f, dim=1)
    rows = torch.full((f.shape[0], 256), 0xFFFF, dtype=torch.int64, device=f.device)
    rows[:, :254] = c[:, :254]
    return rows.to(torch.int32)


def cross_device_decode(logits: dict, codes: dict, chunk: int = 256) -> dict:
    """The paper's cross-platform failure (Sec. 1, Fig. 1b/c) on the float
    variant: each network level's true symbols are range coded with the
    tables the GPU's softmax makes from the float logits, in substreams of
    `chunk` nodes as the codec does, and every substream is decoded twice:
    with those same tables (the decoder on the same device: must round trip)
    and with the tables the CPU's softmax makes from the same logits (the
    decoder on another device).  logits: {d: float [N_d, 255] on the GPU};
    codes: {d: u8 occupancy codes [N_d]} (symbol = code - 1).  Returns per
    level the rows whose tables differ, the substreams whose decode reports a
    corrupt stream or returns other symbols, and the symbols that come out
    wrong; `cloud_differs` is true when any level decodes wrong (its
    children, and so the decoded cloud, then differ)."""
    from . import lpc

    out = {"levels": {}, "cloud_differs": False, "same_device_round_trip": True}
    for d in sorted(logits):
        g = float_cdf(logits[d]).cpu().numpy().astype(np.uint16)
        c = float_cdf(logits[d].cpu()).numpy().astype(np.uint16)
        syms = (codes[d].cpu().numpy().astype(np.int64) - 1).astype(np.uint8)
        n = syms.shape[0]
        bad_sub = corrupt = wrong = 0
        first = -1
        nbytes = 0
        for s0 in range(0, n, chunk):
            s1 = min(n, s0 + chunk)
            data = lpc.rc_encode_rows(g[s0:s1], syms[s0:s1])
            nbytes += len(data)
            st, same = lpc.rc_decode_rows(g[s0:s1], data)
            if st != lpc.OK or not np.array_equal(same, syms[s0:s1]):
                out["same_device_round_trip"] = False
            st, other = lpc.rc_decode_rows(c[s0:s1], data)
            diff = np.nonzero(other != syms[s0:s1])[0]
            if st != lpc.OK or diff.size:
                bad_sub += 1
                corrupt += int(st != lpc.OK)
                wrong += int(diff.size)
                if first < 0 and diff.size:
                    first = s0 + int(diff[0])
        out["levels"][int(d)] = {
            "nodes": int(n), "rows_differing": int((g != c).any(axis=1).sum()),
            "substreams": -(-n // chunk), "substreams_failing": bad_sub,
            "substreams_reported_corrupt": corrupt, "symbols_wrong": wrong,
            "first_wrong_symbol": first, "bytes": nbytes}
        out["cloud_differs"] |= bad_sub > 0
    return out
