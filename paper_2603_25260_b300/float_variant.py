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
