"""Integer weight blob from the parameters of the quantisation-aware twin.

The paper trains the network in floating point with fake quantisers and
deploys it with integer arithmetic only (Sec. 3.3, Eq. 12-14; supplement,
Training).  The twin (``train.QATModel``) quantises every INT8 activation
with the fixed scale s_a = 1/32 (zero point 0) and every weight tensor
symmetrically with s_w = max|W| / 127; the export turns each layer into the
blob record the integer codec reads:

- weights      W_q = clip(round(W / s_w), -127, 127);
- bias         b_q = round(b / (s_w s_a)), in units of the accumulator;
- multiplier   m = round(s_w s_a / s_out 2^r) with r = 24: requantisation
  (Eq. 14) maps the accumulator to the output scale s_out = s_a, or to the
  logit scale s_l = 1/16 nat per step of the exp table for the predictor's
  last layer;
- PReLU slope  round(a 2^15) (Q15; PReLU commutes with the positive scale,
  so it acts on the accumulator);
- residual merge (the ResBlock reading): round(m_a 2^15), round(m_b 2^15) with a 15-bit
  rounding shift, inputs and output at s_a;
- embeddings   clip(round(E / s_a), -128, 127).

``python -m paper_2603_25260_b300.export --steps N --out PATH`` trains the
twin for N AdamW steps on the seeded 8-frame training batch of the 64-beam
generator (rate loss in bits per point, fake quantisers on) and writes the
blob; ``--arch gred|baseline`` and ``--t-off 3`` train and export the
ablation architectures of Sec. 4.3 instead.
"""

from __future__ import annotations

import argparse
import os

import numpy as np

from . import synth

# A blob exported after 400 steps (lr 1e-3, seed 0) of
# `python -m paper_2603_25260_b300.export --steps 400 --out <path>`: 34.7 ->
# 13.1 bits per point on the network levels of the training batch.
TRAINED_BLOB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                            "trained_synth_c32.blob")

ACT_SCALE = 1.0 / 32.0
LOGIT_SCALE = 1.0 / 16.0  # the exp table's step (synth.exp_lut)
SHIFT = 24


def _wq(W: np.ndarray) -> tuple[np.ndarray, float]:
    s = max(float(np.abs(W).max()), 1e-12) / 127.0
    return np.clip(np.round(W / s), -127, 127).astype(np.int8), s


def _q15(a: np.ndarray) -> np.ndarray:
    return np.clip(np.round(np.asarray(a, dtype=np.float64) * 32768.0), -32768, 32767).astype(np.int16)


def quantize_twin(P: dict, C: int = 32, arch: int = synth.ARCH_XFP, t_off: int = 4) -> bytes:
    """The integer blob of twin parameters P (name -> float array) of the
    given architecture."""
    P = {k: np.asarray(v, dtype=np.float64) for k, v in P.items()}
    recs = []
    for (name, kind, S, cin, cout, prelu, ins, out) in synth.network_records(C, arch, t_off):
        rec = synth.Record(name, kind, S, cin, cout, prelu)  # every zero point is 0
        if kind == synth.KIND_EMBED:
            tab = np.clip(np.round(P[name] / ACT_SCALE), -128, 127)
            tab[0, :] = 0  # code 0 never occurs
            rec.W = tab.astype(np.int8)
        elif kind in (synth.KIND_SUM, synth.KIND_SELECT):
            Wq, sw = _wq(P[name + ".W"])
            rec.W = Wq.reshape(S, cout, cin)
            rows = S if kind == synth.KIND_SELECT else 1
            b = np.broadcast_to(P[name + ".b"].reshape(-1, cout), (rows, cout))
            rec.shift = SHIFT
            s_out = LOGIT_SCALE if name.startswith("P2_") else ACT_SCALE
            rec.bias = np.clip(np.round(b / (sw * ACT_SCALE)), -(1 << 30) + 1,
                               (1 << 30) - 1).astype(np.int32)
            m = round(sw * ACT_SCALE / s_out * (1 << SHIFT))
            rec.mult = np.full((rows, cout), min(max(m, 1), (1 << 31) - 1), dtype=np.int32)
            if prelu:
                rec.slope = np.broadcast_to(_q15(P[name + ".a"]), (rows, cout)).copy()
            else:
                rec.slope = np.zeros((rows, cout), dtype=np.int16)
        else:  # residual merge
            rec.shift = 15
            ma = np.clip(np.round(P[name + ".ma"] * 32768.0), 0, (1 << 16) - 1)
            mb = np.clip(np.round(P[name + ".mb"] * 32768.0), 0, (1 << 16) - 1)
            rec.mult = np.stack([ma, mb]).astype(np.int32)
            rec.slope = _q15(P[name + ".a"])
        recs.append(rec)
    return synth.pack_blob(recs, synth.exp_lut(LOGIT_SCALE), C, arch, t_off)


def train(steps: int, lr: float = 1e-3, seed: int = 0, log_every: int = 50,
          arch: int = synth.ARCH_XFP, t_off: int = 4) -> tuple[dict, list]:
    """AdamW on the rate loss of the 8-frame training batch, fake quantisers
    and fp32 operands, for one architecture; returns the parameters and the
    loss history."""
    import torch

    from . import train as T

    specs = synth.training_specs()
    frames = [T.BatchFrame([T.Frame(torch.from_numpy(synth.make_frame(s)).cuda(), s.L)
                            for s in specs])]
    model = T.QATModel(synth.twin_params(seed, arch=arch, t_off=t_off), qat=True, bf16=False,
                       arch=arch, t_off=t_off)
    opt = torch.optim.AdamW(model.parameters(), lr=lr, weight_decay=1e-4)
    hist = []
    for k in range(steps):
        loss = T.train_step(model, opt, frames)
        hist.append(loss)
        if log_every and (k % log_every == 0 or k == steps - 1):
            print(f"step {k}: {loss:.4f} bits/point (network levels)", flush=True)
    params = {n: model.P(n).detach().cpu().numpy().astype(np.float32) for n in model.names}
    return params, hist


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--arch", choices=sorted(synth.ARCHS), default="gred_xfp")
    ap.add_argument("--t-off", type=int, choices=(3, 4), default=4)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    arch = synth.ARCHS[a.arch]
    params, hist = train(a.steps, a.lr, a.seed, arch=arch, t_off=a.t_off)
    blob = quantize_twin(params, arch=arch, t_off=a.t_off)
    with open(a.out, "wb") as f:
        f.write(blob)
    np.savez(a.out + ".params.npz", **params)
    print(f"wrote {a.out} ({len(blob)} bytes); loss {hist[0]:.3f} -> {hist[-1]:.3f} "
          f"bits/point over {len(hist)} steps")


if __name__ == "__main__":
    main()
