"""Seeded synthetic inputs: spinning-LiDAR frames and integer weight blobs.

This module generates inputs only.  It holds none of the codec's arithmetic
(no octree, no network, no softmax, no entropy coding) and it is the one
module that both the CPU oracle's tests and the CUDA path's tests draw their
inputs from.

Frames stand in for the KITTI and Ford scans the paper evaluates on
(Sec. 4.1), which are not available here.  A frame is a ray cast of a
spinning multi-beam sensor at the origin against a seeded scene (ground plane,
axis-aligned boxes, vertical cylinders), then quantised to a 2^L grid over a
cube centred on the sensor, following the coordinate quantisation of the
supplement ("Quantization of KITTI Dataset": normalise into a cube, scale by
2^L, quantise).

Weight blobs carry every integer parameter of the network (INT8 weights,
INT32 biases, fixed-point multipliers and shifts, zero points, Q15 PReLU
slopes, and the exp lookup table of the integer softmax, Sec. 3.3).  The
paper's trained weights are not available, so the blob is drawn from a seeded
generator with analytic scales that keep activations in range.

Blob layout (little endian):
  header (32 B): "LPCW", u32 version=1, u32 C, u32 n_records, u32 lut_len=256,
                 u32 arch (0 GRED + XFP, 1 GRED only, 2 baseline), u32 t_off (t = L - t_off;
                 3 or 4, 0 reads as 4), u32 pad
  u32 lut[256]                     exp table over the non-positive domain, lut[0] = 2^16
  n_records x record, in network order (see ``network_records``); each record is
  a 48-byte header  u32 kind, S, cin, cout; i32 z_in, z_in2, z_out, shift;
  u32 flags (bit0 = PReLU); 3 x u32 pad; followed by 16-byte padded arrays:
    kind 1 (summed slices: sparse 3x3x3 conv S = 27, stride-2 down conv S = 8,
            plain linear S = 1; one output row sums slice products):
        i8 W[S][cout][cin], i32 bias[cout], i32 mult[cout], i16 slope[cout]
    kind 2 (occupancy-code embedding, cin = 256 table rows):
        i8 table[256][cout]
    kind 3 (residual merge, S = 2, cin = cout):
        i32 mult[2][cout] (the two branch multipliers), i16 slope[cout]
    kind 4 (selected slices: the 8x channel-expanding up-sampling linear layer;
            child c of a parent uses slice c only):
        i8 W[S][cout][cin], i32 bias[S][cout], i32 mult[S][cout], i16 slope[S][cout]
"""

from __future__ import annotations

import dataclasses
import math
import struct

import numpy as np

# ----------------------------------------------------------------------------
# Frames
# ----------------------------------------------------------------------------

GROUND_Z = -1.73
MAX_RANGE = 80.0
RANGE_SIGMA = 0.02


@dataclasses.dataclass(frozen=True)
class FrameSpec:
    beams: int
    bins: int
    elev_lo: float  # degrees
    elev_hi: float
    n_boxes: int
    n_cyl: int
    dropout: float
    L: int
    cube: float  # metres
    seed: int
    target_points: int | None = None  # subsample to exactly this many (batched mix)


# The three single-frame workloads and the gradient-check frame.
C1 = FrameSpec(16, 512, -15.0, 15.0, 20, 10, 0.0, 12, 160.0, 1001)
C2 = FrameSpec(64, 2048, -24.8, 2.0, 60, 30, 0.10, 16, 160.0, 1002)
C3 = FrameSpec(128, 2048, -25.0, 15.0, 120, 60, 0.0, 18, 200.0, 1003)
GRADCHECK = FrameSpec(16, 128, -15.0, 15.0, 20, 10, 0.0, 10, 160.0, 4000)

_BEAM_FAMILIES = {
    16: (-15.0, 15.0, 20, 10, 0.0),
    64: (-24.8, 2.0, 60, 30, 0.10),
    128: (-25.0, 15.0, 120, 60, 0.0),
}


def batch_specs(n_frames: int = 64, base_seed: int = 2000) -> list[FrameSpec]:
    """The mixed-size batch: beams drawn from {16, 64, 128}, target point
    counts log-uniform in [8k, 230k], depth uniform in 12..18."""
    out = []
    for i in range(n_frames):
        seed = base_seed + i
        rng = np.random.Generator(np.random.PCG64(seed + 10_000_000))
        beams = int(rng.choice([16, 64, 128]))
        lo, hi, nb, nc, drop = _BEAM_FAMILIES[beams]
        target = int(round(math.exp(rng.uniform(math.log(8000), math.log(230000)))))
        bins = int(min(max(round(target / (beams * 0.9)), 256), 8192))
        L = int(rng.integers(12, 19))
        cube = 160.0 if L <= 16 else 200.0
        out.append(FrameSpec(beams, bins, lo, hi, nb, nc, drop, L, cube, seed, target))
    return out


def training_specs() -> list[FrameSpec]:
    return [dataclasses.replace(C2, seed=3000 + i) for i in range(8)]


def _scene(rng: np.random.Generator, n_boxes: int, n_cyl: int):
    def centres(n):
        # uniform in the disc r <= 50 m, rejecting r < 4 m
        xs = []
        while len(xs) < n:
            r = math.sqrt(rng.uniform(0.0, 1.0)) * 50.0
            if r < 4.0:
                continue
            a = rng.uniform(0.0, 2 * math.pi)
            xs.append((r * math.cos(a), r * math.sin(a)))
        return np.array(xs, dtype=np.float64).reshape(n, 2)

    bc = centres(n_boxes)
    sides = rng.uniform(1.0, 5.0, size=(n_boxes, 3))
    bmin = np.stack([bc[:, 0] - sides[:, 0] / 2, bc[:, 1] - sides[:, 1] / 2,
                     np.full(n_boxes, GROUND_Z)], 1)
    bmax = np.stack([bc[:, 0] + sides[:, 0] / 2, bc[:, 1] + sides[:, 1] / 2,
                     GROUND_Z + sides[:, 2]], 1)
    cc = centres(n_cyl)
    cr = rng.uniform(0.1, 0.5, size=n_cyl)
    ch = rng.uniform(1.0, 6.0, size=n_cyl)
    return bmin, bmax, cc, cr, ch


def _cast(dirs: np.ndarray, bmin, bmax, cc, cr, ch) -> np.ndarray:
    """Nearest positive hit distance along unit rays from the origin (inf = miss)."""
    n = dirs.shape[0]
    t = np.full(n, np.inf)
    dz = dirs[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = np.where(dz < -1e-9, GROUND_Z / dz, np.inf)
    t = np.minimum(t, np.where(tg > 0, tg, np.inf))
    inv = np.where(np.abs(dirs) > 1e-12, 1.0 / np.where(np.abs(dirs) > 1e-12, dirs, 1.0), np.inf)
    for i in range(bmin.shape[0]):
        with np.errstate(invalid="ignore"):
            t1 = bmin[i][None, :] * inv
            t2 = bmax[i][None, :] * inv
        tlo = np.nanmax(np.minimum(t1, t2), axis=1)
        thi = np.nanmin(np.maximum(t1, t2), axis=1)
        hit = (thi >= tlo) & (thi > 0)
        th = np.where(tlo > 0, tlo, thi)
        t = np.where(hit & (th < t), th, t)
    dx, dy = dirs[:, 0], dirs[:, 1]
    a = dx * dx + dy * dy
    for i in range(cc.shape[0]):
        cx, cy = cc[i]
        bq = -2.0 * (dx * cx + dy * cy)
        cq = cx * cx + cy * cy - cr[i] * cr[i]
        disc = bq * bq - 4 * a * cq
        ok = (disc >= 0) & (a > 1e-12)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        with np.errstate(divide="ignore", invalid="ignore"):
            r1 = (-bq - sq) / (2 * a)
            r2 = (-bq + sq) / (2 * a)
        for th in (r1, r2):
            z = th * dz
            good = ok & (th > 0) & (z >= GROUND_Z) & (z <= GROUND_Z + ch[i]) & (th < t)
            t = np.where(good, th, t)
    return t


def lidar_points(spec: FrameSpec) -> np.ndarray:
    """Float64 [n, 3] points of one synthetic sweep."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    bmin, bmax, cc, cr, ch = _scene(rng, spec.n_boxes, spec.n_cyl)
    elev = np.deg2rad(np.linspace(spec.elev_lo, spec.elev_hi, spec.beams))
    az = 2 * np.pi * np.arange(spec.bins) / spec.bins
    E, A = np.meshgrid(elev, az, indexing="ij")
    dirs = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    ts = []
    for s in range(0, dirs.shape[0], 16384):
        ts.append(_cast(dirs[s:s + 16384], bmin, bmax, cc, cr, ch))
    t = np.concatenate(ts)
    t = t + rng.normal(0.0, RANGE_SIGMA, size=t.shape)
    keep = np.isfinite(t) & (t > 0) & (t <= MAX_RANGE)
    if spec.dropout > 0:
        keep &= rng.uniform(size=t.shape) >= spec.dropout
    pts = dirs[keep] * t[keep, None]
    if spec.target_points is not None and pts.shape[0] > spec.target_points:
        idx = rng.choice(pts.shape[0], size=spec.target_points, replace=False)
        pts = pts[np.sort(idx)]
    return pts


def quantize(points: np.ndarray, L: int, cube: float) -> np.ndarray:
    """Grid coordinates in [0, 2^L): floor((p + S/2) / S * 2^L), clamped, cube
    of side S centred on the sensor.  Duplicates are kept (the codec removes them)."""
    q = np.floor((points + cube / 2.0) / cube * float(1 << L))
    q = np.clip(q, 0, (1 << L) - 1)
    return np.ascontiguousarray(q.astype(np.int32))


def make_frame(spec: FrameSpec) -> np.ndarray:
    """int32 [n, 3] quantised coordinates for one frame."""
    return quantize(lidar_points(spec), spec.L, spec.cube)


def make_frames(specs: list[FrameSpec], workers: int | None = None) -> list[np.ndarray]:
    """make_frame for many specs on a thread pool (the ray caster's array
    operations release the GIL); every frame has its own seeded generator, so
    the result does not depend on the number of workers."""
    import concurrent.futures as cf
    import os

    workers = workers or min(len(specs), os.cpu_count() or 1)
    if workers <= 1 or len(specs) <= 1:
        return [make_frame(s) for s in specs]
    with cf.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(make_frame, specs))


def random_cloud(n: int, L: int, seed: int, clustered: bool = True) -> np.ndarray:
    """Small random int32 [n, 3] clouds for unit tests (optionally clustered so
    that 3x3x3 neighbourhoods are populated)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = 1 << L
    if not clustered or n == 0:
        return rng.integers(0, side, size=(n, 3), dtype=np.int64).astype(np.int32)
    k = max(1, n // 64)
    centres = rng.integers(0, side, size=(k, 3))
    which = rng.integers(0, k, size=n)
    spread = max(1.0, side / 64.0)
    pts = centres[which] + np.round(rng.normal(0.0, spread, size=(n, 3)))
    return np.clip(pts, 0, side - 1).astype(np.int32)


# ----------------------------------------------------------------------------
# Weight blob
# ----------------------------------------------------------------------------

KIND_SUM, KIND_EMBED, KIND_RESADD, KIND_SELECT = 1, 2, 3, 4
N_REL_LEVELS = 5
N_SYMBOLS = 255


@dataclasses.dataclass
class Record:
    name: str
    kind: int
    S: int
    cin: int
    cout: int
    prelu: bool
    z_in: int = 0
    z_in2: int = 0
    z_out: int = 0
    shift: int = 0
    W: np.ndarray | None = None
    bias: np.ndarray | None = None
    mult: np.ndarray | None = None
    slope: np.ndarray | None = None


# Architectures: the paper's model and the two ablations of Sec. 4.3 (Table 4),
# all on the same five network-coded levels b = L-5 .. L-1 and the same ops.
ARCH_XFP = 0   # GRED + XFP (Sec. 3.1-3.2, Eq. 4-11)
ARCH_GRED = 1  # GRED only: no feature propagated between levels
ARCH_BASE = 2  # neither: every level's features extracted at its parent level
ARCHS = {"gred_xfp": ARCH_XFP, "gred": ARCH_GRED, "baseline": ARCH_BASE}


def check_arch(arch: int, t_off: int) -> None:
    if arch not in (ARCH_XFP, ARCH_GRED, ARCH_BASE) or t_off not in (3, 4):
        raise ValueError(f"architecture {arch} with t = L - {t_off} is not defined")


def dense_span(arch: int, t_off: int, j: int) -> int:
    """m = d - k: the number of up-sampling steps from the level k whose
    features a non-propagating level d = b + j (j >= 1) extracts.  GRED
    re-densifies the levels below t to k = t (Eq. 4-6); the baseline and the
    levels down to t extract at k = d - 1."""
    d_minus_t = j - (5 - t_off)
    return d_minus_t if (arch == ARCH_GRED and d_minus_t > 0) else 1


def network_records(C: int, arch: int = ARCH_XFP, t_off: int = 4) -> list[tuple]:
    """(name, kind, S, cin, cout, prelu, input tensor(s), output tensor) in blob order.

    Tensor names are used only to give every activation tensor one zero point,
    shared by its producers and consumers (concatenated halves share one)."""
    check_arch(arch, t_off)
    n_sh = 5 - t_off  # relative levels 1..n_sh lie at or above t
    r = []
    # j = 0 : level b, shallow, no ResBlock input yet (coarse levels are frequency coded)
    r += [("E_0", KIND_EMBED, 1, 256, C, False, ("X0",), "X0"),
          ("UP_0", KIND_SELECT, 8, C, C, True, ("X0",), "F_b"),
          ("P1_0", KIND_SUM, 1, C, C, True, ("F_b",), "h_0"),
          ("P2_0", KIND_SUM, 1, C, N_SYMBOLS, False, ("h_0",), "logit_0")]
    for j in range(1, N_REL_LEVELS):
        if arch == ARCH_XFP and j <= n_sh:
            # shallow level d <= t: S^{d-1} = ResBlock(F^{d-1});
            # F^d = Up(Concat(S^{d-1}, X^{d-1}))
            src = "F_b" if j == 1 else f"F_{j - 1}"
            dst = "Xt" if j == n_sh else f"F_{j}"
            r += [(f"RA_{j}", KIND_SUM, 27, C, C, True, (src,), f"y1_{j}"),
                  (f"RB_{j}", KIND_SUM, 27, C, C, False, (f"y1_{j}",), f"y2_{j}"),
                  (f"RM_{j}", KIND_RESADD, 2, C, C, True, (f"y1_{j}", f"y2_{j}"), f"X{j}"),
                  (f"E_{j}", KIND_EMBED, 1, 256, C, False, (f"X{j}",), f"X{j}"),
                  (f"UP_{j}", KIND_SELECT, 8, 2 * C, C, True, (f"X{j}",), dst),
                  (f"P1_{j}", KIND_SUM, 1, C, C, True, (dst,), f"h_{j}"),
                  (f"P2_{j}", KIND_SUM, 1, C, N_SYMBOLS, False, (f"h_{j}",), f"logit_{j}")]
            continue
        if arch == ARCH_XFP:
            # deep level t + m, re-densified to level t and fused with F^t
            m, cat, gk = j - n_sh, 2, "Xt"
        else:
            # no propagation: features of level d from X^{d-1} alone
            m, cat, gk = dense_span(arch, t_off, j), 1, f"gk_{j}"
        r.append((f"G_{j}", KIND_EMBED, 1, 256, C, False, (gk,) if m == 1 else (f"g_{j}_0",),
                  gk if m == 1 else f"g_{j}_0"))
        for i in range(1, m):
            src = f"g_{j}_{i - 1}"
            dst = gk if i == m - 1 else f"g_{j}_{i}"
            r.append((f"D_{j}_{i}", KIND_SUM, 8, C, C, True, (src,), dst))
        r += [(f"RA_{j}", KIND_SUM, 27, cat * C, C, True, (gk,), f"y1_{j}"),
              (f"RB_{j}", KIND_SUM, 27, C, C, False, (f"y1_{j}",), f"y2_{j}"),
              (f"RM_{j}", KIND_RESADD, 2, C, C, True, (f"y1_{j}", f"y2_{j}"), f"H_{j}_0")]
        for k in range(m):
            if cat == 2:
                r.append((f"E_{j}_{k}", KIND_EMBED, 1, 256, C, False, (f"H_{j}_{k}",),
                          f"H_{j}_{k}"))
            r.append((f"UP_{j}_{k}", KIND_SELECT, 8, cat * C, C, True, (f"H_{j}_{k}",),
                      f"H_{j}_{k + 1}"))
        r += [(f"P1_{j}", KIND_SUM, 1, C, C, True, (f"H_{j}_{m}",), f"h_{j}"),
              (f"P2_{j}", KIND_SUM, 1, C, N_SYMBOLS, False, (f"h_{j}",), f"logit_{j}")]
    return r


def exp_lut(logit_scale: float = 1.0 / 16.0) -> np.ndarray:
    """lut[i] = round(2^16 exp(-i * s)) for i = 0..255: the softmax numerator
    over the non-positive domain l - max(l) = -i (Sec. 3.3, integer softmax)."""
    i = np.arange(256, dtype=np.float64)
    lut = np.round(65536.0 * np.exp(-i * logit_scale)).astype(np.int64)
    lut[0] = 65536
    return lut.astype(np.uint32)


def make_blob_records(C: int = 32, seed: int = 7, act_sigma: float = 30.0, arch: int = ARCH_XFP,
                      t_off: int = 4) -> tuple[list[Record], np.ndarray]:
    rng = np.random.Generator(np.random.PCG64(seed))
    zp: dict[str, int] = {}

    def z_of(name):
        if name not in zp:
            zp[name] = int(rng.integers(-12, 13))
        return zp[name]

    sigma_w = 127.0 / math.sqrt(3.0)
    recs = []
    for (name, kind, S, cin, cout, prelu, ins, out) in network_records(C, arch, t_off):
        rec = Record(name, kind, S, cin, cout, prelu)
        rec.z_out = z_of(out)
        if kind == KIND_EMBED:
            rec.z_in = rec.z_out
            tab = np.round(rng.normal(rec.z_out, act_sigma, size=(256, cout)))
            tab[0, :] = rec.z_out
            rec.W = np.clip(tab, -128, 127).astype(np.int8)
        elif kind in (KIND_SUM, KIND_SELECT):
            rec.z_in = z_of(ins[0])
            P = S if kind == KIND_SELECT else 1
            if S == 27:
                fan = 27 * cin * 0.3
            elif S == 8 and name.startswith("D_"):
                fan = cin * 8 * 0.35
            else:
                fan = cin
            sigma_acc = math.sqrt(fan) * act_sigma * sigma_w
            target = act_sigma * (1.6 if prelu else 1.0)
            if name.startswith("P2_"):
                target = 24.0
            rec.shift = 24
            ratio = target / sigma_acc
            rec.W = rng.integers(-127, 128, size=(S, cout, cin)).astype(np.int8)
            rec.bias = np.clip(np.round(rng.normal(0.0, 0.3 * sigma_acc, size=(P, cout))),
                               -(1 << 29), 1 << 29).astype(np.int32)
            m = np.round((1 << rec.shift) * ratio * rng.uniform(0.8, 1.2, size=(P, cout)))
            rec.mult = np.clip(m, 1, (1 << 31) - 1).astype(np.int32)
            if prelu:
                rec.slope = np.round(rng.uniform(0.05, 0.35, size=(P, cout)) * 32768).astype(np.int16)
            else:
                rec.slope = np.zeros((P, cout), dtype=np.int16)
        else:  # residual merge
            rec.z_in = z_of(ins[0])
            rec.z_in2 = z_of(ins[1])
            rec.shift = 15
            m = np.round(32768 * 0.7 * rng.uniform(0.8, 1.2, size=(2, cout)))
            rec.mult = np.clip(m, 0, (1 << 16) - 1).astype(np.int32)
            rec.slope = np.round(rng.uniform(0.05, 0.35, size=(cout,)) * 32768).astype(np.int16)
        recs.append(rec)
    return recs, exp_lut()


def _pad16(b: bytes) -> bytes:
    return b + b"\0" * ((-len(b)) % 16)


def pack_blob(recs: list[Record], lut: np.ndarray, C: int, arch: int = ARCH_XFP,
              t_off: int = 4) -> bytes:
    check_arch(arch, t_off)
    out = [struct.pack("<4sIIIIII4x", b"LPCW", 1, C, len(recs), 256, arch,
                       0 if t_off == 4 else t_off)]
    out.append(lut.astype("<u4").tobytes())
    for r in recs:
        out.append(struct.pack("<IIIIiiiiI12x", r.kind, r.S, r.cin, r.cout, r.z_in, r.z_in2,
                               r.z_out, r.shift, 1 if r.prelu else 0))
        if r.kind in (KIND_SUM, KIND_SELECT):
            out.append(_pad16(r.W.astype(np.int8).tobytes()))
            out.append(_pad16(r.bias.astype("<i4").tobytes()))
            out.append(_pad16(r.mult.astype("<i4").tobytes()))
            out.append(_pad16(r.slope.astype("<i2").tobytes()))
        elif r.kind == KIND_EMBED:
            out.append(_pad16(r.W.astype(np.int8).tobytes()))
        else:
            out.append(_pad16(r.mult.astype("<i4").tobytes()))
            out.append(_pad16(r.slope.astype("<i2").tobytes()))
    return b"".join(out)


def make_blob(C: int = 32, seed: int = 7, arch: int = ARCH_XFP, t_off: int = 4) -> bytes:
    """The seeded weight blob (default: C = 32, seed 7, GRED + XFP, t = L - 4)."""
    recs, lut = make_blob_records(C, seed, arch=arch, t_off=t_off)
    return pack_blob(recs, lut, C, arch, t_off)


# ----------------------------------------------------------------------------
# Parameters of the differentiable twin (names, shapes, seeded initial values)
# ----------------------------------------------------------------------------

def twin_param_shapes(C: int = 32, arch: int = ARCH_XFP, t_off: int = 4) -> dict:
    """Parameter names and shapes of the twin: the float counterparts of the
    blob records, in record order (PReLU slopes per output channel)."""
    s = {}
    for (name, kind, S, cin, cout, prelu, _, _) in network_records(C, arch, t_off):
        if kind == KIND_EMBED:
            s[name] = (256, C)
        elif kind == KIND_RESADD:
            s[name + ".ma"] = (C,)
            s[name + ".mb"] = (C,)
            s[name + ".a"] = (C,)
        else:
            s[name + ".W"] = (S, cout, cin) if S > 1 else (cout, cin)
            s[name + ".b"] = (S, cout) if kind == KIND_SELECT else (cout,)
            if prelu:
                s[name + ".a"] = (cout,)
    return s


def twin_params(seed: int = 0, C: int = 32, arch: int = ARCH_XFP, t_off: int = 4) -> dict:
    """Seeded float parameters (numpy float32) for both implementations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, shape in twin_param_shapes(C, arch, t_off).items():
        if name.endswith(".W"):
            fan = shape[-1] * (shape[0] if len(shape) == 3 and shape[0] == 27 else 1)
            if len(shape) == 3 and shape[0] == 8 and name.startswith("D_"):
                fan = shape[-1] * 3
            v = rng.normal(0.0, 1.0 / math.sqrt(fan), size=shape)
        elif name.endswith(".a"):
            v = rng.uniform(0.05, 0.35, size=shape)
        elif name.endswith(".ma") or name.endswith(".mb"):
            v = rng.uniform(0.5, 0.9, size=shape)
        elif name.endswith(".b"):
            v = rng.normal(0.0, 0.05, size=shape)
        else:  # embeddings
            v = rng.normal(0.0, 0.5, size=shape)
        out[name] = v.astype(np.float32)
    return out
