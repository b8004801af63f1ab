"""Architecture switches of the ablations (Sec. 4.3, Table 4; supplement,
choice of t): GRED + XFP, GRED only and the baseline, each with t = L - 4 or
L - 3, on the CPU oracle.

Pins of the oracle's integer network in each architecture:
- its logits equal the FP64 twin's (a separate PyTorch implementation of the
  same architecture) up to quantisation rounding, on the integer blob
  exported from the twin's parameters; a wrong wiring (features taken at the
  wrong level, a missing concatenation) moves the logits by several steps;
- levels whose structure two architectures share give byte-identical logits
  when their parameters are the same;
- lossless round trip, the stream header's t, and blob validation."""

import numpy as np
import pytest

import oracle as O
from oracle import train_ref as T
from paper_2603_25260_b300 import export, synth

VARIANTS = [(a, t) for a in (synth.ARCH_XFP, synth.ARCH_GRED, synth.ARCH_BASE) for t in (4, 3)]


@pytest.fixture(scope="module")
def gframe():
    spec = synth.GRADCHECK
    xyz = synth.make_frame(spec)
    return xyz, spec.L, T.Frame(xyz, spec.L)


def _blob(arch, t_off, seed=5):
    P = synth.twin_params(seed, arch=arch, t_off=t_off)
    return P, export.quantize_twin(P, arch=arch, t_off=t_off)


@pytest.mark.parametrize("arch,t_off", VARIANTS)
def test_logits_match_twin(gframe, arch, t_off):
    """Integer logits (steps of 1/16 nat) against the fake-quantised FP64
    twin: mean difference under half a step, none above 4 steps, on logits
    that spread over several steps per level."""
    xyz, L, fr = gframe
    P, blob = _blob(arch, t_off)
    assert O.check_blob(blob) == 0
    lg = T.level_logits(T.to_torch(P, requires_grad=False), fr, qat=True, arch=arch, t_off=t_off)
    for d in range(L - 5, L):
        li = O.logits_level(blob, xyz, L, d).astype(np.float64)
        lf = lg[d].detach().numpy() / export.LOGIT_SCALE
        assert li.shape == lf.shape
        e = np.abs(li - lf)
        assert lf.std() > 1.0
        assert e.mean() < 0.45 and e.max() < 4.0, (d, e.mean(), e.max())


def test_twin_wiring_mistake_is_seen(gframe):
    """The comparison above separates the architectures: with the last
    layers' weights scaled up (logits spread over tens of steps), the GRED
    blob's logits at the re-densified levels are three times closer to the
    GRED twin's than to the twin run as the baseline on the same parameters
    (deep levels' features taken at their parent level instead of at t)."""
    xyz, L, fr = gframe
    P = {k: v.copy() for k, v in synth.twin_params(5, arch=synth.ARCH_GRED).items()}
    for j in range(5):
        P[f"P2_{j}.W"] *= 6.0
    blob = export.quantize_twin(P, arch=synth.ARCH_GRED)
    Pt = T.to_torch(P, requires_grad=False)
    right = T.level_logits(Pt, fr, qat=True, arch=synth.ARCH_GRED)
    wrong = T.level_logits(Pt, fr, qat=True, arch=synth.ARCH_BASE)
    for d in (L - 2, L - 1):
        li = O.logits_level(blob, xyz, L, d).astype(np.float64)
        e_r = np.abs(li - right[d].detach().numpy() / export.LOGIT_SCALE).mean()
        e_w = np.abs(li - wrong[d].detach().numpy() / export.LOGIT_SCALE).mean()
        assert e_w > 3.0 * e_r, (d, e_r, e_w)


def test_shared_levels_identical(gframe):
    """Same seed, same records up to a level => same parameters => the same
    integer logits: level b in every architecture; GRED and the baseline
    agree on every level extracted at its parent level (j = 1, 2 with
    t = L - 4; j = 1..3 with t = L - 3); the baseline ignores t."""
    xyz, L, _ = gframe
    lg = {(a, t): {d: O.logits_level(_blob(a, t)[1], xyz, L, d) for d in range(L - 5, L)}
          for a, t in VARIANTS}
    b = L - 5
    for v in VARIANTS:
        assert np.array_equal(lg[v][b], lg[VARIANTS[0]][b])
    for d in range(L - 5, L):
        assert np.array_equal(lg[(synth.ARCH_BASE, 3)][d], lg[(synth.ARCH_BASE, 4)][d])
    for t_off, shared in ((4, 2), (3, 3)):
        for j in range(shared + 1):
            assert np.array_equal(lg[(synth.ARCH_GRED, t_off)][b + j],
                                  lg[(synth.ARCH_BASE, t_off)][b + j])
        assert not np.array_equal(lg[(synth.ARCH_GRED, t_off)][L - 1],
                                  lg[(synth.ARCH_BASE, t_off)][L - 1])
    # XFP's propagated level b + 1 is not the baseline's
    assert not np.array_equal(lg[(synth.ARCH_XFP, 4)][b + 1], lg[(synth.ARCH_BASE, 4)][b + 1])


@pytest.mark.parametrize("arch,t_off", VARIANTS)
def test_round_trip_and_header(arch, t_off):
    blob = synth.make_blob(arch=arch, t_off=t_off)
    assert O.check_blob(blob) == 0
    for n, L, seed in ((1500, 9, 21), (300, 6, 22)):
        xyz = synth.random_cloud(n, L, seed)
        data = O.encode(blob, xyz, L, 200)
        assert data[5] == L and data[6] == L - 5 and data[7] == L - t_off
        dec = O.decode(blob, data, n)
        assert np.array_equal(O.leaf_keys(dec, L), O.leaf_keys(xyz, L))
    other = synth.make_blob(arch=(arch + 1) % 3, t_off=t_off)
    with pytest.raises(O.OracleError) as e:
        O.decode(other, data, n)
    assert e.value.status == -5


def test_blob_header_validation():
    recs, lut = synth.make_blob_records(arch=synth.ARCH_GRED)
    good = synth.pack_blob(recs, lut, 32, synth.ARCH_GRED)
    assert O.check_blob(good) == 0
    # the records of one architecture under another's header
    assert O.check_blob(synth.pack_blob(recs, lut, 32, synth.ARCH_XFP)) != 0
    assert O.check_blob(synth.pack_blob(recs, lut, 32, synth.ARCH_GRED, 3)) != 0
    for off, v in ((20, 3), (24, 2), (24, 5)):
        bad = bytearray(good)
        bad[off:off + 4] = int(v).to_bytes(4, "little")
        assert O.check_blob(bytes(bad)) != 0
    # t_off 0 reads as 4: the default blob is unchanged by the field
    assert synth.make_blob()[20:32] == bytes(12)
    with pytest.raises(ValueError):
        synth.network_records(32, 3, 4)
    with pytest.raises(ValueError):
        synth.network_records(32, 0, 5)
