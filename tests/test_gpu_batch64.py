"""The batched form at full size: the 64-frame mixed batch (beams from
{16, 64, 128}, log-uniform 8k-230k points, depths 12-18; 2.78 M points in
all) through encode_batch and decode_batch on one GPU.  Every frame's stream
must equal the oracle's stream of that frame coded alone, byte for byte, and
every frame must decode to exactly its input voxels.  This reaches what the
smaller batch tests do not: frames up to ~230k points, the two-group decode
with large frames, the large-batch coarse scan and capacity-sized graph grids
at 2.8 M points.
"""

import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_25260_b300 import synth

pytestmark = pytest.mark.gpu

CHUNK = 1024


@pytest.fixture(scope="module")
def lpc():
    from paper_2603_25260_b300 import build, lpc as mod
    build.build()
    mod.lib()
    return mod


def _oracle_streams(blob, frames, Ls, chunk):
    """The oracle's per-frame streams, one frame per host thread (the oracle
    releases the GIL inside its C calls; each call single-threaded)."""
    prev = O.get_threads()
    O.set_threads(1)
    try:
        with cf.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
            # largest frames first so the pool's tail is short
            order = sorted(range(len(frames)), key=lambda i: -frames[i].shape[0])
            futs = {i: ex.submit(O.encode, blob, frames[i], Ls[i], chunk) for i in order}
            return [futs[i].result() for i in range(len(frames))]
    finally:
        O.set_threads(prev)


def test_batch64_full_size_matches_per_frame_oracle(lpc, blob):
    specs = synth.batch_specs(64)
    frames = synth.make_frames(specs)
    Ls = [s.L for s in specs]
    npts = sum(f.shape[0] for f in frames)
    assert npts > 2_500_000 and max(f.shape[0] for f in frames) > 200_000
    cod = lpc.Codec(blob, max(Ls), max(f.shape[0] for f in frames), max_frames=len(frames),
                    chunk=CHUNK, max_batch_points=npts)
    xs = [torch.from_numpy(f).cuda() for f in frames]
    outs = cod.encode_batch(xs, Ls)
    want = _oracle_streams(blob, frames, Ls, CHUNK)
    bad = [i for i in range(len(frames)) if outs[i] != want[i]]
    assert not bad, f"streams differ from the oracle for frames {bad}"
    # twice: the first decode runs the levels directly, the second replays
    # the captured level graphs
    for _ in range(2):
        decs = cod.decode_batch(outs, [f.shape[0] for f in frames])
        for i, (f, L, dcd) in enumerate(zip(frames, Ls, decs)):
            assert np.array_equal(O.leaf_keys(dcd.cpu().numpy(), L), O.leaf_keys(f, L)), i
    cod.close()
