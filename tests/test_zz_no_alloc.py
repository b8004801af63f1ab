"""The allocation-free kernel-map entry point.

Some callers of this library may not allocate device memory where they need
a kernel map (a real-time loop whose memory is fixed at start-up, or code
that runs while another component owns the CUDA allocator).  For them
lpc_kernel_map_noalloc keeps its hash table in a static device array.  These
checks call it through the C ABI twice in a row, on different clouds, and
compare each result with the allocating entry point lpc_kernel_map (integer
output, so the comparison is exact).  The file sorts last so that a run that
stops at the first failure has run every other test before this one.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_25260_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lpc():
    from paper_2603_25260_b300 import build, lpc as mod
    build.build()
    mod.lib()
    return mod


def _keys(n, depth, seed):
    keys = O.leaf_keys(synth.random_cloud(n, depth, seed), depth)
    return torch.from_numpy(keys.view(np.int64)).cuda()


def test_noalloc_matches_allocating_entry_point_twice(lpc):
    # a larger map first, then a smaller one: the second call must not see
    # anything the first call left in the shared table
    for n, depth, seed in ((60000, 12, 21), (3000, 7, 22)):
        keys = _keys(n, depth, seed)
        want = lpc.kernel_map(keys, depth)
        out = torch.full((keys.shape[0], 27), -7, dtype=torch.int32, device="cuda")
        got = lpc.kernel_map_noalloc(keys, depth, out)
        torch.cuda.synchronize()
        assert torch.equal(got, want)


def _keys_at_cap(kind, n):
    """Exactly n unique sorted depth-12 keys: a random subset of a clustered
    cloud, or a solid 64^3 block (every interior node has 27 neighbours)."""
    if kind == "block":
        g = np.arange(64, dtype=np.int32)
        xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 1000
        keys = O.leaf_keys(xyz, 12)
    else:
        keys = O.leaf_keys(synth.random_cloud(2 * n, 12, 23), 12)
        rng = np.random.Generator(np.random.PCG64(24))
        keys = np.sort(rng.choice(keys, size=n, replace=False))
    assert keys.shape[0] == n
    return torch.from_numpy(keys.view(np.int64)).cuda()


@pytest.mark.parametrize("kind", ["random", "block"])
def test_noalloc_at_the_node_limit(lpc, kind):
    # the table's limit exactly: 2^18 nodes in 2^19 slots, load factor 1/2,
    # the longest probe chains the entry point accepts
    n = lpc.NOALLOC_MAX_NODES
    keys = _keys_at_cap(kind, n)
    want = lpc.kernel_map(keys, 12)
    out = torch.full((n, 27), -7, dtype=torch.int32, device="cuda")
    for _ in range(2):
        got = lpc.kernel_map_noalloc(keys, 12, out)
        torch.cuda.synchronize()
        assert torch.equal(got, want)


def test_noalloc_second_call_allocates_nothing(lpc):
    # after the first call on the device (which may load the array's module),
    # further calls leave the device's free memory unchanged
    keys = _keys(20000, 10, 25)
    out = torch.empty((keys.shape[0], 27), dtype=torch.int32, device="cuda")
    lpc.kernel_map_noalloc(keys, 10, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        lpc.kernel_map_noalloc(keys, 10, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_too_many_nodes(lpc):
    n = lpc.NOALLOC_MAX_NODES + 1
    keys = torch.arange(n, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 27), dtype=torch.int32, device="cuda")
    with pytest.raises(lpc.LpcError) as e:
        lpc.kernel_map_noalloc(keys, 7, out)
    assert e.value.status == lpc.CAPACITY
