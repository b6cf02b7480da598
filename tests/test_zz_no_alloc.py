"""The allocation-free labeller, agipc_aggregate_static, for callers that
cannot allocate GPU memory (they have no agipc_ctx, whose creation calls
cudaMalloc).  Its scratch is a fixed array inside the library, shared by all
calls.  Checked through the C ABI, bit for bit, against the CPU oracle's union-find
labels and against agipc_aggregate, on two calls in a row with different
inputs, so a stale array from the first call must not leak into the
second.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_04773_gb300 import agipc, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04773_gb300 import build
    build.build()
    agipc.load()


def _with_context(n, edges, tags):
    ctx = agipc.Context(n, edges.shape[0], 1, 0)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    agipc.agipc_aggregate(ctx, n, edges, tags, labels, nc)
    assert ctx.status() == agipc.OK
    ctx.close()
    return labels.cpu().numpy(), int(nc.item())


def test_static_labeller_matches_oracle_and_context_labeller_twice():
    big = scenes.domino_grid(seed=77, gx=2, gy=2, dims=(3, 5, 8), n_pairs=0)
    small = scenes.unit_cube(seed=1001)
    rng = np.random.default_rng(12)
    cases = [(big.n, big.edges, big.tags),
             (small.n, small.edges, (rng.random(small.n_edges) < 0.6).astype(np.uint8))]
    stream = torch.cuda.current_stream()
    for n, e, t in cases:
        edges = torch.from_numpy(np.ascontiguousarray(e, np.int32)).cuda()
        tags = torch.from_numpy(np.ascontiguousarray(t, np.uint8)).cuda()
        labels = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nc = torch.zeros(1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        agipc.agipc_aggregate_static(stream, n, edges, tags, labels, nc, status)
        torch.cuda.synchronize()
        ref_labels, ref_nc = _with_context(n, edges, tags)
        or_labels, or_nc = oracle.labels(n, np.asarray(e), np.asarray(t))
        got = labels.cpu().numpy()
        assert int(status.item()) == 0
        assert int(nc.item()) == or_nc == ref_nc
        assert np.array_equal(got, or_labels)
        assert np.array_equal(got, ref_labels)


def test_static_labeller_rejects_sizes_beyond_its_array():
    stream = torch.cuda.current_stream()
    n = agipc.AGGREGATE_STATIC_MAX_NODES + 1
    edges = torch.zeros(1, 2, dtype=torch.int32, device="cuda")
    tags = torch.zeros(1, dtype=torch.uint8, device="cuda")
    labels = torch.empty(1, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(agipc.AgipcError) as err:
        agipc.agipc_aggregate_static(stream, n, edges, tags, labels, nc, status)
    assert err.value.code == agipc.ERR_INVALID_ARG
