"""The allocation-free Hilbert seed ranking (slt_seed_rank_noalloc) against the ranking that
slt_inspect computes for its partition (the existing entry point), bit for bit.

Callers that cannot allocate device memory where they need the ordering (a framework owning every
allocation through its own pool, code where cudaMalloc would synchronise or is not permitted) use
the allocation-free entry point; it keeps its scratch in one fixed device array, shared by all
calls, so two calls in a row must each give the right answer (the second may not see the
first's leftovers)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_POINTS = 1 << 20


def _inspect_rank(lib, xy):
    ch = lib.slt_chain_create()
    s = lib.slt_set(ch, xy.shape[0])
    lib.slt_set_points(ch, s, xy)
    lib.slt_loop(ch, s, [(-1, "r")])
    sched = lib.slt_inspect(ch, tile_size=1024, renumber=1)
    return lib.slt_schedule_export(sched, "rank", 0)


def _noalloc_rank(lib, xy):
    import torch
    d_xy = torch.tensor(xy, dtype=torch.float64, device="cuda")
    d_rank = torch.full((xy.shape[0],), -1, dtype=torch.int32, device="cuda")
    lib.slt_seed_rank_noalloc(d_xy, d_rank)
    torch.cuda.synchronize()
    return d_rank.cpu().numpy()


def test_noalloc_rank_matches_inspector_on_consecutive_calls(lib):
    import synth
    m = synth.make_mesh(16, 16, seed=0)
    centroids = ((m["cellxy"][:, 0] + m["cellxy"][:, 1]) + m["cellxy"][:, 2]) / 3.0
    rng = np.random.default_rng(5)
    big = np.stack([rng.uniform(0, 300, MAX_POINTS), rng.uniform(0, 150, MAX_POINTS)], 1)
    small = rng.uniform(-1, 1, size=(3000, 2))
    # consecutive calls with different sizes and bounding boxes: full size, then smaller ones
    for xy in (big, centroids, small, centroids):
        got = _noalloc_rank(lib, xy)
        want = _inspect_rank(lib, xy)
        assert np.array_equal(got, want)
        assert np.array_equal(np.sort(got), np.arange(xy.shape[0]))


def test_noalloc_rank_rejects_more_points_than_its_scratch(lib):
    import torch
    n = MAX_POINTS + 1
    d_xy = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    d_rank = torch.zeros((n,), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.SltError) as e:
        lib.slt_seed_rank_noalloc(d_xy, d_rank)
    assert e.value.code == -1 and "at most" in str(e.value)
