"""The allocation-free seeding search gives the same lists as ff_seed_knn.

ff_seed_knn_static exists for callers that cannot allocate device memory: a
plug-in inside a host program that owns every allocation and gives libraries
a fixed budget, or a real-time loop that must never wait on the allocator
(cudaMalloc and cudaFree can synchronise the device).  It keeps its scratch in
the library's static device memory instead of a context.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu


def _padded_level0(ctx, slot: int, channels: int):
    """Level-0 features in the library's padded layout [H][W][16 | 32]."""
    import torch
    dense = ctx.features_of(slot, 0)
    H, W, D = dense.shape
    out = torch.zeros((H, W, 16 if channels == 1 else 32), dtype=torch.int8,
                      device=dense.device)
    out[..., :D] = dense
    return out.contiguous()


@pytest.mark.parametrize("name,stride", [("sintel1024x436", 1), ("tiny128x96", 1),
                                         ("tiny128x96", 2)])
def test_static_seeding_equals_context_seeding_twice(name, stride):
    import torch
    pair, prm = workloads.make_workload(name)
    C, S = prm["channels"], prm["scales"]
    W, H = pair.width, pair.height
    cfg = ff.Config(channels=C, scales=S, iters=prm["iters"], radius_q3=prm["radius_q3"],
                    max_width=W, max_height=H, seed_stride=stride)
    ctx = ff.Context(cfg)
    ctx.features(0, torch.from_numpy(pair.img1).cuda())
    ctx.features(1, torch.from_numpy(pair.img2).cuda())
    f0 = _padded_level0(ctx, 0, C)
    f1 = _padded_level0(ctx, 1, C)
    for direction, (fs, fd) in enumerate(((f0, f1), (f1, f0))):
        ref_idx, ref_dist = ctx.seed_knn(direction)
        torch.cuda.synchronize()
        for _ in range(2):   # two calls in a row share the static scratch
            idx = torch.full_like(ref_idx, -7)
            dist = torch.full_like(ref_dist, -7)
            ff.ff_seed_knn_static(fs, fd, W, H, C, S, cfg.seed_leaf, cfg.seed_stride, idx, dist,
                                  torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert torch.equal(idx, ref_idx)
            assert torch.equal(dist, ref_dist)
        if name == "tiny128x96":
            # and both equal the oracle's exact search on the same features
            import oracle as O
            a = fs[..., :9 * C].cpu().numpy()
            b = fd[..., :9 * C].cpu().numpy()
            oi, od = O.seed_knn(a, b, S, cfg.seed_leaf, stride)
            np.testing.assert_array_equal(idx.cpu().numpy().reshape(oi.shape), oi)
            np.testing.assert_array_equal(dist.cpu().numpy().reshape(od.shape), od)
    ctx.close()


def test_static_seeding_rejects_sizes_beyond_its_scratch():
    import torch
    feat = torch.zeros((436, 1024, 32), dtype=torch.int8, device="cuda")
    out = torch.zeros((436, 1024, 8), dtype=torch.int32, device="cuda")
    # one scale: every pixel is a query, 446464 > 131072 lists
    with pytest.raises(ff.FFError) as e:
        ff.ff_seed_knn_static(feat, feat, 1024, 436, 3, 1, 8, 1, out, out)
    assert e.value.status == ff.FF_EINVAL
    assert "static scratch" in str(e.value)
