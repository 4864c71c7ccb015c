"""The benchmark's own launch at full size: 160 letter pages (2550 x 3300) x
28 page-operations in one graph-captured batch launch, exactly what bench.py
times.  Every page-operation of the first page and a seeded sample of the
others are checked bit for bit against the oracle."""
import numpy as np
import pytest
import torch

import bench
import oracle

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import NCORES, unpack_words  # noqa: E402


def test_bench_launch_sampled_against_oracle():
    B = 160
    pages = bench.make_pages(B)
    dev_in = torch.empty((B, bench.H, bench.NW), dtype=torch.int64, device="cuda")
    for k, p in enumerate(pages):
        dev_in[k].copy_(M.pack(p, 64).words)
    srcs = [M.Packed(dev_in[k], bench.W) for k in range(B)]
    jobs, dev_out = bench.build_jobs(M, srcs, ("packed", "rle"))
    dev_out.fill_(-1)  # an unwritten result cannot pass
    graph = M.Batch(jobs, rle_runs_per_row=64).capture()
    graph.replay()
    graph.replay()  # a replay recomputes the same results
    torch.cuda.synchronize()
    assert M.sync_status() == M.MORPH_OK
    per_page = len(jobs) // B
    assert per_page == 28
    rng = np.random.default_rng(20261204)
    picks = set(range(per_page)) | {len(jobs) - 1} | set(rng.choice(len(jobs), 16, replace=False).tolist())
    for k in sorted(picks):
        j = jobs[k]
        sw, sh = j["se"]
        ref = oracle.apply(j["op"], pages[k // per_page], sw, sh, mode="separable", threads=NCORES)
        got = unpack_words(dev_out[k], bench.W)
        assert np.array_equal(got, ref), "page %d %s %s %s" % (k // per_page, j["op"], j["se"], j["path"])
