"""Serving loop on the GPU: every result of the continuous-batching server
is the same, bit for bit, as the pipeline computed alone (single launches),
and matches the oracle on sampled requests."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from paper_0712_0121_gb300.serve import (BatchExecutor, PerPageExecutor, Server,  # noqa: E402
                                          poisson_arrivals)
from gpu_helpers import NCORES  # noqa: E402

W, H = 1275, 1650


@pytest.fixture(scope="module")
def pool():
    pages = []
    for k, kind in enumerate(synth.CONFIG3_KINDS):
        img = synth.config3_page(kind, page=k, W=W, H=H)[0]
        pages.append((img, M.pack(img, 64)))
    return pages


def alone(src, rpr):
    cur = src
    for op, (sw, sh) in (("close", (31, 1)), ("open", (3, 3)), ("dilate", (1, 15))):
        nxt = M.Packed.empty(W, H, 64)
        M.morph_rect(op, nxt, cur, sw, sh)
        cur = nxt
    out = M.Rle.empty(W, H, H * rpr)
    M.rle_from_bitmap(out, cur)
    return out.to_numpy()


@pytest.mark.parametrize("path", ["packed", "rle"])
def test_served_results_equal_alone(pool, path):
    rpr = W // 8 + 4
    ex = BatchExecutor([p for _, p in pool], W, H, n_slots=48, n_streams=3, runs_per_row=rpr, path=path)
    srv = Server(ex, budget_bytes=40e9)
    n = 40
    # 16 requests arrive together, the rest as a fast Poisson stream: they
    # are admitted in shared rounds and are on the GPU at the same time
    arr = np.concatenate([np.zeros(16), 1e-3 + poisson_arrivals(3000.0, n - 16, seed=11)])
    pages = np.arange(n) % len(pool)
    st = srv.run(arr, pages)
    torch.cuda.synchronize()
    assert M.sync_status() == M.MORPH_OK
    assert st.completed == n
    assert max(st.batch_sizes) > 1, "no admission round held more than one request"
    assert st.max_in_flight > 1, "no two requests were in flight together"
    # results live in the slots until reused: check the last occupant of each slot
    last = {}
    for r in srv.requests:
        last[r.slot] = r
    refs = {k: alone(pool[k][1], rpr) for k in range(len(pool))}
    for slot, r in last.items():
        rp, runs = ex.result(r).to_numpy()
        rrp, rruns = refs[r.page]
        assert np.array_equal(rp, rrp) and np.array_equal(runs, rruns), "request %d" % r.rid


def test_pipeline_matches_oracle(pool):
    img, src = pool[1]
    rp, runs = alone(src, W // 8 + 4)
    ref = img
    for op, (sw, sh) in (("close", (31, 1)), ("open", (3, 3)), ("dilate", (1, 15))):
        ref = oracle.apply(op, ref, sw, sh, mode="separable", threads=NCORES)
    orp, oruns = oracle.rle_encode(ref)
    assert np.array_equal(rp, orp) and np.array_equal(runs, oruns)


def test_per_page_baseline_runs(pool):
    ex = PerPageExecutor([p for _, p in pool], W, H)
    st = Server(ex, budget_bytes=40e9).run(poisson_arrivals(500.0, 10, seed=2), np.arange(10) % 4)
    assert st.completed == 10 and st.max_in_flight == 1
