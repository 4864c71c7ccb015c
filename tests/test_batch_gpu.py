"""The persistent batch launch: mixed page sizes, operations, rectangles and
paths in one launch, each page bit-exact against the oracle, the same alone
and in the mix, replayable from a CUDA graph; overflow and time-out reported
through the device status without harming the context."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import NCORES, unpack_words  # noqa: E402


def make_jobs(specs):
    jobs, imgs = [], []
    for k, (W, H, op, se, path, dens) in enumerate(specs):
        img = synth.text_page(W, H, 9000 + k, dens, glyph=(4, 12, 6, 14), gap=(2, 6), ncols=2)[0]
        src = M.pack(img, 64 if k % 3 else 32)
        dst = M.Packed.empty(W, H, 32 if k % 2 else 64)
        dst.words.fill_(-1)
        jobs.append(dict(op=op, se=se, path=path, src=src, dst=dst))
        imgs.append(img)
    return jobs, imgs


SPECS = [
    (300, 200, "erode", (3, 3), "packed", 0.2),
    (301, 177, "dilate", (5, 5), "rle", 0.1),
    (517, 333, "open", (9, 9), "packed", 0.25),
    (517, 333, "close", (9, 9), "rle", 0.25),
    (1000, 50, "open", (41, 1), "rle", 0.15),
    (1000, 50, "close", (1, 41), "packed", 0.15),
    (77, 640, "dilate", (101, 1), "packed", 0.05),
    (77, 640, "erode", (1, 31), "rle", 0.4),
    (200, 120, "close", (15, 15), "rle", 0.02),
    (200, 120, "open", (31, 31), "packed", 0.3),
    (64, 64, "erode", (1, 1), "rle", 0.5),
    (2550, 400, "close", (51, 51), "packed", 0.08),
]


def check_all(jobs, imgs):
    for k, (j, img) in enumerate(zip(jobs, imgs)):
        sw, sh = j["se"]
        ref = oracle.apply(j["op"], img, sw, sh, mode="separable", threads=NCORES)
        got = unpack_words(j["dst"].words, img.shape[1])
        assert np.array_equal(got, ref), "job %d %s %s %s" % (k, j["op"], j["se"], j["path"])


def test_mixed_batch_matches_oracle():
    jobs, imgs = make_jobs(SPECS)
    b = M.Batch(jobs)
    b.launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)


def test_alone_equals_in_the_mix_and_graph_replay():
    jobs, imgs = make_jobs(SPECS)
    b = M.Batch(jobs)
    g = b.capture()
    for j in jobs:
        j["dst"].words.fill_(0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)
    mixed = [j["dst"].words.clone() for j in jobs]
    for k, j in enumerate(jobs):
        alone = M.Packed.empty(j["dst"].width, j["dst"].height, j["dst"].word_bits)
        one = M.Batch([dict(j, dst=alone)])
        one.launch()
        assert torch.equal(alone.words, mixed[k]), "job %d differs alone" % k
        single = M.Packed.empty(j["dst"].width, j["dst"].height, j["dst"].word_bits)
        M.morph_rect(j["op"], single, j["src"], *j["se"])
        assert torch.equal(single.words, mixed[k]), "job %d differs from the single-op launch" % k


def test_rle_buffer_overflow_is_reported_and_packed_jobs_survive():
    specs = [(400, 100, "open", (3, 3), "rle", 0.5), (400, 100, "open", (3, 3), "packed", 0.5)]
    jobs, imgs = make_jobs(specs)
    b = M.Batch(jobs, rle_runs_per_row=2)
    b.launch()
    assert M.sync_status() == M.MORPH_ECAPACITY
    ref = oracle.opening(imgs[1], 3, 3)
    assert np.array_equal(unpack_words(jobs[1]["dst"].words, 400), ref)
    assert M.sync_status() == M.MORPH_OK


def test_wait_time_out_is_reported_and_device_stays_usable():
    specs = [(300, 90, "erode", (3, 3), "rle", 0.3), (300, 90, "dilate", (3, 3), "packed", 0.3)]
    jobs, imgs = make_jobs(specs)
    # the second phase of the RLE job waits for one item more than exist
    b = M.Batch(jobs, debug=[(0, 200_000_000), (1, 1)])
    b.launch()
    assert M.sync_status() == M.MORPH_ETIMEOUT
    ok = M.Batch(jobs)
    ok.launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)


def test_config4_like_sample():
    """Twelve pages drawn like the uneven batch workload (sizes scaled down)."""
    specs = []
    for k, j in enumerate(synth.config4_jobs(12)):
        W, H = j["W"] // 4, j["H"] // 4
        specs.append((W, H, j["op"], j["se"], "rle" if k % 2 else "packed", j["density"]))
    jobs, imgs = make_jobs(specs)
    M.Batch(jobs).launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)


def test_rle_jobs_on_one_page_share_its_encode():
    """RLE-path jobs on the same source page encode it once: every job, the
    encoder and the jobs that read its runs (including two-stage run passes,
    which write their second stage into their own buffer), is exact."""
    W, H = 700, 450
    img = synth.text_page(W, H, 4242, 0.15, glyph=(4, 12, 6, 14), gap=(2, 6), ncols=2)[0]
    src = M.pack(img, 64)
    ops = [("open", (1, 1)), ("close", (9, 1)), ("open", (1, 7)), ("erode", (5, 5)), ("close", (31, 3)),
           ("dilate", (15, 15)), ("open", (41, 1)), ("close", (3, 3))]
    jobs = []
    for op, se in ops:
        dst = M.Packed.empty(W, H, 64)
        dst.words.fill_(-1)
        jobs.append(dict(op=op, se=se, path="rle", src=src, dst=dst))
    pdst = M.Packed.empty(W, H, 64)
    jobs.append(dict(op="close", se=(7, 7), path="packed", src=src, dst=pdst))
    b = M.Batch(jobs)
    for _ in range(2):  # a relaunch recomputes the shared encode
        b.launch()
        assert M.sync_status() == M.MORPH_OK
        for j in jobs:
            sw, sh = j["se"]
            ref = oracle.apply(j["op"], img, sw, sh, mode="separable", threads=NCORES)
            assert np.array_equal(unpack_words(j["dst"].words, W), ref), (j["op"], j["se"], j["path"])


def test_shared_encode_overflow_is_reported():
    W, H = 400, 100
    img = synth.random_bits((H, W), 99, 0.5)
    src = M.pack(img, 64)
    jobs = [dict(op=op, se=(3, 3), path="rle", src=src, dst=M.Packed.empty(W, H, 64))
            for op in ("open", "close", "erode")]
    b = M.Batch(jobs, rle_runs_per_row=2)
    b.launch()
    assert M.sync_status() == M.MORPH_ECAPACITY
    ok = M.Batch(jobs, rle_runs_per_row=W // 2 + 1)  # room for any row
    ok.launch()
    assert M.sync_status() == M.MORPH_OK
    for j in jobs:
        ref = oracle.apply(j["op"], img, 3, 3)
        assert np.array_equal(unpack_words(j["dst"].words, W), ref)


def test_dependency_chains_across_grouped_and_persistent_jobs():
    """Chains whose links run on different parts of the launch: packed jobs
    grouped level by level (0, 1, 2), an RLE job reading a grouped job's
    result, a packed job reading an RLE job's result (run by the persistent
    kernel), and a conversion of a chain's last page to runs."""
    rng_pages = [synth.text_page(640, 480, 9300 + k, 0.12, glyph=(4, 12, 6, 14), gap=(2, 6), ncols=2)[0]
                 for k in range(2)]
    a, b = rng_pages
    P = lambda img: M.pack(img, 64)  # noqa: E731
    E = lambda: M.Packed.empty(640, 480, 64)  # noqa: E731
    src_a, src_b = P(a), P(b)
    a1, a2, a3, a4 = E(), E(), E(), E()
    b1, b2 = E(), E()
    rle_out = M.Rle.empty(640, 480, 480 * 321)
    jobs = [
        dict(op="close", se=(15, 15), path="packed", src=src_a, dst=a1),                    # 0, level 0
        dict(op="open", se=(3, 3), path="packed", src=a1, dst=a2, depends_on=0),             # 1, level 1
        dict(op="dilate", se=(1, 15), path="packed", src=a2, dst=a3, depends_on=1),          # 2, level 2
        dict(op="erode", se=(5, 5), path="rle", src=a3, dst=a4, depends_on=2),               # 3, persistent
        dict(op="open", se=(7, 7), path="rle", src=src_b, dst=b1),                           # 4, persistent
        dict(op="close", se=(3, 3), path="packed", src=b1, dst=b2, depends_on=4),            # 5, persistent
        dict(op="to_rle", src=a4, dst=rle_out, depends_on=3),                                # 6, persistent
    ]
    bt = M.Batch(jobs)
    assert bt.kernels >= 4  # three packed levels and the persistent kernel
    for _ in range(2):  # a replay gives the same pages
        bt.launch()
        assert M.sync_status() == M.MORPH_OK
        ra = a
        for op, (sw, sh) in (("close", (15, 15)), ("open", (3, 3)), ("dilate", (1, 15)), ("erode", (5, 5))):
            ra = oracle.apply(op, ra, sw, sh, mode="separable", threads=NCORES)
        rb = oracle.apply("close", oracle.apply("open", b, 7, 7, mode="separable", threads=NCORES), 3, 3,
                          mode="separable", threads=NCORES)
        assert np.array_equal(unpack_words(a4.words, 640), ra)
        assert np.array_equal(unpack_words(b2.words, 640), rb)
        g_rp, g_runs = rle_out.to_numpy()
        o_rp, o_runs = oracle.rle_encode(ra)
        assert np.array_equal(g_rp, o_rp)
        assert np.array_equal(g_runs.reshape(-1, 2), o_runs.reshape(-1, 2))


def test_groups_only_launch_reuses_the_encodes():
    """The timing hook (morph_batch_plan_debug 2) launches the tile groups
    without the persistent kernel: after one full launch the RLE groups read
    the encodes left in the workspace and write the same pages."""
    specs = [(640, 480, "open", (7, 7), "rle", 0.12), (640, 480, "close", (15, 15), "rle", 0.12),
             (640, 480, "open", (31, 31), "packed", 0.12)]
    jobs, imgs = make_jobs(specs)
    b = M.Batch(jobs)
    full = b.kernels
    b.launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)
    for j in jobs:
        j["dst"].words.fill_(-1)
    b.debug(2, 1)
    assert b.kernels == full - 1
    b.launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)
    b.debug(2, 0)
    assert b.kernels == full


def test_batch_between_host_buffers_on_two_calls():
    """morph_batch_launch_host: the pages go in from pinned host memory, the
    batch runs, the results come back to pinned host memory — all queued on
    one stream; the second call with other pages in the same host buffer
    gives that input's results."""
    W, H, K = 700, 333, 3
    ops = [("open", (7, 7), "packed"), ("close", (15, 15), "rle"), ("erode", (51, 1), "packed")]
    d_in = torch.empty((K, H, (W + 63) // 64), dtype=torch.int64, device="cuda")
    d_out = torch.empty((K, H, (W + 63) // 64), dtype=torch.int64, device="cuda")
    jobs = [dict(op=op, se=se, path=path, src=M.Packed(d_in[k], W), dst=M.Packed(d_out[k], W))
            for k, (op, se, path) in enumerate(ops)]
    b = M.Batch(jobs)
    h_in = torch.empty(d_in.shape, dtype=torch.int64, pin_memory=True)
    h_out = torch.empty(d_out.shape, dtype=torch.int64, pin_memory=True)
    for call in range(2):
        imgs = [synth.text_page(W, H, 9500 + 10 * call + k, 0.15, glyph=(4, 12, 6, 14), gap=(2, 6))[0]
                for k in range(K)]
        for k, img in enumerate(imgs):
            h_in[k].copy_(M.pack(img, 64).words.cpu())
        h_out.fill_(-1)
        b.launch_host(h_in, d_in, h_out, d_out)
        assert M.sync_status() == M.MORPH_OK
        for k, (img, (op, (sw, sh), _)) in enumerate(zip(imgs, ops)):
            ref = oracle.apply(op, img, sw, sh, mode="separable", threads=NCORES)
            assert np.array_equal(unpack_words(h_out[k], W), ref), (call, k, op)


@pytest.mark.parametrize("words", [2, 4])
def test_word_tile_per_job(words):
    """A job's words_per_thread picks the packed tile's word tile; every
    operation and window class stays bit-exact (a tiling the tile cannot
    hold falls back to the persistent kernel, also exact)."""
    specs = [(300, 200, "erode", (3, 3), "packed", 0.2), (517, 333, "open", (9, 9), "packed", 0.25),
             (1000, 50, "close", (1, 41), "packed", 0.15), (77, 640, "dilate", (101, 1), "packed", 0.05),
             (200, 120, "open", (31, 31), "packed", 0.3), (2550, 400, "close", (51, 51), "packed", 0.08),
             (640, 480, "open", (15, 15), "packed", 0.12)]
    jobs, imgs = make_jobs(specs)
    for j in jobs:
        j["words_per_thread"] = words
    b = M.Batch(jobs)
    b.launch()
    assert M.sync_status() == M.MORPH_OK
    check_all(jobs, imgs)


def test_word_tile_out_of_range_is_rejected():
    jobs, _ = make_jobs([(64, 64, "erode", (3, 3), "packed", 0.3)])
    jobs[0]["words_per_thread"] = 3
    with pytest.raises(M.MorphError):
        M.Batch(jobs)
