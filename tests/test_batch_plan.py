"""Host logic of the batch planner (``morph_batch_plan_*``), on the CPU.

Planning reads only the job descriptors: page pointers are checked for
alignment and overlap but never dereferenced, so the plans here are built
from made-up, well-aligned device addresses and no GPU is needed.  What a
plan holds is checked through the C ABI's queries: the kernel launches one
call makes (one grouped launch per rectangle-tile variant and dependency
level, one per run-length-source-tile variant, plus the persistent kernel
when it has work items), its work items, its workspace, and the job checks.
"""
import ctypes

import pytest

W, H = 2550, 3300              # a letter page at 300 dpi
NW = (W + 63) // 64            # 64-bit words per row
PAGE = H * NW * 8              # bytes of one packed page
BASE = 1 << 32                 # made-up device addresses, far apart


@pytest.fixture(scope="module")
def M():
    from paper_0712_0121_gb300 import build
    build.build_morph()
    from paper_0712_0121_gb300 import morph
    return morph


def page(M, k, W_=W, H_=H, fmt=1, stride=None, offset=0):
    """Descriptor of made-up packed page k (pages never overlap)."""
    d = M.morph_image()
    d.fmt, d.width, d.height, d.reserved = fmt, W_, H_, 0
    d.words = BASE + k * 2 * PAGE + offset
    d.stride_words = stride if stride is not None else ((W_ + 63) // 64 if fmt == 1 else (W_ + 31) // 32)
    return d


def rle_image(M, k, W_=W, H_=H, cap=H * 64):
    d = M.morph_image()
    d.fmt, d.width, d.height, d.reserved = 2, W_, H_, 0
    d.row_ptr = BASE + (1000 + k) * 2 * PAGE
    d.runs = d.row_ptr + 4 * (H_ + 1) + 12
    d.capacity_runs = cap
    d.n_runs = d.runs + 4 * cap
    return d


def job(M, op, src, dst, se=(3, 3), path=0, depends_on=-1, words=0, tile_rows=0, origin=None):
    j = M.morph_job()
    j.op, j.path = op, path
    j.se_w, j.se_h = se
    j.origin_x, j.origin_y = origin if origin is not None else (se[0] // 2, se[1] // 2)
    j.depends_on, j.tile_rows, j.words_per_thread = depends_on, tile_rows, words
    j.src, j.dst = src, dst
    return j


class Plan:
    def __init__(self, M, jobs, tile_rows=0, runs_per_row=0):
        L = M.lib()
        arr = (M.morph_job * len(jobs))(*jobs)
        self.nbytes = int(L.morph_batch_plan_bytes(arr, len(jobs), tile_rows, runs_per_row))
        assert self.nbytes > 0, L.morph_last_error()
        self.buf = ctypes.create_string_buffer(self.nbytes)
        st = L.morph_batch_plan_build(self.buf, self.nbytes, arr, len(jobs), tile_rows, runs_per_row)
        assert st == M.MORPH_OK, L.morph_last_error()
        self.L = L

    @property
    def kernels(self):
        return self.L.morph_batch_kernels(self.buf)

    @property
    def items(self):
        return self.L.morph_batch_items(self.buf)

    @property
    def workspace(self):
        return self.L.morph_batch_workspace_size(self.buf)


def rejected(M, jobs):
    """plan_bytes gives 0 and plan_build MORPH_EINVAL; returns the message."""
    L = M.lib()
    arr = (M.morph_job * len(jobs))(*jobs)
    assert L.morph_batch_plan_bytes(arr, len(jobs), 0, 0) == 0
    buf = ctypes.create_string_buffer(1 << 16)
    assert L.morph_batch_plan_build(buf, len(buf), arr, len(jobs), 0, 0) == M.MORPH_EINVAL
    return L.morph_last_error().decode()


ERODE, DILATE, OPEN, CLOSE, TO_RLE = 0, 1, 2, 3, 4


def test_packed_jobs_of_one_variant_are_one_grouped_launch(M):
    jobs = [job(M, ERODE, page(M, 2 * k), page(M, 2 * k + 1)) for k in range(6)]
    p = Plan(M, jobs)
    assert p.kernels == 1
    assert p.items == 0                      # nothing for the persistent kernel
    assert p.workspace > 0                   # its counters are still cleared


def test_one_launch_per_variant_and_per_dependency_level(M):
    narrow = [job(M, ERODE, page(M, 0), page(M, 1)), job(M, ERODE, page(M, 2), page(M, 3))]
    assert Plan(M, narrow).kernels == 1
    # a 51x51 erosion takes another tile variant than a 3x3 one
    mixed = narrow + [job(M, ERODE, page(M, 4), page(M, 5), se=(51, 51))]
    assert Plan(M, mixed).kernels == 2
    # a chain page 0 -> 1 -> 2 of the same variant: one level per link
    chain = [job(M, CLOSE, page(M, 0), page(M, 1), se=(31, 1)),
             job(M, CLOSE, page(M, 1), page(M, 2), se=(31, 1), depends_on=0)]
    p = Plan(M, chain)
    assert p.kernels == 2 and p.items == 0


def test_word_tiles_are_separate_variants(M):
    a = job(M, ERODE, page(M, 0), page(M, 1), words=2)
    b = job(M, ERODE, page(M, 2), page(M, 3), words=4)
    c = job(M, ERODE, page(M, 4), page(M, 5), words=2)
    assert Plan(M, [a, c]).kernels == 1
    assert Plan(M, [a, b, c]).kernels == 2


def test_rle_jobs_on_one_page_share_its_encode(M):
    one = Plan(M, [job(M, OPEN, page(M, 0), page(M, 1), se=(7, 7), path=1)])
    # the persistent kernel encodes the page; the tile group reads the runs
    assert one.kernels == 2 and one.items > 0
    same_page = Plan(M, [job(M, OPEN, page(M, 0), page(M, 1), se=(7, 7), path=1),
                         job(M, CLOSE, page(M, 0), page(M, 2), se=(7, 7), path=1),
                         job(M, OPEN, page(M, 0), page(M, 3), se=(15, 15), path=1)])
    assert same_page.items == one.items      # one encode of page 0 for all three
    two_pages = Plan(M, [job(M, OPEN, page(M, 0), page(M, 1), se=(7, 7), path=1),
                         job(M, OPEN, page(M, 2), page(M, 3), se=(7, 7), path=1)])
    assert two_pages.items == 2 * one.items
    assert two_pages.kernels == 2            # one RLE group of one variant
    assert two_pages.workspace > one.workspace


def test_packed_and_rle_groups_and_the_persistent_kernel(M):
    jobs = [job(M, OPEN, page(M, 0), page(M, 1), se=(3, 3)),
            job(M, OPEN, page(M, 0), page(M, 2), se=(51, 51)),
            job(M, OPEN, page(M, 0), page(M, 3), se=(7, 7), path=1)]
    p = Plan(M, jobs)
    assert p.kernels == 2 + 1 + 1            # two packed groups, the encodes, one RLE group


def test_to_rle_and_dependent_rle_jobs_run_in_the_persistent_kernel(M):
    conv = Plan(M, [job(M, TO_RLE, page(M, 0), rle_image(M, 0))])
    assert conv.kernels == 1 and conv.items > 0
    # an RLE job that another job depends on stays inside the persistent kernel
    dep = Plan(M, [job(M, CLOSE, page(M, 0), page(M, 1), se=(5, 5), path=1),
                   job(M, TO_RLE, page(M, 1), rle_image(M, 1), depends_on=0)])
    assert dep.kernels == 1
    assert dep.items > conv.items


def test_groups_only_hook_drops_the_persistent_kernel(M):
    L = M.lib()
    p = Plan(M, [job(M, OPEN, page(M, 0), page(M, 1), se=(7, 7), path=1)])
    assert p.kernels == 2
    assert L.morph_batch_plan_debug(p.buf, 2, 1) == M.MORPH_OK
    assert p.kernels == 1
    assert L.morph_batch_plan_debug(p.buf, 2, 0) == M.MORPH_OK
    assert p.kernels == 2
    assert L.morph_batch_plan_debug(p.buf, 0, 5) == M.MORPH_OK      # wait limit (clamped to 1 ms)
    assert L.morph_batch_plan_debug(p.buf, 9, 0) == M.MORPH_EINVAL
    packed = Plan(M, [job(M, ERODE, page(M, 0), page(M, 1))])
    assert L.morph_batch_plan_debug(packed.buf, 1, 1) == M.MORPH_EINVAL  # no multi-phase job
    assert b"more than one phase" in L.morph_last_error()


def test_plan_queries_reject_a_buffer_that_is_not_a_plan(M):
    L = M.lib()
    junk = ctypes.create_string_buffer(4096)
    assert L.morph_batch_kernels(junk) == -1
    assert L.morph_batch_items(junk) == -1
    assert L.morph_batch_workspace_size(junk) == 0
    assert L.morph_batch_kernels(None) == -1
    assert L.morph_batch_plan_debug(junk, 2, 1) == M.MORPH_EINVAL


def test_plan_buffer_too_small(M):
    L = M.lib()
    jobs = [job(M, ERODE, page(M, 0), page(M, 1))]
    arr = (M.morph_job * 1)(*jobs)
    n = int(L.morph_batch_plan_bytes(arr, 1, 0, 0))
    buf = ctypes.create_string_buffer(n)
    assert L.morph_batch_plan_build(buf, n - 1, arr, 1, 0, 0) == M.MORPH_ENOMEM
    assert L.morph_batch_plan_build(buf, n, arr, 1, 0, 0) == M.MORPH_OK
    assert L.morph_batch_plan_build(None, n, arr, 1, 0, 0) == M.MORPH_EINVAL
    assert L.morph_batch_plan_build(buf, n, arr, 0, 0, 0) == M.MORPH_EINVAL


def test_plan_rejects_bad_jobs(M):
    ok = lambda **kw: job(M, kw.pop("op", ERODE), kw.pop("src", page(M, 0)),  # noqa: E731
                          kw.pop("dst", page(M, 1)), **kw)
    good = ok()
    assert Plan(M, [good]).kernels == 1
    cases = [
        (ok(op=7), "bad op"),
        (ok(words=3), "words_per_thread"),
        (ok(tile_rows=-1), "tile_rows"),
        (ok(depends_on=0), "earlier job"),                 # itself
        (ok(depends_on=-2), "earlier job"),
        (ok(path=5), "path must be"),
        (ok(se=(0, 3)), "structuring element"),
        (ok(se=(3, 3), origin=(3, 1)), "structuring element"),
        (ok(dst=page(M, 1, W_=W - 1)), "sizes"),
        (ok(src=page(M, 0, offset=4)), "misaligned"),      # 64-bit words on a 4-byte boundary
        (ok(dst=page(M, 0, offset=8 * NW * 100)), "overlaps"),
        (ok(src=page(M, 0, stride=NW - 1)), "stride"),
        (ok(src=page(M, 0, W_=70000, H_=8), dst=page(M, 1, W_=70000, H_=8), path=1), "65535"),
        (ok(op=TO_RLE, dst=page(M, 1)), "MORPH_TO_RLE"),
    ]
    for bad, words in cases:
        msg = rejected(M, [bad])
        assert msg.startswith("job 0:") and words in msg, (words, msg)
    # the failing job is named when it is not the first one
    msg = rejected(M, [good, ok(src=page(M, 2), dst=page(M, 3), op=9)])
    assert msg.startswith("job 1:")


def test_a_dependency_on_a_grouped_job_waits_for_every_level(M):
    """A persistent-kernel job after a grouped packed job is ordered by the
    stream (groups first), not by a wait inside the kernel: the plan still
    builds and keeps both launches."""
    jobs = [job(M, CLOSE, page(M, 0), page(M, 1), se=(3, 3)),
            job(M, TO_RLE, page(M, 1), rle_image(M, 0), depends_on=0)]
    p = Plan(M, jobs)
    assert p.kernels == 2
    alone = Plan(M, [job(M, TO_RLE, page(M, 1), rle_image(M, 0))])
    assert p.items == alone.items
