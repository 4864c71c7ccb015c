#!/usr/bin/env python3
"""Benchmark of the rectangular-morphology hot path on GB300.

Workload (letter pages at 300 dpi): B distinct seeded 2550 x 3300 document
pages (8 % ink, 2-3 columns, ruled lines, boxes) resident in HBM.  One step =
one batch launch (captured as a CUDA graph) that opens and closes every page
with each of the rectangles 3x3, 7x7, 15x15, 31x31, 51x51, 1x51 and 51x1,
once on the packed path and once on the RLE path, i.e. 28 page-operations per
page.  The batch planner groups the packed jobs by tile variant (one launch of
the rectangle tile per group), encodes each page to runs once in the
persistent batch kernel, and runs the RLE jobs as groups of the run-length
source tile that read those runs (the algorithmic bytes count the encode once
per page): ten kernel launches per step on the letter workload.

Metric: page-operation pixels per second (Gpix/s) over the whole step.  The
JSON line also carries pages/s, the packed-only and RLE-only rates (timed as
separate batches), the roofline of the dominant kernel (the grouped launch of
the two-stage tile with counter vertical passes: open / close by 15x15, 31x31
and 51x51 on the packed path, timed alone with CUDA events, algorithmic
bytes against the measured HBM copy bandwidth), the same ratio for the whole
step, an end-to-end figure through the same API with host buffers (H2D of the
pages and D2H of every result inside the timed region), sampled SM clocks,
and the CPU oracle timed on a bounded sample of the same workload on this
host's cores.

--impl reference times the CPU oracle (plain C on unpacked bytes) on the same
workload, a bounded sample per step.
"""
import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

W, H = 2550, 3300
SES = [(3, 3), (7, 7), (15, 15), (31, 31), (51, 51), (1, 51), (51, 1)]
OPS = ["open", "close"]
METRIC = "Gpix/s rect erode/dilate (packed, RLE) vs HBM peak; batched pages/s; p50/p99 ms"
UNIT = "Gpix/s"
WORKLOAD = ("letter-300dpi: 2550x3300 text pages, open+close x {3,7,15,31,51 squares, "
            "1x51, 51x1}, packed and RLE paths (a page's RLE jobs share one bitmap->RLE "
            "encode per step), one batch launch per step (grouped tile kernels and the "
            "persistent encode kernel, one CUDA graph)")


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------ host cores
def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(pages, seconds_cap, threads):
    """Run the CPU oracle on pages until the op list is done or the cap is
    hit; returns (pixel-ops, seconds, description)."""
    import oracle
    t0 = time.perf_counter()
    pix, nops = 0, 0
    for img in pages:
        rp, runs = oracle.rle_encode(img)
        for path in ("packed", "rle"):
            for (sw, sh) in SES:
                for op in OPS:
                    if path == "packed":
                        oracle.apply(op, img, sw, sh, mode="separable", threads=threads)
                    else:
                        oracle.rle_apply(op, rp, runs, W, H, sw, sh, mode="separable", threads=threads)
                    pix += W * H
                    nops += 1
                    if time.perf_counter() - t0 > seconds_cap:
                        dt = time.perf_counter() - t0
                        return pix, dt, "%d page-ops (separable mode) on %d letter page(s)" % (nops, len(pages))
    dt = time.perf_counter() - t0
    return pix, dt, "%d page-ops (separable mode) on %d letter page(s)" % (nops, len(pages))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling (every 100 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- workload
def pmap(fn, items):
    """Map on host threads (the C page generator releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(32, cpu_count())) as ex:
        return list(ex.map(fn, items))


def make_pages(n, seed_base=0):
    from paper_0712_0121_gb300 import synth
    return pmap(lambda k: synth.document_page(W, H, synth.seed_for(2, seed_base + k), 0.08)[0], range(n))


NW = (W + 63) // 64  # 64-bit words per row




def build_jobs(M, srcs, paths):
    """Jobs over the pages; every result in one contiguous device tensor."""
    import torch
    n = len(srcs) * len(paths) * len(SES) * len(OPS)
    out = torch.empty((n, H, NW), dtype=torch.int64, device="cuda")
    jobs, k = [], 0
    for src in srcs:
        for path in paths:
            for (sw, sh) in SES:
                for op in OPS:
                    jobs.append(dict(op=op, se=(sw, sh), path=path, src=src, dst=M.Packed(out[k], W)))
                    k += 1
    return jobs, out


def alg_bytes(job_path, runs_in, runs_out_per_op):
    """Algorithmic bytes of one page-operation (roofline numerator)."""
    page = H * NW * 8
    if job_path == "packed":
        return 2 * page
    # bitmap in, runs written and read back, result runs, bitmap out
    return 2 * page + 4 * (2 * runs_in + 2 * runs_out_per_op) + 4 * 4 * (H + 1)


def encode_bytes(runs_in):
    """Algorithmic bytes of one bitmap -> runs encode of a page."""
    return H * NW * 8 + 4 * runs_in + 4 * (H + 1)


def max_over_ranks(x: float) -> float:
    """Max of a float over the ranks of the default process group (the step
    time every rank reports is the slowest rank's); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units processed by all ranks per second, timed by the slowest rank."""
    return units_per_rank * world / (ms_max * 1e-3)


# The dominant kernel of a step (the largest share of the step's launch
# list, profiles/bench_step_letter300_launch_list.md): the run-length-source
# tile's grouped launch that runs the RLE open / close jobs of these
# rectangles (two stages, van Herk / Gil-Werman rings, doubling second
# horizontal pass).
DOMINANT_PATH = "rle"
DOMINANT_SES = ((7, 7), (15, 15))
DOMINANT_KERNEL = ("k_rle_rect<2 stages, 2 words/thread, ring vertical, log horizontal>: the grouped "
                   "launch of the RLE open/close jobs by 7x7 and 15x15 (runs in, bitmap out), timed "
                   "without the persistent encode kernel")
# Sources that kernel and its planner are built from.
DOMINANT_SOURCES = ("rle_rect.cuh", "rle_rect_kernels.cuh", "rle_rect_w2.cu", "rect_tile.cuh", "rect.cu",
                    "rle_tile.cuh", "counters.cuh", "morph_internal.cuh", "batch.cu")


def csrc_digest():
    """SHA-256 over the sources of the dominant kernel (ties a profile record
    of that kernel to the code it was taken from)."""
    import hashlib
    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_0712_0121_gb300", "csrc", f) for f in DOMINANT_SOURCES]
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + b"\0" + fh.read())
    return h.hexdigest()


def profile_traffic(name, pages):
    """DRAM bytes per launch from a committed ncu record (profiles/<name>),
    scaled to `pages` pages, or None when the record is missing or was taken
    from other kernel sources."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("|"):
                    k, v = line.split(":", 1)
                    kv[k.strip().strip("-* `")] = v.strip().strip("`")
        if kv.get("csrc_sha256") != csrc_digest():
            return None
        return int(float(kv["dram_bytes_per_launch"]) * pages / float(kv["pages"]))
    except (OSError, KeyError, ValueError):
        return None


def measured_peak():
    """(HBM GB/s, source) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# A device-side delay queued before every timed launch (about 0.5 ms at a
# 2.07 GHz SM clock): the start event and the launch are enqueued while it
# runs, so the host's time to enqueue them (binding, plan, launch call) falls
# outside the event pair, which then brackets the device work alone.
QUEUE_AHEAD_CYCLES = 1_000_000


def time_launches(fn, steps, stream):
    import torch
    times = []
    for _ in range(steps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            torch.cuda._sleep(QUEUE_AHEAD_CYCLES)
        s.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        times.append(s.elapsed_time(e))
    return times


# Rectangles of the letter-page and 600-dpi workloads, timed one by one.
PER_OP_SES = [(3, 3), (5, 5), (7, 7), (15, 15), (31, 31), (51, 51), (1, 51), (51, 1), (101, 1), (1, 61)]
DENSITY_KINDS = ("blank", "text", "halftone", "noise")
DENSITY_OPS = (("dilate", 101, 1), ("dilate", 1, 61), ("open", 5, 5))
DENSITY_DISCS = (3, 12, 25)


def median_ms(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    return statistics.median(time_launches(fn, reps, stream))


def run_per_op(M, dev_in, peak, stream, reps):
    """Each rectangle of the letter-page and 600-dpi workloads alone, erode /
    dilate / open / close on the packed path, over the B resident pages seen
    as one 2550 x (B * 3300) image (more than L2; windows cross the page
    seams, the same work per pixel).  Algorithmic bytes: one read and one
    write of the bitmap (2 bits per pixel)."""
    import torch
    B = dev_in.shape[0]
    stack = M.Packed(dev_in.view(B * H, NW), W)
    dst = M.Packed.empty(W, B * H, 64)
    page_bytes = B * H * NW * 8
    out = []
    for (sw, sh) in PER_OP_SES:
        row = {"se": "%dx%d" % (sw, sh)}
        for op in ("erode", "dilate", "open", "close"):
            ws = torch.empty(max(1, M.workspace_size(op, dst, stack, sw, sh)), dtype=torch.uint8, device="cuda")
            ms = median_ms(lambda: M.morph_rect(op, dst, stack, sw, sh, workspace=ws), reps, stream)
            gbs = 2 * page_bytes / (ms * 1e-3) / 1e9
            row[op] = {"ms": round(ms, 4), "gpix_s": round(W * B * H / (ms * 1e-3) / 1e9, 1),
                       "alg_gb_s": round(gbs, 1), "frac": round(gbs / peak, 3)}
        out.append(row)
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d after the per-op table" % st)
    del dst
    torch.cuda.empty_cache()
    return out


def rle_bytes(W_, H_, runs):
    return 4 * runs + 4 * (H_ + 1)


def run_density_sweep(M, peak, stream, reps, copies):
    """600-dpi pages (5100 x 6600) of four kinds — near-blank 0.5 %, text 8 %,
    halftone 45 %, salt-and-pepper 5 % — each stacked `copies` times into one
    tall image (distinct memory, more than L2).  For each op: the packed path,
    and the RLE path with runs in and out (bitmap -> runs and runs -> bitmap
    timed on their own).  Algorithmic bytes: packed 2 bits per pixel; RLE op 4
    bytes per run in and out plus the row offsets."""
    import torch
    from paper_0712_0121_gb300 import synth
    Wd, Hd = 5100, 6600
    nwd = (Wd + 63) // 64
    rows = Hd * copies
    out = []
    for kind in DENSITY_KINDS:
        img, ink = synth.config3_page(kind)
        one = M.pack(img, 64).words
        stack_t = one.repeat(copies, 1)
        stack = M.Packed(stack_t, Wd)
        dst = M.Packed.empty(Wd, rows, 64)
        cap = rows * (Wd // 2 + 1)
        a, b = M.Rle.empty(Wd, rows, cap), M.Rle.empty(Wd, rows, cap)
        cws = torch.empty(M.convert_workspace_size(rows), dtype=torch.uint8, device="cuda")
        bmp_bytes = rows * nwd * 8
        t_enc = median_ms(lambda: M.rle_from_bitmap(a, stack, cws), reps, stream)
        runs_in = int(a.n_runs.item())
        t_dec = median_ms(lambda: M.rle_to_bitmap(dst, a), reps, stream)
        enc_b = bmp_bytes + rle_bytes(Wd, rows, runs_in)
        rec = {"kind": kind, "ink": round(float(ink), 4), "runs_per_row": round(runs_in / rows, 1),
               "to_rle": {"ms": round(t_enc, 4), "gpix_s": round(Wd * rows / (t_enc * 1e-3) / 1e9, 1),
                          "alg_gb_s": round(enc_b / (t_enc * 1e-3) / 1e9, 1),
                          "frac": round(enc_b / (t_enc * 1e-3) / 1e9 / peak, 3)},
               "to_bitmap": {"ms": round(t_dec, 4), "gpix_s": round(Wd * rows / (t_dec * 1e-3) / 1e9, 1),
                             "alg_gb_s": round(enc_b / (t_dec * 1e-3) / 1e9, 1),
                             "frac": round(enc_b / (t_dec * 1e-3) / 1e9 / peak, 3)},
               "ops": []}
        for op, sw, sh in DENSITY_OPS:
            pws = torch.empty(max(1, M.workspace_size(op, dst, stack, sw, sh)), dtype=torch.uint8, device="cuda")
            t_p = median_ms(lambda: M.morph_rect(op, dst, stack, sw, sh, workspace=pws), reps, stream)
            rws = torch.empty(max(1, M.workspace_size(op, b, a, sw, sh)), dtype=torch.uint8, device="cuda")
            t_r = median_ms(lambda: M.morph_rect(op, b, a, sw, sh, workspace=rws), reps, stream)
            runs_out = int(b.n_runs.item())
            pb = 2 * bmp_bytes
            rb = rle_bytes(Wd, rows, runs_in) + rle_bytes(Wd, rows, runs_out)
            rec["ops"].append({
                "op": "%s %dx%d" % (op, sw, sh),
                "packed": {"ms": round(t_p, 4), "gpix_s": round(Wd * rows / (t_p * 1e-3) / 1e9, 1),
                           "frac": round(pb / (t_p * 1e-3) / 1e9 / peak, 3)},
                "rle": {"ms": round(t_r, 4), "gpix_s": round(Wd * rows / (t_r * 1e-3) / 1e9, 1),
                        "alg_gb_s": round(rb / (t_r * 1e-3) / 1e9, 1),
                        "frac": round(rb / (t_r * 1e-3) / 1e9 / peak, 3), "runs_out_per_row": round(runs_out / rows, 1),
                        "with_conversions_gpix_s": round(Wd * rows / ((t_r + t_enc + t_dec) * 1e-3) / 1e9, 1)},
            })
            del pws, rws
        # closing by discs (section "Experiments", circular masks): the
        # packed path and the RLE path (runs in, runs out)
        rec["disc_close"] = []
        for r in DENSITY_DISCS:
            disc = np.zeros((2 * r + 1, 2 * r + 1), np.uint8)
            jj, ii = np.mgrid[0:2 * r + 1, 0:2 * r + 1]
            disc[((ii - r) ** 2 + (jj - r) ** 2) <= r * r] = 1
            pws = torch.empty(max(1, M.mask_workspace_size("close", dst, stack, disc, r, r)), dtype=torch.uint8,
                              device="cuda")
            t_p = median_ms(lambda: M.morph_mask("close", dst, stack, disc, r, r, workspace=pws), reps, stream)
            rws = torch.empty(max(1, M.mask_workspace_size("close", b, a, disc, r, r)), dtype=torch.uint8,
                              device="cuda")
            t_r = median_ms(lambda: M.morph_mask("close", b, a, disc, r, r, workspace=rws), reps, stream)
            rec["disc_close"].append({"r": r, "element_runs": 2 * r + 1,
                                      "packed_ms": round(t_p, 4), "rle_ms": round(t_r, 4),
                                      "runs_out_per_row": round(int(b.n_runs.item()) / rows, 1)})
            del pws, rws
        st = M.sync_status()
        if st != M.MORPH_OK:
            raise RuntimeError("device status %d in the density sweep (%s)" % (st, kind))
        out.append(rec)
        del stack_t, stack, dst, a, b, cws
        torch.cuda.empty_cache()
    return {"pages": "one seeded page per kind, stacked %d times (%d rows, %.0f MB packed)"
                     % (copies, rows, rows * nwd * 8 / 1e6), "results": out}


def run_config1(M, stream, reps):
    """512 x 512 text page (packed u32 rows): erode / dilate by 3x3, 11x1 and
    1x11 on the packed and RLE paths, and the RLE round trip.  One page is
    32 KB and stays in L2: device times of single launches (a page this
    small leaves most SMs idle)."""
    import torch
    from paper_0712_0121_gb300 import synth
    img, ink = synth.config1_page()
    Hc, Wc = img.shape
    src = M.pack(img, 32)
    dst = M.Packed.empty(Wc, Hc, 32)
    cap = Hc * (Wc // 2 + 1)
    a, b = M.Rle.empty(Wc, Hc, cap), M.Rle.empty(Wc, Hc, cap)
    cws = torch.empty(M.convert_workspace_size(Hc), dtype=torch.uint8, device="cuda")
    rec = {"ink": round(float(ink), 4), "ops": []}
    t_enc = median_ms(lambda: M.rle_from_bitmap(a, src, cws), reps, stream)
    t_dec = median_ms(lambda: M.rle_to_bitmap(dst, a), reps, stream)
    rec["to_rle_us"], rec["to_bitmap_us"] = round(t_enc * 1e3, 2), round(t_dec * 1e3, 2)
    for op in ("erode", "dilate"):
        for sw, sh in ((3, 3), (11, 1), (1, 11)):
            t_p = median_ms(lambda: M.morph_rect(op, dst, src, sw, sh), reps, stream)
            rws = torch.empty(max(1, M.workspace_size(op, b, a, sw, sh)), dtype=torch.uint8, device="cuda")
            t_r = median_ms(lambda: M.morph_rect(op, b, a, sw, sh, workspace=rws), reps, stream)
            rec["ops"].append({"op": "%s %dx%d" % (op, sw, sh), "packed_us": round(t_p * 1e3, 2),
                               "rle_us": round(t_r * 1e3, 2)})
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d in config 1" % st)
    return rec


def run_uneven_batch(M, args, stream):
    """Uneven batch: seeded pages of four sizes, ink density U(1,30) %, each
    with its own rectangle and op; per-page path, band and word tile from
    the autotuner (tuned per page size); one batch launch (CUDA graph) vs the same
    per-page launches captured in one CUDA graph, and vs a host loop of
    them."""
    import torch
    from paper_0712_0121_gb300 import autotune, synth
    t0 = time.perf_counter()
    specs = synth.config4_jobs(args.batch_pages)
    tuner = autotune.Tuner(cache_path=args.tune_cache, pages_per_class=4, reps=2)
    sizes = sorted({(j["W"], j["H"]) for j in specs})
    if not all(tuner.tuned(W_, H_) for W_, H_ in sizes):
        # every page size of the workload is its own class
        for W_, H_ in sizes:
            tuner.tune_grid(W_, H_, synth.CONFIG4_OPS, synth.CONFIG4_SES,
                            densities=(0.01, 0.05, 0.15, 0.3), bands=(64, 128, 256, 512))
        tuner.save()
    t_tune = time.perf_counter() - t0
    imgs = pmap(lambda j: synth.config4_page(j)[0], specs)
    jobs, npix, nrle = [], 0, 0
    wchosen = {}  # packed pages per size by the word tile the tuner chose
    for j, img in zip(specs, imgs):
        src = M.pack(img, 64)
        dst = M.Packed.empty(j["W"], j["H"], 64)
        path, band = tuner.choose(j["W"], j["H"], j["op"], j["se"], j["density"])
        words = tuner.words(j["W"], j["H"], j["op"], j["se"])
        nrle += path == "rle"
        if path == "packed":
            wkey = "%dx%d" % (j["W"], j["H"])
            wchosen.setdefault(wkey, {"planner": 0, "2": 0, "4": 0})[str(words) if words else "planner"] += 1
        jobs.append(dict(op=j["op"], se=j["se"], path=path, tile_rows=band, words_per_thread=words, src=src, dst=dst))
        npix += j["W"] * j["H"]
    del imgs
    batch = M.Batch(jobs)
    graph = batch.capture()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    tb = statistics.mean(time_launches(graph.replay, 5, stream))
    ws = torch.empty(max(M.convert_workspace_size(6600), 1 << 20), dtype=torch.uint8, device="cuda")
    rles = {}

    def loop():
        for j in jobs:
            if j["path"] == "rle":
                key = (j["src"].width, j["src"].height)
                if key not in rles:
                    cap = key[1] * (key[0] // 16 + 4)
                    rles[key] = (M.Rle.empty(key[0], key[1], cap), M.Rle.empty(key[0], key[1], cap))
                a, b = rles[key]
                M.rle_from_bitmap(a, j["src"], ws)
                M.morph_rect(j["op"], b, a, *j["se"])
                M.rle_to_bitmap(j["dst"], b)
            else:
                M.morph_rect(j["op"], j["dst"], j["src"], *j["se"])

    for _ in range(2):
        loop()
    torch.cuda.synchronize()
    tl = statistics.mean(time_launches(loop, 3, stream))
    # the fair baseline: the same per-page launches captured once in a CUDA
    # graph (no host work per page left in the timed region)
    pg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pg):
        loop()
    for _ in range(2):
        pg.replay()
    torch.cuda.synchronize()
    tg = statistics.mean(time_launches(pg.replay, 5, stream))
    st = M.sync_status()
    peak = measured_peak()[0]
    alg = sum(2 * j["src"].height * ((j["src"].width + 63) // 64) * 8 for j in jobs)
    return {"pages": len(jobs), "rle_path_pages": nrle, "megapixels": round(npix / 1e6, 1),
            "size_classes_tuned": [list(sz) for sz in sizes],
            "words_per_thread_chosen": wchosen,
            "batch_ms": round(tb, 3), "batch_pages_s": round(len(jobs) / tb * 1e3, 1),
            "batch_gpix_s": round(npix / tb / 1e6, 1),
            "batch_roofline": {"alg_bytes": int(alg), "alg_gb_s": round(alg / tb / 1e6, 1),
                               "frac": round(alg / tb / 1e6 / peak, 3),
                               "note": "2 bits per pixel per page-operation (bitmap in and out)"},
            "graph_per_page_ms": round(tg, 3), "graph_per_page_pages_s": round(len(jobs) / tg * 1e3, 1),
            "speedup_vs_graph": round(tg / tb, 2),
            "per_page_loop_ms": round(tl, 3), "per_page_loop_pages_s": round(len(jobs) / tl * 1e3, 1),
            "speedup_vs_host_loop": round(tl / tb, 2), "status": st, "tune_s": round(t_tune, 1)}


SERVE_RATES = (50, 200, 1000, 5000, 20000)


def run_serving(M, args):
    """Poisson arrivals of 5100x6600 pages (near-blank, text, halftone,
    noise), pipeline close(31x1) -> open(3x3) -> dilate(1x15) -> RLE, 40 GB
    budget: continuous batching vs an unbatched per-page server.  The pool
    holds 256 device-resident pages (64 copies of each kind in distinct
    memory, 1.08 GB: far more than L2), so requests read HBM.  Rates beyond
    what one page at a time can sustain (5000 and 20000 pages/s) show the
    batching at work; each run stops admitting after its arrival window plus
    half of it again, and sustained pages/s counts completed requests."""
    import torch
    from paper_0712_0121_gb300 import synth
    from paper_0712_0121_gb300.serve import BatchExecutor, PerPageExecutor, Server, poisson_arrivals
    PW, PH = 5100, 6600
    kinds = [M.pack(synth.config3_page(kind, page=0)[0], 64) for kind in synth.CONFIG3_KINDS]
    pool = [M.Packed(kinds[k % len(kinds)].words.clone(), PW) for k in range(args.serve_pool)]
    bex = BatchExecutor(pool, PW, PH, n_slots=64, n_streams=4)
    pex = PerPageExecutor(pool, PW, PH)
    # warm-up both paths
    Server(bex, 40e9).run(poisson_arrivals(2000.0, 64, 1), np.arange(64) % len(pool))
    Server(pex, 40e9).run(poisson_arrivals(2000.0, 4, 1), np.arange(4) % len(pool))
    torch.cuda.synchronize()
    out = {"pool_pages": len(pool), "pool_bytes": int(sum(p.words.numel() * 8 for p in pool)),
           "slot_bytes": int(bex.slot_bytes), "slots": bex.n_slots, "budget_bytes": int(40e9)}
    keep = ("p50_ms", "p99_ms", "queue_p99_ms", "sustained_pages_s", "mean_batch", "max_in_flight", "completed")
    best = {"batched": 0.0, "per_page": 0.0}
    for rate in SERVE_RATES:
        n = max(20, int(rate * args.serve_seconds))
        arr = poisson_arrivals(float(rate), n, seed=5000 + rate)
        pages = np.random.default_rng(rate).integers(0, len(pool), size=n)
        limit = 1.5 * float(arr[-1])
        # the garbage collector stays off while requests are timed (both
        # modes alike): its pauses are host noise, not serving latency
        gc.collect()
        gc.disable()
        try:
            sb = Server(bex, 40e9).run(arr, pages, time_limit=limit).summary()
            sp = Server(pex, 40e9).run(arr, pages, time_limit=limit).summary()
        finally:
            gc.enable()
        rec = {"requests": n}
        for name, sm in (("batched", sb), ("per_page", sp)):
            rec[name] = {k: (round(sm[k], 3) if isinstance(sm[k], float) else sm[k]) for k in keep}
            # highest offered rate served in full with p99 under 50 ms
            if sm["completed"] == n and sm["p99_ms"] is not None and sm["p99_ms"] < 50.0:
                best[name] = max(best[name], float(rate))
        out[str(rate)] = rec
    out["max_rate_p99_under_50ms"] = best
    st = M.sync_status()
    out["status"] = st
    return out


def run_probe(args):
    """Standalone operations, repeated, on a tall stack of distinct letter
    pages (more than L2): a target for ncu captures of a single kernel, and
    a timing of each kernel alone (CUDA events, median of the repetitions)
    with its algorithmic bytes against the measured HBM copy bandwidth."""
    import torch
    from paper_0712_0121_gb300 import morph as M
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    pages = make_pages(16)
    img = np.concatenate([pages[k % 16] for k in range(args.probe_pages)], axis=0)
    Ht, Wt = img.shape
    src = M.pack(img, 64)
    page_bytes = src.words.numel() * 8
    peak = 6782.1
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    results = []
    if args.probe == "cc":
        return run_probe_cc(args, M, src, Wt, Ht, peak, stream)
    if args.probe == "layout":
        return run_probe_layout(args, M, stream)
    if args.probe == "line":
        return run_probe_line(args, M, src, Wt, Ht, page_bytes, peak, stream)
    if args.probe == "xpose":
        return run_probe_xpose(args, M, src, Wt, Ht, page_bytes, peak, stream)
    for se in args.probe_se.split(","):
        if args.probe == "mask":
            # "d<r>": digital disc of radius r; "WxH": the full rectangle as a mask
            if se.startswith("d"):
                r = int(se[1:])
                jj, ii = np.mgrid[0:2 * r + 1, 0:2 * r + 1]
                mask = (((ii - r) ** 2 + (jj - r) ** 2) <= r * r).astype(np.uint8)
            else:
                mw, mh = (int(v) for v in se.split("x"))
                mask = np.ones((mh, mw), np.uint8)
            dst = M.Packed.empty(Wt, Ht, 64)
            ox, oy = mask.shape[1] // 2, mask.shape[0] // 2
            ws = torch.empty(max(1, M.mask_workspace_size(args.probe_op, dst, src, mask, ox, oy)),
                             dtype=torch.uint8, device="cuda")
            fn = lambda: M.morph_mask(args.probe_op, dst, src, mask, ox, oy, workspace=ws)  # noqa: E731
            alg = 2 * page_bytes
        elif args.probe == "packed":
            sw, sh = (int(v) for v in se.split("x"))
            dst = M.Packed.empty(Wt, Ht, 64)
            fn = lambda: M.morph_rect(args.probe_op, dst, src, sw, sh)  # noqa: E731
            alg = 2 * page_bytes
        else:
            sw, sh = (int(v) for v in se.split("x"))
            cap = Ht * args.rle_runs_per_row
            a, b = M.Rle.empty(Wt, Ht, cap), M.Rle.empty(Wt, Ht, cap)
            out = M.Packed.empty(Wt, Ht, 64)
            ws = torch.empty(M.workspace_size(args.probe_op, b, a, sw, sh), dtype=torch.uint8, device="cuda")
            cws = torch.empty(M.convert_workspace_size(Ht), dtype=torch.uint8, device="cuda")

            def fn():
                M.rle_from_bitmap(a, src, cws)
                M.morph_rect(args.probe_op, b, a, sw, sh, workspace=ws)
                M.rle_to_bitmap(out, b)
            alg = 2 * page_bytes
        fn()
        torch.cuda.synchronize()
        ms = statistics.median(time_launches(fn, args.probe_reps, stream))
        st = M.sync_status()
        results.append({"se": se, "ms": round(ms, 4), "gpix_s": round(Wt * Ht / ms / 1e6, 1),
                        "alg_gb_s": round(alg / ms / 1e6, 1), "frac": round(alg / ms / 1e6 / peak, 3),
                        "status": st})
        if st != M.MORPH_OK:
            print(json.dumps(results[-1]))
            raise SystemExit(1)
    print(json.dumps({"probe": args.probe, "op": args.probe_op, "width": Wt, "height": Ht,
                      "peak_gb_s": peak, "results": results}))


def run_probe_cc(args, M, src, Wt, Ht, peak, stream):
    """Connected components (connectivity 4 or 8, with statistics) and the
    run-length histograms of the RLE form of the stack; --probe-se lists
    "4", "8" and "hist".  Algorithmic bytes: the runs and row offsets read
    once, one label written per run and one record per component."""
    import torch
    cap = Ht * args.rle_runs_per_row
    rle = M.Rle.empty(Wt, Ht, cap)
    M.rle_from_bitmap(rle, src)
    n_runs = int(rle.n_runs.item())
    labels = torch.empty(max(n_runs, 1), dtype=torch.int32, device="cuda")
    ws = torch.empty(M.components_workspace_size(rle), dtype=torch.uint8, device="cuda")
    nc = torch.zeros(1, dtype=torch.int64, device="cuda")
    base = 4 * n_runs + 4 * (Ht + 1)
    results = []
    for tok in args.probe_se.split(","):
        if tok == "hist":
            black = torch.empty(Wt + 1, dtype=torch.int64, device="cuda")
            white = torch.empty(Wt + 1, dtype=torch.int64, device="cuda")
            fn = lambda: M.run_length_hist(rle, black, white)  # noqa: E731
            alg, extra = base, {}
        else:
            conn = int(tok)
            M.rle_components(rle, conn, labels=labels, stats=False, n_components=nc, workspace=ws)
            n = int(nc.item())
            stats = torch.empty((max(n, 1), 7), dtype=torch.int64, device="cuda")
            fn = lambda: M.rle_components(rle, conn, labels=labels, stats=stats,  # noqa: E731
                                          n_components=nc, workspace=ws)
            alg, extra = base + 4 * n_runs + 56 * n, {"components": n}
        fn()
        torch.cuda.synchronize()
        ms = statistics.median(time_launches(fn, args.probe_reps, stream))
        st = M.sync_status()
        r = {"se": tok, "ms": round(ms, 4), "gpix_s": round(Wt * Ht / ms / 1e6, 1),
             "gruns_s": round(n_runs / ms / 1e6, 2), "alg_gb_s": round(alg / ms / 1e6, 1),
             "frac": round(alg / ms / 1e6 / peak, 3), "status": st}
        r.update(extra)
        results.append(r)
        if st != M.MORPH_OK:
            print(json.dumps(r))
            raise SystemExit(1)
    print(json.dumps({"probe": "cc", "width": Wt, "height": Ht, "runs": n_runs, "peak_gb_s": peak,
                      "results": results}))


def run_probe_layout(args, M, stream):
    """Layout analysis of single letter pages (2550 x 3300), one call per
    page (each call reads two histograms back to the host), as pages/s over
    16 distinct pages."""
    import torch
    pages = [M.pack(p, 64) for p in make_pages(16)]
    ws = torch.empty(M.layout_workspace_size(pages[0]), dtype=torch.uint8, device="cuda")
    boxes = torch.empty((65536, 7), dtype=torch.int64, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    found = []
    for pg in pages:
        _, _, gaps = M.layout_boxes(pg, 90, boxes=boxes, n_boxes=nb, workspace=ws)
        found.append((gaps, int(nb.item())))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = max(1, args.probe_reps)
    for _ in range(reps):
        for pg in pages:
            M.layout_boxes(pg, 90, boxes=boxes, n_boxes=nb, workspace=ws)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / (reps * len(pages))
    st = M.sync_status()
    print(json.dumps({"probe": "layout", "width": W, "height": H, "ms_per_page": round(dt * 1e3, 4),
                      "pages_s": round(1.0 / dt, 1), "gaps_and_blocks": found[:4], "status": st}))
    if st != M.MORPH_OK:
        raise SystemExit(1)


def run_probe_line(args, M, src, Wt, Ht, page_bytes, peak, stream):
    """Line elements of half length 12 at the angles (degrees) listed in
    --probe-se, --probe-op erode / dilate / open / close, on the stack
    (skew, axis-parallel line, skew back; the transposed case for lines
    nearer the x axis).  Algorithmic bytes: the page read and written once."""
    import torch
    results = []
    dst = M.Packed.empty(Wt, Ht, 64)
    for tok in args.probe_se.split(","):
        angle = float(tok)
        shift, L, o, horizontal = M.line_element(angle, 12, Wt, Ht)
        n = M.sheared_line_workspace_size(args.probe_op, src, shift, L, horizontal)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        fn = lambda: M.sheared_line(args.probe_op, dst, src, shift, L, o, horizontal,  # noqa: E731
                                    workspace=ws)
        fn()
        torch.cuda.synchronize()
        ms = statistics.median(time_launches(fn, args.probe_reps, stream))
        st = M.sync_status()
        alg = 2 * page_bytes
        results.append({"se": tok, "length": L, "horizontal": bool(horizontal), "ms": round(ms, 4),
                        "gpix_s": round(Wt * Ht / ms / 1e6, 1), "alg_gb_s": round(alg / ms / 1e6, 1),
                        "frac": round(alg / ms / 1e6 / peak, 3), "status": st})
        if st != M.MORPH_OK:
            print(json.dumps(results[-1]))
            raise SystemExit(1)
    print(json.dumps({"probe": "line", "op": args.probe_op, "width": Wt, "height": Ht,
                      "peak_gb_s": peak, "results": results}))


def run_probe_xpose(args, M, src, Wt, Ht, page_bytes, peak, stream):
    """Transposition (section "Efficient Transpose") of the stack, or of its
    first 65535 rows for RLE (the transpose's width must fit 16-bit runs);
    --probe-se lists "packed", "rle" and "rletH" (a 1 x H erosion done as the
    H x 1 erosion of the transpose, transposed back, next to the direct RLE
    erosion).  Algorithmic bytes: the packed page read and written once; for
    RLE the runs and row offsets of input and output."""
    import torch
    results = []
    for tok in args.probe_se.split(","):
        extra = {}
        if tok == "packed":
            dst = M.Packed.empty(Ht, Wt, 64)
            fn = lambda: M.transpose(dst, src)  # noqa: E731
            W, H, alg = Wt, Ht, 2 * page_bytes
        else:
            H = min(Ht, 65535)
            W = Wt
            sub = M.Packed(src.words[:H], Wt)
            a = M.Rle.empty(W, H, H * args.rle_runs_per_row)
            M.rle_from_bitmap(a, sub)
            n_in = int(a.n_runs.item())
            cap_t = W * (H // 2 + 1)
            t = M.Rle.empty(H, W, cap_t)
            ws = torch.empty(M.rle_transpose_workspace_size(a), dtype=torch.uint8, device="cuda")
            M.rle_transpose(t, a, ws)
            n_out = int(t.n_runs.item())
            extra = {"runs_in": n_in, "runs_out": n_out}
            if tok == "rle":
                fn = lambda: M.rle_transpose(t, a, ws)  # noqa: E731
                alg = 4 * (n_in + n_out) + 4 * (H + 1) + 4 * (W + 1)
            else:
                h = int(tok[4:])
                t2 = M.Rle.empty(H, W, cap_t)
                back = M.Rle.empty(W, H, H * args.rle_runs_per_row)
                ws_b = torch.empty(M.rle_transpose_workspace_size(t2), dtype=torch.uint8, device="cuda")
                direct = M.Rle.empty(W, H, H * args.rle_runs_per_row)
                wsd = torch.empty(M.workspace_size("erode", direct, a, 1, h), dtype=torch.uint8,
                                  device="cuda")
                wst = torch.empty(M.workspace_size("erode", t2, t, h, 1), dtype=torch.uint8,
                                  device="cuda")

                def fn():
                    M.rle_transpose(t, a, ws)
                    M.morph_rect("erode", t2, t, h, 1, workspace=wst)
                    M.rle_transpose(back, t2, ws_b)
                fd = lambda: M.morph_rect("erode", direct, a, 1, h, workspace=wsd)  # noqa: E731
                fd()
                torch.cuda.synchronize()
                extra["direct_ms"] = round(statistics.median(time_launches(fd, args.probe_reps, stream)), 4)
                alg = 8 * n_in + 4 * (H + 1)
        fn()
        torch.cuda.synchronize()
        ms = statistics.median(time_launches(fn, args.probe_reps, stream))
        st = M.sync_status()
        r = {"se": tok, "width": W, "height": H, "ms": round(ms, 4),
             "gpix_s": round(W * H / ms / 1e6, 1), "alg_gb_s": round(alg / ms / 1e6, 1),
             "frac": round(alg / ms / 1e6 / peak, 3), "status": st}
        r.update(extra)
        results.append(r)
        if st != M.MORPH_OK:
            print(json.dumps(r))
            raise SystemExit(1)
    print(json.dumps({"probe": "xpose", "peak_gb_s": peak, "results": results}))


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_0712_0121_gb300 import morph as M

    B = args.pages
    t_gen = time.perf_counter()
    pages = make_pages(B, seed_base=rank * B)
    t_gen = time.perf_counter() - t_gen
    dev_in = torch.empty((B, H, NW), dtype=torch.int64, device="cuda")
    for k, p in enumerate(pages):
        dev_in[k].copy_(M.pack(p, 64).words)
    srcs = [M.Packed(dev_in[k], W) for k in range(B)]
    torch.cuda.synchronize()

    jobs, dev_out = build_jobs(M, srcs, ("packed", "rle"))
    batch = M.Batch(jobs, rle_runs_per_row=args.rle_runs_per_row)
    graph = batch.capture()
    stream = torch.cuda.current_stream()

    # warm-up
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d after warm-up" % st)

    # timed region: K steps, barrier + synchronize on both sides, CUDA events
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    times = time_launches(graph.replay, args.steps, stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d after the timed steps" % st)
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms)

    n_jobs = len(jobs)
    pix_step_rank = n_jobs * W * H
    value = whole_job_rate(pix_step_rank, world, ms_max) / 1e9
    pages_per_s = whole_job_rate(B, world, ms_max)

    # algorithmic bytes per launch (run counts from the oracle-free device encode)
    rle_probe = M.Rle.empty(W, H, H * args.rle_runs_per_row)
    runs_in = []
    for s in srcs[: min(8, B)]:
        M.rle_from_bitmap(rle_probe, s)
        runs_in.append(int(rle_probe.n_runs.item()))
    mean_runs_in = float(np.mean(runs_in))
    # output run counts: one page, every (op, se)
    out_runs = {}
    tmp = M.Rle.empty(W, H, H * args.rle_runs_per_row)
    M.rle_from_bitmap(rle_probe, srcs[0])
    for (sw, sh) in SES:
        for op in OPS:
            M.morph_rect(op, tmp, rle_probe, sw, sh)
            out_runs[(op, sw, sh)] = int(tmp.n_runs.item())
    bytes_launch = 0
    for j in jobs:
        bytes_launch += alg_bytes(j["path"], mean_runs_in, out_runs[(j["op"],) + j["se"]])
    # a page's RLE jobs share one encode: count its bitmap read, runs write
    # and row offsets once per page, not once per job
    rle_per_page = sum(1 for j in jobs if j["path"] == "rle") // B
    bytes_launch -= B * max(0, rle_per_page - 1) * encode_bytes(mean_runs_in)
    step_achieved = bytes_launch / (ms * 1e-3) / 1e9

    # the dominant kernel alone: a batch of just its jobs; one full launch
    # leaves the sources' encodes in the workspace, then the tile group runs
    # by itself (forked onto an auxiliary stream and joined back, so events
    # on this stream bracket it), timed like the steps
    dom = [j for j in jobs if j["path"] == DOMINANT_PATH and tuple(j["se"]) in DOMINANT_SES]
    bdom = M.Batch(dom, rle_runs_per_row=args.rle_runs_per_row)
    bdom.launch(stream=stream)
    torch.cuda.synchronize()
    bdom.debug(2, 1)  # the tile groups alone
    gdom = bdom.capture()
    for _ in range(3):
        gdom.replay()
    torch.cuda.synchronize()
    dom_ms = statistics.mean(time_launches(gdom.replay, max(5, args.steps // 2), stream))
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d after the dominant-kernel launches" % st)
    page_bytes = H * NW * 8
    if DOMINANT_PATH == "rle":
        # runs and row offsets of the page read, the bitmap written
        dom_unit = 4 * mean_runs_in + 4 * (H + 1) + page_bytes
    else:
        dom_unit = 2 * page_bytes
    dom_bytes = len(dom) * dom_unit
    dom_kernels = bdom.kernels
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    del bdom, gdom

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6782.1, "fallback"
    try:
        with open(peaks_path) as f:
            peak = float(json.load(f)["hbm_gbs"])
            peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak = 6800.0

    # per-path rates (separate batches, same pages)
    sub = {}
    for path in ("packed", "rle"):
        jb, ob = build_jobs(M, srcs, (path,))
        b2 = M.Batch(jb, rle_runs_per_row=args.rle_runs_per_row)
        g2 = b2.capture()
        for _ in range(2):
            g2.replay()
        torch.cuda.synchronize()
        tt = time_launches(g2.replay, max(2, args.steps // 2), stream)
        sub[path] = len(jb) * W * H / (statistics.mean(tt) * 1e-3) / 1e9
        del b2, g2, jb, ob
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # each rectangle alone, the 600-dpi density sweep and the 512 x 512
    # config, timed standalone (after the batch numbers, before the e2e run)
    tables = {}
    if not args.no_tables:
        tables["per_op"] = {"image": "the %d resident pages as one 2550 x %d image (%.0f MB packed, > L2)"
                                     % (B, B * H, B * H * NW * 8 / 1e6),
                            "results": run_per_op(M, dev_in, peak, stream, args.table_reps)}
        tables["density_sweep"] = run_density_sweep(M, peak, stream, args.table_reps, args.density_copies)
        tables["config1"] = run_config1(M, stream, max(10, args.table_reps))
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: morph_batch_launch_host
    # copies the step's pages in from pinned host memory, runs the batch and
    # copies every result back, on one stream
    host_in = torch.empty((B, H, NW), dtype=torch.int64, pin_memory=True)
    host_in.copy_(dev_in)
    host_out = torch.empty((n_jobs, H, NW), dtype=torch.int64, pin_memory=True)
    e2e_steps = max(2, args.steps // 2)
    batch.launch_host(host_in, dev_in, host_out, dev_out, stream=stream)  # warm-up
    torch.cuda.synchronize()
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_t = []
    for _ in range(e2e_steps):
        s_ev.record(stream)
        batch.launch_host(host_in, dev_in, host_out, dev_out, stream=stream)
        e_ev.record(stream)
        e_ev.synchronize()
        e2e_t.append(s_ev.elapsed_time(e_ev))
    e2e_serial_ms = statistics.mean(e2e_t)
    h2d = host_in.numel() * 8
    d2h = host_out.numel() * 8

    # The same calls pipelined the way a serving host runs them: two sets of
    # device buffers (each with its own batch plan) and host result buffers,
    # consecutive steps' calls on two streams, so that one step's copies run
    # while the other's kernels do.  Every step still copies its inputs from
    # pinned host memory and reads all its results back.
    dev_in2 = torch.empty_like(dev_in)
    srcs2 = [M.Packed(dev_in2[k], W) for k in range(B)]
    jobs2, dev_out2 = build_jobs(M, srcs2, ("packed", "rle"))
    batch2 = M.Batch(jobs2, rle_runs_per_row=args.rle_runs_per_row)
    host_out2 = torch.empty(host_out.shape, dtype=host_out.dtype, pin_memory=True)
    bufs = [(dev_in, dev_out, batch, host_out), (dev_in2, dev_out2, batch2, host_out2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]

    def pipelined_steps(n):
        for k in range(n):
            din, dout, bat, hout = bufs[k % 2]
            bat.launch_host(host_in, din, hout, dout, stream=streams[k % 2])

    pipelined_steps(2)  # warm-up of the second plan and the streams
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(streams[0])
    streams[1].wait_event(p0)
    pipelined_steps(e2e_steps)
    streams[0].wait_stream(streams[1])
    p1.record(streams[0])
    p1.synchronize()
    e2e_ms = p0.elapsed_time(p1) / e2e_steps
    st = M.sync_status()
    if st != M.MORPH_OK:
        raise RuntimeError("device status %d after the end-to-end steps" % st)
    del batch2, jobs2, dev_out2, dev_in2, srcs2, host_out2
    e2e_value = pix_step_rank * world / (e2e_ms * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 rows, 32-bit word lanes, exact bitwise",
        "data": "synthetic (seeded document pages; UW3 scans are not available)",
        "config": {"workload": WORKLOAD, "pages_per_gpu": B, "page_ops_per_step": n_jobs,
                   "parallelism": "pages sharded across GPUs, no collective" if world > 1 else "1 GPU",
                   "l2": "inputs %.0f MB + outputs %.0f MB per step > 129 MB L2, no flush needed"
                         % (B * H * NW * 8 / 1e6, n_jobs * H * NW * 8 / 1e6)},
        "pages_per_s": round(pages_per_s, 1),
        "packed_gpix_s": round(sub["packed"], 1), "rle_gpix_s": round(sub["rle"], 1),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": profile_traffic("k_rle_rect_open_close_letter_dram.md", B),
                     "kernel": DOMINANT_KERNEL, "peak_source": peak_src,
                     "page_ops_per_launch": len(dom), "launches": dom_kernels,
                     "alg_bytes_per_launch": int(dom_bytes), "ms_per_launch": round(dom_ms, 4),
                     "alg_bytes_per_page_op": int(dom_unit)},
        "step_roofline": {"alg_bytes_per_step": int(bytes_launch), "achieved": round(step_achieved, 1),
                          "unit": "GB/s", "frac": round(step_achieved / peak, 4),
                          "kernels_per_step": batch.kernels},
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 3),
                "steps": e2e_steps, "api": "morph_batch_launch_host (copy in, batch, copy out; C ABI)",
                "pipelined": "calls of neighbouring steps on two streams: copies overlap kernels",
                "unpipelined_ms_per_step": round(e2e_serial_ms, 3),
                "unpipelined_value": round(pix_step_rank * world / (e2e_serial_ms * 1e-3) / 1e9, 2)},
        "gpu_launches": args.steps * batch.kernels,
        "clocks": clocks,
        "generation_s": round(t_gen, 2),
    }
    line.update(tables)
    if not args.no_batch:
        line["uneven_batch"] = run_uneven_batch(M, args, stream)
    if not args.no_serve:
        line["serving"] = run_serving(M, args)
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = cpu_count()
        pix, dt, desc = oracle_sample(pages[:2], args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": round(pix / dt / 1e9, 5), "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": desc + ", %.1f s" % dt}
        pix1, dt1, desc1 = oracle_sample(pages[:1], args.cpu_seconds / 2, 1)
        line["cpu_baseline_1core"] = {"value": round(pix1 / dt1 / 1e9, 5), "unit": UNIT, "cores": 1,
                                      "kind": "oracle", "sample": desc1 + ", %.1f s" % dt1}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    cores = cpu_count()
    pages = make_pages(1)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(pages, per_step, cores)
    pix_t, dt_t, desc = 0, 0.0, ""
    for _ in range(args.steps):
        pix, dt, desc = oracle_sample(pages, per_step, cores)
        pix_t += pix
        dt_t += dt
    value = pix_t / dt_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt_t / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded document pages)",
        "config": {"workload": WORKLOAD, "pages_per_gpu": 1},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc + " per step, bounded to %.1f s" % per_step},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)  # ~0.7 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pages", type=int, default=160, help="pages per GPU (inputs > L2 from 128 up)")
    ap.add_argument("--rle-runs-per-row", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch section")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving section")
    ap.add_argument("--batch-pages", type=int, default=256)
    ap.add_argument("--no-tables", action="store_true",
                    help="skip the per-rectangle, density-sweep and 512x512 tables")
    ap.add_argument("--table-reps", type=int, default=5)
    ap.add_argument("--density-copies", type=int, default=48,
                    help="copies of each 5100x6600 page in the density-sweep stack (48: 203 MB)")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window per rate")
    ap.add_argument("--serve-pool", type=int, default=256, help="device-resident pages the requests draw from")
    ap.add_argument("--tune-cache", default=os.path.join("/tmp", "morph_tune_cache.json"))
    ap.add_argument("--probe", choices=["packed", "rle", "mask", "cc", "xpose", "line", "layout"], default=None,
                    help="run one standalone op on a tall page stack (ncu target) and exit")
    ap.add_argument("--probe-op", default="erode")
    ap.add_argument("--probe-se", default="3x3")
    ap.add_argument("--probe-pages", type=int, default=160)
    ap.add_argument("--probe-reps", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
