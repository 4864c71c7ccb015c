"""Autotuner for the batch launch: per page class it measures

* the row-band height of packed tiles (``tile_rows``),
* the packed tile's word tile (2 or 4 32-bit words per thread, or the
  planner's own choice), and
* packed path versus RLE path, over a grid of ink densities,

and answers :func:`Tuner.choose` (path, tile_rows) and :func:`Tuner.words`
(words per thread) for a page from its size,
operation, rectangle and ink density — the runtime algorithm selection the
paper proposes between bit blit and run-length methods (section
"Experiments", choosing by mask size or output complexity), measured on this
GPU instead of assumed.  Results are cached in a JSON file keyed by the GPU
name, so tuning runs once per machine.

Measurements use the library's own batch launch on seeded synthetic pages;
nothing here computes pixels.
"""
from __future__ import annotations

import json
import os
import statistics

DENSITIES = (0.005, 0.02, 0.05, 0.1, 0.2, 0.3)
BANDS = (32, 64, 128, 256, 512)
WORDS = (2, 4)  # 32-bit words per thread of the packed tile, besides the planner's choice


def _key(W, H, op, se):
    return "%dx%d:%s:%dx%d" % (W, H, op, se[0], se[1])


class Tuner:
    """``min_pixels``: every timed batch repeats the class's pages until it
    holds at least this many pixels, so that both paths are timed at full
    occupancy (a few pages leave most CTAs idle on the packed path, whose
    tiles are few and large, and time latency instead of throughput)."""

    def __init__(self, cache_path=None, pages_per_class=8, reps=3, min_pixels=1_000_000_000):
        self.cache_path = cache_path
        self.pages_per_class = pages_per_class
        self.reps = reps
        self.min_pixels = min_pixels
        self.table = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = json.load(f)

    # ------------------------------------------------------------ timing
    def _time_batch(self, jobs, reps):
        import torch
        from . import morph as M
        b = M.Batch(jobs)
        b.launch()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            b.launch()
            e.record()
            e.synchronize()
            ts.append(s.elapsed_time(e))
        if M.sync_status() != M.MORPH_OK:
            return float("inf")
        return statistics.median(ts)

    def _pages(self, W, H, density, n):
        from . import morph as M
        from . import synth
        out = []
        for k in range(n):
            img = synth.document_page(W, H, 0x7A11 + 97 * k + int(density * 1e4), density)[0]
            out.append(M.pack(img, 64))
        return out

    def tune_grid(self, W, H, ops, ses, densities=DENSITIES, bands=BANDS):
        """Measure every (op, rectangle) class of one page size; the seeded
        pages of each density are generated once and shared."""
        from . import morph as M
        n = self.pages_per_class
        pages = {d: self._pages(W, H, d, n) for d in densities}
        mid = self._pages(W, H, 0.08, n)
        total = n * max(1, -(-self.min_pixels // (n * W * H)))
        outs = [M.Packed.empty(W, H, 64) for _ in range(total)]
        for op in ops:
            for se in ses:
                self.tune_class(W, H, op, se, densities, bands, pages, mid, outs)
        return self.table

    def tune_class(self, W, H, op, se, densities=DENSITIES, bands=BANDS, pages=None, mid=None,
                   outs=None):
        """Measure one (size, op, rectangle) class; returns its table entry."""
        from . import morph as M
        n = self.pages_per_class
        total = n * max(1, -(-self.min_pixels // (n * W * H)))  # page-ops per timed batch
        entry = {"density": [], "packed_ms": [], "rle_ms": [], "band": None}
        mid = mid if mid is not None else self._pages(W, H, 0.08, n)
        if outs is None or len(outs) < total:
            outs = [M.Packed.empty(W, H, 64) for _ in range(total)]

        def jobs_of(srcs, **kw):
            return [dict(op=op, se=se, src=srcs[k % n], dst=outs[k], **kw) for k in range(total)]

        best_band, best_t = 0, float("inf")
        for band in bands:
            t = self._time_batch(jobs_of(mid, path="packed", tile_rows=band), self.reps)
            if t < best_t:
                best_band, best_t = band, t
        entry["band"] = best_band
        # the word tile at that band: the planner's choice (0) unless 2 or 4
        # words per thread measure faster
        best_words = 0
        for words in WORDS:
            t = self._time_batch(jobs_of(mid, path="packed", tile_rows=best_band, words_per_thread=words),
                                 self.reps)
            if t < best_t:
                best_words, best_t = words, t
        entry["words"] = best_words
        for dens in densities:
            pg = pages[dens] if pages is not None else self._pages(W, H, dens, n)
            tp = self._time_batch(jobs_of(pg, path="packed", tile_rows=best_band, words_per_thread=best_words),
                                  self.reps)
            tr = self._time_batch(jobs_of(pg, path="rle"), self.reps)
            entry["density"].append(dens)
            entry["packed_ms"].append(tp / total)
            entry["rle_ms"].append(tr / total)
        self.table[_key(W, H, op, se)] = entry
        return entry

    def save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1)
            os.replace(tmp, self.cache_path)

    # ------------------------------------------------------------ decision
    def tuned(self, W, H) -> bool:
        """Whether any class of this page size has been measured."""
        return any(k.startswith("%dx%d:" % (W, H)) for k in self.table)

    def words(self, W, H, op, se, ref_size=None) -> int:
        """Words per thread of the packed tile for the class (0 = the
        planner's choice, also for untuned classes and older caches)."""
        if ref_size is not None:
            W, H = ref_size
        e = self.table.get(_key(W, H, op, se))
        return int(e.get("words", 0)) if e else 0

    def choose(self, W, H, op, se, density, ref_size=None):
        """(path, tile_rows) for one page; ``ref_size`` maps the page to the
        size its class was tuned at; untuned classes take the packed path with
        the default band."""
        if ref_size is not None:
            W, H = ref_size
        e = self.table.get(_key(W, H, op, se))
        if not e:
            return "packed", 0
        ds = e["density"]
        # nearest measured density (log scale)
        import math
        k = min(range(len(ds)), key=lambda i: abs(math.log(ds[i]) - math.log(max(density, 1e-4))))
        path = "rle" if e["rle_ms"][k] < e["packed_ms"][k] else "packed"
        return path, e["band"] or 0

    def crossover(self, W, H, op, se):
        """Densities at which the RLE path was measured faster."""
        e = self.table.get(_key(W, H, op, se))
        if not e:
            return []
        return [d for d, p, r in zip(e["density"], e["packed_ms"], e["rle_ms"]) if r < p]
