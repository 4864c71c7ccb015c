// Persistent batch launch (K8): many uneven pages, each with its own
// operation, rectangle and path, in ONE kernel launch.
//
// The host builds a plan: a job table and a list of work items.  A packed
// job is one phase of independent tiles (the fused tile of packed_tile.cuh).
// An RLE job is a chain of phases — bitmap->RLE count, scan, write (shared:
// RLE jobs on the same source page read one job's encode); per erosion stage
// the run pass (count, scan, write) or the between-line pass (rows to a
// bitmap; for a first stage of two, its run counts, scan and encode; the
// last stage's rows go straight to the job's packed output); RLE->bitmap
// after a run-pass stage — whose items depend on every item of the job's
// previous phase.  Items are listed by level (a job's phase index, shifted
// past the phase of the job it depends on) and claimed in list order from a
// device queue by persistent CTAs.  An item waits (bounded spin with acquire loads) only
// for items of smaller index, which running CTAs have already claimed, so
// the launch cannot deadlock; a wait that exceeds the time limit latches
// MORPH_ETIMEOUT and makes every CTA stop.
//
// The kernel reads the plan from device memory (the caller copies it there)
// and keeps its counters and RLE buffers in the caller's workspace, so one
// launch can be captured in a CUDA graph and replayed.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "packed_tile.cuh"
#include "rle_rect.cuh"
#include "rle_tile.cuh"

namespace morph {
namespace {

constexpr uint32_t PLAN_MAGIC = 0x4d425031u;  // "MBP1"
constexpr int MAX_PH = 11;
// Phases of the bitmap -> runs encode that starts an RLE-path job.
constexpr int ENCODE_PHASES = 3;

struct SrcKey {  // a source page, for sharing its encode between jobs
    const void *words;
    int64_t stride;
    int fmt, W, H;
    bool operator<(const SrcKey &o) const {
        if (words != o.words) return words < o.words;
        if (stride != o.stride) return stride < o.stride;
        if (fmt != o.fmt) return fmt < o.fmt;
        if (W != o.W) return W < o.W;
        return H < o.H;
    }
};

// Rows per row-range item (bitmap <-> runs, row pass, runs -> bitmap): a
// multiple of 64 up to 1024, chosen per job at plan time.
constexpr int BATCH_ROWS_MIN = 64, BATCH_ROWS_MAX = 1024;
// Row-range items per phase that keep two CTAs on each of 152 SMs busy
// several times over.
constexpr int64_t ROW_ITEMS_TARGET = 8 * 2 * 152;
constexpr int BATCH_THREADS = 256;
constexpr long long WAIT_LIMIT_NS = 4000000000ll;  // default 4 s

enum ItemKind : int {
    IK_PACKED = 0,
    IK_B2R_COUNT,
    IK_SCAN,
    IK_B2R_WRITE,
    IK_ROW_COUNT,
    IK_ROW_WRITE,
    IK_V_BMP,      // between-line pass: rows to a bitmap
    IK_BCOUNT,     // run counts of the stored bitmap rows
    IK_BWRITE,     // encode the stored bitmap rows into runs
    IK_R2B,
    IK_OUT_SCAN,   // MORPH_TO_RLE: scan into the caller's RLE dst
    IK_OUT_WRITE,  // MORPH_TO_RLE: write the caller's runs
};

struct BatchJob {
    int32_t path;               // MORPH_PATH_PACKED / MORPH_PATH_RLE
    int32_t dep;                // job that must finish first, or -1
    int32_t level0;             // queue level of phase 0 (items sorted by level)
    RleOut out;                 // MORPH_TO_RLE destination
    int32_t variant;            // packed tile variant
    int32_t nphase;
    int32_t phase_items[MAX_PH];
    int32_t phase_kind[MAX_PH];
    int32_t phase_stage[MAX_PH];  // erosion stage (0/1) of run / between-line phases
    int32_t gx;                 // packed: tiles along x of the grid
    PackedArgs pa;              // packed path
    // RLE path
    const uint32_t *src;
    int64_t sstride;
    uint32_t *dst;
    int64_t dstride;
    int32_t W, H, nw_cover, nst;
    RowOp rop[2];
    VArgs va[2];                // pointers are filled on the device from ws offsets
    int32_t vkind[2];           // between-line variant (nwt, kmax)
    int64_t off_counts, off_rpA, off_runsA, off_rpB, off_runsB, off_nA, off_nB, off_bmp;
    int64_t off_srp, off_sruns;  // the RLE source the first stage reads (own A, or a shared one)
    int32_t src_job;             // job whose encode produced that source (itself if not shared)
    int32_t dep_phase;           // phase of `dep` whose completion gates this job's phase 0
    int64_t cap;                // runs capacity of each RLE buffer
    int rows;                   // rows per row-range item
};

struct BatchItem {
    int32_t job;
    int16_t phase;
    int16_t kind;
    int32_t idx;
};

struct BatchHeader {
    uint32_t magic;
    int32_t n_jobs, n_items, smem_bytes;
    int64_t jobs_off, items_off, plan_bytes;
    int64_t ws_ctrl_bytes, ws_bytes;
    int64_t wait_limit_ns;
    int32_t n_groups;
    int32_t kb_after_groups;  // a persistent-kernel job reads a grouped packed job's result
    int32_t groups_only;      // timing hook: launch the tile groups alone (morph_batch_plan_debug 2)
    int32_t pad0;
    int64_t groups_off;
};

// Jobs run outside the persistent kernel as launches of the rectangle tiles
// over job tables, one group per tile variant and CTA size: packed jobs whose
// dependency (if any) is itself such a packed job, level by level before the
// persistent kernel; RLE-path jobs that neither depend on another job nor are
// depended on (source runs -> both stages -> the job's bitmap) after it, once
// it has encoded their sources.
struct TileGroup {
    int32_t rle;         // 0: packed tile (before the persistent kernel); 1: RLE-source tile (after)
    int32_t njobs, ctas;
    int32_t level;       // packed: dependency level (a job's dependency runs at a lower level)
    int64_t smem;        // dynamic shared memory of the launch
    int64_t jobs_off;    // RectArgs[njobs] (packed) or RleJob[njobs] (RLE) in the plan
    int64_t starts_off;  // int[njobs + 1]: first CTA of each job
    RectArgs proto;      // variant and CTA size of the group
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------- device side
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0: wait until *ctr >= target.  false on abort or time-out.
__device__ bool wait_count(const int *ctr, int target, int *abort_flag, int *status,
                           unsigned long long limit_ns) {
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0;; ++it) {
        if (ld_acquire(ctr) >= target) return true;
        if (*(volatile int *)abort_flag) return false;
        if ((it & 63) == 63 && now_ns() - t0 > limit_ns) {
            latch_status(status, MORPH_ETIMEOUT);
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(200);
    }
}

// Packed tile variants reachable from the batch: stages {1, 2} x column
// counters {none, 2-row register, 6 planes, 16 planes} x horizontal
// {none, reach<=1, halo 1, 2, 4 words}.
template <int NST, bool HS, int KMAX, int HALO, bool HX1>
__device__ __noinline__ void tile_fn(const PackedArgs &a, int bx, int by, uint32_t *sm) {
    packed_tile<NST, HS, KMAX, HALO, HX1, false>(a, bx, by, sm);
}

template <int NST, int KMAX>
__device__ __forceinline__ void tile_h(int h, const PackedArgs &a, int bx, int by, uint32_t *sm) {
    switch (h) {
    case 0: tile_fn<NST, false, KMAX, 1, false>(a, bx, by, sm); break;
    case 1: tile_fn<NST, true, KMAX, 1, true>(a, bx, by, sm); break;
    case 2: tile_fn<NST, true, KMAX, 1, false>(a, bx, by, sm); break;
    case 3: tile_fn<NST, true, KMAX, 2, false>(a, bx, by, sm); break;
    default: tile_fn<NST, true, KMAX, 4, false>(a, bx, by, sm); break;
    }
}

template <int NST>
__device__ __forceinline__ void tile_k(int k, int h, const PackedArgs &a, int bx, int by, uint32_t *sm) {
    switch (k) {
    case 0: tile_h<NST, 0>(h, a, bx, by, sm); break;
    case 1: tile_h<NST, 2>(h, a, bx, by, sm); break;
    case 2: tile_h<NST, 6>(h, a, bx, by, sm); break;
    default: tile_h<NST, 16>(h, a, bx, by, sm); break;
    }
}

__device__ void run_packed_tile(int variant, const PackedArgs &a, int bx, int by, uint32_t *sm) {
    const int h = variant % 5, k = (variant / 5) % 4, nst = variant / 20;
    if (nst == 0) tile_k<1>(k, h, a, bx, by, sm);
    else tile_k<2>(k, h, a, bx, by, sm);
}

template <int NWT, int KMAX>
__device__ __noinline__ void vpass_fn(const VArgs &a, int bx, uint32_t *sm) {
    vpass_tile<NWT, KMAX>(a, bx, sm);
}

template <int KMAX>
__device__ __noinline__ void vband_fn(const VArgs &a, int bx, uint32_t *sm) {
    vband_tile<2, KMAX>(a, bx, sm);
}

__device__ void run_vpass(int vkind, const VArgs &a, int bx, uint32_t *sm) {
    switch (vkind) {
    case 0: vpass_fn<2, 2>(a, bx, sm); break;
    case 1: vpass_fn<2, 3>(a, bx, sm); break;
    case 2: vpass_fn<2, 6>(a, bx, sm); break;
    case 3: vpass_fn<2, 16>(a, bx, sm); break;
    case 4: vpass_fn<8, 2>(a, bx, sm); break;
    case 5: vpass_fn<8, 3>(a, bx, sm); break;
    case 6: vpass_fn<8, 6>(a, bx, sm); break;
    case 7: vpass_fn<8, 16>(a, bx, sm); break;
    case 8: vband_fn<2>(a, bx, sm); break;
    case 9: vband_fn<3>(a, bx, sm); break;
    case 10: vband_fn<6>(a, bx, sm); break;
    default: vband_fn<16>(a, bx, sm); break;
    }
}

struct Ctrl {
    int head, abort_flag;
    int pad[62];
    // followed by int done[n_jobs][MAX_PH] and int overflow[n_jobs]
};

__global__ void __launch_bounds__(BATCH_THREADS, 2) k_batch(const uint8_t *plan, uint8_t *ws,
                                                           int *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int s_next[2], s_ok;
    const BatchHeader *hdr = reinterpret_cast<const BatchHeader *>(plan);
    const BatchJob *jobs = reinterpret_cast<const BatchJob *>(plan + hdr->jobs_off);
    const BatchItem *items = reinterpret_cast<const BatchItem *>(plan + hdr->items_off);
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(ws);
    int *done = reinterpret_cast<int *>(ws + sizeof(Ctrl));
    int *overflow = done + (size_t)hdr->n_jobs * MAX_PH;
    const int n_items = hdr->n_items;

    // Thread 0 reserves the CTA's next item as soon as the current one may
    // start, and publishes it when the current one ends: the queue atomic's
    // latency hides behind the work.  A CTA holds at most one reserved item
    // besides the one it runs, and items are reserved in list (level)
    // order, so the lowest unfinished item can always proceed.
    if (threadIdx.x == 0)
        s_next[0] = *(volatile int *)&ctrl->abort_flag ? n_items : atomicAdd(&ctrl->head, 1);
    __syncthreads();
    for (int k = 0;; ++k) {
        const int i = s_next[k & 1];
        if (i >= n_items) break;
        const BatchItem it = items[i];
        const BatchJob &J = jobs[it.job];
        int nxt = n_items;
        if (threadIdx.x == 0) {
            bool ok = true;
            if (it.phase > 0) {
                ok = wait_count(done + (size_t)it.job * MAX_PH + it.phase - 1,
                                J.phase_items[it.phase - 1], &ctrl->abort_flag, status,
                                (unsigned long long)hdr->wait_limit_ns);
            } else if (J.dep >= 0) {
                const BatchJob &D = jobs[J.dep];
                ok = wait_count(done + (size_t)J.dep * MAX_PH + J.dep_phase,
                                D.phase_items[J.dep_phase], &ctrl->abort_flag, status,
                                (unsigned long long)hdr->wait_limit_ns);
            }
            s_ok = ok;
            if (ok && !*(volatile int *)&ctrl->abort_flag) nxt = atomicAdd(&ctrl->head, 1);
        }
        __syncthreads();
        if (!s_ok) break;
        __threadfence();

        // overflow: bit 0 = one of the job's RLE buffers, bit 1 = its source
        // encode (which jobs sharing that encode check too)
        const bool ovf = (it.phase > 0 && *(volatile int *)(overflow + it.job) != 0) ||
                         (J.src_job != it.job && (*(volatile int *)(overflow + J.src_job) & 2));
        switch (it.kind) {
        case IK_PACKED:
            run_packed_tile(J.variant, J.pa, it.idx % J.gx, it.idx / J.gx, sm);
            break;
        case IK_B2R_COUNT: {
            const int r0 = it.idx * J.rows;
            b2r_count_rows(J.src, J.sstride, J.W, r0, min(J.H, r0 + J.rows),
                           reinterpret_cast<int32_t *>(ws + J.off_counts));
            break;
        }
        case IK_B2R_WRITE: {
            if (ovf) break;
            const int r0 = it.idx * J.rows;
            b2r_write_rows<3>(J.src, J.sstride, J.W, r0, min(J.H, r0 + J.rows),
                           reinterpret_cast<const int32_t *>(ws + J.off_rpA),
                           reinterpret_cast<uint16_t *>(ws + J.off_runsA));
            break;
        }
        case IK_SCAN: {
            if (ovf) break;
            // output buffer of the phase that this scan completes
            const int st = J.phase_stage[it.phase];
            const bool toA = st < 0 || st == 1;
            int32_t *rp = reinterpret_cast<int32_t *>(ws + (toA ? J.off_rpA : J.off_rpB));
            int64_t *nr = reinterpret_cast<int64_t *>(ws + (toA ? J.off_nA : J.off_nB));
            scan_rows_block(reinterpret_cast<const int32_t *>(ws + J.off_counts), J.H, rp, nr, J.cap,
                            status);
            if (threadIdx.x == 0 && rp[J.H] > J.cap) atomicOr(overflow + it.job, st < 0 ? 3 : 1);
            break;
        }
        case IK_ROW_COUNT:
        case IK_ROW_WRITE: {
            if (ovf) break;
            const int st = J.phase_stage[it.phase];
            const bool fromA = st == 0;  // stage 0 reads the source, writes B; stage 1 B -> A
            const RleIn in{reinterpret_cast<const int32_t *>(ws + (fromA ? J.off_srp : J.off_rpB)),
                           reinterpret_cast<const uint16_t *>(ws + (fromA ? J.off_sruns : J.off_runsB)),
                           J.W, J.H};
            const int r0 = it.idx * J.rows;
            const bool write = it.kind == IK_ROW_WRITE;
            rowpass_rows(in, J.rop[st], write, reinterpret_cast<int32_t *>(ws + J.off_counts),
                         reinterpret_cast<const int32_t *>(ws + (fromA ? J.off_rpB : J.off_rpA)),
                         reinterpret_cast<uint16_t *>(ws + (fromA ? J.off_runsB : J.off_runsA)), r0,
                         min(J.H, r0 + J.rows));
            break;
        }
        case IK_V_BMP: {
            if (ovf) break;
            const int st = J.phase_stage[it.phase];
            const bool fromA = st == 0;
            VArgs va = J.va[st];
            va.in.row_ptr = reinterpret_cast<const int32_t *>(ws + (fromA ? J.off_srp : J.off_rpB));
            va.in.runs = reinterpret_cast<const uint16_t *>(ws + (fromA ? J.off_sruns : J.off_runsB));
            if (st == J.nst - 1) {
                // last stage: the rows go straight to the job's packed output
                va.bmp = J.dst;
                va.bmp_stride = J.dstride;
                va.bmp_words = J.nw_cover;
                va.counts = nullptr;
            } else {
                va.bmp = reinterpret_cast<uint32_t *>(ws + J.off_bmp);
                va.bmp_stride = (J.W + 31) / 32;
                va.bmp_words = (J.W + 31) / 32;
                va.counts = nullptr;
            }
            run_vpass(J.vkind[st], va, it.idx, sm);
            break;
        }
        case IK_BCOUNT: {
            if (ovf) break;
            const int r0 = it.idx * J.rows;
            b2r_count_rows(reinterpret_cast<const uint32_t *>(ws + J.off_bmp), (J.W + 31) / 32, J.W, r0,
                           min(J.H, r0 + J.rows), reinterpret_cast<int32_t *>(ws + J.off_counts));
            break;
        }
        case IK_BWRITE: {
            if (ovf) break;
            const int r0 = it.idx * J.rows;
            b2r_write_rows<3>(reinterpret_cast<const uint32_t *>(ws + J.off_bmp), (J.W + 31) / 32, J.W, r0,
                           min(J.H, r0 + J.rows),
                           reinterpret_cast<const int32_t *>(ws + J.off_rpB),
                           reinterpret_cast<uint16_t *>(ws + J.off_runsB));
            break;
        }
        case IK_OUT_SCAN: {
            scan_rows_block(reinterpret_cast<const int32_t *>(ws + J.off_counts), J.H, J.out.row_ptr,
                            J.out.n_runs, J.out.capacity, status);
            if (threadIdx.x == 0 && J.out.row_ptr[J.H] > J.out.capacity) atomicExch(overflow + it.job, 1);
            break;
        }
        case IK_OUT_WRITE: {
            if (ovf) break;
            const int r0 = it.idx * J.rows;
            b2r_write_rows<3>(J.src, J.sstride, J.W, r0, min(J.H, r0 + J.rows),
                           J.out.row_ptr, J.out.runs);
            break;
        }
        case IK_R2B: {
            if (ovf) break;
            const bool fromA = J.nst == 2;  // last stage wrote A (two stages) or B (one)
            const RleIn in{reinterpret_cast<const int32_t *>(ws + (fromA ? J.off_rpA : J.off_rpB)),
                           reinterpret_cast<const uint16_t *>(ws + (fromA ? J.off_runsA : J.off_runsB)),
                           J.W, J.H};
            const int r0 = it.idx * J.rows;
            r2b_rows(in, J.dst, J.dstride, J.nw_cover, r0, min(J.H, r0 + J.rows), sm);
            break;
        }
        default:
            break;
        }
        __threadfence();
        if (threadIdx.x == 0) s_next[(k + 1) & 1] = nxt;
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + (size_t)it.job * MAX_PH + it.phase, 1);
    }
}

// ------------------------------------------------------------ host side
int bitlen(int v) {
    int k = 0;
    while (v) { ++k; v >>= 1; }
    return k;
}

// Column-counter class of the batch's packed variants for sh: index into
// {0, 2, 6, 16} planes.
int batch_kidx(int km) {
    if (km == 0) return 0;
    if (km == 2) return 1;  // sh == 3 window
    if (km <= 6) return 2;
    return 3;
}
constexpr int BATCH_KMAX[4] = {0, 2, 6, 16};

int packed_variant(const PackedArgs &a) {
    const int kidx = batch_kidx(packed_kmax(a));
    int h;
    if (!a.hmode) h = 0;
    else if (a.sw <= 3 && a.ex[0] <= 1 && a.sw - 1 - a.ex[0] <= 1) h = 1;
    else {
        const int halo = packed_halo(a.sw, a.ex[0]);
        h = halo == 1 ? 2 : (halo == 2 ? 3 : 4);
    }
    return ((a.nst - 1) * 4 + kidx) * 5 + h;
}

struct Clip {
    int sw, sh, ox, oy;
};
Clip clip_rect(int W, int H, int sw, int sh, int ox, int oy) {
    int l = ox, r = sw - 1 - ox, u = oy, d = sh - 1 - oy;
    if (l > W - 1) l = W - 1;
    if (r > W - 1) r = W - 1;
    if (u > H - 1) u = H - 1;
    if (d > H - 1) d = H - 1;
    return {l + r + 1, u + d + 1, l, u};
}

morph_status berr(morph_status st, const char *msg, int job) {
    set_error("job %d: %s", job, msg);
    return st;
}

// Build jobs and items; returns MORPH_OK and fills the vectors.
struct GroupPlan {
    TileGroup g;
    std::vector<RectArgs> rect;
    std::vector<RleJob> rle;
    std::vector<int> starts;
};

bool same_variant(const RectArgs &x, const RectArgs &y) {
    return x.nst == y.nst && x.nwt == y.nwt && x.vmode == y.vmode && x.hmode == y.hmode && x.halo == y.halo &&
           x.threads == y.threads;
}

void add_to_group(std::vector<GroupPlan> &G, int rle, int level, const RectArgs &ra, const RleJob *rj,
                  size_t smem_bytes) {
    GroupPlan *gp = nullptr;
    for (auto &x : G)
        if (x.g.rle == rle && x.g.level == level && same_variant(x.g.proto, ra)) gp = &x;
    if (!gp) {
        G.emplace_back();
        gp = &G.back();
        memset(&gp->g, 0, sizeof(gp->g));
        gp->g.rle = rle;
        gp->g.level = level;
        gp->g.proto = ra;
        gp->starts.push_back(0);
    }
    const int ctas = (int)(rect_grid(ra).x * rect_grid(ra).y);
    if (rle) gp->rle.push_back(*rj);
    else gp->rect.push_back(ra);
    gp->starts.push_back(gp->starts.back() + ctas);
    gp->g.njobs += 1;
    gp->g.ctas += ctas;
    if ((int64_t)smem_bytes > gp->g.smem) gp->g.smem = (int64_t)smem_bytes;
}

morph_status build(const morph_job *jobs, int n, int tile_rows, int rle_runs_per_row,
                   std::vector<BatchJob> &J, std::vector<BatchItem> &I, int64_t &ws_ctrl,
                   int64_t &ws_total, int &smem, std::vector<GroupPlan> &G, int *kb_after_groups = nullptr) {
    J.assign(n, BatchJob{});
    G.clear();
    smem = 0;
    if (kb_after_groups) *kb_after_groups = 0;
    // jobs another job depends on stay inside the persistent kernel
    std::vector<char> depended(n, 0);
    for (int j = 0; j < n; ++j)
        if (jobs[j].depends_on >= 0 && jobs[j].depends_on < j) depended[jobs[j].depends_on] = 1;
    std::vector<int> glevel(n, -1);  // level of a packed job run as a grouped launch
    // Default rows per row-range item: larger items amortise the per-item
    // cost (claim, dependency check, job fields) once the plan has enough
    // row-range work to keep every CTA busy with the larger items too.
    int64_t rle_rows = 0;
    for (int j = 0; j < n; ++j)
        if (jobs[j].op == MORPH_TO_RLE || jobs[j].path == MORPH_PATH_RLE) rle_rows += jobs[j].src.height;
    int auto_rows = BATCH_ROWS_MIN;
    while (auto_rows < BATCH_ROWS_MAX && rle_rows / (2 * auto_rows) >= ROW_ITEMS_TARGET) auto_rows *= 2;
    auto item_rows = [&](const morph_job &q) {
        const int want = q.tile_rows ? q.tile_rows : (tile_rows ? tile_rows : auto_rows);
        int r = (want + BATCH_ROWS_MIN - 1) / BATCH_ROWS_MIN * BATCH_ROWS_MIN;
        return r > BATCH_ROWS_MAX ? BATCH_ROWS_MAX : r;
    };
    int64_t off = al(sizeof(Ctrl) + (size_t)n * MAX_PH * sizeof(int) + (size_t)n * sizeof(int));
    ws_ctrl = off;
    std::map<SrcKey, int> encoders;  // source page -> job that encodes it to runs
    for (int j = 0; j < n; ++j) {
        const morph_job &q = jobs[j];
        BatchJob &b = J[j];
        memset(&b, 0, sizeof(b));
        const morph_image &s = q.src, &d = q.dst;
        auto packed = [](const morph_image &m) { return m.fmt == MORPH_PACKED32 || m.fmt == MORPH_PACKED64; };
        if (q.tile_rows < 0) return berr(MORPH_EINVAL, "tile_rows must be >= 0", j);
        if (q.words_per_thread != 0 && q.words_per_thread != 2 && q.words_per_thread != 4)
            return berr(MORPH_EINVAL, "words_per_thread must be 0, 2 or 4", j);
        if (q.depends_on < -1 || q.depends_on >= j)
            return berr(MORPH_EINVAL, "depends_on must be -1 or an earlier job", j);
        b.dep = q.depends_on;
        b.dep_phase = b.dep >= 0 ? J[b.dep].nphase - 1 : 0;
        // a job that waits for a grouped packed job runs after every group
        // level in stream order: no wait inside the persistent kernel
        if (b.dep >= 0 && glevel[b.dep] >= 0) {
            b.dep = -1;
            b.dep_phase = 0;
            if (kb_after_groups) *kb_after_groups = 1;
        }
        b.src_job = j;
        if (q.op == MORPH_TO_RLE) {
            if (!packed(s) || d.fmt != MORPH_RLE) return berr(MORPH_EINVAL, "MORPH_TO_RLE needs a packed src and an RLE dst", j);
            if (s.width < 1 || s.height < 1 || s.width != d.width || s.height != d.height || s.width > 65535)
                return berr(MORPH_EINVAL, "bad or different sizes (RLE width <= 65535)", j);
            const int Bs = s.fmt == MORPH_PACKED32 ? 32 : 64;
            if (!s.words || s.stride_words < (s.width + Bs - 1) / Bs || (uintptr_t)s.words % (Bs / 8) ||
                !d.row_ptr || d.capacity_runs < 0 || (d.capacity_runs > 0 && !d.runs) || (uintptr_t)d.runs % 4 ||
                s.reserved || d.reserved)
                return berr(MORPH_EINVAL, "bad descriptor", j);
            b.path = -1;
            b.src = (const uint32_t *)s.words;
            b.sstride = s.stride_words * (Bs / 32);
            b.W = s.width;
            b.H = s.height;
            b.out = RleOut{d.row_ptr, d.runs, d.capacity_runs, d.n_runs};
            b.off_counts = off;
            off += al((size_t)b.H * 4);
            b.rows = item_rows(q);
            const int rows_items = (b.H + b.rows - 1) / b.rows;
            b.nphase = 3;
            b.phase_kind[0] = IK_B2R_COUNT; b.phase_items[0] = rows_items; b.phase_stage[0] = -1;
            b.phase_kind[1] = IK_OUT_SCAN;  b.phase_items[1] = 1;          b.phase_stage[1] = -1;
            b.phase_kind[2] = IK_OUT_WRITE; b.phase_items[2] = rows_items; b.phase_stage[2] = -1;
            continue;
        }
        if (!packed(s) || !packed(d)) return berr(MORPH_EINVAL, "src and dst must be packed", j);
        if (s.width < 1 || s.height < 1 || s.width != d.width || s.height != d.height)
            return berr(MORPH_EINVAL, "bad or different sizes", j);
        if (!s.words || !d.words || s.reserved || d.reserved) return berr(MORPH_EINVAL, "bad descriptor", j);
        const int Bs = s.fmt == MORPH_PACKED32 ? 32 : 64, Bd = d.fmt == MORPH_PACKED32 ? 32 : 64;
        if (s.stride_words < (s.width + Bs - 1) / Bs || d.stride_words < (d.width + Bd - 1) / Bd)
            return berr(MORPH_EINVAL, "stride too small", j);
        if ((uintptr_t)s.words % (Bs / 8) || (uintptr_t)d.words % (Bd / 8))
            return berr(MORPH_EINVAL, "misaligned words", j);
        if (q.op < MORPH_ERODE || q.op > MORPH_CLOSE) return berr(MORPH_EINVAL, "bad op", j);
        if (q.se_w < 1 || q.se_h < 1 || q.se_w > 65535 || q.se_h > 65535 || q.origin_x < 0 ||
            q.origin_x >= q.se_w || q.origin_y < 0 || q.origin_y >= q.se_h)
            return berr(MORPH_EINVAL, "bad structuring element", j);
        {
            const uintptr_t slo = (uintptr_t)s.words, dlo = (uintptr_t)d.words;
            const uintptr_t shi = slo + (uintptr_t)((int64_t)(s.height - 1) * s.stride_words * (Bs / 8) + (s.width + Bs - 1) / Bs * (Bs / 8));
            const uintptr_t dhi = dlo + (uintptr_t)((int64_t)(d.height - 1) * d.stride_words * (Bd / 8) + (d.width + Bd - 1) / Bd * (Bd / 8));
            if (slo < dhi && dlo < shi) return berr(MORPH_EINVAL, "dst overlaps src", j);
        }
        const int W = s.width, H = s.height;
        const Clip c = clip_rect(W, H, q.se_w, q.se_h, q.origin_x, q.origin_y);
        const int nw_cover = d.fmt == MORPH_PACKED32 ? (W + 31) / 32 : 2 * ((W + 63) / 64);
        b.path = q.path;
        const bool independent = q.depends_on < 0 && !depended[j];
        const int band_hint = q.tile_rows ? q.tile_rows : tile_rows;
        const bool chainable = q.depends_on < 0 || glevel[q.depends_on] >= 0;
        if (q.path == MORPH_PATH_PACKED && chainable) {
            RectArgs ra;
            memset(&ra, 0, sizeof(ra));
            ra.src = (const uint32_t *)s.words;
            ra.sstride = s.stride_words * (Bs / 32);
            ra.dst = (uint32_t *)d.words;
            ra.dstride = d.stride_words * (Bd / 32);
            ra.W = W;
            ra.H = H;
            ra.nw_valid = (W + 31) / 32;
            ra.nw_cover = nw_cover;
            if (rect_plan(ra, q.op, c.sw, c.sh, c.ox, c.oy, band_hint, 0, q.words_per_thread, 0) == 0) {
                ra.band_auto = 0;
                b.path = q.path;
                b.nphase = 0;  // no work in the persistent kernel
                glevel[j] = q.depends_on < 0 ? 0 : glevel[q.depends_on] + 1;
                add_to_group(G, 0, glevel[j], ra, nullptr, rect_smem_words(ra) * 4);
                continue;
            }
        }
        if (q.path == MORPH_PATH_PACKED) {
            PackedArgs &a = b.pa;
            memset(&a, 0, sizeof(a));
            a.src = (const uint32_t *)s.words;
            a.sstride = s.stride_words * (Bs / 32);
            a.dst = (uint32_t *)d.words;
            a.dstride = d.stride_words * (Bd / 32);
            a.W = W;
            a.H = H;
            a.nw_valid = (W + 31) / 32;
            a.nw_cover = nw_cover;
            const int kmax_class = [&] {
                // packed_kmax() of this rectangle, mapped to the batch's classes
                PackedArgs t{};
                t.sh = c.sh;
                int k = 0;
                for (int v = c.sh; v; v >>= 1) ++k;
                t.K = k;
                return BATCH_KMAX[batch_kidx(packed_kmax(t))];
            }();
            if (packed_plan(a, q.op, c.sw, c.sh, c.ox, c.oy, q.tile_rows ? q.tile_rows : tile_rows,
                            MAX_THREADS, kmax_class, false) != 0)
                return berr(MORPH_EINVAL, "rectangle reaches more than 128 pixels sideways", j);
            b.variant = packed_variant(a);
            const dim3 g = packed_grid(a);
            b.gx = g.x;
            b.nphase = 1;
            b.phase_kind[0] = IK_PACKED;
            b.phase_items[0] = g.x * g.y;
            b.phase_stage[0] = -1;
            const int sb = (int)packed_smem_bytes(a);
            if (sb > smem) smem = sb;
        } else if (q.path == MORPH_PATH_RLE) {
            if (W > 65535) return berr(MORPH_EINVAL, "RLE path needs width <= 65535", j);
            b.src = (const uint32_t *)s.words;
            b.sstride = s.stride_words * (Bs / 32);
            b.dst = (uint32_t *)d.words;
            b.dstride = d.stride_words * (Bd / 32);
            b.W = W;
            b.H = H;
            b.nw_cover = nw_cover;
            b.nst = (q.op == MORPH_OPEN || q.op == MORPH_CLOSE) ? 2 : 1;
            const int rpr = rle_runs_per_row > 0 ? rle_runs_per_row : W / 16 + 4;
            b.cap = (int64_t)H * (rpr < (W + 1) / 2 ? rpr : (W + 1) / 2);
            if (b.cap < 1) b.cap = 1;
            // Jobs on the same source page share one bitmap -> RLE encode: the
            // first eligible job encodes into its buffer A (which it then
            // only reads), later ones read that buffer and wait for its
            // encode phases instead of encoding again.  Only jobs without a
            // user dependency share, and only encoders whose A stays intact
            // (a two-stage run pass writes its second stage into A).
            // independent jobs: the run-length-source tile after the
            // persistent kernel (which only encodes their source pages)
            bool fused = false;
            RectArgs fra;
            if (independent) {
                memset(&fra, 0, sizeof(fra));
                fra.dst = (uint32_t *)d.words;
                fra.dstride = d.stride_words * (Bd / 32);
                fra.W = W;
                fra.H = H;
                fra.nw_valid = (W + 31) / 32;
                fra.nw_cover = nw_cover;
                if (rect_plan(fra, q.op, c.sw, c.sh, c.ox, c.oy, band_hint, 0, 0, 0, true) == 0) {
                    fra.band_auto = 0;
                    fused = true;
                }
            }
            const bool a_rewritten = b.nst == 2 && c.sh == 1 && !fused;
            int enc = -1;
            if (q.depends_on < 0) {
                const SrcKey key{s.words, s.stride_words, s.fmt, W, H};
                auto f = encoders.find(key);
                if (f != encoders.end()) enc = f->second;
                else if (!a_rewritten) encoders[key] = j;
            }
            b.off_counts = off; off += al((size_t)H * 4);
            b.off_nA = off; off += al(8);
            if (!fused) {
                b.off_nB = off; off += al(8);
                b.off_rpB = off; off += al((size_t)(H + 1) * 4);
                b.off_runsB = off; off += al((size_t)b.cap * 4);
            }
            if (enc < 0 || a_rewritten) {
                b.off_rpA = off; off += al((size_t)(H + 1) * 4);
                b.off_runsA = off; off += al((size_t)b.cap * 4);
            }
            if (enc >= 0) {
                b.src_job = enc;
                b.dep = enc;
                b.dep_phase = ENCODE_PHASES - 1;
                b.off_srp = J[enc].off_rpA;
                b.off_sruns = J[enc].off_runsA;
            } else {
                b.off_srp = b.off_rpA;
                b.off_sruns = b.off_runsA;
            }
            if (b.nst == 2 && c.sh > 1 && !fused) {
                b.off_bmp = off;
                off += al((size_t)H * ((W + 31) / 32) * 4);
            }
            b.rows = item_rows(q);
            const int rows_items = (H + b.rows - 1) / b.rows;
            int p = 0;
            auto add = [&](int kind, int items, int stage) {
                b.phase_kind[p] = kind;
                b.phase_items[p] = items;
                b.phase_stage[p] = stage;
                ++p;
            };
            if (b.src_job == j) {  // encode the source: ENCODE_PHASES phases
                add(IK_B2R_COUNT, rows_items, -1);
                add(IK_SCAN, 1, -1);
                add(IK_B2R_WRITE, rows_items, -1);
            }
            if (fused) {
                RleJob rj;
                rj.a = fra;
                rj.off_row_ptr = b.off_srp;
                rj.off_runs = b.off_sruns;
                rj.op1 = RowOp{(q.op == MORPH_DILATE || q.op == MORPH_CLOSE) ? 1 : 0, c.sw, c.ox, W};
                rj.cap = b.src_job == j ? b.cap : J[b.src_job].cap;
                add_to_group(G, 1, 0, fra, &rj, rle_rect_smem_words(fra) * 4);
                b.nphase = p;  // the encode, if this job is its page's encoder
                continue;
            }
            for (int st = 0; st < b.nst; ++st) {
                // stage order: open = erode then dilate; close = dilate then erode
                const bool dil = (q.op == MORPH_DILATE) || (q.op == MORPH_OPEN && st == 1) ||
                                 (q.op == MORPH_CLOSE && st == 0);
                b.rop[st] = RowOp{dil ? 1 : 0, c.sw, c.ox, W};
                if (c.sh == 1) {
                    add(IK_ROW_COUNT, rows_items, st);
                    add(IK_SCAN, 1, st);
                    add(IK_ROW_WRITE, rows_items, st);
                } else {
                    VArgs &v = b.va[st];
                    memset(&v, 0, sizeof(v));
                    v.in.W = W;
                    v.in.H = H;
                    v.op = b.rop[st];
                    v.inv = dil;
                    v.sh = c.sh;
                    v.ey = dil ? c.sh - 1 - c.oy : c.oy;
                    v.K = bitlen(c.sh);
                    for (int k = 0; k < 16; ++k) v.eqm[k] = ((c.sh >> k) & 1) ? 0u : ONES;
                    const int km = vpass_kmax(c.sh);
                    const int kk = km == 2 ? 0 : (km == 3 ? 1 : (km == 6 ? 2 : 3));
                    int sb, grid;
                    if (vband_plan(v, W, H, c.sh, VBAND_SMEM_BUDGET)) {
                        b.vkind[st] = 8 + kk;
                        sb = (int)vband_smem_bytes(v);
                        grid = vband_grid(v);
                    } else {
                        vpass_plan(v, W, H, c.sh);
                        b.vkind[st] = (v.nwt == 2 ? 0 : 4) + kk;
                        sb = (int)vpass_smem_bytes(v);
                        grid = vpass_grid(v);
                    }
                    v.capacity = b.cap;
                    if (sb > smem) smem = sb;
                    // rows -> bitmap; an intermediate stage is then encoded
                    // into runs (its run pass input for the next stage), the
                    // last stage's bitmap is the job's output
                    add(IK_V_BMP, grid, st);
                    if (st < b.nst - 1) {
                        add(IK_BCOUNT, rows_items, st);
                        add(IK_SCAN, 1, st);
                        add(IK_BWRITE, rows_items, st);
                    }
                }
            }
            if (c.sh == 1) add(IK_R2B, rows_items, -1);
            b.nphase = p;
            const int sb = 8 * nw_cover * 4;
            if (sb > smem) smem = sb;
        } else {
            return berr(MORPH_EINVAL, "path must be MORPH_PATH_PACKED or MORPH_PATH_RLE", j);
        }
    }
    ws_total = off;
    // Level order: phase p of job j sits at level level0_j + p, where a job
    // that depends on job i starts one level after i's last phase.  Items are
    // listed by level, so every item a wait refers to comes earlier in the
    // list (and is already held by a running CTA when the wait starts).
    I.clear();
    int maxlevel = 0;
    for (int j = 0; j < n; ++j) {
        J[j].level0 = J[j].dep >= 0 ? J[J[j].dep].level0 + J[j].dep_phase + 1 : 0;
        const int top = J[j].level0 + J[j].nphase;
        if (top > maxlevel) maxlevel = top;
    }
    for (int lv = 0; lv < maxlevel; ++lv)
        for (int j = 0; j < n; ++j) {
            const int p = lv - J[j].level0;
            if (p >= 0 && p < J[j].nphase)
                for (int k = 0; k < J[j].phase_items[p]; ++k)
                    I.push_back(BatchItem{j, (int16_t)p, (int16_t)J[j].phase_kind[p], k});
        }
    return MORPH_OK;
}

// Streams the batch launch forks its tile groups onto (per device, created
// once, never destroyed), with the events of the fork and of the join.  The
// launch sequence holds the device's mutex, so one set serves every caller.
// Streams 0 .. AUX_PACKED - 1 run the packed groups, the others the RLE
// groups, so that the two kinds overlap (the packed tiles are bound by
// integer logic, the run-length-source tiles by latency).
constexpr int AUX_STREAMS = 8;
constexpr int AUX_PACKED = 4;
struct AuxStreams {
    std::mutex mu;
    bool made = false;
    cudaStream_t st[AUX_STREAMS];
    cudaEvent_t fork, kb_done, join[AUX_STREAMS], level[AUX_PACKED];
};
AuxStreams *aux_streams(int dev, cudaError_t &e) {
    static AuxStreams a[64];
    e = cudaSuccess;
    if (dev < 0 || dev >= 64) {
        e = cudaErrorInvalidDevice;
        return nullptr;
    }
    return &a[dev];
}
cudaError_t make_aux(AuxStreams &a) {
    if (a.made) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < AUX_STREAMS && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&a.st[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.kb_done, cudaEventDisableTiming);
    for (int k = 0; k < AUX_STREAMS && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&a.join[k], cudaEventDisableTiming);
    for (int k = 0; k < AUX_PACKED && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&a.level[k], cudaEventDisableTiming);
    if (e == cudaSuccess) a.made = true;
    return e;
}

size_t group_tables_bytes(const GroupPlan &g) {
    const size_t tab = g.g.rle ? g.rle.size() * sizeof(RleJob) : g.rect.size() * sizeof(RectArgs);
    return al(tab) + al(g.starts.size() * sizeof(int));
}

size_t plan_size(const std::vector<BatchJob> &J, const std::vector<BatchItem> &I, const std::vector<GroupPlan> &G) {
    size_t n = al(sizeof(BatchHeader)) + al(J.size() * sizeof(BatchJob)) + al(I.size() * sizeof(BatchItem)) +
               al(G.size() * sizeof(TileGroup));
    for (const auto &g : G) n += group_tables_bytes(g);
    return n;
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" {

size_t morph_batch_plan_bytes(const morph_job *jobs, int n_jobs, int tile_rows,
                              int rle_runs_per_row) {
    if (!jobs || n_jobs < 1) return 0;
    std::vector<BatchJob> J;
    std::vector<BatchItem> I;
    std::vector<GroupPlan> G;
    int64_t c, t;
    int smem;
    if (build(jobs, n_jobs, tile_rows, rle_runs_per_row, J, I, c, t, smem, G) != MORPH_OK) return 0;
    return plan_size(J, I, G);
}

morph_status morph_batch_plan_build(void *host_plan, size_t plan_bytes, const morph_job *jobs,
                                    int n_jobs, int tile_rows, int rle_runs_per_row) {
    if (!host_plan || !jobs || n_jobs < 1) {
        set_error("NULL plan or jobs, or n_jobs < 1");
        return MORPH_EINVAL;
    }
    std::vector<BatchJob> J;
    std::vector<BatchItem> I;
    std::vector<GroupPlan> G;
    int64_t ctrl, total;
    int smem, kb_after = 0;
    morph_status st = build(jobs, n_jobs, tile_rows, rle_runs_per_row, J, I, ctrl, total, smem, G, &kb_after);
    if (st != MORPH_OK) return st;
    BatchHeader h;
    memset(&h, 0, sizeof(h));
    h.kb_after_groups = kb_after;
    h.magic = PLAN_MAGIC;
    h.n_jobs = n_jobs;
    h.n_items = (int32_t)I.size();
    h.smem_bytes = smem;
    h.jobs_off = (int64_t)al(sizeof(BatchHeader));
    h.items_off = h.jobs_off + (int64_t)al(J.size() * sizeof(BatchJob));
    h.groups_off = h.items_off + (int64_t)al(I.size() * sizeof(BatchItem));
    h.n_groups = (int32_t)G.size();
    int64_t toff = h.groups_off + (int64_t)al(G.size() * sizeof(TileGroup));
    for (auto &g : G) {
        g.g.jobs_off = toff;
        toff += (int64_t)al(g.g.rle ? g.rle.size() * sizeof(RleJob) : g.rect.size() * sizeof(RectArgs));
        g.g.starts_off = toff;
        toff += (int64_t)al(g.starts.size() * sizeof(int));
    }
    h.plan_bytes = toff;
    h.ws_ctrl_bytes = ctrl;
    h.ws_bytes = total;
    h.wait_limit_ns = WAIT_LIMIT_NS;
    if ((int64_t)plan_bytes < h.plan_bytes) {
        set_error("plan buffer of %zu bytes < %lld needed", plan_bytes, (long long)h.plan_bytes);
        return MORPH_ENOMEM;
    }
    uint8_t *p = (uint8_t *)host_plan;
    memset(p, 0, (size_t)h.plan_bytes);
    memcpy(p, &h, sizeof(h));
    memcpy(p + h.jobs_off, J.data(), J.size() * sizeof(BatchJob));
    memcpy(p + h.items_off, I.data(), I.size() * sizeof(BatchItem));
    for (size_t k = 0; k < G.size(); ++k) {
        const GroupPlan &g = G[k];
        memcpy(p + h.groups_off + k * sizeof(TileGroup), &g.g, sizeof(TileGroup));
        if (g.g.rle) memcpy(p + g.g.jobs_off, g.rle.data(), g.rle.size() * sizeof(RleJob));
        else memcpy(p + g.g.jobs_off, g.rect.data(), g.rect.size() * sizeof(RectArgs));
        memcpy(p + g.g.starts_off, g.starts.data(), g.starts.size() * sizeof(int));
    }
    return MORPH_OK;
}

int morph_batch_kernels(const void *host_plan) {
    const BatchHeader *h = (const BatchHeader *)host_plan;
    if (!h || h->magic != PLAN_MAGIC) return -1;
    return h->n_groups + (h->n_items > 0 && !h->groups_only ? 1 : 0);
}

size_t morph_batch_workspace_size(const void *host_plan) {
    const BatchHeader *h = (const BatchHeader *)host_plan;
    if (!h || h->magic != PLAN_MAGIC) return 0;
    return (size_t)h->ws_bytes;
}

morph_status morph_batch_plan_debug(void *host_plan, int what, long long value) {
    BatchHeader *h = (BatchHeader *)host_plan;
    if (!h || h->magic != PLAN_MAGIC) {
        set_error("NULL or invalid plan");
        return MORPH_EINVAL;
    }
    if (what == 0) {
        if (value < 1000000) value = 1000000;
        h->wait_limit_ns = value;
        return MORPH_OK;
    }
    if (what == 1) {
        BatchJob *J = (BatchJob *)((uint8_t *)host_plan + h->jobs_off);
        for (int j = 0; j < h->n_jobs; ++j)
            if (J[j].nphase > 1) {
                J[j].phase_items[0] += (int32_t)value;
                return MORPH_OK;
            }
        set_error("no job with more than one phase");
        return MORPH_EINVAL;
    }
    if (what == 2) {
        h->groups_only = value != 0;
        return MORPH_OK;
    }
    set_error("unknown debug request %d", what);
    return MORPH_EINVAL;
}

int morph_batch_items(const void *host_plan) {
    const BatchHeader *h = (const BatchHeader *)host_plan;
    if (!h || h->magic != PLAN_MAGIC) return -1;
    return h->n_items;
}

morph_status morph_batch_launch(const void *dev_plan, const void *host_plan, void *workspace,
                                size_t workspace_bytes, int n_ctas, void *stream) {
    const BatchHeader *h = (const BatchHeader *)host_plan;
    if (!dev_plan || !h || h->magic != PLAN_MAGIC) {
        set_error("NULL or invalid plan");
        return MORPH_EINVAL;
    }
    if (!workspace || (int64_t)workspace_bytes < h->ws_bytes) {
        set_error("workspace of %zu bytes < %lld needed", workspace ? workspace_bytes : (size_t)0,
                  (long long)h->ws_bytes);
        return MORPH_ENOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int smem = h->smem_bytes;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && n_ctas <= 0) {
        // resident CTAs for this shared-memory size, cached per device
        static std::mutex mu;
        static int cached_smem[128], cached_ctas[128];
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess && dev >= 0 && dev < 128) {
            std::lock_guard<std::mutex> lk(mu);
            if (cached_ctas[dev] > 0 && cached_smem[dev] == smem) {
                n_ctas = cached_ctas[dev];
            } else {
                e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BATCH_THREADS, smem);
                n_ctas = sms * (per_sm > 0 ? per_sm : 1);
                cached_smem[dev] = smem;
                cached_ctas[dev] = n_ctas;
            }
        }
    }
    const uint8_t *dp = (const uint8_t *)dev_plan, *hp = (const uint8_t *)host_plan;
    const TileGroup *groups = reinterpret_cast<const TileGroup *>(hp + h->groups_off);
    int npk = 0, nrl = 0;
    for (int k = 0; k < h->n_groups; ++k) {
        if (groups[k].ctas < 1) continue;
        if (groups[k].rle) ++nrl;
        else ++npk;
    }
    // Tile groups run on the device's auxiliary streams, forked from and
    // joined back into the caller's stream, ordered only by what they read:
    //  - packed groups on streams 0 .. AUX_PACKED - 1, level by level (the
    //    packed streams meet at an event barrier between levels);
    //  - the persistent kernel on the caller's stream, at once, or after the
    //    last packed level when one of its jobs reads a grouped job's result;
    //  - RLE groups on the other streams once the persistent kernel has
    //    encoded their sources.
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    AuxStreams *ax = nullptr;
    if (e == cudaSuccess) ax = aux_streams(dev, e);
    if (e == cudaSuccess && npk + nrl == 0) ax = nullptr;
    // a plan with at most one group per level and at most one RLE group (a
    // single request's chain of jobs, say) has nothing to overlap: it runs in
    // stream order on the caller's stream, without the fork, the level
    // barriers and the join (dozens of event calls per launch)
    {
        int per_level[64] = {}, maxper = 0;
        bool deep = false;
        for (int k = 0; k < h->n_groups; ++k) {
            if (groups[k].rle || groups[k].ctas < 1) continue;
            if (groups[k].level >= 64) { deep = true; continue; }
            const int c = ++per_level[groups[k].level];
            if (c > maxper) maxper = c;
        }
        if (!deep && maxper <= 1 && nrl <= 1) ax = nullptr;
    }
    std::unique_lock<std::mutex> lk;
    if (ax) {
        lk = std::unique_lock<std::mutex>(ax->mu);
        e = make_aux(*ax);
    }
    const int np = ax && npk > 0 ? AUX_PACKED : 0;                  // packed streams in use
    const int nr = ax && nrl > 0 ? AUX_STREAMS - AUX_PACKED : 0;    // RLE streams in use
    // every packed stream waits for every other one's last launch
    auto packed_barrier = [&]() {
        cudaError_t r = cudaSuccess;
        for (int k = 0; r == cudaSuccess && k < np; ++k) r = cudaEventRecord(ax->level[k], ax->st[k]);
        for (int k = 0; r == cudaSuccess && k < np; ++k)
            for (int q = 0; r == cudaSuccess && q < np; ++q)
                if (q != k) r = cudaStreamWaitEvent(ax->st[k], ax->level[q], 0);
        return r;
    };
    if (ax && e == cudaSuccess) {
        e = cudaEventRecord(ax->fork, s);
        for (int k = 0; e == cudaSuccess && k < np; ++k) e = cudaStreamWaitEvent(ax->st[k], ax->fork, 0);
    }
    int maxlevel = -1;
    for (int k = 0; k < h->n_groups; ++k)
        if (!groups[k].rle && groups[k].ctas > 0 && groups[k].level > maxlevel) maxlevel = groups[k].level;
    int gi = 0;
    for (int lv = 0; e == cudaSuccess && lv <= maxlevel; ++lv) {
        if (lv > 0 && ax) e = packed_barrier();
        for (int k = 0; e == cudaSuccess && k < h->n_groups; ++k) {
            const TileGroup &g = groups[k];
            if (g.rle || g.ctas < 1 || g.level != lv) continue;
            const RectJobs mj{reinterpret_cast<const RectArgs *>(dp + g.jobs_off),
                              reinterpret_cast<const int *>(dp + g.starts_off), g.njobs, g.ctas, (size_t)g.smem};
            e = launch_rect(g.proto, ax ? ax->st[gi++ % AUX_PACKED] : s, &mj);
            if (e != cudaSuccess) {
                set_error("batch launch: packed group %d (stages %d, %d words, modes %d/%d/%d, %d threads, %d "
                          "CTAs, %lld bytes shared): %s", k, g.proto.nst, g.proto.nwt, g.proto.vmode,
                          g.proto.hmode, g.proto.halo, g.proto.threads, g.ctas, (long long)g.smem,
                          cudaGetErrorString(e));
                return MORPH_ECUDA;
            }
        }
    }
    if (h->n_items > 0 && !h->groups_only) {
        if (np > 0 && h->kb_after_groups && e == cudaSuccess) {
            // the persistent kernel reads results of the packed groups
            for (int k = 0; e == cudaSuccess && k < np; ++k) e = cudaEventRecord(ax->level[k], ax->st[k]);
            for (int k = 0; e == cudaSuccess && k < np; ++k) e = cudaStreamWaitEvent(s, ax->level[k], 0);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(workspace, 0, (size_t)h->ws_ctrl_bytes, s);
        if (e == cudaSuccess) {
            k_batch<<<n_ctas, BATCH_THREADS, smem, s>>>(dp, (uint8_t *)workspace, device_status_ptr());
            e = cudaGetLastError();
        }
    }
    // RLE groups read the encodes of the persistent kernel: fork after it
    if (nr > 0 && e == cudaSuccess) {
        e = cudaEventRecord(ax->kb_done, s);
        for (int k = AUX_PACKED; e == cudaSuccess && k < AUX_STREAMS; ++k)
            e = cudaStreamWaitEvent(ax->st[k], ax->kb_done, 0);
    }
    int ri = 0;
    for (int k = 0; e == cudaSuccess && k < h->n_groups; ++k) {
        const TileGroup &g = groups[k];
        if (!g.rle || g.ctas < 1) continue;
        const RleJobs mj{reinterpret_cast<const RleJob *>(dp + g.jobs_off),
                         reinterpret_cast<const int *>(dp + g.starts_off), (const uint8_t *)workspace, g.njobs,
                         g.ctas, (size_t)g.smem};
        e = launch_rle_rect_tile(g.proto, RleSrc{}, ax ? ax->st[AUX_PACKED + ri++ % (AUX_STREAMS - AUX_PACKED)] : s,
                                 &mj);
        if (e != cudaSuccess) {
            set_error("batch launch: RLE group %d (stages %d, %d words, modes %d/%d/%d, %d threads, %d CTAs, "
                      "%lld bytes shared): %s", k, g.proto.nst, g.proto.nwt, g.proto.vmode, g.proto.hmode,
                      g.proto.halo, g.proto.threads, g.ctas, (long long)g.smem, cudaGetErrorString(e));
            return MORPH_ECUDA;
        }
    }
    // join every stream that was forked back into the caller's stream
    for (int k = 0; e == cudaSuccess && k < np; ++k) {
        e = cudaEventRecord(ax->join[k], ax->st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ax->join[k], 0);
    }
    for (int k = AUX_PACKED; e == cudaSuccess && k < AUX_PACKED + nr; ++k) {
        e = cudaEventRecord(ax->join[k], ax->st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ax->join[k], 0);
    }
    if (e != cudaSuccess) {
        set_error("batch launch: %s", cudaGetErrorString(e));
        return MORPH_ECUDA;
    }
    return MORPH_OK;
}

morph_status morph_batch_launch_host(const void *dev_plan, const void *host_plan, void *workspace,
                                     size_t workspace_bytes, const void *h_in, void *d_in, size_t in_bytes,
                                     void *h_out, const void *d_out, size_t out_bytes, void *stream) {
    if ((in_bytes && (!h_in || !d_in)) || (out_bytes && (!h_out || !d_out))) {
        set_error("batch host launch: NULL buffer with a nonzero size");
        return MORPH_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (in_bytes) {
        const cudaError_t e = cudaMemcpyAsync(d_in, h_in, in_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            set_error("batch host launch: copy in: %s", cudaGetErrorString(e));
            return MORPH_ECUDA;
        }
    }
    const morph_status st = morph_batch_launch(dev_plan, host_plan, workspace, workspace_bytes, 0, stream);
    if (st != MORPH_OK) return st;
    if (out_bytes) {
        const cudaError_t e = cudaMemcpyAsync(h_out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            set_error("batch host launch: copy out: %s", cudaGetErrorString(e));
            return MORPH_ECUDA;
        }
    }
    return MORPH_OK;
}

}  // extern "C"
