// Connected components and run-length statistics of RLE images (the paper's
// section "Connected Component Extraction and Statistics" and the run-length
// statistics of section "Other Operations").
//
// Components: every run is a node of a union-find forest stored in the
// caller's label array (parent indices, parent[k] <= k always, so a tree's
// root is its smallest run index = the component's first run in raster
// order).  The image is cut into bands of CC_BAND lines; a band's runs are
// one contiguous index range, so every per-band kernel walks them as a flat
// array (thread per run, the line found by binary search over the band's
// row offsets in shared memory).  Launches:
//   band     one CTA per band, cut into sub-bands of at most CC_CAP runs:
//            each sub-band's runs and union-find forest sit in shared
//            memory; every run of a line is united with the runs of the line
//            above that it touches (binary search over the ascending runs
//            above); parent = the sub-band root is written out, then the
//            seams between its sub-bands are joined in global memory
//   seams    the first line of every band joined with the line above it in
//            global memory (lock-free union: the larger root is hooked under
//            the smaller by compare-and-swap; a failed swap means the root
//            was hooked meanwhile and the union retries from there; finds
//            halve paths)
//   flatten  parent[k] = root(k) (read-only walks, so every entry ends at
//            its root); roots per band counted
//   scan     roots per band -> first component number of each band
//   rank     roots get their component number (raster order of roots) and
//            reset their statistics record
//   label    label[k] = number of root(k); statistics gathered in a shared-
//            memory table of the band's components (neighbouring lanes with
//            one label and line summed first by a segmented shuffle scan)
//            and added to the records once per component and band.
// Run-length histograms: persistent CTAs over the bands, shared-memory bins
// for runs shorter than RLH_BINS, global atomics for longer ones.
#include "morph_internal.cuh"

namespace morph {
namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_WARPS = CC_THREADS / 32;
constexpr int CC_UNITE_LIMIT = 1 << 20;  // retries of one union (lock-free: never reached)
constexpr int CC_BAND = 64;              // lines per band
constexpr int CC_CAP = 4096;             // runs per shared-memory sub-band
constexpr int CC_TABLE = 1024;           // components per band in the statistics table
constexpr int RLH_BINS = 2048;           // shared-memory bins per histogram

__device__ __forceinline__ int run_start(uint32_t r) { return (int)(r & 0xFFFFu); }
__device__ __forceinline__ int run_end(uint32_t r) { return (int)(r >> 16); }

__host__ __device__ __forceinline__ int nbands(int H) { return (H + CC_BAND - 1) / CC_BAND; }

// row offsets of the band's lines r0..r1 (r1 - r0 + 1 entries)
__device__ __forceinline__ void load_band_rows(const RleIn &in, int r0, int r1, int *s_rp) {
    for (int i = threadIdx.x; i <= r1 - r0; i += blockDim.x) s_rp[i] = in.row_ptr[r0 + i];
}

// local line l of run k: the last l in [0, nl) with s_rp[l] <= k
__device__ __forceinline__ int band_line(const int *s_rp, int nl, int k) {
    int lo = 0, hi = nl;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_rp[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------- union-find
// global forest: entries change under other threads, read through L2
__device__ __forceinline__ int ld_parent(const int32_t *p, int k) { return __ldcg(p + k); }

__device__ __forceinline__ int find_root(int32_t *parent, int x) {
    while (true) {
        const int p = ld_parent(parent, x);
        if (p == x) return x;
        const int gp = ld_parent(parent, p);
        if (gp == p) return p;
        __stcg(parent + x, gp);  // an ancestor of x: never breaks a tree
        x = gp;
    }
}

// read-only walk to the root: used once the forest no longer changes, where
// the only writes are entries set to their final root (a halving write
// racing with such a write could leave a non-root ancestor behind)
__device__ __forceinline__ int root_of(const int32_t *parent, int x) {
    int p = ld_parent(parent, x);
    while (p != x) {
        x = p;
        p = ld_parent(parent, x);
    }
    return x;
}

__device__ __forceinline__ bool unite(int32_t *parent, int a, int b) {
    for (int it = 0; it < CC_UNITE_LIMIT; ++it) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return true;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + a, a, b);
        if (old == a) return true;
        a = old;
    }
    return false;
}

// shared-memory forest of one sub-band (indices relative to its first run)
__device__ __forceinline__ int sfind(volatile int32_t *sp, int x) {
    while (true) {
        const int p = sp[x];
        if (p == x) return x;
        const int gp = sp[p];
        if (gp == p) return p;
        sp[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ bool sunite(int32_t *sp, int a, int b) {
    volatile int32_t *vp = sp;
    for (int it = 0; it < CC_UNITE_LIMIT; ++it) {
        a = sfind(vp, a);
        b = sfind(vp, b);
        if (a == b) return true;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(sp + a, a, b);
        if (old == a) return true;
        a = old;
    }
    return false;
}

// The lanes of one warp take the runs [a1, b1) of a line and unite each with
// the touching runs of the line above, [a0, a1).  runs is indexed in the same
// index space as the bounds; unite_fn(k, j) joins two of those indices.
template <typename U>
__device__ __forceinline__ void link_runs(const uint32_t *runs, int a0, int a1, int b1, int d,
                                          U unite_fn) {
    for (int k = a1 + (int)(threadIdx.x & 31); k < b1; k += 32) {
        const uint32_t r = runs[k];
        const int s = run_start(r), e = run_end(r);
        // first run above whose end reaches this start (ends ascend)
        int lo = a0, hi = a1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (run_end(runs[mid]) + d <= s) lo = mid + 1;
            else hi = mid;
        }
        for (int j = lo; j < a1; ++j) {
            if (run_start(runs[j]) >= e + d) break;
            unite_fn(k, j);
        }
    }
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_band(RleIn in, int d, int32_t *parent, int *status) {
    __shared__ int32_t sp[CC_CAP];
    __shared__ uint32_t sr[CC_CAP];
    __shared__ unsigned char sline[CC_CAP];  // band line of each window run
    __shared__ int s_rp[CC_BAND + 1];
    __shared__ int s_sub[CC_BAND + 1];
    __shared__ unsigned char s_gh[CC_BAND];
    __shared__ int s_nsub;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r0 = blockIdx.x * CC_BAND, r1 = min(in.H, r0 + CC_BAND), nl = r1 - r0;
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    load_band_rows(in, r0, r1, s_rp);
    __syncthreads();
    if (s_rp[nl] - s_rp[0] <= CC_CAP) {
        // the whole band fits (the common case): one sub-band
        if (tid == 0) {
            s_sub[0] = 0;
            s_sub[1] = nl;
            s_gh[0] = 0;
            s_nsub = 1;
        }
    } else if (tid == 0) {
        // Greedy cut into sub-bands that fit CC_CAP runs together with the
        // previous sub-band's last line ("ghost" runs: the line above is then
        // joined in shared memory too).  Ghosts are dropped when they do not
        // fit (that seam is joined in global memory); a line with more runs
        // than CC_CAP is a sub-band of its own, kept in global memory.
        int n = 0, l = 0;
        bool prev_smem = false;
        s_sub[0] = 0;
        while (l < nl) {
            int g = (l > 0 && prev_smem) ? s_rp[l] - s_rp[l - 1] : 0;
            if (g + s_rp[l + 1] - s_rp[l] > CC_CAP) g = 0;
            int l2 = l + 1;
            while (l2 < nl && g + s_rp[l2 + 1] - s_rp[l] <= CC_CAP) ++l2;
            s_gh[n] = g > 0 ? 1 : 0;
            prev_smem = g + s_rp[l2] - s_rp[l] <= CC_CAP;
            s_sub[++n] = l2;
            l = l2;
        }
        s_nsub = n;
    }
    __syncthreads();
    const int nsub = s_nsub;
    for (int sb = 0; sb < nsub; ++sb) {
        const int la = s_sub[sb], lb = s_sub[sb + 1];
        const int g = s_gh[sb] ? s_rp[la] - s_rp[la - 1] : 0;
        const int G = s_rp[la] - g, n = s_rp[lb] - G;  // window: runs [G, G + n)
        if (n <= CC_CAP) {
            for (int i = tid; i < n; i += CC_THREADS) {
                sp[i] = i;
                sr[i] = runs[G + i];
            }
            for (int l = la - (g > 0 ? 1 : 0) + warp; l < lb; l += CC_WARPS)
                for (int k = s_rp[l] + (tid & 31); k < s_rp[l + 1]; k += 32) sline[k - G] = (unsigned char)l;
            __syncthreads();
            // one thread per run of the lines whose line above is in the
            // window (balanced over the warps whatever the lines hold), in
            // rounds of CC_THREADS runs top to bottom: a round's runs hook
            // under trees the rounds above have finished, which keeps the
            // trees shallow (lines linked all at once would chain a vertical
            // stroke run under run, one line per level)
            const int kend = s_rp[lb];
            for (int k0 = s_rp[g > 0 ? la : la + 1]; k0 < kend; k0 += CC_THREADS) {
                const int k = k0 + tid;
                if (k0 > s_rp[g > 0 ? la : la + 1]) __syncthreads();
                if (k >= kend) continue;
                const int kk = k - G;
                const int l = sline[kk];
                const int a0 = s_rp[l - 1] - G, a1 = s_rp[l] - G;
                const uint32_t r = sr[kk];
                const int rs = run_start(r), re = run_end(r);
                int lo = a0, hi = a1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (run_end(sr[mid]) + d <= rs) lo = mid + 1;
                    else hi = mid;
                }
                for (int j = lo; j < a1; ++j) {
                    if (run_start(sr[j]) >= re + d) break;
                    if (!sunite(sp, kk, j)) latch_status(status, MORPH_ETIMEOUT);
                }
            }
            __syncthreads();
            for (int i = tid; i < n; i += CC_THREADS) {
                int x = i, p = sp[x];
                while (p != x) {
                    x = p;
                    p = sp[x];
                }
                if (i >= g) {
                    // a root among the ghosts: continue with that ghost's
                    // parent, written when the sub-band above was finished
                    parent[G + i] = x >= g ? G + x : parent[G + x];
                } else if (x != i) {
                    // two ghosts that this sub-band connects (rare: a U shape
                    // closing): their components above are joined globally
                    if (!unite(parent, G + i, G + x)) latch_status(status, MORPH_ETIMEOUT);
                }
            }
            __syncthreads();  // before the next sub-band reuses sp and sr
        } else {
            for (int i = tid; i < n; i += CC_THREADS) parent[G + i] = G + i;
            __syncthreads();
        }
    }
    // seams between sub-bands that carried no ghosts: global memory
    for (int sb = 1 + warp; sb < nsub; sb += CC_WARPS) {
        if (s_gh[sb]) continue;
        const int l = s_sub[sb];
        link_runs(runs, s_rp[l - 1], s_rp[l], s_rp[l + 1], d, [&](int k, int j) {
            if (!unite(parent, k, j)) latch_status(status, MORPH_ETIMEOUT);
        });
    }
}

// first line of every band against the last line of the band above (one warp per seam)
__global__ void __launch_bounds__(CC_THREADS) k_cc_seams(RleIn in, int d, int32_t *parent, int *status) {
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    const int nb = nbands(in.H);
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int b = 1 + w; b < nb; b += nw) {
        const int y = b * CC_BAND;
        link_runs(runs, in.row_ptr[y - 1], in.row_ptr[y], in.row_ptr[y + 1], d, [&](int k, int j) {
            if (!unite(parent, k, j)) latch_status(status, MORPH_ETIMEOUT);
        });
    }
}

// Exclusive count of the flags of the CTA's threads before this one (in
// thread order); total = all flags.  s_w: CC_WARPS ints of shared memory.
__device__ __forceinline__ int block_excl_count(bool f, int *s_w, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) s_w[warp] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < CC_WARPS; ++w) {
        const int c = s_w[w];
        before += w < warp ? c : 0;
        all += c;
    }
    __syncthreads();  // s_w is rewritten by the next call
    total = all;
    return before + __popc(m & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_flatten(RleIn in, int32_t *parent, int32_t *counts) {
    const int r0 = blockIdx.x * CC_BAND, r1 = min(in.H, r0 + CC_BAND);
    const int A = in.row_ptr[r0], B = in.row_ptr[r1];
    int roots = 0;
    for (int i0 = A; i0 < B; i0 += CC_THREADS) {
        const int k = i0 + (int)threadIdx.x;
        bool root = false;
        if (k < B) {
            const int r = root_of(parent, k);
            root = r == k;
            if (!root) __stcg(parent + k, r);
        }
        roots += __syncthreads_count(root);
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = roots;
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_rank(RleIn in, const int32_t *parent,
                                                       const int32_t *bandptr, int32_t *rank,
                                                       morph_component *stats, int64_t max_c) {
    __shared__ int s_rp[CC_BAND + 1];
    __shared__ int s_w[CC_WARPS];
    const int r0 = blockIdx.x * CC_BAND, r1 = min(in.H, r0 + CC_BAND), nl = r1 - r0;
    load_band_rows(in, r0, r1, s_rp);
    __syncthreads();
    const int A = s_rp[0], B = s_rp[nl];
    int base = bandptr[blockIdx.x];
    for (int i0 = A; i0 < B; i0 += CC_THREADS) {
        const int k = i0 + (int)threadIdx.x;
        const bool root = k < B && parent[k] == k;
        int total;
        const int pos = block_excl_count(root, s_w, total);
        if (root) {
            const int c = base + pos;
            rank[k] = c;
            if (stats && c < max_c) {
                // the root is the component's first run: its line is y0
                const int y = r0 + band_line(s_rp, nl, k);
                morph_component &t = stats[c];
                t.x0 = INT64_MAX;
                t.y0 = y;
                t.x1 = INT64_MIN;
                t.y1 = y + 1;
                t.area = 0;
                t.sum_x = 0;
                t.sum_y = 0;
            }
        }
        base += total;
    }
}

__device__ __forceinline__ void add_i64(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// Shared-memory table of the components met in one band (open addressing).
struct CcTable {
    int32_t key[CC_TABLE];
    int32_t x0[CC_TABLE], x1[CC_TABLE], y1[CC_TABLE], area[CC_TABLE];
    unsigned long long sx[CC_TABLE], sy[CC_TABLE];
};

__device__ __forceinline__ int cc_slot(int lab) { return (int)(((unsigned)lab * 2654435761u) >> 22); }

__device__ __forceinline__ void record_add(morph_component &g, int x0, int x1, int y1, int area,
                                           int64_t sx, int64_t sy) {
    atomicMin(reinterpret_cast<long long *>(&g.x0), (long long)x0);
    atomicMax(reinterpret_cast<long long *>(&g.x1), (long long)x1);
    atomicMax(reinterpret_cast<long long *>(&g.y1), (long long)y1);
    add_i64(&g.area, area);
    add_i64(&g.sum_x, sx);
    add_i64(&g.sum_y, sy);
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_label(RleIn in, int32_t *labels,
                                                        const int32_t *rank,
                                                        morph_component *stats, int64_t max_c) {
    static_assert(CC_TABLE == 1024, "cc_slot maps to 10 bits");
    __shared__ CcTable t;
    __shared__ int s_rp[CC_BAND + 1];
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned le = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    const int r0 = blockIdx.x * CC_BAND, r1 = min(in.H, r0 + CC_BAND), nl = r1 - r0;
    load_band_rows(in, r0, r1, s_rp);
    if (stats) {
        for (int i = tid; i < CC_TABLE; i += CC_THREADS) {
            t.key[i] = -1;
            t.x0[i] = INT32_MAX;
            t.x1[i] = 0;
            t.y1[i] = 0;
            t.area[i] = 0;
            t.sx[i] = 0;
            t.sy[i] = 0;
        }
    }
    __syncthreads();
    const int A = s_rp[0], B = s_rp[nl];
    for (int i0 = A; i0 < B; i0 += CC_THREADS) {
        const int k = i0 + tid;
        const bool ok = k < B;
        int lab = -1, y = -1, s = 0, e = 0;
        if (ok) {
            lab = rank[labels[k]];
            labels[k] = lab;
            const uint32_t r = runs[k];
            s = run_start(r);
            e = run_end(r);
            y = r0 + band_line(s_rp, nl, k);
        }
        if (!stats) continue;
        // segments of neighbouring lanes with one label on one line:
        // inclusive sums of area and sum of x up to each lane
        const int prev_lab = __shfl_up_sync(0xFFFFFFFFu, lab, 1);
        const int prev_y = __shfl_up_sync(0xFFFFFFFFu, y, 1);
        const bool head = lane == 0 || prev_lab != lab || prev_y != y;
        const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
        const int seg = __popc(heads & le);
        const int len = e - s;
        int area = len;
        int64_t sx = (int64_t)(s + e - 1) * len / 2;
        int x0 = s;
        bool tail = true;
        if (heads != 0xFFFFFFFFu) {  // some lanes share a segment: sum it first
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int a_up = __shfl_up_sync(0xFFFFFFFFu, area, off);
                const int64_t sx_up = __shfl_up_sync(0xFFFFFFFFu, sx, off);
                const int seg_up = __shfl_up_sync(0xFFFFFFFFu, seg, off);
                const int x0_up = __shfl_up_sync(0xFFFFFFFFu, x0, off);
                if (lane >= off && seg_up == seg) {
                    area += a_up;
                    sx += sx_up;
                    x0 = x0_up;  // runs of a line ascend: the segment's first start
                }
            }
            const int nseg = __shfl_down_sync(0xFFFFFFFFu, seg, 1);
            tail = lane == 31 || nseg != seg;
        }
        if (!(ok && tail && lab < max_c)) continue;
        const int64_t sy = (int64_t)y * area;
        // find or claim the component's slot (linear probing)
        int slot = cc_slot(lab), got = -1;
        for (int probe = 0; probe < CC_TABLE; ++probe) {
            const int cur = atomicCAS(&t.key[slot], -1, lab);
            if (cur == -1 || cur == lab) {
                got = slot;
                break;
            }
            slot = (slot + 1) & (CC_TABLE - 1);
        }
        if (got >= 0) {
            atomicMin(&t.x0[got], x0);
            atomicMax(&t.x1[got], e);
            atomicMax(&t.y1[got], y + 1);
            atomicAdd(&t.area[got], area);
            atomicAdd(&t.sx[got], (unsigned long long)sx);
            atomicAdd(&t.sy[got], (unsigned long long)sy);
        } else {  // table full: straight to the record
            record_add(stats[lab], x0, e, y + 1, area, sx, sy);
        }
    }
    if (!stats) return;
    __syncthreads();
    for (int i = tid; i < CC_TABLE; i += CC_THREADS) {
        const int lab = t.key[i];
        if (lab >= 0)
            record_add(stats[lab], t.x0[i], t.x1[i], t.y1[i], t.area[i], (int64_t)t.sx[i], (int64_t)t.sy[i]);
    }
}

// ------------------------------------------------- run-length histograms
__global__ void __launch_bounds__(CC_THREADS) k_rl_hist(RleIn in, int64_t *black, int64_t *white) {
    __shared__ uint32_t hb[RLH_BINS], hw[RLH_BINS];
    __shared__ int s_rp[CC_BAND + 1];
    for (int i = threadIdx.x; i < RLH_BINS; i += blockDim.x) {
        hb[i] = 0;
        hw[i] = 0;
    }
    const int W = in.W;
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    auto count = [&](uint32_t *sh, int64_t *g, int len) {
        if (!g || len <= 0) return;
        if (len < RLH_BINS) atomicAdd(sh + len, 1u);
        else add_i64(g + len, 1);
    };
    const int nb = nbands(in.H);
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int r0 = b * CC_BAND, r1 = min(in.H, r0 + CC_BAND), nl = r1 - r0;
        __syncthreads();  // the previous band is done with s_rp
        load_band_rows(in, r0, r1, s_rp);
        __syncthreads();
        const int A = s_rp[0], B = s_rp[nl];
        for (int k = A + (int)threadIdx.x; k < B; k += CC_THREADS) {
            const int l = band_line(s_rp, nl, k);
            const uint32_t r = runs[k];
            const int s = run_start(r), e = run_end(r);
            const int pe = k > s_rp[l] ? run_end(runs[k - 1]) : 0;  // end of the run before
            count(hb, black, e - s);
            count(hw, white, s - pe);
            if (k == s_rp[l + 1] - 1) count(hw, white, W - e);  // the line's last run
        }
        for (int l = threadIdx.x; l < nl; l += CC_THREADS)
            if (s_rp[l] == s_rp[l + 1]) count(hw, white, W);  // empty line
    }
    __syncthreads();
    const int nbins = min(RLH_BINS, W + 1);
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        if (black && hb[i]) add_i64(black + i, hb[i]);
        if (white && hw[i]) add_i64(white + i, hw[i]);
    }
}

}  // namespace

cudaError_t launch_rle_components(RleIn in, int conn, MorphCC c, int *status, cudaStream_t s) {
    const int d = conn == 8 ? 1 : 0;
    const int nb = nbands(in.H);
    k_cc_band<<<nb, CC_THREADS, 0, s>>>(in, d, c.labels, status);
    if (nb > 1) {
        int gs = (nb - 1 + CC_WARPS - 1) / CC_WARPS;
        if (gs > 152 * 8) gs = 152 * 8;
        k_cc_seams<<<gs, CC_THREADS, 0, s>>>(in, d, c.labels, status);
    }
    // roots per band -> first component number of each band (counts holds
    // nb <= H entries, rootptr nb + 1)
    k_cc_flatten<<<nb, CC_THREADS, 0, s>>>(in, c.labels, c.counts);
    const int64_t cap = c.stats ? c.max_components : INT64_MAX;
    launch_scan_rows(c.counts, nb, c.rootptr, c.n_components, cap, status, s);
    k_cc_rank<<<nb, CC_THREADS, 0, s>>>(in, c.labels, c.rootptr, c.rank, c.stats, c.max_components);
    k_cc_label<<<nb, CC_THREADS, 0, s>>>(in, c.labels, c.rank, c.stats, c.max_components);
    return cudaGetLastError();
}

cudaError_t launch_run_length_hist(RleIn in, int64_t *black, int64_t *white, cudaStream_t s) {
    const size_t bytes = (size_t)(in.W + 1) * sizeof(int64_t);
    cudaError_t e;
    if (black && (e = cudaMemsetAsync(black, 0, bytes, s)) != cudaSuccess) return e;
    if (white && (e = cudaMemsetAsync(white, 0, bytes, s)) != cudaSuccess) return e;
    int g = nbands(in.H);
    if (g > 152 * 4) g = 152 * 4;
    k_rl_hist<<<g, CC_THREADS, 0, s>>>(in, black, white);
    return cudaGetLastError();
}

}  // namespace morph
