// Connected components and run-length statistics of RLE images (the paper's
// section "Connected Component Extraction and Statistics" and the run-length
// statistics of section "Other Operations").
//
// Components: every run is a node of a union-find forest stored in the
// caller's label array (parent indices, parent[k] <= k always, so a tree's
// root is its smallest run index = the component's first run in raster
// order).  Five launches:
//   init     parent[k] = k
//   link     one warp per line y: each run of y finds, by binary search over
//            the ascending runs of line y-1, the first run above it can
//            touch, and unites with every touching run.  Union is lock-free:
//            the larger of the two roots is hooked under the smaller with a
//            compare-and-swap on its parent entry; a failed swap means the
//            root was hooked meanwhile and the union retries from there.
//            Finds halve paths (a node's parent becomes its grandparent).
//   flatten  parent[k] = root(k) (read-only walks, so every entry ends at
//            its root); roots per line counted
//   scan     roots per line -> first component number of each line
//   rank     roots get their component number (raster order of roots);
//            they also reset their statistics record
//   label    label[k] = number of root(k); statistics accumulated per run,
//            runs of one warp that are neighbours and share a label summed
//            first (segmented shuffle scan) so that one lane per segment
//            issues the atomics.
// Run-length histograms: one warp per line, shared-memory bins for short
// runs, global atomics for long ones.
#include "morph_internal.cuh"

namespace morph {
namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_WARPS = CC_THREADS / 32;
constexpr int CC_UNITE_LIMIT = 1 << 20;  // retries of one union (lock-free: never reached)
constexpr int RLH_BINS = 2048;           // shared-memory bins per histogram

__device__ __forceinline__ int run_start(uint32_t r) { return (int)(r & 0xFFFFu); }
__device__ __forceinline__ int run_end(uint32_t r) { return (int)(r >> 16); }

// parent entries change under other threads: read through L2
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

__device__ __forceinline__ int gwarp() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int nwarps() { return (int)((gridDim.x * blockDim.x) >> 5); }

__global__ void __launch_bounds__(CC_THREADS) k_cc_init(const int32_t *row_ptr, int H, int32_t *parent) {
    const int n = row_ptr[H];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        parent[k] = k;
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_link(RleIn in, int d, int32_t *parent, int *status) {
    const int lane = threadIdx.x & 31;
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    for (int y = 1 + gwarp(); y < in.H; y += nwarps()) {
        const int a0 = in.row_ptr[y - 1], a1 = in.row_ptr[y], b1 = in.row_ptr[y + 1];
        for (int k = a1 + lane; k < b1; k += 32) {
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
                if (!unite(parent, k, j)) latch_status(status, MORPH_ETIMEOUT);
            }
        }
    }
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_flatten(RleIn in, int32_t *parent, int32_t *counts) {
    const int lane = threadIdx.x & 31;
    for (int y = gwarp(); y < in.H; y += nwarps()) {
        const int a = in.row_ptr[y], b = in.row_ptr[y + 1];
        int roots = 0;
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            bool root = false;
            if (k < b) {
                const int r = root_of(parent, k);
                root = r == k;
                if (!root) __stcg(parent + k, r);
            }
            roots += __popc(__ballot_sync(0xFFFFFFFFu, root));
        }
        if (lane == 0) counts[y] = roots;
    }
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_rank(RleIn in, const int32_t *parent,
                                                       const int32_t *rootptr, int32_t *rank,
                                                       morph_component *stats, int64_t max_c) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int y = gwarp(); y < in.H; y += nwarps()) {
        const int a = in.row_ptr[y], b = in.row_ptr[y + 1];
        int base = rootptr[y];
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            const bool root = k < b && parent[k] == k;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, root);
            if (root) {
                const int c = base + __popc(m & lt);
                rank[k] = c;
                if (stats && c < max_c) {
                    // the root is the component's first run: its line is y0
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
            base += __popc(m);
        }
    }
}

__device__ __forceinline__ void add_i64(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_label(RleIn in, int32_t *labels,
                                                        const int32_t *rank,
                                                        morph_component *stats, int64_t max_c) {
    const int lane = threadIdx.x & 31;
    const unsigned le = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    for (int y = gwarp(); y < in.H; y += nwarps()) {
        const int a = in.row_ptr[y], b = in.row_ptr[y + 1];
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            const bool ok = k < b;
            int lab = -1, s = 0, e = 0;
            if (ok) {
                lab = rank[labels[k]];
                labels[k] = lab;
                const uint32_t r = runs[k];
                s = run_start(r);
                e = run_end(r);
            }
            if (!stats) continue;
            // segments of neighbouring lanes with one label: inclusive sums
            // of area and sum of x up to each lane, within its segment
            const int prev = __shfl_up_sync(0xFFFFFFFFu, lab, 1);
            const bool head = lane == 0 || prev != lab;
            const int seg = __popc(__ballot_sync(0xFFFFFFFFu, head) & le);
            const int len = e - s;
            int area = len;
            int64_t sx = (int64_t)(s + e - 1) * len / 2;
            int x0 = s;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int a_up = __shfl_up_sync(0xFFFFFFFFu, area, off);
                const int64_t sx_up = __shfl_up_sync(0xFFFFFFFFu, sx, off);
                const int seg_up = __shfl_up_sync(0xFFFFFFFFu, seg, off);
                const int x0_up = __shfl_up_sync(0xFFFFFFFFu, x0, off);
                if (lane >= off && seg_up == seg) {
                    area += a_up;
                    sx += sx_up;
                    x0 = x0_up;  // runs ascend: the segment's first start
                }
            }
            const int nseg = __shfl_down_sync(0xFFFFFFFFu, seg, 1);
            const bool tail = lane == 31 || nseg != seg;
            if (ok && tail && lab < max_c) {
                morph_component &t = stats[lab];
                atomicMin(reinterpret_cast<long long *>(&t.x0), (long long)x0);
                atomicMax(reinterpret_cast<long long *>(&t.x1), (long long)e);
                atomicMax(reinterpret_cast<long long *>(&t.y1), (long long)(y + 1));
                add_i64(&t.area, area);
                add_i64(&t.sum_x, sx);
                add_i64(&t.sum_y, (int64_t)y * area);
            }
        }
    }
}

// ------------------------------------------------- run-length histograms
__global__ void __launch_bounds__(CC_THREADS) k_rl_hist(RleIn in, int64_t *black, int64_t *white) {
    __shared__ uint32_t hb[RLH_BINS], hw[RLH_BINS];
    for (int i = threadIdx.x; i < RLH_BINS; i += blockDim.x) {
        hb[i] = 0;
        hw[i] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int W = in.W;
    const uint32_t *runs = reinterpret_cast<const uint32_t *>(in.runs);
    auto count = [&](uint32_t *sh, int64_t *g, int len) {
        if (!g || len <= 0) return;
        if (len < RLH_BINS) atomicAdd(sh + len, 1u);
        else add_i64(g + len, 1);
    };
    for (int y = gwarp(); y < in.H; y += nwarps()) {
        const int a = in.row_ptr[y], b = in.row_ptr[y + 1];
        int carry = 0;  // end of the previous run of the line
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            int s = W, e = W;
            if (k < b) {
                const uint32_t r = runs[k];
                s = run_start(r);
                e = run_end(r);
            }
            int pe = __shfl_up_sync(0xFFFFFFFFu, e, 1);
            if (lane == 0) pe = carry;
            if (k < b) {
                count(hb, black, e - s);
                count(hw, white, s - pe);
            }
            carry = __shfl_sync(0xFFFFFFFFu, e, 31);
            if (k0 + 32 >= b) {
                // last chunk: the lane holding the line's last run closes it
                if (k == b - 1) count(hw, white, W - e);
            }
        }
        if (a == b && lane == 0) count(hw, white, W);
    }
    __syncthreads();
    const int nb = min(RLH_BINS, W + 1);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (black && hb[i]) add_i64(black + i, hb[i]);
        if (white && hw[i]) add_i64(white + i, hw[i]);
    }
}

int rows_grid(int H) {
    int g = (H + CC_WARPS - 1) / CC_WARPS;
    if (g > 152 * 8) g = 152 * 8;
    return g < 1 ? 1 : g;
}

}  // namespace

cudaError_t launch_rle_components(RleIn in, int conn, MorphCC c, int *status, cudaStream_t s) {
    const int d = conn == 8 ? 1 : 0;
    const int g = rows_grid(in.H);
    k_cc_init<<<152 * 4, CC_THREADS, 0, s>>>(in.row_ptr, in.H, c.labels);
    k_cc_link<<<g, CC_THREADS, 0, s>>>(in, d, c.labels, status);
    k_cc_flatten<<<g, CC_THREADS, 0, s>>>(in, c.labels, c.counts);
    const int64_t cap = c.stats ? c.max_components : INT64_MAX;
    launch_scan_rows(c.counts, in.H, c.rootptr, c.n_components, cap, status, s);
    k_cc_rank<<<g, CC_THREADS, 0, s>>>(in, c.labels, c.rootptr, c.rank, c.stats, c.max_components);
    k_cc_label<<<g, CC_THREADS, 0, s>>>(in, c.labels, c.rank, c.stats, c.max_components);
    return cudaGetLastError();
}

cudaError_t launch_run_length_hist(RleIn in, int64_t *black, int64_t *white, cudaStream_t s) {
    const size_t bytes = (size_t)(in.W + 1) * sizeof(int64_t);
    cudaError_t e;
    if (black && (e = cudaMemsetAsync(black, 0, bytes, s)) != cudaSuccess) return e;
    if (white && (e = cudaMemsetAsync(white, 0, bytes, s)) != cudaSuccess) return e;
    int g = (in.H + CC_WARPS - 1) / CC_WARPS;
    if (g > 152 * 4) g = 152 * 4;
    k_rl_hist<<<g < 1 ? 1 : g, CC_THREADS, 0, s>>>(in, black, white);
    return cudaGetLastError();
}

}  // namespace morph
