// Single-image launches of the run-length kernels (bodies in rle_tile.cuh):
// bitmap -> RLE (count, scan, write), RLE -> bitmap, and an RLE erosion or
// dilation (within-line run pass for se_h == 1, otherwise the between-line
// pass with the within-line pass fused into its input), each as count ->
// scan -> write.
#include "rle_tile.cuh"

namespace morph {
namespace {

__global__ void __launch_bounds__(256, 3) k_b2r_count(const uint32_t *src, int64_t sstride, int W,
                                                   int H, int32_t *counts) {
    for (int r0 = blockIdx.x * RLE_ROWS_PER_ITEM; r0 < H; r0 += gridDim.x * RLE_ROWS_PER_ITEM)
        b2r_count_rows(src, sstride, W, r0, min(H, r0 + RLE_ROWS_PER_ITEM), counts);
}

__global__ void __launch_bounds__(256, 3) k_b2r_write(const uint32_t *src, int64_t sstride, int W,
                                                   int H, const int32_t *row_ptr, int64_t capacity,
                                                   uint16_t *runs) {
    if ((int64_t)row_ptr[H] > capacity) return;
    for (int r0 = blockIdx.x * RLE_ROWS_PER_ITEM; r0 < H; r0 += gridDim.x * RLE_ROWS_PER_ITEM)
        b2r_write_rows<1>(src, sstride, W, r0, min(H, r0 + RLE_ROWS_PER_ITEM), row_ptr, runs);
}

__global__ void __launch_bounds__(1024) k_scan_rows(const int32_t *counts, int H, int32_t *row_ptr,
                                                    int64_t *n_runs, int64_t capacity, int *status) {
    scan_rows_block(counts, H, row_ptr, n_runs, capacity, status);
}

// Multi-CTA exclusive scan of the per-row counts for tall images, in three
// launches and without scratch memory: row_ptr[i0] of every segment of
// SCAN_SEG rows first holds the segment's sum, then (scanned in place) the
// segment's offset, from which each segment's CTA scans its own rows.
constexpr int SCAN_SEG = 4096;

__global__ void __launch_bounds__(1024) k_scan_seg_sums(const int32_t *counts, int H,
                                                        int32_t *row_ptr) {
    __shared__ int64_t wsum[32];
    const int i0 = blockIdx.x * SCAN_SEG, i1 = min(H, i0 + SCAN_SEG);
    int64_t loc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_SEG / 1024; ++j) {
        const int i = i0 + j * 1024 + threadIdx.x;
        if (i < i1) loc += counts[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) loc += __shfl_xor_sync(FULL_MASK, loc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        if (threadIdx.x == 0) row_ptr[i0] = (int32_t)v;
    }
}

__global__ void __launch_bounds__(1024) k_scan_seg_tops(int H, int nseg, int32_t *row_ptr,
                                                        int64_t *n_runs, int64_t capacity,
                                                        int *status) {
    const int64_t total = scan_block(row_ptr, SCAN_SEG, nseg, row_ptr, SCAN_SEG, 0);
    if (threadIdx.x == 0) {
        row_ptr[H] = (int32_t)total;
        if (n_runs) *n_runs = total;
        if (total > capacity) latch_status(status, MORPH_ECAPACITY);
    }
}

__global__ void __launch_bounds__(1024) k_scan_seg_rows(const int32_t *counts, int H,
                                                        int32_t *row_ptr) {
    const int i0 = blockIdx.x * SCAN_SEG;
    const int64_t off = row_ptr[i0];  // read by every thread before the scan's first write
    scan_block(counts + i0, 1, min(SCAN_SEG, H - i0), row_ptr + i0, 1, off);
}

__global__ void __launch_bounds__(256) k_r2b(RleIn in, uint32_t *dst, int64_t dstride, int nw_cover) {
    extern __shared__ __align__(16) uint32_t sm[];
    for (int r0 = blockIdx.x * RLE_ROWS_PER_ITEM; r0 < in.H; r0 += gridDim.x * RLE_ROWS_PER_ITEM)
        r2b_rows(in, dst, dstride, nw_cover, r0, min(in.H, r0 + RLE_ROWS_PER_ITEM), sm);
}

__global__ void __launch_bounds__(256) k_rowpass(RleIn in, RowOp op, int write, int32_t *counts,
                                                 const int32_t *out_row_ptr, int64_t capacity,
                                                 uint16_t *out) {
    if (write && (int64_t)out_row_ptr[in.H] > capacity) return;
    for (int r0 = blockIdx.x * RLE_ROWS_PER_ITEM; r0 < in.H; r0 += gridDim.x * RLE_ROWS_PER_ITEM)
        rowpass_rows(in, op, write, counts, out_row_ptr, out, r0, min(in.H, r0 + RLE_ROWS_PER_ITEM));
}

template <int KMAX>
__global__ void __launch_bounds__(MAX_THREADS) k_vband(const VArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    vband_tile<2, KMAX>(a, blockIdx.x, sm);
}

template <int NWT, int KMAX>
__global__ void __launch_bounds__(MAX_THREADS) k_vpass(const VArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    if (a.write && (int64_t)a.out_row_ptr[a.in.H] > a.capacity) return;
    vpass_tile<NWT, KMAX>(a, blockIdx.x, sm);
}

int bit_length(int v) {
    int k = 0;
    while (v) { ++k; v >>= 1; }
    return k;
}

int row_items(int H) {
    int n = (H + RLE_ROWS_PER_ITEM - 1) / RLE_ROWS_PER_ITEM;
    if (n > 152 * 16) n = 152 * 16;
    return n < 1 ? 1 : n;
}


template <int NWT, int KMAX>
cudaError_t launch_vt(const VArgs &a, cudaStream_t s) {
    const size_t smem = vpass_smem_bytes(a);
    auto kern = k_vpass<NWT, KMAX>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<vpass_grid(a), vpass_threads(a), smem, s>>>(a);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_bt(const VArgs &a, cudaStream_t s) {
    const size_t smem = vband_smem_bytes(a);
    auto kern = k_vband<KMAX>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<vband_grid(a), vpass_threads(a), smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_band(const VArgs &a, cudaStream_t s) {
    switch (vpass_kmax(a.sh)) {
    case 2: return launch_bt<2>(a, s);
    case 3: return launch_bt<3>(a, s);
    case 6: return launch_bt<6>(a, s);
    default: return launch_bt<16>(a, s);
    }
}

template <int NWT>
cudaError_t launch_vk(const VArgs &a, cudaStream_t s) {
    switch (vpass_kmax(a.sh)) {
    case 2: return launch_vt<NWT, 2>(a, s);
    case 3: return launch_vt<NWT, 3>(a, s);
    case 6: return launch_vt<NWT, 6>(a, s);
    default: return launch_vt<NWT, 16>(a, s);
    }
}

}  // namespace

// counts[0..H) -> row_ptr[0..H], *n_runs, capacity check (see scan_rows_block)
void launch_scan_rows(const int32_t *counts, int H, int32_t *row_ptr, int64_t *n_runs,
                      int64_t capacity, int *status, cudaStream_t s) {
    if (H <= 2 * SCAN_SEG) {
        k_scan_rows<<<1, 1024, 0, s>>>(counts, H, row_ptr, n_runs, capacity, status);
        return;
    }
    const int nseg = (H + SCAN_SEG - 1) / SCAN_SEG;
    k_scan_seg_sums<<<nseg, 1024, 0, s>>>(counts, H, row_ptr);
    k_scan_seg_tops<<<1, 1024, 0, s>>>(H, nseg, row_ptr, n_runs, capacity, status);
    k_scan_seg_rows<<<nseg, 1024, 0, s>>>(counts, H, row_ptr);
}

int vpass_kmax(int sh) {
    const int K = bit_length(sh);
    return sh == 3 ? 2 : (K <= 3 ? 3 : (K <= 6 ? 6 : 16));
}

void vpass_plan(VArgs &a, int W, int H, int sh) {
    a.nw_ext = (W >> 5) + 1;
    a.nwt = a.nw_ext <= 2 * MAX_THREADS ? 2 : 8;
    a.tpr = (a.nw_ext + a.nwt - 1) / a.nwt;
    a.groups = MAX_THREADS / a.tpr;
    if (a.groups < 1) a.groups = 1;
    a.rb = a.nwt == 2 ? 8 : 4;
    int band = 8 * (sh - 1);
    if (band < 64) band = 64;
    if (band > 1024) band = 1024;
    a.band = band;
    if (a.groups * a.band > H) {
        a.groups = (H + a.band - 1) / a.band;
        if (a.groups < 1) a.groups = 1;
    }
    a.slot_words = a.tpr * a.nwt;
}

bool vband_plan(VArgs &a, int W, int H, int sh, size_t budget) {
    a.nw_ext = (W >> 5) + 1;
    a.nwt = 2;
    a.tpr = (a.nw_ext + 1) / 2;
    if (a.tpr > MAX_THREADS) return false;
    a.slot_words = a.tpr * 2;
    a.rb = 0;
    // tile rows + one row offset per row, and the run staging buffer
    const size_t fixed = 64 + (size_t)2 * VBAND_RUN_CHUNK * 4 + 8;
    const size_t row_bytes = (size_t)a.slot_words * 4 + 4;
    if (budget < fixed + row_bytes) return false;
    const long rmax = (long)((budget - fixed) / row_bytes);
    int G = MAX_THREADS / a.tpr;
    long S = 0;
    for (; G >= 1; --G) {
        S = (rmax - (sh - 1)) / G;
        const long want = sh - 1 > 16 ? sh - 1 : 16;  // warm-up at most as long as the segment
        if (S >= want || G == 1) break;
    }
    if (S < 1) return false;
    // no more rows per tile than the image needs
    const long per = (H + G - 1) / G;
    if (S > per) S = per;
    a.groups = G;
    a.band = (int)S;
    return true;
}

// T[R][slot_words] | row offsets int[R + 1] (padded to 16 bytes) | runs uint32[2][CHUNK]
size_t vband_smem_bytes(const VArgs &a) {
    const size_t R = (size_t)a.groups * a.band + a.sh - 1;
    const size_t off = ((R * a.slot_words + R + 1) * 4 + 15) & ~(size_t)15;
    return off + (size_t)2 * VBAND_RUN_CHUNK * 4;
}

int vband_grid(const VArgs &a) { return (a.in.H + a.groups * a.band - 1) / (a.groups * a.band); }

size_t vpass_smem_bytes(const VArgs &a) {
    const size_t nslot = (size_t)a.rb * a.groups;
    return 2 * nslot * a.slot_words * sizeof(uint32_t) + (2 * nslot + 2) * sizeof(int);
}
int vpass_threads(const VArgs &a) { return ((a.groups * a.tpr + 31) / 32) * 32; }
int vpass_grid(const VArgs &a) { return (a.in.H + a.groups * a.band - 1) / (a.groups * a.band); }

cudaError_t launch_rle_from_bitmap(const uint32_t *src, int64_t sstride, int W, int H, RleOut out,
                                   int32_t *counts, int *status, cudaStream_t s) {
    const int grid = row_items(H);
    k_b2r_count<<<grid, 256, 0, s>>>(src, sstride, W, H, counts);
    launch_scan_rows(counts, H, out.row_ptr, out.n_runs, out.capacity, status, s);
    k_b2r_write<<<grid, 256, 0, s>>>(src, sstride, W, H, out.row_ptr, out.capacity, out.runs);
    return cudaGetLastError();
}

cudaError_t launch_rle_to_bitmap(RleIn in, uint32_t *dst, int64_t dstride, int nw_cover,
                                 cudaStream_t s) {
    const size_t smem = (size_t)8 * nw_cover * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_r2b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_r2b<<<row_items(in.H), 256, smem, s>>>(in, dst, dstride, nw_cover);
    return cudaGetLastError();
}

cudaError_t launch_rle_rect(RleIn in, RleOut out, int dilate, int sw, int sh, int ox, int oy,
                            int32_t *counts, uint32_t *bmp_scratch, int *status, cudaStream_t s) {
    RowOp op;
    op.dilate = dilate;
    op.sw = sw;
    op.o = ox;
    op.W = in.W;
    if (sh == 1) {
        const int grid = row_items(in.H);
        k_rowpass<<<grid, 256, 0, s>>>(in, op, 0, counts, nullptr, 0, nullptr);
        launch_scan_rows(counts, in.H, out.row_ptr, out.n_runs, out.capacity, status, s);
        k_rowpass<<<grid, 256, 0, s>>>(in, op, 1, nullptr, out.row_ptr, out.capacity, out.runs);
        return cudaGetLastError();
    }
    VArgs a;
    a.in = in;
    a.op = op;
    a.inv = dilate;
    a.sh = sh;
    a.ey = dilate ? sh - 1 - oy : oy;
    a.K = bit_length(sh);
    for (int k = 0; k < 16; ++k) a.eqm[k] = ((sh >> k) & 1) ? 0u : ONES;
    vpass_plan(a, in.W, in.H, sh);
    a.counts = counts;
    a.bmp = nullptr;
    a.bmp_stride = 0;
    a.bmp_words = 0;
    a.write = 0;
    if (bmp_scratch) {
        // one between-line pass storing the rows as bitmap words; then the
        // run counts of the stored rows, the prefix sum, and their encode
        const int nwv = (in.W + 31) / 32;
        a.bmp = bmp_scratch;
        a.bmp_stride = nwv;
        a.bmp_words = nwv;
        a.counts = nullptr;
        VArgs b = a;
        cudaError_t e;
        if (vband_plan(b, in.W, in.H, sh, VBAND_SMEM_BUDGET)) e = launch_band(b, s);
        else e = a.nwt == 2 ? launch_vk<2>(a, s) : launch_vk<8>(a, s);
        if (e != cudaSuccess) return e;
        k_b2r_count<<<row_items(in.H), 256, 0, s>>>(bmp_scratch, nwv, in.W, in.H, counts);
        launch_scan_rows(counts, in.H, out.row_ptr, out.n_runs, out.capacity, status, s);
        k_b2r_write<<<row_items(in.H), 256, 0, s>>>(bmp_scratch, nwv, in.W, in.H, out.row_ptr,
                                                     out.capacity, out.runs);
        return cudaGetLastError();
    }
    a.out_row_ptr = out.row_ptr;
    a.capacity = out.capacity;
    a.out = out.runs;
    cudaError_t e = a.nwt == 2 ? launch_vk<2>(a, s) : launch_vk<8>(a, s);
    if (e != cudaSuccess) return e;
    launch_scan_rows(counts, in.H, out.row_ptr, out.n_runs, out.capacity, status, s);
    a.write = 1;
    return a.nwt == 2 ? launch_vk<2>(a, s) : launch_vk<8>(a, s);
}

}  // namespace morph
