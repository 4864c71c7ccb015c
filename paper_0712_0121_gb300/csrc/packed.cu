// Single-image launch of the fused packed tile (see packed_tile.cuh for the
// algorithm) and the host-side planner that picks the stage parameters and
// the tiling.
#include "packed_tile.cuh"

namespace morph {
namespace {

template <int NST, bool HS, int KMAX, int HALO, bool HX1>
__global__ void __launch_bounds__(MAX_THREADS) k_packed(const PackedArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    packed_tile<NST, HS, KMAX, HALO, HX1>(a, blockIdx.x, blockIdx.y, sm);
}

template <int NST, bool HS, int KMAX, int HALO, bool HX1 = false>
cudaError_t launch_t(const PackedArgs &a, cudaStream_t s) {
    const size_t smem = packed_smem_bytes(a);
    auto kern = k_packed<NST, HS, KMAX, HALO, HX1>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<packed_grid(a), packed_threads(a), smem, s>>>(a);
    return cudaGetLastError();
}

template <int NST, bool HS, int KMAX>
cudaError_t launch_h(const PackedArgs &a, cudaStream_t s) {
    if constexpr (!HS) {
        return launch_t<NST, HS, KMAX, 1>(a, s);
    } else {
        if (a.sw <= 3 && a.ex[0] <= 1 && a.sw - 1 - a.ex[0] <= 1) return launch_t<NST, HS, KMAX, 1, true>(a, s);
        switch (packed_halo(a.sw, a.ex[0])) {
        case 1: return launch_t<NST, HS, KMAX, 1>(a, s);
        case 2: return launch_t<NST, HS, KMAX, 2>(a, s);
        case 4: return launch_t<NST, HS, KMAX, 4>(a, s);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <int NST, bool HS>
cudaError_t launch_v(const PackedArgs &a, cudaStream_t s) {
    switch (packed_kmax(a)) {
    case 0: return launch_h<NST, HS, 0>(a, s);
    case 2: return launch_h<NST, HS, 2>(a, s);
    case 3: return launch_h<NST, HS, 3>(a, s);
    case 4: return launch_h<NST, HS, 4>(a, s);
    case 6: return launch_h<NST, HS, 6>(a, s);
    default: return launch_h<NST, HS, 16>(a, s);
    }
}

int bit_length(int v) {
    int k = 0;
    while (v) { ++k; v >>= 1; }
    return k;
}

}  // namespace

int packed_halo(int sw, int ex) {
    const int reach = ex > sw - 1 - ex ? ex : sw - 1 - ex;
    const int hw = (reach + 31) / 32;
    if (hw <= 1) return 1;
    if (hw <= 2) return 2;
    if (hw <= 4) return 4;
    return 0;  // wider than the register window supports
}

int packed_kmax(const PackedArgs &a) {
    if (a.sh == 1) return 0;
    if (a.sh == 3) return 2;  // two-row register window
    if (a.K <= 2) return 3;
    if (a.K <= 3) return 3;
    if (a.K <= 4) return 4;
    if (a.K <= 6) return 6;
    return 16;
}

size_t packed_smem_bytes(const PackedArgs &a) {
    if (!a.hmode) return 0;
    if (!a.ring) return (size_t)a.nst * 2 * a.rb * a.groups * a.slot_words * sizeof(uint32_t);
    // ring tile: PK_NBUF1 chunks of input rows, plus one chunk of first-stage
    // rows for open / close
    return (size_t)(PK_NBUF1 + (a.nst == 2 ? 1 : 0)) * pk1_rb(a.nwt) * a.groups * a.slot_words *
           sizeof(uint32_t);
}

int packed_threads(const PackedArgs &a) { return ((a.groups * a.tpr + 31) / 32) * 32; }

dim3 packed_grid(const PackedArgs &a) {
    return dim3((a.H + a.groups * a.band - 1) / (a.groups * a.band), a.nstrips);
}

// Fill the stage and tiling parameters.  Returns 0 on success, -1 if the
// rectangle is too wide for the horizontal register window.
int packed_plan(PackedArgs &a, int op, int sw, int sh, int ox, int oy, int band_hint,
                int threads_hint, int kmax_class, bool ring2) {
    const int rx = sw - 1 - ox, ry = sh - 1 - oy;
    a.sw = sw;
    a.sh = sh;
    switch (op) {
    case MORPH_ERODE: a.nst = 1; a.ex[0] = ox; a.ey[0] = oy; a.inv_in = 0; a.inv_out = 0; break;
    case MORPH_DILATE: a.nst = 1; a.ex[0] = rx; a.ey[0] = ry; a.inv_in = 1; a.inv_out = 1; break;
    case MORPH_OPEN:
        a.nst = 2; a.ex[0] = ox; a.ey[0] = oy; a.ex[1] = rx; a.ey[1] = ry;
        a.inv_in = 0; a.inv_out = 1; break;
    default:
        a.nst = 2; a.ex[0] = rx; a.ey[0] = ry; a.ex[1] = ox; a.ey[1] = oy;
        a.inv_in = 1; a.inv_out = 0; break;
    }
    if (a.nst == 1) { a.ex[1] = a.ex[0]; a.ey[1] = a.ey[0]; }
    a.K = bit_length(sh);
    for (int k = 0; k < 16; ++k) a.eqm[k] = ((sh >> k) & 1) ? 0u : ONES;
    a.hmode = sw == 1 ? 0 : 1;
    a.m = bit_length(sw) - 1;
    const int halo = packed_halo(sw, ox);
    if (halo == 0) return -1;

    int max_threads = threads_hint > 0 ? threads_hint : MAX_THREADS;
    if (max_threads > MAX_THREADS) max_threads = MAX_THREADS;
    if (max_threads < 32) max_threads = 32;
    // words per thread: the ring tile (sw > 1) picks 2 or 4 (see pk1_nwt),
    // the register-prefetch tile moves 2
    const bool one_stage = a.hmode != 0 && (a.nst == 1 || ring2);  // ring tile
    a.ring = one_stage;
    const bool hx1 = sw <= 3 && a.ex[0] <= 1 && sw - 1 - a.ex[0] <= 1;
    const int nwt = one_stage ? pk1_nwt(hx1, kmax_class >= 0 ? kmax_class : packed_kmax(a)) : PK_NWT;
    a.nwt = nwt;
    const int cover_threads = (a.nw_cover + nwt - 1) / nwt;
    if (cover_threads <= max_threads) {
        a.tpr = cover_threads;
        a.groups = max_threads / cover_threads;
        a.strip_words = a.nw_cover;
        a.halo_words = 0;
        a.nstrips = 1;
    } else {
        a.tpr = max_threads;
        a.groups = 1;
        a.halo_words = ((a.nst * halo + nwt - 1) / nwt) * nwt;
        a.strip_words = max_threads * nwt - 2 * a.halo_words;
        a.nstrips = (a.nw_cover + a.strip_words - 1) / a.strip_words;
    }
    a.rb = PK_RB;
    const int wup = a.nst * (sh - 1);
    int band = band_hint > 0 ? band_hint : 4 * wup;
    if (band < 64) band = 64;
    if (band_hint <= 0 && band > 1024) band = 1024;
    a.band = ((band + a.rb - 1) / a.rb) * a.rb;
    const int hcap = ((a.H + a.rb - 1) / a.rb) * a.rb;
    if (a.band > hcap) a.band = hcap;
    if (a.groups * a.band > hcap) {
        a.groups = (hcap + a.band - 1) / a.band;
        if (a.groups < 1) a.groups = 1;
    }
    a.slot_words = a.tpr * nwt + 2 * (one_stage ? pk1_pad(halo, nwt) : pk_pad(halo));
    // vector loads / stores of a thread's words: 16 bytes (one stage) or 8
    const int vb = nwt * 4;
    a.vec = ((uintptr_t)a.src % vb == 0) && ((uintptr_t)a.dst % vb == 0) && (a.sstride % nwt == 0) &&
            (a.dstride % nwt == 0);
    return 0;
}

cudaError_t launch_packed(PackedArgs &a, cudaStream_t s) {
    if (packed_halo(a.sw, a.ex[0]) == 0) return cudaErrorInvalidValue;
    if (a.nst == 1) return a.hmode ? launch_v<1, true>(a, s) : launch_v<1, false>(a, s);
    return a.hmode ? launch_v<2, true>(a, s) : launch_v<2, false>(a, s);
}

}  // namespace morph
