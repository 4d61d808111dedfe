// Register-only throughput probes for the integer roofline.
//
// The cell update of the inter-task kernel is pure integer ALU work (packed
// int16x2 DPX max/add plus one byte permute per cell pair).  NVIDIA does not
// publish the per-SM DPX issue rate of sm_103, so the roofline's denominator
// is measured here: every thread of a grid that exactly fills the GPU runs
// long chains of the instruction mix from registers (and, like the kernels,
// its profile words from shared memory), and the SM cycle counter (clock64)
// gives operations or cells per SM cycle.
//   mode 0: independent __viaddmax_s16x2 chains (raw DPX rate)
//   mode 1: the inter-task kernel's cell-pair sequence as it ships, at 32
//           rows per lane: in the biased unsigned domain, E' and X by
//           __viaddmax_u16x2, H by __vimax3_u16x2 with the zero floor, H - o
//           by a 32-bit subtract, F below by __viaddmax_u16x2, the profile
//           addend by one byte permute, and the running maximum by one
//           __vimax3_u16x2 per two rows; result: cell updates per SM cycle
//   mode 2: the same recurrence with four sequences in the bytes of a word
//           (unsigned saturating byte SIMD, the zero floor from saturation):
//           H - o, E' and F below by __vsubus4 and __vmaxu4, the diagonal by
//           __vaddus4 and __vsubus4 of a biased profile byte, H by two
//           __vmaxu4, the running maximum by one __vmaxu4 per row, and the
//           four sequences' profile bytes gathered by a 4x4 byte transpose
//           (eight permutes per four rows), at 16 rows per lane (three
//           registers per row); result: cell updates per SM cycle
#include "simd16.cuh"
#include "swdb_internal.cuh"

#ifndef PROBE2_ROWS
#define PROBE2_ROWS 32
#endif

namespace swdb {
namespace {

using simd16::pair_sel;

__device__ __forceinline__ uint32_t prmt_p(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__global__ void k_probe_dpx(int iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
    uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    uint32_t a4 = a0 * 11u, a5 = a0 * 13u, a6 = a0 * 17u, a7 = a0 * 19u;
    const uint32_t b = 0xfff5fff5u, c = seed * 0x9e3779b9u;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a0 = __viaddmax_s16x2(a0, b, c); a1 = __viaddmax_s16x2(a1, b, c);
            a2 = __viaddmax_s16x2(a2, b, c); a3 = __viaddmax_s16x2(a3, b, c);
            a4 = __viaddmax_s16x2(a4, b, c); a5 = __viaddmax_s16x2(a5, b, c);
            a6 = __viaddmax_s16x2(a6, b, c); a7 = __viaddmax_s16x2(a7, b, c);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
    const uint32_t r = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
    if (r == 0x12345678u) sink[0] = r;
}

// The shipped cell-pair sequence of k_inter_i16x2 (see k_inter16.cu) with R
// rows held in registers; the two sequences' int8 profile words come from
// shared memory as in the kernel.
template <int R>
__global__ void k_probe_cells(int iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
    __shared__ uint4 tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = make_uint4(seed * 3u + threadIdx.x, seed ^ (threadIdx.x * 77u),
                                                        seed + threadIdx.x * 5u, 0x7f7f0101u ^ threadIdx.x);
    uint32_t E[R], Ho[R];
    const uint32_t BNEG_O2 = 0x7ff67ff6u, ADD_NEG_E = 0xffffffffu, OO = 0x000a000au, BZERO2 = 0x80008000u;
#pragma unroll
    for (int r = 0; r < R; ++r) { E[r] = BNEG_O2 + r; Ho[r] = BNEG_O2 ^ (seed + r); }
    uint32_t hin = seed | 0x80008000u, fin = BNEG_O2, hd = BNEG_O2, mx = BZERO2;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        uint32_t wa[R / 4], wb[R / 4];
#pragma unroll
        for (int v = 0; v < R / 16; ++v) {
            const uint4 x = tab[(i + v) & 63];
            const uint4 y = tab[(i + v + 17) & 63];
            wa[4 * v + 0] = x.x; wa[4 * v + 1] = x.y; wa[4 * v + 2] = x.z; wa[4 * v + 3] = x.w;
            wb[4 * v + 0] = y.x; wb[4 * v + 1] = y.y; wb[4 * v + 2] = y.z; wb[4 * v + 3] = y.w;
        }
        uint32_t f = fin;
        uint32_t d = hd;
        uint32_t yprev = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t p = prmt_p(wa[r / 4], wb[r / 4], pair_sel(r % 4));
            const uint32_t e_r = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
            const uint32_t x = __viaddmax_u16x2(d, p, e_r);
            const uint32_t y = __vimax3_u16x2(f, x, BZERO2);
            const uint32_t ho = y - OO;
            f = __viaddmax_u16x2(f, ADD_NEG_E, ho);
            d = Ho[r];
            E[r] = e_r;
            Ho[r] = ho;
            if (r & 1) mx = __vimax3_u16x2(mx, yprev, y);
            yprev = y;
        }
        hd = hin;
        hin = Ho[R - 1];
        fin = f;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
    if (mx == 0x12345678u) sink[0] = mx;
}

// The shipped sequence with two columns per step: column j's row r and
// column j+1's row r are computed back to back, so two F chains (one per
// column) are in flight instead of one; column j+1 reads E and H - o of
// row r just after column j updated them, and its diagonal is column j's
// H - o of the row above.
template <int R>
__global__ void k_probe_cells2(int iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
    __shared__ uint4 tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = make_uint4(seed * 3u + threadIdx.x, seed ^ (threadIdx.x * 77u),
                                                        seed + threadIdx.x * 5u, 0x7f7f0101u ^ threadIdx.x);
    uint32_t E[R], Ho[R];
    const uint32_t BNEG_O2 = 0x7ff67ff6u, ADD_NEG_E = 0xffffffffu, OO = 0x000a000au, BZERO2 = 0x80008000u;
#pragma unroll
    for (int r = 0; r < R; ++r) { E[r] = BNEG_O2 + r; Ho[r] = BNEG_O2 ^ (seed + r); }
    uint32_t hin = seed | 0x80008000u, fin = BNEG_O2, hd = BNEG_O2, mx = BZERO2;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; i += 2) {
        uint32_t wa[R / 4], wb[R / 4], wc[R / 4], wd[R / 4];
#pragma unroll
        for (int v = 0; v < R / 16; ++v) {
            const uint4 x = tab[(i + v) & 63];
            const uint4 y = tab[(i + v + 17) & 63];
            const uint4 z = tab[(i + v + 29) & 63];
            const uint4 u = tab[(i + v + 41) & 63];
            wa[4 * v + 0] = x.x; wa[4 * v + 1] = x.y; wa[4 * v + 2] = x.z; wa[4 * v + 3] = x.w;
            wb[4 * v + 0] = y.x; wb[4 * v + 1] = y.y; wb[4 * v + 2] = y.z; wb[4 * v + 3] = y.w;
            wc[4 * v + 0] = z.x; wc[4 * v + 1] = z.y; wc[4 * v + 2] = z.z; wc[4 * v + 3] = z.w;
            wd[4 * v + 0] = u.x; wd[4 * v + 1] = u.y; wd[4 * v + 2] = u.z; wd[4 * v + 3] = u.w;
        }
        uint32_t f0 = fin, f1 = fin ^ 0x10001u;
        uint32_t d0 = hd, d1 = hin;
        uint32_t y0prev = 0, y1prev = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t p0 = prmt_p(wa[r / 4], wb[r / 4], pair_sel(r % 4));
            const uint32_t p1 = prmt_p(wc[r / 4], wd[r / 4], pair_sel(r % 4));
            // column j, row r
            const uint32_t e0 = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
            const uint32_t x0 = __viaddmax_u16x2(d0, p0, e0);
            const uint32_t y0 = __vimax3_u16x2(f0, x0, BZERO2);
            const uint32_t ho0 = y0 - OO;
            f0 = __viaddmax_u16x2(f0, ADD_NEG_E, ho0);
            d0 = Ho[r];
            // column j + 1, row r
            const uint32_t e1 = __viaddmax_u16x2(e0, ADD_NEG_E, ho0);
            const uint32_t x1 = __viaddmax_u16x2(d1, p1, e1);
            const uint32_t y1 = __vimax3_u16x2(f1, x1, BZERO2);
            const uint32_t ho1 = y1 - OO;
            f1 = __viaddmax_u16x2(f1, ADD_NEG_E, ho1);
            d1 = ho0;
            E[r] = e1;
            Ho[r] = ho1;
            if (r & 1) { mx = __vimax3_u16x2(mx, y0prev, y0); mx = __vimax3_u16x2(mx, y1prev, y1); }
            y0prev = y0;
            y1prev = y1;
        }
        hd = hin;
        hin = Ho[R - 1];
        fin = f0 ^ f1;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
    if (mx == 0x12345678u) sink[0] = mx;
}

// The recurrence in unsigned saturating byte SIMD: four database sequences
// per 32-bit word, R rows held in registers (H for the diagonal, H - o for
// the next column's E, and E).  Each sequence's profile row (four query rows
// of biased S + b per word) comes from shared memory; a 4x4 byte transpose
// turns four sequences' words into one word per query row.  Per row and
// column (four cells): H - o once, E' and F below (a saturating subtract and
// a max each), the diagonal (a saturating add and the bias subtract), H (two
// maxima), the running maximum, and two permutes of the transpose.
template <int R>
__global__ void k_probe_cells_u8x4(int iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
    __shared__ uint4 tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = make_uint4(seed * 3u + threadIdx.x, seed ^ (threadIdx.x * 77u),
                                                        seed + threadIdx.x * 5u, 0x07070101u ^ threadIdx.x);
    uint32_t E[R], H[R], Ho[R];
    const uint32_t O4 = 0x0a0a0a0au, E4 = 0x01010101u, B4 = 0x04040404u;
#pragma unroll
    for (int r = 0; r < R; ++r) { E[r] = 0; H[r] = (seed + r) & 0x0f0f0f0fu; Ho[r] = 0; }
    uint32_t hin = seed & 0x1f1f1f1fu, fin = 0, hd = 0, mx = 0;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        uint32_t f = fin;
        uint32_t d = hd;
        uint32_t ho_up = __vsubus4(hin, O4);
#pragma unroll
        for (int g = 0; g < R / 4; ++g) {
            // profile words of the four sequences for query rows 4g..4g+3
            const uint4 w = tab[(i + g) & 63];
            const uint32_t lo01 = prmt_p(w.x, w.y, 0x5140), hi01 = prmt_p(w.x, w.y, 0x7362);
            const uint32_t lo23 = prmt_p(w.z, w.w, 0x5140), hi23 = prmt_p(w.z, w.w, 0x7362);
            uint32_t pr[4];
            pr[0] = prmt_p(lo01, lo23, 0x5410);
            pr[1] = prmt_p(lo01, lo23, 0x7632);
            pr[2] = prmt_p(hi01, hi23, 0x5410);
            pr[3] = prmt_p(hi01, hi23, 0x7632);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = 4 * g + u;
                const uint32_t e_r = __vmaxu4(__vsubus4(E[r], E4), Ho[r]);
                f = __vmaxu4(__vsubus4(f, E4), ho_up);
                const uint32_t x = __vsubus4(__vaddus4(d, pr[u]), B4);
                const uint32_t h = __vmaxu4(__vmaxu4(x, e_r), f);
                mx = __vmaxu4(mx, h);
                d = H[r];
                E[r] = e_r;
                H[r] = h;
                ho_up = __vsubus4(h, O4);
                Ho[r] = ho_up;
            }
        }
        hd = hin;
        hin = H[R - 1] ^ i;
        fin = f;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
    if (mx == 0x12345678u) sink[0] = mx;
}

}  // namespace

cudaError_t launch_probe(int mode, int grid, int iters, unsigned long long *cycles, uint32_t *sink,
                         cudaStream_t s) {
    if (mode == 0) k_probe_dpx<<<grid, kCtaThreads, 0, s>>>(iters, 12345u, cycles, sink);
    else if (mode == 1) k_probe_cells<32><<<grid, kCtaThreads, 0, s>>>(iters, 12345u, cycles, sink);
    else if (mode == 2) k_probe_cells_u8x4<16><<<grid, kCtaThreads, 0, s>>>(iters, 12345u, cycles, sink);
    else k_probe_cells2<PROBE2_ROWS><<<grid, kCtaThreads, 0, s>>>(iters, 12345u, cycles, sink);
    return cudaGetLastError();
}

int probe_blocks_per_sm(int mode) {
    int n = 0;
    if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_dpx, kCtaThreads, 0);
    else if (mode == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_cells<32>, kCtaThreads, 0);
    else if (mode == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_cells_u8x4<16>, kCtaThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_cells2<PROBE2_ROWS>, kCtaThreads, 0);
    return n;
}

// Work per thread and loop iteration of each probe mode: DPX operations
// (mode 0) or cell updates (32 rows x 2 sequences; 16 rows x 4 sequences).
double probe_work_per_iteration(int mode) { return mode == 0 ? 64.0 : (mode == 3 ? 2.0 * PROBE2_ROWS : 64.0); }

}  // namespace swdb
