// Register-only throughput probes for the integer roofline.
//
// The cell update of the inter-task kernel is pure integer ALU work (packed
// int16x2 DPX max/add plus one byte permute per cell pair).  NVIDIA does not
// publish the per-SM DPX issue rate of sm_103, so the roofline's denominator
// is measured here: every thread of a grid that exactly fills the GPU runs
// long chains of the instruction mix from registers, and the SM cycle
// counter (clock64) gives operations per SM cycle.
//   mode 0: independent __viaddmax_s16x2 chains (raw DPX rate)
//   mode 1: the inter-task kernel's full cell-pair sequence (5 DPX ops,
//           1 byte permute, and the running max every second row) on
//           register data; the result is cell updates per SM cycle.
#include "swdb_internal.cuh"

namespace swdb {
namespace {

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

// The cell-pair sequence of k_inter_i16x2 with R rows held in registers.
template <int R>
__global__ void k_probe_cells(int iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
    uint32_t E[R], Ho[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { E[r] = 0xfff6fff6u + r; Ho[r] = 0xfff6fff6u ^ (seed + r); }
    const uint32_t NEG_O2 = 0xfff6fff6u, NEG_E2 = 0xffffffffu, MIN2 = 0x80008000u;
    uint32_t wa = seed * 0x9e3779b9u, wb = seed * 0x85ebca6bu;
    uint32_t hin = seed, fin = seed >> 1, hd = NEG_O2, mx = NEG_O2;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        uint32_t f = __viaddmax_s16x2(fin, NEG_E2, hin);
        uint32_t d = hd;
        uint32_t xo_prev = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t p = prmt_p(wa, wb, (r & 3) | (((r & 3) | 8) << 4) | ((4 + (r & 3)) << 8) |
                                                  (((4 + (r & 3)) | 8) << 12));
            const uint32_t e_r = __viaddmax_s16x2(E[r], NEG_E2, Ho[r]);
            const uint32_t x = __viaddmax_s16x2_relu(d, p, e_r);
            if (r > 0) f = __viaddmax_s16x2(f, NEG_E2, xo_prev);
            const uint32_t xo = __viaddmax_s16x2(x, NEG_O2, MIN2);
            const uint32_t ho = __viaddmax_s16x2(f, NEG_O2, xo);
            d = Ho[r];
            E[r] = e_r;
            Ho[r] = ho;
            xo_prev = xo;
        }
#pragma unroll
        for (int r = 0; r < R; r += 2) mx = __vimax3_s16x2(mx, Ho[r], Ho[r + 1]);
        hd = hin;
        hin = Ho[R - 1] ^ wa;
        fin = f;
        wa = wa * 1664525u + 1013904223u;
        wb ^= wa;
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
    else k_probe_cells<16><<<grid, kCtaThreads, 0, s>>>(iters, 12345u, cycles, sink);
    return cudaGetLastError();
}

int probe_blocks_per_sm(int mode) {
    int n = 0;
    if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_dpx, kCtaThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_cells<16>, kCtaThreads, 0);
    return n;
}

}  // namespace swdb
