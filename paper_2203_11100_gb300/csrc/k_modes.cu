// Global, semi-global and overlap scores of one query against the database:
// the non-local alignment modes (SW# offers them besides local, Section 2.3;
// the paper leaves other alignment operations to future work, Section 5).
// Same Gotoh recurrences as the local kernels (Section 2.2, affine gaps of
// Section 4.1) without the zero floor of H; the modes differ only in the
// first row and column and in the cells the score is read from:
//
//   global       H(i,0) = -g(i), H(0,j) = -g(j);  score H(m,n)
//   semi-global  H(i,0) = -g(i), H(0,j) = 0;     score max_j H(m,j)
//   overlap      H(i,0) = H(0,j) = 0;            score max(max_j H(m,j), max_i H(i,n))
//
// with g(k) = o + (k-1)*min(o,e), the first column's own recurrence from
// H(0,0) = 0.  Scores can be negative.  This kernel computes them in exact
// int32 (the host rejects inputs whose values could leave +-2^29) for the
// pairs the packed int16x2 kernel (k_modes16.cu) cannot take exactly (the
// longest sequences), or for every pair when int32 is requested.
//
// One warp per database sequence: lane k holds query rows 8k+1 .. 8k+8 of a
// 256-row strip and runs one column behind lane k-1 (H and F of a lane's
// bottom row reach the next lane by shuffle).  The query profile S(q_i, c) + o
// is a global [code][row] table (it stays in L1/L2); a lane reads its 8 rows
// for the current target code with two 16-byte loads.  Only the strip that
// holds row m picks out H(m, j) (a compile-time variant of the strip loop).  Between strips the
// bottom row (H, F per column) goes through this warp slot's scratch row in
// global memory (H - o of the strip's last row and F of the row below),
// rewritten in place: lane 31 writes column j - 30 while lane 0 prefetches
// column j + 2, so a column is always read before it is rewritten.
// Warps take (query, sequence) items from one atomic counter: the queries'
// entries one after another (the host orders them longest query first), each
// entry's sequences longest first, so the longest items start first and the
// queries' long sequences run side by side rather than one launch after another.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "../../include/swdb.h"
#include "swdb_internal.cuh"

namespace swdb {
namespace {

constexpr int kMR = 8;                   // query rows per lane
constexpr int kMStrip = 32 * kMR;        // rows per strip
constexpr int32_t kMNeg = -(1 << 30);    // -infinity of E and F

__device__ __forceinline__ int32_t lead_gap(int64_t k, int32_t o, int32_t gmin) {
    return k <= 0 ? 0 : int32_t(o + (k - 1) * int64_t(gmin));
}

// H(i, 0) of the mode
__device__ __forceinline__ int32_t col0(int mode, int64_t i, int32_t o, int32_t gmin) {
    return mode == SW_ALIGN_OVERLAP ? 0 : -lead_gap(i, o, gmin);
}

__global__ void __launch_bounds__(kCtaThreads) k_modes_i32(const __grid_constant__ ModeArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp_slot = blockIdx.x * (kCtaThreads / 32) + (threadIdx.x >> 5);
    int2 *bnd = a.boundary + int64_t(warp_slot) * (a.max_cols + 1);
    const int mode = a.mode;
    const int32_t o = a.gap_open, e = a.gap_extend, gmin = e < o ? e : o;

    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = int64_t(atomicAdd(a.work_counter, 1ull));
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        // the entry holding this item: the last with item_start <= item
        int lo = 0, hi = a.n_entries - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.entries[mid].item_start <= item) lo = mid;
            else hi = mid - 1;
        }
        const ModeEntry &en = a.entries[lo];
        const int64_t s = item - en.item_start;
        const int m = en.m;
        const int m_pad = en.m_pad;
        const int32_t *prof = a.prof + en.prof_off;
        int32_t *scores = a.scores + int64_t(en.query) * a.scores_stride;
        const int64_t orig = a.db.perm[s];
        if (orig < 0) continue;                              // padding slot of the last bundle
        const int n = a.db.len[s];
        if (m == 0 || n == 0) {
            if (lane == 0) {
                int32_t v = 0;
                if (mode == SW_ALIGN_GLOBAL) v = -lead_gap(m == 0 ? n : m, o, gmin);
                else if (mode == SW_ALIGN_SEMIGLOBAL) v = (n == 0) ? -lead_gap(m, o, gmin) : 0;
                scores[orig] = v;
            }
            continue;
        }
        // Lane 0 reads the codes 4 columns at a time (one 8-byte word holds 4
        // columns of this sequence and its pair partner), one word ahead of use;
        // the other lanes receive a column's code from the lane before them.
        const uint2 *cptr = reinterpret_cast<const uint2 *>(a.db.codes + a.db.bundle_off[s / kBundleSeqs]) +
                            int((s % kBundleSeqs) >> 1);
        const int hsh = int(s & 1);                           // byte of this sequence within a column pair
        int32_t last_row = kMNeg;      // max over j >= 1 of H(m, j) (the lane holding row m)
        int32_t last_col = kMNeg;      // max over rows <= m of H(i, n)
        int32_t hmn = kMNeg;           // H(m, n)
        auto strip = [&](const int r0, auto last_c) {
            constexpr bool LAST = decltype(last_c)::value;   // this strip holds row m
            __syncwarp();                                    // last strip's boundary writes are visible
            const int row0 = r0 + lane * kMR + 1;            // 1-based first row of this lane
            // Registers carry Ho = H - o (as the local kernels do): then E and
            // F are one add-max each, and the diagonal term is one add-max with
            // the profile S + o.
            int32_t Ho[kMR], E[kMR];
#pragma unroll
            for (int r = 0; r < kMR; ++r) {
                Ho[r] = col0(mode, row0 + r, o, gmin) - o;   // H(i, 0) - o
                E[r] = kMNeg;                                // E(i, 0)
            }
            int32_t hd = ((row0 - 1 == 0) ? 0 : col0(mode, row0 - 1, o, gmin)) - o;   // H(row0-1, 0) - o
            int32_t pub_h = 0, pub_f = kMNeg, pub_c = 0;
            uint2 quad = make_uint2(0, 0), quad_next = make_uint2(0, 0);
            int2 bn_next = make_int2(0, 0);                  // lane 0: boundary entry of its next column
            if (lane == 0) {
                quad_next = __ldg(cptr);
                if (r0 > 0) bn_next = bnd[1];
            }
            const bool more = r0 + kMStrip < m;
            const int rm = m - row0;                         // index of row m in this lane, if 0..7
            const int32_t *prow = prof + r0 + lane * kMR;
            // One column step.  STEADY: every lane inside its sequence and none at
            // the last column (31 <= st <= n - 2), so the range checks fold away.
            auto step = [&](const int st, auto steady_c) {
                constexpr bool STEADY = decltype(steady_c)::value;
                // from lane k-1: Ho of its bottom row at column j, F of our top row
                int32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1);
                int32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1);
                int cin = __shfl_up_sync(0xffffffffu, pub_c, 1);
                const int j = st - lane + 1;
                if (STEADY || (j >= 1 && j <= n)) {
                    if (lane == 0) {                         // column j = st + 1
                        const int u = st & 3;
                        if (u == 0) {
                            quad = quad_next;
                            if (st + 4 < n) quad_next = __ldg(cptr + ((st >> 2) + 1) * kBundlePairs);
                        }
                        const uint32_t w = (u & 2) ? quad.y : quad.x;
                        cin = int((w >> (8 * ((u & 1) * 2 + hsh))) & 0xffu);
                        if (r0 == 0) {                       // H(0, j) - o; F(1, j) = H(0, j) - o
                            hin = ((mode == SW_ALIGN_GLOBAL) ? -lead_gap(j, o, gmin) : 0) - o;
                            fin = hin;
                        } else {                             // H(r0, j) - o, F(r0+1, j)
                            hin = bn_next.x;
                            fin = bn_next.y;
                            if (j < n) bn_next = bnd[j + 1];
                        }
                    }
                    const int c = cin;
                    const int4 *pp = reinterpret_cast<const int4 *>(prow + int64_t(c) * m_pad);
                    int32_t sc[kMR];
#pragma unroll
                    for (int v = 0; v < kMR / 4; ++v) {
                        const int4 x4 = __ldg(pp + v);
                        sc[4 * v] = x4.x; sc[4 * v + 1] = x4.y; sc[4 * v + 2] = x4.z; sc[4 * v + 3] = x4.w;
                    }
                    int32_t f = fin, d = hd, hm = kMNeg;
#pragma unroll
                    for (int r = 0; r < kMR; ++r) {
                        const int32_t e_r = __viaddmax_s32(E[r], -e, Ho[r]);   // E(i,j)
                        const int32_t x = __viaddmax_s32(d, sc[r], e_r);       // max(H(i-1,j-1) + S, E(i,j))
                        const int32_t h = max(x, f);                            // H(i,j)
                        const int32_t ho = h - o;
                        f = __viaddmax_s32(f, -e, ho);                          // F(i+1,j)
                        d = Ho[r];
                        E[r] = e_r;
                        Ho[r] = ho;
                        if (LAST && r == rm) hm = h;
                    }
                    if (LAST) last_row = max(last_row, hm);
                    if (!STEADY && j == n) {
                        int32_t lc = kMNeg;
#pragma unroll
                        for (int r = 0; r < kMR; ++r)
                            if (row0 + r <= m) lc = max(lc, Ho[r] + o);
                        last_col = max(last_col, lc);
                        if (hm != kMNeg) hmn = hm;
                    }
                    hd = hin;
                    pub_h = Ho[kMR - 1];
                    pub_f = f;
                    pub_c = c;
                    if (more && lane == 31) bnd[j] = make_int2(Ho[kMR - 1], f);
                }
            };
            int st = 0;
            for (; st < 31 && st < n + 31; ++st) step(st, std::false_type());
            for (; st <= n - 2; ++st) step(st, std::true_type());
            for (; st < n + 31; ++st) step(st, std::false_type());
        };
        int r0 = 0;
        for (; r0 + kMStrip < m; r0 += kMStrip) strip(r0, std::false_type());
        strip(r0, std::true_type());
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            last_row = max(last_row, __shfl_xor_sync(0xffffffffu, last_row, off));
            last_col = max(last_col, __shfl_xor_sync(0xffffffffu, last_col, off));
            hmn = max(hmn, __shfl_xor_sync(0xffffffffu, hmn, off));
        }
        if (lane == 0) {
            int32_t v;
            if (mode == SW_ALIGN_GLOBAL) v = hmn;
            else if (mode == SW_ALIGN_SEMIGLOBAL) v = max(last_row, -lead_gap(m, o, gmin));   // j = 0 too
            else v = max(max(last_row, last_col), 0);          // H(m,0) = H(0,n) = 0
            scores[orig] = v;
        }
    }
}

}  // namespace

cudaError_t launch_modes_i32(const ModeArgs &a, int grid, cudaStream_t s) {
    if (a.n_items <= 0 || a.n_entries <= 0) return cudaSuccess;
    if (!a.entries || !a.work_counter || grid <= 0) return cudaErrorInvalidValue;
    const int64_t warps = kCtaThreads / 32;
    const int64_t need = (a.n_items + warps - 1) / warps;
    k_modes_i32<<<unsigned(std::min<int64_t>(grid, need)), kCtaThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int modes_slots(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_modes_i32, kCtaThreads, 0) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

int32_t modes_strip_rows() { return kMStrip; }

}  // namespace swdb
