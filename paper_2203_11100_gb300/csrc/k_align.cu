// Traceback of optimal local alignments for chosen (query, database
// sequence) pairs: the alignment behind a score of Section 2.2, read back
// from the Gotoh matrices (affine gaps as in Section 4.1) with the tie rules
// stated in swdb.h.
//
// int32 arithmetic.  A warp works on one 256-row strip at a time: lane k
// holds query rows 8k+1 .. 8k+8 of the strip and runs one column behind lane
// k-1 (a skewed wavefront: H and F of a lane's bottom row reach the next lane
// by shuffle).
//
// Forward pass (k_align_fwd, one CTA of 8 warps per pair): the strips run as
// a wavefront over the warps, each a few dozen columns behind the strip
// above.  The last lane of a strip writes its bottom row's H and F for every
// column (the strip's checkpoint row, the top boundary of the next strip);
// the warp below reads it once published.  The profile S(q_i, c) of each
// query is a global [code][row] table.  The maximum and the first cell in
// row-major order that holds it are kept per lane and reduced over the CTA.
//
// Traceback pass (k_align_bwd, one warp per pair; the strip's int32 profile
// [code][row] in shared memory): starting from the end cell's strip, the
// warp recomputes that strip's rows up to the current row and columns up to
// the current column from the checkpoint row above it, storing one flag byte
// per cell (which of the candidates H equals, whether E and F open at the
// cell); lane 0 then walks the path through the strip.  When the path
// leaves the strip at the top, the strip above is recomputed the same way.
// Every strip is recomputed at most once, so the traceback costs at most
// one more forward pass, and memory is ceil(m/256) checkpoint rows plus one
// strip of flags instead of m x n.
//
// The non-local modes (global, semi-global, overlap; SW# offers them besides
// local alignment, Section 2.3) run the same passes on their own matrices:
// the mode's first row and column (g(k) = o + (k-1) min(o, e) for a leading
// gap), no zero floor, and the end cell the first of the mode's candidates in
// row-major order (global (m, n); semi-global the last row; overlap the last
// column, then the last row) whose H is their maximum.  The walk has no stop
// at H = 0; on reaching the first row or column it emits the leading gap the
// mode prices there (global: both; semi-global: the first column) and stops.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/swdb.h"
#include "swdb_internal.cuh"

namespace swdb {
namespace {

constexpr int kAR = 8;                   // query rows per lane
constexpr int kStrip = 32 * kAR;         // rows per strip
constexpr int32_t kNegInf = -(1 << 29);  // -infinity of the recurrences
constexpr int kFW = 8;                   // warps per pair in the forward pass
constexpr int kPub = 32;                 // forward pass: columns per progress publication
constexpr long long kAlignSpin = 1ll << 25;   // x ~32 ns sleep: about a second

// flag bits of one cell (i, j)
constexpr uint8_t F_ZERO = 1;    // H(i,j) = 0
constexpr uint8_t F_DIAG = 2;    // H(i,j) = H(i-1,j-1) + S(q_i, t_j)
constexpr uint8_t F_HE = 4;      // H(i,j) = E(i,j)
constexpr uint8_t F_HF = 8;      // H(i,j) = F(i,j)
constexpr uint8_t F_EOPEN = 16;  // E(i,j) = H(i,j-1) - o
constexpr uint8_t F_FOPEN = 32;  // F(i,j) = H(i-1,j) - o

// Address of column 0 of sorted database sequence s in the bundle layout;
// column j0 is at base[(j0/4)*64 + (j0%4)*2].
__device__ __forceinline__ const uint8_t *target_base(const DbView &db, int64_t s) {
    const int64_t b = s / kBundleSeqs;
    const int slot = int((s % kBundleSeqs) >> 1);
    const int h = int(s & 1);
    return db.codes + db.bundle_off[b] + slot * kQuadBytes + h;
}

__device__ __forceinline__ int target_code(const uint8_t *base, int j0) {
    return base[int64_t(j0 >> 2) * kBundleRowBytes + (j0 & 3) * 2];
}

// Profile of rows r0 .. r0+255: prof[c][r] = S(q_{r0+r}, c), -inf past m or
// for codes outside the matrix.
__device__ __forceinline__ void load_profile(int32_t (*prof)[kStrip], const int32_t *mat, const uint8_t *q,
                                             int m, int r0, int lane) {
    for (int idx = lane; idx < kProfRows * kStrip; idx += 32) {
        const int c = idx / kStrip, r = idx % kStrip;
        int32_t v = kNegInf;
        if (r0 + r < m) {
            const int qc = q[r0 + r];
            if (qc < kProfRows) v = mat[qc * kProfRows + c];
        }
        prof[c][r] = v;
    }
}

__device__ __forceinline__ int32_t max3(int32_t a, int32_t b, int32_t c) { return __vimax3_s32(a, b, c); }

// Leading gap of k residues on the first row or column of a non-local mode.
__device__ __forceinline__ int32_t lead_gap(int k, int32_t o, int32_t e) {
    return k <= 0 ? 0 : o + (k - 1) * min(o, e);
}

// H(i, 0) and H(0, j) of the mode (local: 0).
__device__ __forceinline__ int32_t first_col(int mode, int i, int32_t o, int32_t e) {
    return (mode == SW_ALIGN_GLOBAL || mode == SW_ALIGN_SEMIGLOBAL) ? -lead_gap(i, o, e) : 0;
}
__device__ __forceinline__ int32_t first_row(int mode, int j, int32_t o, int32_t e) {
    return mode == SW_ALIGN_GLOBAL ? -lead_gap(j, o, e) : 0;
}

// Candidate end cell (1-based i <= m, j <= n) of a non-local mode.
__device__ __forceinline__ bool end_candidate(int mode, int i, int j, int m, int n) {
    if (mode == SW_ALIGN_GLOBAL) return i == m && j == n;
    if (mode == SW_ALIGN_SEMIGLOBAL) return i == m;
    return i == m || j == n;
}

__device__ __forceinline__ int ld_acquire_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" :: "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Forward pass, one CTA of kFW warps per pair.  Warp w takes strips w,
// w + kFW, ... in order.  Strip s reads the bottom row of strip s - 1 from
// its checkpoint row in global memory, column by column, once the warp that
// writes it has published the columns: pub[w] = strip * (n + 1) + columns
// written, monotonic over the warp's strips and released after the writes
// (every kPub columns and at the last column).  Every checkpoint row stays
// in memory, so a writer never waits for a reader, and strips run as a
// wavefront about kPub + 31 columns apart.  Each wait is bounded; when it
// runs out the pair's status records a timeout and the CTA stops waiting.
template <int MODE>
__global__ void __launch_bounds__(kFW * 32) k_align_fwd(const AlignArgs a) {
    __shared__ int pub[kFW];
    __shared__ int abort_flag;
    __shared__ int32_t red_best[kFW];
    __shared__ long long red_key[kFW];
    __shared__ int red_status[kFW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const AlignPairDev P = a.pairs[blockIdx.x];
    AlignResultDev *R = a.results + blockIdx.x;
    const int m = P.m, n = P.n;
    constexpr int mode = MODE;              // a.mode, fixed per instance: no mode tests per cell
    constexpr bool local = mode == SW_ALIGN_LOCAL;
    if (m <= 0 || n <= 0) {
        if (threadIdx.x == 0) {
            // only the first row or column: global ends at (m, n), semi-global
            // at (m, 0) (its first candidate when m = 0), overlap at (0, 0)
            AlignResultDev res{};
            if (mode == SW_ALIGN_GLOBAL || (mode == SW_ALIGN_SEMIGLOBAL && n == 0)) {
                res.i_end = max(m, 0);
                res.j_end = mode == SW_ALIGN_GLOBAL ? max(n, 0) : 0;
                res.score = -lead_gap(max(m, 0) + max(n, 0), a.gap_open, a.gap_extend);
            }
            *R = res;
        }
        return;
    }
    if (threadIdx.x < kFW) pub[threadIdx.x] = -1;
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    const int32_t *prof = a.prof + P.prof_off;        // [code][m_pad] = S(q_i, code)
    const uint8_t *tb = target_base(a.db, P.t_sorted);
    const int32_t o = a.gap_open, e = a.gap_extend;
    const int nstrips = (m + kStrip - 1) / kStrip;
    const int prevw = (warp + kFW - 1) % kFW;         // writes the strip above ours

    // best value and (i << 32) | j of its first cell in row-major order; the
    // non-local modes start from their boundary candidates: H(m, 0) for
    // semi-global, H(0, n) = 0 for overlap
    int32_t best = local ? 0 : INT32_MIN;
    int64_t bkey = INT64_MAX;
    if (mode == SW_ALIGN_SEMIGLOBAL) {
        best = first_col(mode, m, o, e);
        bkey = int64_t(m) << 32;
    } else if (mode == SW_ALIGN_OVERLAP) {
        best = 0;
        bkey = int64_t(n);
    }
    int status = 0;
    for (int strip = warp; strip < nstrips && status == 0; strip += kFW) {
        const int r0 = strip * kStrip;
        const int row0 = r0 + lane * kAR + 1;          // 1-based first row of this lane
        int32_t H[kAR], E[kAR];
#pragma unroll
        for (int r = 0; r < kAR; ++r) { H[r] = first_col(mode, row0 + r, o, e); E[r] = kNegInf; }
        int32_t hd = first_col(mode, row0 - 1, o, e), pub_h = 0, pub_f = kNegInf;
        const int2 *ck_in = strip > 0 ? a.ckpt + P.ckpt_off + int64_t(strip - 1) * (n + 1) : nullptr;
        int2 *ck_out = a.ckpt + P.ckpt_off + int64_t(strip) * (n + 1);
        const bool write_ck = r0 + kStrip < m;
        const int32_t *prow = prof + r0 + lane * kAR;
        const int need_base = (strip - 1) * (n + 1);
        int avail = 0;                                 // columns of ck_in known to be written
        if (write_ck && lane == 31) ck_out[0] = make_int2(first_col(mode, r0 + kStrip, o, e), kNegInf);
        for (int s = 0; s < n + 31; ++s) {
            if (strip > 0 && s + 1 <= n && s + 1 > avail) {   // warp-uniform
                const int want = min(s + kPub, n);
                bool ok = false;
                for (long long it = 0; it < kAlignSpin; ++it) {
                    if (ld_acquire_cta(&pub[prevw]) >= need_base + want) { ok = true; break; }
                    if (*reinterpret_cast<volatile int *>(&abort_flag)) break;
                    __nanosleep(32);
                }
                if (!ok) {
                    status = 5;                        // timeout (or another warp's)
                    if (lane == 0) *reinterpret_cast<volatile int *>(&abort_flag) = 1;
                    break;
                }
                avail = want;
            }
            int32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1);
            int32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1);
            const int j = s - lane + 1;                 // 1-based column
            if (j >= 1 && j <= n) {
                if (lane == 0) {
                    if (strip == 0) { hin = first_row(mode, j, o, e); fin = kNegInf; }
                    else { const int2 v = ck_in[j]; hin = v.x; fin = v.y; }
                }
                const int c = target_code(tb, j - 1);
                const int4 *pp = reinterpret_cast<const int4 *>(prow + int64_t(c) * P.m_pad);
                const int4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
                const int32_t sc[kAR] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                int32_t f = fin, up = hin, d = hd;
#pragma unroll
                for (int r = 0; r < kAR; ++r) {
                    const int32_t e_r = __viaddmax_s32(E[r], -e, H[r] - o);     // E(i,j)
                    f = __viaddmax_s32(f, -e, up - o);                           // F(i,j)
                    const int32_t h = max3(d + sc[r], e_r, local ? max(f, 0) : f);   // H(i,j)
                    d = H[r];
                    E[r] = e_r;
                    H[r] = h;
                    up = h;
                    const int i = row0 + r;
                    if (h >= best && i <= m && (local ? h > 0 : end_candidate(mode, i, j, m, n))) {
                        const int64_t key = (int64_t(i) << 32) | uint32_t(j);
                        if (h > best || key < bkey) { best = h; bkey = key; }
                    }
                }
                hd = hin;
                pub_h = H[kAR - 1];
                pub_f = f;
                if (write_ck && lane == 31) {
                    ck_out[j] = make_int2(H[kAR - 1], f);
                    if (j % kPub == 0 || j == n) st_release_cta(&pub[warp], strip * (n + 1) + j);
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const int32_t ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t ok = __shfl_xor_sync(0xffffffffu, bkey, off);
        if (ob > best || (ob == best && ok < bkey)) { best = ob; bkey = ok; }
    }
    if (lane == 0) {
        red_best[warp] = best;
        red_key[warp] = bkey;
        red_status[warp] = status;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int st = 0;
        for (int w = 0; w < kFW; ++w) {
            if (red_best[w] > best || (red_best[w] == best && red_key[w] < bkey)) { best = red_best[w]; bkey = red_key[w]; }
            st = max(st, red_status[w]);
        }
        AlignResultDev res{};
        res.score = best;
        if (best > 0 || !local) {
            res.i_end = int32_t(bkey >> 32);
            res.j_end = int32_t(bkey & 0xffffffff);
        }
        res.status = st;
        *R = res;
    }
}

template <int MODE>
__global__ void __launch_bounds__(32) k_align_bwd(const AlignArgs a) {
    __shared__ __align__(16) int32_t prof[kProfRows][kStrip];
    __shared__ int32_t mat[kProfRows * kProfRows];
    const int lane = threadIdx.x;
    const AlignPairDev P = a.pairs[blockIdx.x];
    AlignResultDev *R = a.results + blockIdx.x;
    for (int i = lane; i < kProfRows * kProfRows; i += 32) mat[i] = a.mat[i];
    const int m = P.m, n = P.n;
    constexpr int mode = MODE;              // a.mode, fixed per instance: no mode tests per cell
    constexpr bool local = mode == SW_ALIGN_LOCAL;
    if (local && (R->score <= 0 || m <= 0 || n <= 0)) return;   // empty alignment, written by the forward pass
    const uint8_t *q = a.queries + P.q_off;
    const uint8_t *tb = target_base(a.db, P.t_sorted);
    const int32_t o = a.gap_open, e = a.gap_extend;
    uint8_t *flags = a.flags + P.flags_off;          // [column j-1][row within the strip]
    uint8_t *rev = a.rev + P.rev_off;
    const int64_t max_ops = int64_t(m) + n;

    int i = R->i_end, j = R->j_end, state = 0;        // state 0 = H, 1 = E, 2 = F
    int64_t k = 0;
    int done = 0, status = 0;
    int64_t cells = 0;
    // State H on the first row or column of a non-local mode: the leading gap
    // the mode prices there (global: either; semi-global: the first column),
    // then stop.
    auto boundary = [&]() {
        if (i == 0 && mode == SW_ALIGN_GLOBAL)
            while (j > 0 && k < max_ops) { rev[k++] = SW_OP_D; --j; }
        if (j == 0 && (mode == SW_ALIGN_GLOBAL || mode == SW_ALIGN_SEMIGLOBAL))
            while (i > 0 && k < max_ops) { rev[k++] = SW_OP_I; --i; }
    };
    if (!local && (i == 0 || j == 0)) {               // end cell on the boundary (or an empty side)
        if (lane == 0) boundary();
        done = 1;
        i = __shfl_sync(0xffffffffu, i, 0);
        j = __shfl_sync(0xffffffffu, j, 0);
        k = __shfl_sync(0xffffffffu, k, 0);
    }
    while (!done) {
        if (i < 1) { status = 4; break; }             // not reached: a gap opens at row 1
        const int strip = (i - 1) / kStrip;
        const int r0 = strip * kStrip;
        const int cols = j;
        __syncwarp();
        load_profile(prof, mat, q, m, r0, lane);
        __syncwarp();
        const int row0 = r0 + lane * kAR + 1;
        int32_t H[kAR], E[kAR];
#pragma unroll
        for (int r = 0; r < kAR; ++r) { H[r] = first_col(mode, row0 + r, o, e); E[r] = kNegInf; }
        int32_t hd = first_col(mode, row0 - 1, o, e), pub_h = 0, pub_f = kNegInf;
        const int2 *ck_in = strip > 0 ? a.ckpt + P.ckpt_off + int64_t(strip - 1) * (n + 1) : nullptr;
        const bool lane_used = row0 <= i;             // rows below the path's row are never read
        for (int s = 0; s < cols + 31; ++s) {
            int32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1);
            int32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1);
            const int jj = s - lane + 1;
            if (jj >= 1 && jj <= cols && lane_used) {
                if (lane == 0) {
                    if (strip == 0) { hin = first_row(mode, jj, o, e); fin = kNegInf; }
                    else { const int2 v = ck_in[jj]; hin = v.x; fin = v.y; }
                }
                const int c = target_code(tb, jj - 1);
                const int4 p0 = *reinterpret_cast<const int4 *>(&prof[c][lane * kAR]);
                const int4 p1 = *reinterpret_cast<const int4 *>(&prof[c][lane * kAR + 4]);
                const int32_t sc[kAR] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                int32_t f = fin, up = hin, d = hd;
                uint32_t fl[2] = {0u, 0u};
#pragma unroll
                for (int r = 0; r < kAR; ++r) {
                    const int32_t hleft_o = H[r] - o;
                    const int32_t e_r = __viaddmax_s32(E[r], -e, hleft_o);
                    const int32_t up_o = up - o;
                    f = __viaddmax_s32(f, -e, up_o);
                    const int32_t diag = d + sc[r];
                    const int32_t h = max3(diag, e_r, local ? max(f, 0) : f);
                    uint32_t b = 0;
                    if (local && h == 0) b |= F_ZERO;
                    if (h == diag) b |= F_DIAG;
                    if (h == e_r) b |= F_HE;
                    if (h == f) b |= F_HF;
                    if (e_r == hleft_o) b |= F_EOPEN;
                    if (f == up_o) b |= F_FOPEN;
                    fl[r >> 2] |= b << (8 * (r & 3));
                    d = H[r];
                    E[r] = e_r;
                    H[r] = h;
                    up = h;
                }
                *reinterpret_cast<uint2 *>(flags + int64_t(jj - 1) * kStrip + lane * kAR) = make_uint2(fl[0], fl[1]);
                hd = hin;
                pub_h = H[kAR - 1];
                pub_f = f;
            }
        }
        cells += int64_t(min(i, m) - r0) * cols;
        __syncwarp();
        if (lane == 0) {
            // Walk the path through rows r0+1 .. i of this strip.
            for (;;) {
                if (k >= max_ops) { status = 1; done = 1; break; }
                if (state == 0) {
                    if (i == 0 || j == 0) {
                        if (!local) boundary();
                        done = 1;
                        break;
                    }
                    if (i <= r0) break;                // continue in the strip above
                    const uint8_t b = flags[int64_t(j - 1) * kStrip + (i - r0 - 1)];
                    if (b & F_ZERO) { done = 1; break; }
                    if (b & F_DIAG) { rev[k++] = SW_OP_M; --i; --j; }
                    else if (b & F_HE) state = 1;
                    else if (b & F_HF) state = 2;
                    else { status = 2; done = 1; break; }
                } else if (state == 1) {
                    if (j == 0) { status = 3; done = 1; break; }
                    const uint8_t b = flags[int64_t(j - 1) * kStrip + (i - r0 - 1)];
                    rev[k++] = SW_OP_D;
                    if (b & F_EOPEN) state = 0;
                    --j;
                } else {
                    if (i <= r0) break;                // continue in the strip above
                    const uint8_t b = flags[int64_t(j - 1) * kStrip + (i - r0 - 1)];
                    rev[k++] = SW_OP_I;
                    if (b & F_FOPEN) state = 0;
                    --i;
                }
            }
        }
        i = __shfl_sync(0xffffffffu, i, 0);
        j = __shfl_sync(0xffffffffu, j, 0);
        state = __shfl_sync(0xffffffffu, state, 0);
        k = __shfl_sync(0xffffffffu, k, 0);
        done = __shfl_sync(0xffffffffu, done, 0);
        status = __shfl_sync(0xffffffffu, status, 0);
    }
    __syncwarp();
    uint8_t *ops = a.ops + P.ops_off;
    for (int64_t x = lane; x < k; x += 32) ops[x] = rev[k - 1 - x];
    if (lane == 0) {
        R->i_begin = i;
        R->j_begin = j;
        R->n_ops = int32_t(k);
        R->status = status;
        R->cells = cells;
    }
}

}  // namespace

cudaError_t launch_align(const AlignArgs &a, int which, cudaStream_t s) {
    if (a.n_pairs <= 0) return cudaSuccess;
    if (a.n_pairs > 0x7fffffff) return cudaErrorInvalidValue;
    auto go = [&](auto mode_c) {
        constexpr int M = decltype(mode_c)::value;
        if (which == 0) k_align_fwd<M><<<unsigned(a.n_pairs), kFW * 32, 0, s>>>(a);
        else k_align_bwd<M><<<unsigned(a.n_pairs), 32, 0, s>>>(a);
    };
    switch (a.mode) {
        case SW_ALIGN_LOCAL: go(std::integral_constant<int, SW_ALIGN_LOCAL>()); break;
        case SW_ALIGN_GLOBAL: go(std::integral_constant<int, SW_ALIGN_GLOBAL>()); break;
        case SW_ALIGN_SEMIGLOBAL: go(std::integral_constant<int, SW_ALIGN_SEMIGLOBAL>()); break;
        case SW_ALIGN_OVERLAP: go(std::integral_constant<int, SW_ALIGN_OVERLAP>()); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int64_t align_checkpoint_rows(int32_t m) { return m <= 0 ? 0 : (int64_t(m) + kStrip - 1) / kStrip; }
int32_t align_strip_rows() { return kStrip; }

}  // namespace swdb
