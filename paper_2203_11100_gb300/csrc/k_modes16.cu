// Global, semi-global and overlap scores in packed int16x2 DPX arithmetic.
//
// The modes are those of k_modes.cu (SW# offers global and semi-global
// alignment besides local, Section 2.3; the paper leaves other alignment
// operations to future work, Section 5): the Gotoh recurrences of Section 2.2
// without the zero floor of H, differing in the first row and column and in
// the cells the score is read from.  This kernel gives them the inter-task
// organisation of the local int16x2 kernel (Section 2.2; SW#db's kernel for
// short database sequences, Section 3.2):
//
// * A subwarp of T lanes scores one pair of database sequences, one in each
//   int16 half; lane k owns R query rows of a T*R-row strip and runs one
//   column behind lane k-1.  The int8 profile S + o of the strip sits in
//   shared memory; one byte permute per cell pair builds the packed addend.
// * Values are held in offset binary, B(v) = v + 32768 per half, so unsigned
//   DPX add-max orders them, adding a negative constant is a modular add and
//   subtracting o is a plain 32-bit subtraction.  Per cell pair:
//       E' = max(E - e, Ho_left)             viaddmax
//       X  = max(Ho_diag + S + o, E')        viaddmax
//       H  = max(F, X)                       vimax3 (no zero floor)
//       Ho = H - o                           32-bit subtract
//       F_below = max(F - e, Ho)             viaddmax
// * Exactness is decided on the host, not checked here: every H lies
//   between H(i, 0) - g(j) (the E chain along row i alone, whatever the
//   profile) and max(S, 0) * min(m, n) (each diagonal step adds at most
//   max(S); every boundary value is <= 0), so the host sends a pair here only
//   when both bounds, widened by the largest addend, fit int16.  The other
//   pairs (the longest) go to the int32 kernel.
// * The query is padded at the TOP with P virtual rows so that m + P fills
//   whole strips, the last of which may be short (8, 16 or 24 rows per lane
//   instead of R: the fewest that cover the rest), and row m is always the
//   last row of the last lane: the last-row maximum and H(m, n) then read one
//   fixed register.  The virtual
//   rows reproduce the mode's first row exactly:
//     semi-global, overlap: S = 0 and H(v, 0) = 0 give H(v, j) = 0 and
//                           F(P + 1, j) = -o, as below a first row of zeros;
//     global:               S = -min(o, e), H(v, 0) = -(o - min(o, e)) and
//                           H(P, 0) = 0 give H(v, j) = -g(j) for j >= 1, the
//                           global first row, with H(P, 0) = H(0, 0) as the
//                           first real row's diagonal.
//   Here g(k) = o + (k - 1) min(o, e), the cost of a leading gap of k.
//   E(i, 0) is set to H(i, 0) - o, which stands in for minus infinity
//   (E(i, 1) = max(E(i, 0) - e, H(i, 0) - o) = H(i, 0) - o).
// * Scores: global reads H(m, n) of each half at its own column n; semi-
//   global keeps the maximum of H(m, j) over j <= n (columns past a half's
//   own length are masked off); overlap adds the maximum of H(i, n) over the
//   rows, taken at column n by every lane.
// * Persistent grid: resident CTAs pull chunks of 256/T pairs (longest
//   first) from an atomic counter; each subwarp keeps its strip-boundary row
//   in its CTA slot's scratch, reused chunk after chunk.
#include <algorithm>
#include <type_traits>

#include "../../include/swdb.h"
#include "simd16.cuh"
#include "swdb_internal.cuh"

namespace swdb {
namespace {

using simd16::cp_async16;
using simd16::cp_async_commit;
using simd16::cp_async_wait1;
using simd16::pack2;
using simd16::pair_sel;
using simd16::prmt;

// Per-half unsigned max of two packed words (the three-input DPX max with a
// repeated operand: one instruction).
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) { return __vimax3_u16x2(a, b, b); }

template <int T, int R, int MODE>
__global__ void __launch_bounds__(kCtaThreads, (R <= 16 ? 3 : 2)) k_modes_i16x2(const __grid_constant__ Mode16Args a) {
    static_assert(R % 8 == 0, "rows per lane must be a multiple of 8");
    static_assert(32 % T == 0 && T >= 4, "lanes must divide the warp");
    constexpr bool GLOBAL = MODE == SW_ALIGN_GLOBAL;
    constexpr bool OVERLAP = MODE == SW_ALIGN_OVERLAP;
    constexpr int PAIRS_PER_CTA = kCtaThreads / T;
    constexpr int TR = T * R;
    constexpr int H16 = (R + 15) / 16;                // 16-row groups per lane (the last may hold 8)
    constexpr int SLOT = T * 16 * H16;                // profile bytes per residue
    constexpr int PROF_BYTES = kProfRows * SLOT;

    __shared__ __align__(16) int8_t prof[PROF_BYTES];
    __shared__ int8_t mat[kProfRows * kProfRows];
    __shared__ __align__(16) uint2 bstage[PAIRS_PER_CTA][8];
    __shared__ int sh_chunk;

    const int tid = threadIdx.x;
    const int k = tid % T;               // lane within the subwarp
    const int sub = tid / T;             // subwarp within the CTA
    // staged transposed, [db code][query code]: the profile fill reads one db code
    // against many query codes at once, which then fall in distinct banks
    for (int i = tid; i < kProfRows * kProfRows; i += kCtaThreads)
        mat[(i % kProfRows) * kProfRows + i / kProfRows] = (&a.prof8[0][0])[i];
    const int n_chunks = int((a.pair_end - a.pair_begin + PAIRS_PER_CTA - 1) / PAIRS_PER_CTA);
    const int o = a.gap_open;
    const int gmin = min(a.gap_open, a.gap_extend);
    const int P = a.virt_rows;
    const int npass = (a.m + P + TR - 1) / TR;
    const int rest = a.m + P - (npass - 1) * TR;     // rows of the last strip: T x 8, 16, 24 or R
    const int g_m = o + (a.m - 1) * gmin;             // g(m), m >= 1

    // H(i, 0) of padded row i (row 0 is the strip above the first virtual row)
    auto col0 = [&](int i) -> int {
        const int ir = i - P;
        if (ir >= 1) return OVERLAP ? 0 : -(o + (ir - 1) * gmin);
        if (ir == 0) return 0;
        return GLOBAL ? -(o - gmin) : 0;
    };

    for (;;) {
        __syncthreads();                 // the previous chunk is done with shared state
        if (tid == 0) sh_chunk = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        const int chunk = sh_chunk;
        if (chunk >= n_chunks) break;
        const int64_t pair0 = a.pair_begin + int64_t(chunk) * PAIRS_PER_CTA + sub;
        const bool valid = pair0 < a.pair_end;
        int na = 0, nb = 0;              // lengths of the two halves (na >= nb: sorted, longest first)
        const uint2 *cptr = nullptr;
        uint4 *bnd = nullptr;
        if (valid) {
            na = a.db.len[2 * pair0];
            nb = a.db.len[2 * pair0 + 1];
            const int64_t b = pair0 / kBundlePairs;
            cptr = reinterpret_cast<const uint2 *>(a.db.codes + a.db.bundle_off[b]) + int(pair0 % kBundlePairs);
            if (a.boundary)
                bnd = reinterpret_cast<uint4 *>(a.boundary + int64_t(blockIdx.x) * a.slot_stride +
                                                int64_t(sub) * a.max_cols);
        }
        const int Lp = (na + 3) & ~3;
        const int Lw = __reduce_max_sync(0xffffffffu, Lp);   // warp-uniform column count
        const int Lmin = __reduce_min_sync(0xffffffffu, Lp);

        const uint32_t ADD_NEG_E = pack2(-a.gap_extend);      // modular addend "- e"
        const uint32_t OO = uint32_t(o) | (uint32_t(o) << 16);
        // GLOBAL: B(H(m, n)) of each half, captured at its column n.  Otherwise the
        // running maximum of B(H(m, j)), from j = 0: H(m, 0) = -g(m) (semi-global), 0 (overlap).
        uint32_t res = GLOBAL ? 0u : pack2(32768 + (OVERLAP ? 0 : -g_m));
        uint32_t mcol = 0;               // OVERLAP: maximum of B(H(i, n)) over this lane's rows

        // One pass (strip): padded rows pass*TR .. pass*TR + T*RP - 1, RP rows per
        // lane (RP = R but in the last pass, which may be shorter).
        auto run_pass = [&](const int pass, auto last_c, auto rp_c) {
            constexpr bool LAST = decltype(last_c)::value;
            constexpr int RP = decltype(rp_c)::value;
            constexpr int TRP = T * RP;
            __syncthreads();
            // Profile of padded rows pass*TR .. pass*TR+TRP-1, layout [residue][16-row
            // group][lane][16 rows] as in the local kernel; virtual rows (above the
            // query) score S = 0 (semi-global, overlap) or -min(o, e) (global).
            const int pv = GLOBAL ? (o - gmin) : o;
            for (int w = tid; w < kProfRows * TRP / 4; w += kCtaThreads) {
                const int e0 = w * 4;
                const int res_code = e0 / TRP;
                const int within = e0 % TRP;
                const int row0 = pass * TR + within - P;     // query row of the first of the 4
                const int kk = within / RP, rr = within % RP;
                const int phys = res_code * SLOT + (rr >> 4) * (T * 16) + kk * 16 + (rr & 15);
                uint32_t word = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = row0 + c;
                    int v = pv;
                    if (row >= 0) {
                        v = -128;
                        if (row < a.m) {
                            // device-resident queries are not validated on the host:
                            // codes outside the table score as padding
                            const int qc = a.query[row];
                            if (qc < kProfRows) v = mat[res_code * kProfRows + qc];
                        }
                    }
                    word |= (uint32_t(uint8_t(int8_t(v)))) << (8 * c);
                }
                reinterpret_cast<uint32_t *>(prof)[phys / 4] = word;
            }
            __syncthreads();
            if (Lw == 0) return;

            const int i0 = pass * TR + k * RP;            // padded row above this lane's first row
            uint32_t E[RP], Ho[RP];
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                Ho[r] = pack2(32768 + col0(i0 + r + 1) - o);
                E[r] = Ho[r];
            }
            uint32_t hd = pack2(32768 + col0(i0) - o);   // B(Ho(top - 1, j - 1))
            uint32_t pub_h = hd, pub_f = hd, pub_c = 0;
            // lane 0, first pass: B(H(0, j) - o) of the column about to start
            uint32_t top = GLOBAL ? pack2(32768 + gmin - 2 * o) : pack2(32768 - o);
            const uint32_t GM2 = pack2(gmin);
            const int steps = Lw + T - 1;
            uint2 quad = make_uint2(0, 0), quad_next = make_uint2(0, 0);
            uint2 *stg = bstage[sub];
            constexpr int gstride = 2;                    // uint4 per 4-column group of the slot scratch
            if (Lp > 0) quad_next = __ldg(cptr);          // every lane of the subwarp: one broadcast load
            if (k == 0 && Lp > 0 && pass > 0) {
                cp_async16(stg + 0, bnd);
                cp_async16(stg + 2, bnd + 1);
                cp_async_commit();
                if (4 < Lp) {
                    cp_async16(stg + 4, bnd + gstride);
                    cp_async16(stg + 6, bnd + gstride + 1);
                }
                cp_async_commit();
            }

            // The cell work of column j (0-based) for this lane's RP rows, with the
            // mode's bookkeeping of the last row and of column n.
            auto cells = [&](const int j, const uint32_t hin, const uint32_t fin, const uint32_t cin) {
                const int ta = int(cin & 0xffu), tb = int((cin >> 8) & 0xffu);
                const uint4 *pa = reinterpret_cast<const uint4 *>(prof + ta * SLOT + k * 16);
                const uint4 *pb = reinterpret_cast<const uint4 *>(prof + tb * SLOT + k * 16);
                uint32_t wa[RP / 4], wb[RP / 4];
#pragma unroll
                for (int v = 0; v < RP / 16; ++v) {
                    const uint4 x = pa[v * T];
                    const uint4 y = pb[v * T];
                    wa[4 * v + 0] = x.x; wa[4 * v + 1] = x.y; wa[4 * v + 2] = x.z; wa[4 * v + 3] = x.w;
                    wb[4 * v + 0] = y.x; wb[4 * v + 1] = y.y; wb[4 * v + 2] = y.z; wb[4 * v + 3] = y.w;
                }
                if (RP % 16) {                            // last group of 8 rows: an 8-byte load
                    const uint2 x = *reinterpret_cast<const uint2 *>(pa + (RP / 16) * T);
                    const uint2 y = *reinterpret_cast<const uint2 *>(pb + (RP / 16) * T);
                    wa[RP / 4 - 2] = x.x; wa[RP / 4 - 1] = x.y;
                    wb[RP / 4 - 2] = y.x; wb[RP / 4 - 1] = y.y;
                }
                uint32_t f = fin;                         // B(F) of this lane's top row
                uint32_t d = hd;
                uint32_t ylast = 0;
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const uint32_t p = prmt(wa[r / 4], wb[r / 4], pair_sel(r % 4));
                    const uint32_t e_r = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
                    const uint32_t x = __viaddmax_u16x2(d, p, e_r);
                    const uint32_t y = vmax2(f, x);                    // B(H)
                    const uint32_t ho = y - OO;                         // B(H - o), no borrow
                    f = __viaddmax_u16x2(f, ADD_NEG_E, ho);           // B(F) of the row below
                    d = Ho[r];
                    E[r] = e_r;
                    Ho[r] = ho;
                    if (r == RP - 1) ylast = y;
                }
                if (LAST) {                               // lane T-1: ylast = B(H(m, j + 1))
                    if (GLOBAL) {
                        if (j == na - 1) res = (res & 0xffff0000u) | (ylast & 0xffffu);
                        if (j == nb - 1) res = (res & 0xffffu) | (ylast & 0xffff0000u);
                    } else {
                        const uint32_t mask = (j < na ? 0xffffu : 0u) | (j < nb ? 0xffff0000u : 0u);
                        res = vmax2(res, ylast & mask);
                    }
                }
                if (OVERLAP && (j == na - 1 || j == nb - 1)) {   // column n of a half: its rows here
                    uint32_t cm = Ho[0];
#pragma unroll
                    for (int r = 1; r < RP; ++r) cm = vmax2(cm, Ho[r]);
                    cm += OO;                             // B(H) = B(Ho) + o, no carry
                    const uint32_t mask = (j == na - 1 ? 0xffffu : 0u) | (j == nb - 1 ? 0xffff0000u : 0u);
                    mcol = vmax2(mcol, cm & mask);
                }
                hd = hin;
                pub_h = Ho[RP - 1];
                pub_f = f;
                pub_c = cin;
                if (!LAST && k == T - 1)                  // 4 consecutive columns fill one 32-byte sector
                    reinterpret_cast<uint2 *>(bnd)[size_t(j >> 2) * (gstride * 2) + (j & 3)] = make_uint2(pub_h, pub_f);
            };

            // One column step with every check (lanes starting or finishing).
            auto step = [&](const int s) {
                uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
                uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
                uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
                const int j = s - k;                      // 0-based column (column number j + 1)
                const bool act = (j >= 0) && (j < Lp);
                if (k == 0 && act) {
                    const int s3 = s & 3;
                    if (s3 == 0) {
                        quad = quad_next;
                        if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
                        if (pass > 0) cp_async_wait1();   // group s/4 has landed
                    }
                    const uint32_t w = (s3 & 2) ? quad.y : quad.x;
                    cin = (s3 & 1) ? (w >> 16) : (w & 0xffffu);
                    if (pass == 0) {                      // F(1, j) = H(0, j) - o
                        if (GLOBAL) top -= GM2;           // H(0, j) = -g(j)
                        hin = top;
                        fin = top;
                    } else {
                        const uint2 bv = stg[((s >> 2) & 1) * 4 + s3];
                        hin = bv.x;
                        fin = bv.y;
                        if (s3 == 3) {                    // buffer of group s/4 is free: fetch group s/4 + 2
                            if (s + 5 < Lp) {
                                const uint4 *g = bnd + size_t((s >> 2) + 2) * gstride;
                                cp_async16(stg + ((s >> 2) & 1) * 4, g);
                                cp_async16(stg + ((s >> 2) & 1) * 4 + 2, g + 1);
                            }
                            cp_async_commit();
                        }
                    }
                }
                if (act) cells(j, hin, fin, cin);
            };

            // One steady column step (every lane of the warp inside its pair),
            // U = s % 4: lane 0 takes its code from quad and its top-row inputs
            // from the running top row (first pass) or the broadcast load ib[U],
            // by select instead of a branch.
            auto sstep = [&](const int s, const uint2 *ib, auto u_c) {
                constexpr int U = decltype(u_c)::value;
                uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
                uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
                uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
                const uint32_t w = (U & 2) ? quad.y : quad.x;
                const uint32_t c0 = (U & 1) ? (w >> 16) : (w & 0xffffu);
                uint32_t h0, f0;
                if (pass == 0) {
                    if (GLOBAL) top -= GM2;
                    h0 = top;
                    f0 = top;
                } else {
                    const uint2 v = ib[U];
                    h0 = v.x;
                    f0 = v.y;
                }
                const bool lane0 = k == 0;
                hin = lane0 ? h0 : hin;
                fin = lane0 ? f0 : fin;
                cin = lane0 ? c0 : cin;
                cells(s + U - k, hin, fin, cin);
            };
            using U0 = std::integral_constant<int, 0>;
            using U1 = std::integral_constant<int, 1>;
            using U2 = std::integral_constant<int, 2>;
            using U3 = std::integral_constant<int, 3>;
            const int s_steady = (T + 2) & ~3;
            int s = 0;
            for (; s < s_steady && s < steps; ++s) step(s);
            for (; s + 3 < Lmin; s += 4) {
                quad = quad_next;
                if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
                const uint2 *ib = stg;
                if (pass > 0) {
                    cp_async_wait1();                     // group s/4 has landed
                    ib = stg + ((s >> 2) & 1) * 4;
                }
                sstep(s, ib, U0());
                sstep(s, ib, U1());
                sstep(s, ib, U2());
                sstep(s, ib, U3());
                if (pass > 0) {                           // fetch group s/4 + 2 into the freed half
                    if (k == 0 && s + 5 < Lp) {
                        const uint4 *g = bnd + size_t((s >> 2) + 2) * gstride;
                        cp_async16(stg + ((s >> 2) & 1) * 4, g);
                        cp_async16(stg + ((s >> 2) & 1) * 4 + 2, g + 1);
                    }
                    cp_async_commit();
                }
            }
            for (; s < steps; ++s) step(s);
        };
        using RFull = std::integral_constant<int, R>;
        for (int pass = 0; pass + 1 < npass; ++pass) run_pass(pass, std::false_type(), RFull());
        bool ran = false;
        if constexpr (R > 8) {
            if (rest == T * 8) { run_pass(npass - 1, std::true_type(), std::integral_constant<int, 8>()); ran = true; }
        }
        if constexpr (R > 16) {
            if (rest == T * 16) { run_pass(npass - 1, std::true_type(), std::integral_constant<int, 16>()); ran = true; }
        }
        if constexpr (R > 24) {
            if (rest == T * 24) { run_pass(npass - 1, std::true_type(), std::integral_constant<int, 24>()); ran = true; }
        }
        if (!ran) run_pass(npass - 1, std::true_type(), RFull());

        const uint32_t rlast = __shfl_sync(0xffffffffu, res, T - 1, T);   // lane T-1 holds row m
        if (OVERLAP) {
#pragma unroll
            for (int dd = T / 2; dd >= 1; dd >>= 1) mcol = vmax2(mcol, __shfl_xor_sync(0xffffffffu, mcol, dd, T));
        }
        if (valid && k == 0) {
            const uint32_t sc = OVERLAP ? __vimax3_u16x2(rlast, mcol, 0x80008000u) : rlast;
            // an empty target: H(m, 0) = -g(m) (global, semi-global), 0 (overlap)
            const int empty = OVERLAP ? 0 : -g_m;
            const int64_t oA = a.db.perm[2 * pair0];
            const int64_t oB = a.db.perm[2 * pair0 + 1];
            if (oA >= 0) a.scores[oA] = na > 0 ? int(sc & 0xffffu) - 32768 : empty;
            if (oB >= 0) a.scores[oB] = nb > 0 ? int(sc >> 16) - 32768 : empty;
        }
    }
}

template <int T, int R, int MODE>
cudaError_t launch_one(const Mode16Args &a, int grid, cudaStream_t s) {
    constexpr int PAIRS_PER_CTA = kCtaThreads / T;
    const int64_t pairs = a.pair_end - a.pair_begin;
    if (pairs <= 0) return cudaSuccess;
    // m + virt_rows: whole strips of T*R rows, then a last one of T x 8, 16, 24 or R rows
    const int64_t padded = int64_t(a.m) + a.virt_rows;
    const int64_t last_rows = padded - (padded - 1) / (T * R) * (T * R);
    if (!a.chunk_counter || grid <= 0 || a.m <= 0 || a.virt_rows < 0 || a.virt_rows >= T * R ||
        last_rows % (T * 8) != 0 || (padded > T * R && !a.boundary))
        return cudaErrorInvalidValue;
    const int64_t chunks = (pairs + PAIRS_PER_CTA - 1) / PAIRS_PER_CTA;
    k_modes_i16x2<T, R, MODE><<<unsigned(std::min<int64_t>(grid, chunks)), kCtaThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int T, int R>
cudaError_t launch_tr(const Mode16Args &a, int mode, int grid, cudaStream_t s) {
    switch (mode) {
        case SW_ALIGN_GLOBAL: return launch_one<T, R, SW_ALIGN_GLOBAL>(a, grid, s);
        case SW_ALIGN_SEMIGLOBAL: return launch_one<T, R, SW_ALIGN_SEMIGLOBAL>(a, grid, s);
        case SW_ALIGN_OVERLAP: return launch_one<T, R, SW_ALIGN_OVERLAP>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int T, int R, int MODE>
int slots_one(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_modes_i16x2<T, R, MODE>, kCtaThreads, 0) !=
        cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <int T, int R>
int slots_tr(int sms) {
    return std::max({slots_one<T, R, SW_ALIGN_GLOBAL>(sms), slots_one<T, R, SW_ALIGN_SEMIGLOBAL>(sms),
                     slots_one<T, R, SW_ALIGN_OVERLAP>(sms)});
}

}  // namespace

bool modes16_config_supported(int lanes, int rows) {
    return lanes == 8 && (rows == 16 || rows == 24 || rows == 32);
}

cudaError_t launch_modes_i16x2(const Mode16Args &a, int mode, int lanes, int rows, int grid, cudaStream_t s) {
    switch (lanes * 100 + rows) {
        case 816: return launch_tr<8, 16>(a, mode, grid, s);
        case 824: return launch_tr<8, 24>(a, mode, grid, s);
        case 832: return launch_tr<8, 32>(a, mode, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int modes16_slots(int lanes, int rows, int sms) {
    switch (lanes * 100 + rows) {
        case 816: return slots_tr<8, 16>(sms);
        case 824: return slots_tr<8, 24>(sms);
        case 832: return slots_tr<8, 32>(sms);
        default: return 0;
    }
}

}  // namespace swdb
