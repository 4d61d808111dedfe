// Inter-task Smith-Waterman/Gotoh scoring in packed int16x2 DPX arithmetic.
//
// Section 2.2 (inter-task parallelism: many alignment matrices computed at
// once with no communication between them) and Section 2.3 (SW#db's GPU
// kernel for short database sequences, "solveShort" in Section 3.2).  The
// design here is this library's own, for sm_103a:
//
// * A subwarp of T lanes scores ONE PAIR of database sequences at once: the
//   low int16 half of every register belongs to sequence 2p, the high half
//   to 2p+1, so one DPX instruction updates two cells.
// * Lane k owns R consecutive query rows (a strip of T*R rows per pass) and
//   walks the database columns one step behind lane k-1 (an anti-diagonal
//   skew).  The bottom row's H and F and the column's residue codes move to
//   the next lane with one shuffle each; nothing goes through memory inside
//   a pass.  Queries longer than T*R rows take several passes; lane T-1
//   writes the strip's bottom row (H-o and F per column) to scratch and
//   lane 0 of the next pass reads it back.
// * The query profile of the current strip lives in shared memory as int8
//   S(q_i, a) + o, laid out [residue a][lane k][row r], so each lane fetches
//   its R rows for one database residue with 128-bit loads that are free of
//   bank conflicts (row stride T*R bytes is a multiple of 128 for T*R >= 128).
// * Values are kept shifted and biased: every int16 quantity v is held as
//   the unsigned halfword v + 32768 (offset binary), so unsigned DPX max/add
//   orders them correctly, adding a negative constant is a modular add, and
//   subtracting the gap-open penalty from a non-negative H is a plain 32-bit
//   integer subtraction that never borrows across the halves.  That last
//   operation runs outside the ALU pipe the DPX instructions saturate.  The
//   registers carry Ho = H - o and E per row; F flows down the rows.  Per
//   cell pair:   E' = max(E - e, Ho_left)            (viaddmax)
//                X  = max(Ho_diag + S + o, E')       (viaddmax)
//                H  = max(F, X, 0)                   (vimax3)
//                Ho = H - o                          (32-bit subtract)
//                F_below = max(F - e, Ho)            (viaddmax)
//   which is the recurrence H = max(0, Hdiag + S, E, F) with Hdiag + S =
//   Ho_diag + (S + o).  The running maximum takes two rows per vimax3.
// * The grid is either one CTA per chunk of 256/T pairs, or persistent: the
//   resident CTAs pull chunks (longest first) from an atomic counter and each
//   keeps its strip-boundary rows in its own scratch slot, reused chunk after
//   chunk, so those rows stay in L2 instead of being written back to HBM.
// * Saturation: every value stays below the running maximum of H plus the
//   largest matrix entry, so if that maximum stays below
//   32767 - max(S) no int16 operation overflowed and the score is exact.
//   Sequences at or above that limit are appended to a list and rescored
//   in int32 by another kernel.
#include <algorithm>
#include <type_traits>

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

// SLOTS = true: persistent grid, chunks pulled from *a.chunk_counter, strip
// boundary in per-slot scratch.  SLOTS = false: one CTA per chunk, per-pair
// boundary in the database layout's shape.
template <int T, int R, bool SLOTS>
__global__ void __launch_bounds__(kCtaThreads, (R <= 16 ? 3 : 2)) k_inter_i16x2(const __grid_constant__ InterArgs a) {
    static_assert(R % 8 == 0, "rows per lane must be a multiple of 8");
    static_assert(32 % T == 0 && T >= 4, "lanes must divide the warp");
    constexpr int PAIRS_PER_CTA = kCtaThreads / T;
    constexpr int TR = T * R;
    constexpr int H16 = (R + 15) / 16;                // 16-row groups per lane (the last may hold 8)
    constexpr int SLOT = T * 16 * H16;                // profile bytes per residue
    constexpr int PROF_BYTES = kProfRows * SLOT;

    __shared__ __align__(16) int8_t prof[PROF_BYTES];
    __shared__ int8_t mat[kProfRows * kProfRows];
    // Per subwarp: two 4-column groups of the previous strip's bottom row
    // (B(Ho), B(F) per column), filled by lane 0 with cp.async one group ahead.
    __shared__ __align__(16) uint2 bstage[PAIRS_PER_CTA][8];

    __shared__ int sh_chunk;
    __shared__ uint2 top4[4];            // the top row's inputs B(H-o), B(F) = B(-o), for broadcast reads

    const int tid = threadIdx.x;
    const int k = tid % T;               // lane within the subwarp
    const int sub = tid / T;             // subwarp within the CTA
    // staged transposed, [db code][query code]: the profile fill reads one db code
    // against many query codes at once, which then fall in distinct banks
    for (int i = tid; i < kProfRows * kProfRows; i += kCtaThreads)
        mat[(i % kProfRows) * kProfRows + i / kProfRows] = (&a.prof8[0][0])[i];
    if (tid < 4) top4[tid] = make_uint2(pack2(32768 - a.gap_open), pack2(32768 - a.gap_open));
    const int n_chunks = int((a.pair_end - a.pair_begin + PAIRS_PER_CTA - 1) / PAIRS_PER_CTA);

  for (;;) {
    int chunk = int(blockIdx.x);
    if (SLOTS) {
        __syncthreads();                 // the previous chunk is done with shared state
        if (tid == 0) sh_chunk = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        chunk = sh_chunk;
    }
    if (chunk >= n_chunks) break;
    // The pair index is not kept across the passes (registers are tight at
    // R = 32); the epilogue derives it again from the chunk.
    const int64_t pair0 = a.pair_begin + int64_t(chunk) * PAIRS_PER_CTA + sub;
    const bool valid = pair0 < a.pair_end;

    int64_t b = 0;
    int slot = 0;
    int Lp = 0;
    if (valid) {
        b = pair0 / kBundlePairs;
        slot = int(pair0 % kBundlePairs);
        Lp = (a.db.len[2 * pair0] + 3) & ~3;   // longest of the pair (sorted, longest first)
    }
    const int Lw = __reduce_max_sync(0xffffffffu, Lp);   // warp-uniform column count

    const int o = a.gap_open;
    // Biased constants (see the header comment): B(v) = v + 32768 per half.
    const uint32_t BNEG_O2 = pack2(32768 - o);        // B(-o)
    const uint32_t ADD_NEG_E = pack2(-a.gap_extend);  // modular addend "- e"
    const uint32_t OO = uint32_t(o) | (uint32_t(o) << 16);
    const uint32_t BZERO2 = 0x80008000u;              // B(0)

    // Boundary scratch of this pair, grouped by 4 columns so lane 0 reads a
    // group with two 16-byte loads: either the bundle's region (8*Lb uint2
    // entries at uint2 index off/2, [column/4][slot][column%4]) or this CTA
    // slot's region (max_cols entries per subwarp, [column]).
    const uint2 *cptr = nullptr;
    uint4 *bnd = nullptr;
    constexpr int gstride = SLOTS ? 2 : kBundlePairs * 2;   // uint4 per 4-column group
    if (valid) {
        const int64_t off = a.db.bundle_off[b];
        cptr = reinterpret_cast<const uint2 *>(a.db.codes + off) + slot;
        if (a.boundary) {
            if (SLOTS)
                bnd = reinterpret_cast<uint4 *>(a.boundary + int64_t(blockIdx.x) * a.slot_stride +
                                                int64_t(sub) * a.max_cols);
            else
                bnd = reinterpret_cast<uint4 *>(a.boundary + off / 2) + slot * 2;
        }
    }

    const int npass = (a.m + TR - 1) / TR;
    uint32_t mx = BZERO2;                  // running max of B(H), both halves

    // One pass (strip) of the query: rows pass*TR .. pass*TR + T*RP - 1, RP rows
    // per lane.  Every pass but the last is a full strip (RP = R); the last one
    // takes the fewest rows per lane (a multiple of 8) that cover the rest of
    // the query, which cuts the padded rows a query's final strip computes.
    auto run_pass = [&](const int pass, auto rp_c) {
        constexpr int RP = decltype(rp_c)::value;
        constexpr int TRP = T * RP;
        constexpr int SLOTP = T * 16 * ((RP + 15) / 16);   // profile bytes per residue in this pass
            __syncthreads();
            // Profile strip for rows pass*TR .. pass*TR+TRP-1, layout
            // [residue a][group h][lane k][16 rows]: lane k's rows 16h..16h+15 sit at
            // a*SLOTP + h*T*16 + k*16, so the 8 lanes of a quarter-warp read 8
            // consecutive 16-byte slots (no bank conflicts) and a lane's later
            // groups are compile-time offsets from its first.  With RP = 24 the
            // second group holds 8 rows in the first half of its slot.
            for (int w = tid; w < kProfRows * TRP / 4; w += kCtaThreads) {
                const int e0 = w * 4;
                const int res = e0 / TRP;
                const int within = e0 % TRP;
                const int row0 = pass * TR + within;
                const int kk = within / RP, rr = within % RP;
                const int phys = res * SLOTP + (rr >> 4) * (T * 16) + kk * 16 + (rr & 15);
                uint32_t word = 0;
    #pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = row0 + c;
                    int v = -128;
                    if (row < a.m) {
                        // device-resident queries are not validated on the host:
                        // codes outside the table score as padding
                        const int qc = a.query[row];
                        if (qc < kProfRows) v = mat[res * kProfRows + qc];
                    }
                    word |= (uint32_t(uint8_t(int8_t(v)))) << (8 * c);
                }
                reinterpret_cast<uint32_t *>(prof)[phys / 4] = word;
            }
            __syncthreads();
            if (Lw == 0) return;

            uint32_t E[RP], Ho[RP];
    #pragma unroll
            for (int r = 0; r < RP; ++r) { E[r] = BNEG_O2; Ho[r] = BNEG_O2; }
            uint32_t hd = BNEG_O2;             // B(Ho(top-1, j-1))
            // pub_h: B(Ho) of this lane's bottom row; pub_f: B(F) of the next lane's top row
            uint32_t pub_h = BNEG_O2, pub_f = BNEG_O2, pub_c = 0;
            const bool last_pass = (pass + 1 == npass);
            const int steps = Lw + T - 1;
            // Lane 0 reads codes and (after the first pass) the previous strip's
            // bottom row in groups of 4 columns, one group ahead of use, so the
            // global-load latency stays off the per-column critical path.
            uint2 quad = make_uint2(0, 0), quad_next = make_uint2(0, 0);
            uint2 *stg = bstage[sub];
            if (Lp > 0) quad_next = __ldg(cptr);     // every lane of the subwarp: one broadcast load
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

            // Lane T-1's store of the strip's bottom row (H - o, F) at column jl;
            // 4 consecutive columns fill one 32-byte sector.
            auto bottom_index = [&](const int jl) -> size_t {
                if (SLOTS) return size_t(jl);                           // per subwarp, [column]
                return size_t(jl >> 2) * (gstride * 2) + (jl & 3);      // [column/4][slot][column%4]
            };

            // The cell work of one column step for this lane's RP rows.
            auto cells = [&](const uint32_t hin, const uint32_t fin, const uint32_t cin) {
                const int ta = int(cin & 0xffu), tb = int((cin >> 8) & 0xffu);
                const uint4 *pa = reinterpret_cast<const uint4 *>(prof + ta * SLOTP + k * 16);
                const uint4 *pb = reinterpret_cast<const uint4 *>(prof + tb * SLOTP + k * 16);
                uint32_t wa[RP / 4], wb[RP / 4];
    #pragma unroll
                for (int v = 0; v < RP / 16; ++v) {
                    const uint4 x = pa[v * T];
                    const uint4 y = pb[v * T];
                    wa[4 * v + 0] = x.x; wa[4 * v + 1] = x.y; wa[4 * v + 2] = x.z; wa[4 * v + 3] = x.w;
                    wb[4 * v + 0] = y.x; wb[4 * v + 1] = y.y; wb[4 * v + 2] = y.z; wb[4 * v + 3] = y.w;
                }
                if (RP % 16) {                     // last group of 8 rows: an 8-byte load
                    const uint2 x = *reinterpret_cast<const uint2 *>(pa + (RP / 16) * T);
                    const uint2 y = *reinterpret_cast<const uint2 *>(pb + (RP / 16) * T);
                    wa[RP / 4 - 2] = x.x; wa[RP / 4 - 1] = x.y;
                    wb[RP / 4 - 2] = y.x; wb[RP / 4 - 1] = y.y;
                }
                uint32_t f = fin;                 // B(F) of this lane's top row
                uint32_t d = hd;
                uint32_t yprev = 0;
    #pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const uint32_t p = prmt(wa[r / 4], wb[r / 4], pair_sel(r % 4));
                    const uint32_t e_r = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
                    const uint32_t x = __viaddmax_u16x2(d, p, e_r);
                    const uint32_t y = __vimax3_u16x2(f, x, BZERO2);   // B(H)
                    const uint32_t ho = y - OO;                         // B(H - o), no borrow: y >= 0x8000
                    f = __viaddmax_u16x2(f, ADD_NEG_E, ho);           // B(F) of the row below
                    d = Ho[r];
                    E[r] = e_r;
                    Ho[r] = ho;
                    if (r & 1) mx = __vimax3_u16x2(mx, yprev, y);
                    yprev = y;
                }
                hd = hin;
                pub_h = Ho[RP - 1];
                pub_f = f;
                pub_c = cin;
            };

            // One column step of the subwarp with every check (lanes starting or
            // finishing): the first and last columns.
            auto step = [&](const int s) {
                uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
                uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
                uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
                const int j = s - k;
                const bool act = (j >= 0) && (j < Lp);
                if (k == 0 && act) {
                    const int s3 = s & 3;
                    if (s3 == 0) {
                        quad = quad_next;
                        if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
                        if (pass > 0) cp_async_wait1();      // group s/4 has landed
                    }
                    const uint32_t w = (s3 & 2) ? quad.y : quad.x;
                    cin = (s3 & 1) ? (w >> 16) : (w & 0xffffu);
                    if (pass == 0) {          // H(0,j) = 0, F(1,j) = -o
                        hin = BNEG_O2;
                        fin = BNEG_O2;
                    } else {
                        const uint2 bv = stg[((s >> 2) & 1) * 4 + s3];
                        hin = bv.x;
                        fin = bv.y;
                        if (s3 == 3) {        // buffer of group s/4 is free: fetch group s/4 + 2 into it
                            if (s + 5 < Lp) {
                                const uint4 *g = bnd + size_t((s >> 2) + 2) * gstride;
                                cp_async16(stg + ((s >> 2) & 1) * 4, g);
                                cp_async16(stg + ((s >> 2) & 1) * 4 + 2, g + 1);
                            }
                            cp_async_commit();
                        }
                    }
                }
                if (act) {
                    cells(hin, fin, cin);
                    if (k == T - 1 && !last_pass)
                        reinterpret_cast<uint2 *>(bnd)[bottom_index(s - (T - 1))] = make_uint2(pub_h, pub_f);
                }
            };

            // One steady column step (every lane of the warp inside its sequence),
            // U = s % 4: lane 0 takes its codes from quad and its top-row inputs
            // from the broadcast load ib[U] with selects instead of a branch.
            auto sstep = [&](const int s, const uint2 *ib, auto u_c) {
                constexpr int U = decltype(u_c)::value;
                uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
                uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
                uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
                const uint2 v = ib[U];
                const uint32_t w = (U & 2) ? quad.y : quad.x;
                const uint32_t c0 = (U & 1) ? (w >> 16) : (w & 0xffffu);
                const bool lane0 = k == 0;
                hin = lane0 ? v.x : hin;
                fin = lane0 ? v.y : fin;
                cin = lane0 ? c0 : cin;
                cells(hin, fin, cin);
                if (k == T - 1 && !last_pass)
                    reinterpret_cast<uint2 *>(bnd)[bottom_index(s + U - (T - 1))] = make_uint2(pub_h, pub_f);
            };
            using U0 = std::integral_constant<int, 0>;
            using U1 = std::integral_constant<int, 1>;
            using U2 = std::integral_constant<int, 2>;
            using U3 = std::integral_constant<int, 3>;
            // Steady columns: s >= T-1 (every lane started) and s + 3 < Lmin (no lane
            // of any subwarp in the warp has finished), in groups of 4 aligned to s % 4 == 0.
            const int Lmin = __reduce_min_sync(0xffffffffu, Lp);
            const int s_steady = (T + 2) & ~3;
            int s = 0;
            for (; s < s_steady && s < steps; ++s) step(s);
            for (; s + 3 < Lmin; s += 4) {
                quad = quad_next;
                if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
                const uint2 *ib = top4;
                if (pass > 0) {
                    cp_async_wait1();                              // group s/4 has landed
                    ib = stg + ((s >> 2) & 1) * 4;
                }
                sstep(s, ib, U0());
                sstep(s, ib, U1());
                sstep(s, ib, U2());
                sstep(s, ib, U3());
                if (pass > 0) {                                    // fetch group s/4 + 2 into the freed half
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
    for (int pass = 0; pass + 1 < npass; ++pass) run_pass(pass, RFull());
    if (npass > 0) {
        const int rest = a.m - (npass - 1) * TR;           // rows of the last strip, 1 .. TR
        bool ran = false;
        if constexpr (R > 8) {
            if (rest <= T * 8) { run_pass(npass - 1, std::integral_constant<int, 8>()); ran = true; }
        }
        if constexpr (R > 16) {
            if (!ran && rest <= T * 16) { run_pass(npass - 1, std::integral_constant<int, 16>()); ran = true; }
        }
        if constexpr (R > 24) {
            if (!ran && rest <= T * 24) { run_pass(npass - 1, std::integral_constant<int, 24>()); ran = true; }
        }
        if (!ran) run_pass(npass - 1, RFull());
    }
#pragma unroll
    for (int dd = T / 2; dd >= 1; dd >>= 1) {
        const uint32_t other = __shfl_xor_sync(0xffffffffu, mx, dd, T);
        mx = __vimax3_u16x2(mx, other, other);
    }
    const int chunk_end = SLOTS ? *reinterpret_cast<volatile int *>(&sh_chunk) : int(blockIdx.x);
    const int64_t pair = a.pair_begin + int64_t(chunk_end) * PAIRS_PER_CTA + sub;
    if (pair < a.pair_end && k == 0) {
        const int hA = int(mx & 0xffffu) - 32768;
        const int hB = int(mx >> 16) - 32768;
        const int64_t tA = 2 * pair;
        int mask = 0;
        const int64_t oA = a.db.perm[tA];
        const int64_t oB = a.db.perm[tA + 1];
        if (oA >= 0) {
            if (hA >= a.sat_limit) mask |= 1;
            else a.scores[oA] = hA;
        }
        if (oB >= 0) {
            if (hB >= a.sat_limit) mask |= 2;
            else a.scores[oB] = hB;
        }
        if (mask) {
            const int idx = atomicAdd(a.ovf_count, 1);
            a.ovf_list[idx] = int32_t(pair * 4 + mask);
            atomicAdd(a.ovf_seqs, __popc(mask));
        }
    }
    if (!SLOTS) break;
  }
}

template <int T, int R>
cudaError_t launch_tr(const InterArgs &a, cudaStream_t s, int grid_slots, int priority) {
    constexpr int PAIRS_PER_CTA = kCtaThreads / T;
    const int64_t pairs = a.pair_end - a.pair_begin;
    if (pairs <= 0) return cudaSuccess;
    const int64_t chunks = (pairs + PAIRS_PER_CTA - 1) / PAIRS_PER_CTA;
    if (grid_slots > 0) {
        if (!a.chunk_counter) return cudaErrorInvalidValue;
        const cudaError_t e = launch_with_priority(k_inter_i16x2<T, R, true>,
                                                   dim3(unsigned(std::min<int64_t>(grid_slots, chunks))),
                                                   dim3(kCtaThreads), 0, s, priority, a);
        if (e != cudaSuccess) return e;
    } else {
        k_inter_i16x2<T, R, false><<<unsigned(chunks), kCtaThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int T, int R>
int slots_tr(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inter_i16x2<T, R, true>, kCtaThreads, 0) !=
        cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace

bool inter_config_supported(int lanes, int rows) {
    switch (lanes * 100 + rows) {
        case 416: case 424: case 432: case 816: case 1616: case 3216: case 824: case 832: case 1632: case 3232:
        case 3208: return true;
        default: return false;
    }
}

cudaError_t launch_inter_i16x2(const InterArgs &a, int lanes, int rows, cudaStream_t s, int grid_slots,
                               int priority) {
    switch (lanes * 100 + rows) {
        case 416: return launch_tr<4, 16>(a, s, grid_slots, priority);
        case 424: return launch_tr<4, 24>(a, s, grid_slots, priority);
        case 432: return launch_tr<4, 32>(a, s, grid_slots, priority);
        case 816: return launch_tr<8, 16>(a, s, grid_slots, priority);
        case 824: return launch_tr<8, 24>(a, s, grid_slots, priority);
        case 1616: return launch_tr<16, 16>(a, s, grid_slots, priority);
        case 3208: return launch_tr<32, 8>(a, s, grid_slots, priority);
        case 3216: return launch_tr<32, 16>(a, s, grid_slots, priority);
        case 832: return launch_tr<8, 32>(a, s, grid_slots, priority);
        case 1632: return launch_tr<16, 32>(a, s, grid_slots, priority);
        case 3232: return launch_tr<32, 32>(a, s, grid_slots, priority);
        default: return cudaErrorInvalidValue;
    }
}

int inter_slots(int lanes, int rows, int sms) {
    switch (lanes * 100 + rows) {
        case 416: return slots_tr<4, 16>(sms);
        case 424: return slots_tr<4, 24>(sms);
        case 432: return slots_tr<4, 32>(sms);
        case 816: return slots_tr<8, 16>(sms);
        case 824: return slots_tr<8, 24>(sms);
        case 1616: return slots_tr<16, 16>(sms);
        case 3208: return slots_tr<32, 8>(sms);
        case 3216: return slots_tr<32, 16>(sms);
        case 832: return slots_tr<8, 32>(sms);
        case 1632: return slots_tr<16, 32>(sms);
        case 3232: return slots_tr<32, 32>(sms);
        default: return 0;
    }
}

}  // namespace swdb
