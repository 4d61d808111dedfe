// Batched inter-task scoring: many queries in one persistent launch.
//
// Same recurrences and biased int16x2 arithmetic as k_inter16.cu (Section
// 2.2 inter-task parallelism; affine gaps as in Section 4.1), packed the
// other way round: the two halves of a register hold TWO QUERIES (of similar
// length, paired by the host) against the SAME database sequence.  Their
// profile is then one int16x2 word per (residue, row) -- S(q1_i, a) + o in
// the low half, S(q2_i, a) + o in the high half -- loaded ready to add, so
// the byte permute the sequence-pair packing needs disappears.
//
// The launch is persistent: one CTA per resident slot pulls tiles
// (database chunk, query pair) from an atomic counter, longest chunks first
// and all query pairs of a chunk together (the chunk's codes stay in L2).
// A chunk is 256/T consecutive sorted sequences, one per subwarp of T lanes.
// Queries longer than one strip (T*R rows) take several passes; the strip
// boundary of each subwarp goes to a scratch region owned by the CTA slot,
// reused tile after tile, so it stays in L2.  A pair's last pass takes the
// fewest rows per lane (8, 16, 24 or R) that cover its longer query.
//
// Saturated (query, sequence) results are appended to per-query lists, with
// the two sequences of a database pair merged into one entry (pair*4 + mask)
// because the int32 rescore uses the pair's boundary region for both.
#include <type_traits>

#include "simd16.cuh"
#include "swdb_internal.cuh"

namespace swdb {
namespace {

using simd16::cp_async16;
using simd16::cp_async_commit;
using simd16::cp_async_wait1;
using simd16::pack2;

template <int T, int R>
__global__ void __launch_bounds__(kCtaThreads, (R <= 16 ? 3 : 2)) k_batch_i16x2(const __grid_constant__ BatchArgs a) {
    static_assert(R % 4 == 0, "rows per lane must be a multiple of 4");
    constexpr int SPC = kCtaThreads / T;        // sequences per chunk (one per subwarp)
    constexpr int TR = T * R;
    extern __shared__ __align__(16) uint32_t prof[];   // [32 residues][TR words], see the fill
    __shared__ int8_t mat[kProfRows * kProfRows];
    __shared__ __align__(16) uint2 bstage[SPC][8];
    __shared__ int sh_tile;
    __shared__ int sh_mask[SPC / 2];
    __shared__ uint2 top4[4];        // the top row's inputs B(H-o), B(F) = B(-o), for broadcast reads

    const int tid = threadIdx.x;
    const int k = tid % T;
    const int sub = tid / T;
    // staged transposed, [db code][query code]: the profile fill reads one db code
    // against many query codes at once, which then fall in distinct banks
    for (int i = tid; i < kProfRows * kProfRows; i += kCtaThreads)
        mat[(i % kProfRows) * kProfRows + i / kProfRows] = (&a.prof8[0][0])[i];
    if (tid < 4) top4[tid] = make_uint2(pack2(32768 - a.gap_open), pack2(32768 - a.gap_open));

    const int o = a.gap_open;
    const uint32_t BNEG_O2 = pack2(32768 - o);
    const uint32_t ADD_NEG_E = pack2(-a.gap_extend);
    const uint32_t OO = uint32_t(o) | (uint32_t(o) << 16);
    const uint32_t BZERO2 = 0x80008000u;
    const int64_t n_tiles = int64_t(a.n_chunks) * a.n_qp;
    uint2 *slot_scratch = a.scratch ? a.scratch + int64_t(blockIdx.x) * a.scratch_stride + int64_t(sub) * a.max_cols
                                    : nullptr;

    for (;;) {
        __syncthreads();   // previous tile done with shared state
        if (tid == 0) sh_tile = atomicAdd(a.tile_counter, 1);
        if (tid < SPC / 2) sh_mask[tid] = 0;
        __syncthreads();
        const int64_t tile = sh_tile;
        if (tile >= n_tiles) break;
        const int chunk = int(tile / a.n_qp);
        const int qp = int(tile % a.n_qp);
        const int qa = a.qp_a[qp], qb = a.qp_b[qp];
        const int64_t qa0 = a.q_off[qa];
        const int ma = int(a.q_off[qa + 1] - qa0);
        int64_t qb0 = 0;
        int mb = 0;
        if (qb >= 0) {
            qb0 = a.q_off[qb];
            mb = int(a.q_off[qb + 1] - qb0);
        }
        const int m = ma > mb ? ma : mb;
        const int npass = (m + TR - 1) / TR;

        const int64_t t = a.seq_begin + int64_t(chunk) * SPC + sub;   // this subwarp's sorted sequence
        const bool valid = t < a.seq_end;
        int Lp = 0;
        int64_t pair = 0;
        int h = 0;
        const uint2 *cptr = nullptr;
        if (valid) {
            pair = t >> 1;
            h = int(t & 1);
            Lp = (a.db.len[t] + 3) & ~3;
            const int64_t b = pair / kBundlePairs;
            cptr = reinterpret_cast<const uint2 *>(a.db.codes + a.db.bundle_off[b]) + int(pair % kBundlePairs);
        }
        const int Lw = __reduce_max_sync(0xffffffffu, Lp);
        uint32_t mx = BZERO2;

        // One pass (strip) of the pair: rows pass*TR .. pass*TR + T*RP - 1, RP
        // rows per lane.  Every pass but the last is a full strip (RP = R); the
        // last one takes the fewest rows per lane (a multiple of 8) that cover
        // the rest of the longer query, which cuts the padded rows it computes.
        auto run_pass = [&](const int pass, auto rp_c) {
            constexpr int RP = decltype(rp_c)::value;
            constexpr int TRP = T * RP;
            __syncthreads();
            // Profile strip, word layout [a][row group v][lane k][row%4]: lane k's
            // rows 4v..4v+3 are one 16-byte slot at a*TRP + v*4T + 4k (quarter-warp
            // lanes read consecutive slots).  Word = S(qa_i, a)+o | S(qb_i, a)+o << 16.
            for (int w = tid; w < kProfRows * TRP; w += kCtaThreads) {
                const int res = w / TRP;
                const int rem = w % TRP;
                const int v = rem / (4 * T);
                const int rem2 = rem % (4 * T);
                const int kk = rem2 >> 2;
                const int row = pass * TR + kk * RP + v * 4 + (rem2 & 3);
                int lo = -128, hi = -128;
                if (row < ma) {
                    const int c = a.queries[qa0 + row];
                    if (c < kProfRows) lo = mat[res * kProfRows + c];
                }
                if (row < mb) {
                    const int c = a.queries[qb0 + row];
                    if (c < kProfRows) hi = mat[res * kProfRows + c];
                }
                prof[w] = (uint32_t(lo) & 0xffffu) | (uint32_t(hi) << 16);
            }
            __syncthreads();
            if (Lw == 0) return;

            uint32_t E[RP], Ho[RP];
#pragma unroll
            for (int r = 0; r < RP; ++r) { E[r] = BNEG_O2; Ho[r] = BNEG_O2; }
            uint32_t hd = BNEG_O2;
            uint32_t pub_h = BNEG_O2, pub_f = BNEG_O2, pub_c = 0;
            const bool last_pass = (pass + 1 == npass);
            uint2 quad = make_uint2(0, 0), quad_next = make_uint2(0, 0);
            uint2 *stg = bstage[sub];
            const uint4 *gsrc = reinterpret_cast<const uint4 *>(slot_scratch);
            if (Lp > 0) quad_next = __ldg(cptr);     // every lane of the subwarp: one broadcast load
            if (k == 0 && Lp > 0 && pass > 0) {
                cp_async16(stg + 0, gsrc);
                cp_async16(stg + 2, gsrc + 1);
                cp_async_commit();
                if (4 < Lp) {
                    cp_async16(stg + 4, gsrc + 2);
                    cp_async16(stg + 6, gsrc + 3);
                }
                cp_async_commit();
            }
            const int steps = Lw + T - 1;

            // The cell work of one column step for this lane's RP rows (both
            // queries of the pair in the two halves; cin = the sequence's code).
            auto cells = [&](const uint32_t hin, const uint32_t fin, const uint32_t cin) {
                const uint4 *pp = reinterpret_cast<const uint4 *>(prof + cin * TRP + k * 4);
                uint32_t P[RP];
#pragma unroll
                for (int v = 0; v < RP / 4; ++v) {
                    const uint4 x = pp[v * T];
                    P[4 * v + 0] = x.x; P[4 * v + 1] = x.y; P[4 * v + 2] = x.z; P[4 * v + 3] = x.w;
                }
                uint32_t f = fin;
                uint32_t d = hd;
                uint32_t yprev = 0;
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const uint32_t e_r = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
                    const uint32_t x = __viaddmax_u16x2(d, P[r], e_r);
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
                pub_h = Ho[RP - 1];
                pub_f = f;
                pub_c = cin;
            };

            // One column step with every check (lanes starting or finishing).
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
                        if (pass > 0) cp_async_wait1();
                    }
                    const uint32_t wd = (s3 & 2) ? quad.y : quad.x;
                    cin = (wd >> (16 * (s3 & 1) + 8 * h)) & 0xffu;
                    if (pass == 0) {
                        hin = BNEG_O2;
                        fin = BNEG_O2;
                    } else {
                        const uint2 bv = stg[((s >> 2) & 1) * 4 + s3];
                        hin = bv.x;
                        fin = bv.y;
                        if (s3 == 3) {
                            if (s + 5 < Lp) {
                                const uint4 *g = gsrc + size_t((s >> 2) + 2) * 2;
                                cp_async16(stg + ((s >> 2) & 1) * 4, g);
                                cp_async16(stg + ((s >> 2) & 1) * 4 + 2, g + 1);
                            }
                            cp_async_commit();
                        }
                    }
                }
                if (act) {
                    cells(hin, fin, cin);
                    if (k == T - 1 && !last_pass) slot_scratch[s - (T - 1)] = make_uint2(pub_h, pub_f);
                }
            };

            // One steady column step (every lane of the warp inside its
            // sequence), U = s % 4: lane 0 takes its code from quad and its
            // top-row inputs from the broadcast load ib[U] by select.
            auto sstep = [&](const int s, const uint2 *ib, auto u_c) {
                constexpr int U = decltype(u_c)::value;
                uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
                uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
                uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
                const uint2 v = ib[U];
                const uint32_t wd = (U & 2) ? quad.y : quad.x;
                const uint32_t c0 = (wd >> (16 * (U & 1) + 8 * h)) & 0xffu;
                const bool lane0 = k == 0;
                hin = lane0 ? v.x : hin;
                fin = lane0 ? v.y : fin;
                cin = lane0 ? c0 : cin;
                cells(hin, fin, cin);
                if (k == T - 1 && !last_pass) slot_scratch[s + U - (T - 1)] = make_uint2(pub_h, pub_f);
            };
            using U0 = std::integral_constant<int, 0>;
            using U1 = std::integral_constant<int, 1>;
            using U2 = std::integral_constant<int, 2>;
            using U3 = std::integral_constant<int, 3>;
            const int Lmin = __reduce_min_sync(0xffffffffu, Lp);
            const int s_steady = (T + 2) & ~3;
            int s = 0;
            for (; s < s_steady && s < steps; ++s) step(s);
            for (; s + 3 < Lmin; s += 4) {
                quad = quad_next;
                if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
                const uint2 *ib = top4;
                if (pass > 0) {
                    cp_async_wait1();                          // group s/4 has landed
                    ib = stg + ((s >> 2) & 1) * 4;
                }
                sstep(s, ib, U0());
                sstep(s, ib, U1());
                sstep(s, ib, U2());
                sstep(s, ib, U3());
                if (pass > 0) {                                // fetch group s/4 + 2 into the freed half
                    if (k == 0 && s + 5 < Lp) {
                        const uint4 *g = gsrc + size_t((s >> 2) + 2) * 2;
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
            const int rest = m - (npass - 1) * TR;             // rows of the last strip, 1 .. TR
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
        int64_t orig = -1;
        if (valid && k == 0) {
            orig = a.db.perm[t];
            if (orig >= 0) {
                const int ha = int(mx & 0xffffu) - 32768;
                const int hb = int(mx >> 16) - 32768;
                if (ha >= a.sat_limit) atomicOr(&sh_mask[sub >> 1], 1 << (2 * h));
                else a.scores[int64_t(qa) * a.db.n_seqs + orig] = ha;
                if (qb >= 0) {
                    if (hb >= a.sat_limit) atomicOr(&sh_mask[sub >> 1], 2 << (2 * h));
                    else a.scores[int64_t(qb) * a.db.n_seqs + orig] = hb;
                }
            }
        }
        __syncthreads();
        // One list entry per (query, database pair) with the mask of saturated halves.
        if (tid < SPC / 2 && sh_mask[tid]) {
            const int mk = sh_mask[tid];
            const int64_t p = (a.seq_begin + int64_t(chunk) * SPC) / 2 + tid;
            const int m_a = (mk & 1) | ((mk >> 1) & 2);          // bits for query qa: halves 0,1
            const int m_b = ((mk >> 1) & 1) | ((mk >> 2) & 2);   // bits for query qb
            if (m_a) {
                const int idx = atomicAdd(a.ovf_count + qa, 1);
                a.ovf_list[int64_t(qa) * a.list_stride + idx] = int32_t(p * 4 + m_a);
                atomicAdd(a.ovf_seqs + qa, __popc(m_a));
            }
            if (m_b) {
                const int idx = atomicAdd(a.ovf_count + qb, 1);
                a.ovf_list[int64_t(qb) * a.list_stride + idx] = int32_t(p * 4 + m_b);
                atomicAdd(a.ovf_seqs + qb, __popc(m_b));
            }
        }
    }
}

template <int T, int R>
size_t batch_smem() {
    return size_t(kProfRows) * T * R * sizeof(uint32_t);
}

template <int T, int R>
cudaError_t launch_tr(const BatchArgs &a, int grid, cudaStream_t s, int priority) {
    const size_t smem = batch_smem<T, R>();   // attribute set by batch_slots at planning
    const cudaError_t e = launch_with_priority(k_batch_i16x2<T, R>, dim3(grid), dim3(kCtaThreads), smem, s, priority, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int T, int R>
int slots_tr(int sms) {
    int per_sm = 0;
    const size_t smem = batch_smem<T, R>();
    if (cudaFuncSetAttribute(k_batch_i16x2<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_i16x2<T, R>, kCtaThreads, smem) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace

bool batch_config_supported(int lanes, int rows) {
    switch (lanes * 100 + rows) {
        case 816: case 824: case 832: case 1616: case 1624: case 1632: return true;
        default: return false;
    }
}

int batch_slots(int lanes, int rows, int sms) {
    switch (lanes * 100 + rows) {
        case 816: return slots_tr<8, 16>(sms);
        case 824: return slots_tr<8, 24>(sms);
        case 832: return slots_tr<8, 32>(sms);
        case 1624: return slots_tr<16, 24>(sms);
        case 1616: return slots_tr<16, 16>(sms);
        case 1632: return slots_tr<16, 32>(sms);
        default: return 0;
    }
}

cudaError_t launch_batch_i16x2(const BatchArgs &a, int lanes, int rows, int grid, cudaStream_t s, int priority) {
    switch (lanes * 100 + rows) {
        case 816: return launch_tr<8, 16>(a, grid, s, priority);
        case 824: return launch_tr<8, 24>(a, grid, s, priority);
        case 832: return launch_tr<8, 32>(a, grid, s, priority);
        case 1624: return launch_tr<16, 24>(a, grid, s, priority);
        case 1616: return launch_tr<16, 16>(a, grid, s, priority);
        case 1632: return launch_tr<16, 32>(a, grid, s, priority);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swdb
