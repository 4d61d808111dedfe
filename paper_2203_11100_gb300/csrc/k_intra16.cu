// Intra-task Smith-Waterman/Gotoh scoring of long database sequences.
//
// Section 2.2 (intra-task parallelism: all processing elements work on one
// alignment matrix and exchange border elements) and Section 2.3 (SW#db
// uses it for long sequences; "solveLong" in Section 3.2).  This kernel is
// this library's own design for sm_103a:
//
// * A pipeline of NW warps scores one PAIR of long database sequences
//   (packed int16x2, as in the inter-task kernel: the database is sorted, so
//   the two sequences of a pair have similar lengths).  A CTA runs P such
//   pipelines on P consecutive pairs.
// * The warps of a pipeline split the query: in each super-pass of NW*32*R
//   rows, warp w owns rows [w*32*R, (w+1)*32*R) and its 32 lanes own R rows
//   each.  Warp w of every pipeline reads the same profile slice, so the
//   CTA's shared memory holds NW slices for P pairs (the profile is 32 bytes
//   per query row, and shared memory, not registers, bounds occupancy here).
//   Inside a warp the lanes form the same skewed wavefront as the inter-task
//   kernel (lane k works on column j one step after lane k-1; H/F/codes move
//   lane to lane by shuffle).
// * Between warps of a pipeline the bottom row of warp w (H-o and F per
//   column) goes to warp w+1 through a shared-memory ring of D chunks of C
//   columns: a bounded producer/consumer pipeline with acquire/release
//   flags, so the warps advance as a wavefront of their own.  Between
//   super-passes the last warp's bottom row goes through global scratch
//   (one contiguous row per pair, staged back with cp.async) and a CTA
//   barrier.
// * Steady columns (every lane inside the sequence) run in groups of four
//   with no per-column bookkeeping: lane 0's inputs (the column's codes and
//   the boundary value from the ring, the staging buffer or the top row) are
//   read by every lane as one broadcast load and taken by lane 0 with a
//   select, the ring's waits and releases happen in the fixed groups where a
//   chunk starts or ends, and the input and output addresses advance once
//   per group.  The first 32 columns (lanes starting) and the last ones
//   (lanes finishing, a partly filled chunk) take a general per-column path.
// * Every wait is bounded: if a flag does not arrive within the spin limit
//   the kernel records SW_ERR_TIMEOUT in a status word, tells the other
//   warps to stop waiting, and finishes without hanging.
// Per cell pair the arithmetic is the same biased-domain sequence as the
// inter-task kernel (four DPX operations, one 32-bit subtraction, one byte
// permute and half a running max; see k_inter16.cu for the derivation).
#include <type_traits>

#include "simd16.cuh"
#include "swdb_internal.cuh"

namespace swdb {
namespace {

constexpr int kChunk = 64;      // columns per ring chunk
constexpr int kDepth = 4;       // chunks per ring
constexpr long long kSpinLimit = 1ll << 25;   // x ~32 ns sleep: about a second

using simd16::cp_async16;
using simd16::cp_async_commit;
using simd16::cp_async_wait1;
using simd16::pack2;
using simd16::pair_sel;
using simd16::prmt;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" :: "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Spin (all lanes of a warp) until *flag >= target, the CTA aborts, or the
// spin limit runs out (then record a timeout and abort the CTA).
__device__ bool wait_flag(const int *flag, int target, int *abort_flag, int32_t *status,
                          long long limit = kSpinLimit) {
    for (long long it = 0; it < limit; ++it) {
        if (ld_acquire(flag) >= target) return true;
        if (*reinterpret_cast<volatile int *>(abort_flag)) return false;
        __nanosleep(32);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicExch(status, int32_t(4));   // SW_ERR_TIMEOUT
        *reinterpret_cast<volatile int *>(abort_flag) = 1;
    }
    __syncwarp();
    return false;
}

template <int R, int NW, int P>
__global__ void __launch_bounds__(NW * P * 32, 2) k_intra_i16x2(const __grid_constant__ IntraArgs a) {
    static_assert(R % 8 == 0, "rows per lane must be a multiple of 8");
    constexpr int T = 32;
    constexpr int TR = T * R;
    constexpr int SPR = NW * TR;
    constexpr int C = kChunk;
    constexpr int D = kDepth;
    constexpr int NT = NW * P * 32;
    constexpr int SLOT = T * 16 * ((R + 15) / 16);                             // bytes per residue (16-row groups)
    constexpr int SLICE = kProfRows * SLOT;                                    // bytes per profile slice
    extern __shared__ __align__(16) uint8_t smem[];
    int8_t *prof_all = reinterpret_cast<int8_t *>(smem);                      // [NW][32][SLOT]
    uint2 *ring_all = reinterpret_cast<uint2 *>(smem + NW * SLICE);           // [P][NW][D*C], link into warp w
    uint2 *stage_all = ring_all + P * NW * D * C;                             // [P][8] boundary staging
    int8_t *mat = reinterpret_cast<int8_t *>(stage_all + P * 8);              // [32*32]
    int *full = reinterpret_cast<int *>(mat + kProfRows * kProfRows);         // [P][NW] chunks written into link w
    int *empty = full + P * NW;                                               // [P][NW] chunks read from link w
    int *abort_flag = empty + P * NW;
    __shared__ uint32_t red[P * NW];
    __shared__ uint2 top4[4];          // the top row's inputs B(H-o), B(F) = B(-o), for broadcast reads

    const int warp = threadIdx.x >> 5;
    const int pl = warp / NW;          // pipeline (pair) within the CTA
    const int w = warp % NW;           // warp within the pipeline
    const int k = threadIdx.x & 31;
    // Pair-major order: the longest pair groups of every query are dispatched first.
    const int64_t group = blockIdx.x / a.n_q;
    const int q = int(blockIdx.x % a.n_q);
    const int64_t q0 = a.q_off[q];
    const int m = int(a.q_off[q + 1] - q0);
    if (m == 0) return;   // the host writes zero scores for empty queries
    const uint8_t *query = a.queries + q0;
    int32_t *scores = a.scores + int64_t(q) * a.db.n_seqs;
    int32_t *ovf_list = a.ovf_list + int64_t(q) * a.list_stride;

    // staged transposed, [db code][query code]: the profile fill reads one db code
    // against many query codes at once, which then fall in distinct banks
    for (int i = threadIdx.x; i < kProfRows * kProfRows; i += NT)
        mat[(i % kProfRows) * kProfRows + i / kProfRows] = (&a.prof8[0][0])[i];
    if (threadIdx.x < P * NW) {
        full[threadIdx.x] = 0;
        empty[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) *abort_flag = 0;
    if (threadIdx.x < 4) top4[threadIdx.x] = make_uint2(pack2(32768 - a.gap_open), pack2(32768 - a.gap_open));

    const int64_t pair = a.pair_begin + group * P + pl;
    const bool valid = pair < a.pair_end;
    int Lp = 0;
    const uint2 *cptr = nullptr;
    uint2 *gbnd2 = nullptr;              // this pair's global boundary row, one entry per column
    if (valid) {
        const int64_t b = pair / kBundlePairs;
        const int slot = int(pair % kBundlePairs);
        Lp = (a.db.len[2 * pair] + 3) & ~3;
        const int64_t off = a.db.bundle_off[b];
        cptr = reinterpret_cast<const uint2 *>(a.db.codes + off) + slot;
        // the bundle's region holds 8 * bundle_len entries: pair slot s owns
        // [s * bundle_len, (s + 1) * bundle_len)
        if (a.boundary)
            gbnd2 = a.boundary + int64_t(q) * a.boundary_stride + off / 2 + int64_t(slot) * a.db.bundle_len[b];
    }

    const int o = a.gap_open;
    const uint32_t BNEG_O2 = pack2(32768 - o);
    const uint32_t ADD_NEG_E = pack2(-a.gap_extend);
    const uint32_t OO = uint32_t(o) | (uint32_t(o) << 16);
    const uint32_t BZERO2 = 0x80008000u;

    const int8_t *prof = prof_all + w * SLICE;
    uint2 *ring_in = ring_all + (pl * NW + w) * D * C;
    uint2 *ring_out = ring_all + (pl * NW + (w + 1) % NW) * D * C;
    int *full_in = &full[pl * NW + w];
    int *empty_in = &empty[pl * NW + w];
    int *full_out = &full[pl * NW + (w + 1) % NW];
    int *empty_out = &empty[pl * NW + (w + 1) % NW];
    uint2 *stg = stage_all + pl * 8;

    const int nsp = (m + SPR - 1) / SPR;
    uint32_t mx = BZERO2;      // running max of B(H)
    int g_in = 0, g_out = 0;   // chunk sequence numbers on the incoming / outgoing link

    for (int sp = 0; sp < nsp; ++sp) {
        __syncthreads();
        // All NW profile slices of this super-pass.  Within a slice the layout is
        // [residue a][16-row group h][lane k][16 rows]: lane k's rows 16h..16h+15 sit
        // at a*SLOT + h*32*16 + k*16 (quarter-warp lanes read consecutive 16-byte
        // slots); with R = 8 a lane's one group fills half its slot.
        for (int wi = threadIdx.x; wi < NW * kProfRows * TR / 4; wi += NT) {
            const int slice = wi / (kProfRows * TR / 4);
            const int e0 = (wi % (kProfRows * TR / 4)) * 4;
            const int res = e0 / TR;
            const int within = e0 % TR;                 // kk * R + r
            const int kk = within / R, rl = within % R;
            const int phys = slice * SLICE + res * SLOT + (rl >> 4) * (T * 16) + kk * 16 + (rl & 15);
            const int rr = sp * SPR + slice * TR + within;
            uint32_t word = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int row = rr + c;
                int v = -128;
                if (row < m) {
                    const int qc = query[row];
                    if (qc < kProfRows) v = mat[res * kProfRows + qc];
                }
                word |= (uint32_t(uint8_t(int8_t(v)))) << (8 * c);
            }
            reinterpret_cast<uint32_t *>(prof_all)[phys / 4] = word;
        }
        __syncthreads();
        const int row0 = sp * SPR + w * TR;
        if (row0 >= m || Lp == 0) continue;
        const bool from_ring = w > 0;
        const bool to_ring = (w + 1 < NW) && (row0 + TR < m);
        const bool from_global = (w == 0) && sp > 0;
        const bool to_global = !to_ring && (sp + 1 < nsp);

        uint32_t E[R], Ho[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { E[r] = BNEG_O2; Ho[r] = BNEG_O2; }
        uint32_t hd = BNEG_O2;
        // pub_h: B(Ho) of this lane's bottom row; pub_f: B(F) of the next lane's top row
        uint32_t pub_h = BNEG_O2, pub_f = BNEG_O2, pub_c = 0;
        uint2 quad = make_uint2(0, 0), quad_next = make_uint2(0, 0);
        const uint4 *gsrc = reinterpret_cast<const uint4 *>(gbnd2);   // 2 uint4 per 4 columns
        quad_next = __ldg(cptr);         // every lane: one broadcast load
        if (k == 0 && from_global) {
            cp_async16(stg + 0, gsrc);
            cp_async16(stg + 2, gsrc + 1);
            cp_async_commit();
            if (4 < Lp) {
                cp_async16(stg + 4, gsrc + 2);
                cp_async16(stg + 6, gsrc + 3);
            }
            cp_async_commit();
        }
        const int steps = Lp + T - 1;

        // The cell work of one column step for this lane's R rows, given the
        // top-row inputs (hin, fin) and the column's residue codes cin.
        auto cells = [&](const uint32_t hin, const uint32_t fin, const uint32_t cin) {
            const int ta = int(cin & 0xffu), tb = int((cin >> 8) & 0xffu);
            const uint4 *pa = reinterpret_cast<const uint4 *>(prof + ta * SLOT + k * 16);
            const uint4 *pb = reinterpret_cast<const uint4 *>(prof + tb * SLOT + k * 16);
            uint32_t wa[R / 4], wb[R / 4];
#pragma unroll
            for (int v = 0; v < R / 16; ++v) {
                const uint4 x = pa[v * T];
                const uint4 y = pb[v * T];
                wa[4 * v + 0] = x.x; wa[4 * v + 1] = x.y; wa[4 * v + 2] = x.z; wa[4 * v + 3] = x.w;
                wb[4 * v + 0] = y.x; wb[4 * v + 1] = y.y; wb[4 * v + 2] = y.z; wb[4 * v + 3] = y.w;
            }
            if (R % 16) {                     // last group of 8 rows: an 8-byte load
                const uint2 x = *reinterpret_cast<const uint2 *>(pa + (R / 16) * T);
                const uint2 y = *reinterpret_cast<const uint2 *>(pb + (R / 16) * T);
                wa[R / 4 - 2] = x.x; wa[R / 4 - 1] = x.y;
                wb[R / 4 - 2] = y.x; wb[R / 4 - 1] = y.y;
            }
            uint32_t f = fin;
            uint32_t d = hd;
            uint32_t yprev = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t pr = prmt(wa[r / 4], wb[r / 4], pair_sel(r % 4));
                const uint32_t e_r = __viaddmax_u16x2(E[r], ADD_NEG_E, Ho[r]);
                const uint32_t x = __viaddmax_u16x2(d, pr, e_r);
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
            pub_h = Ho[R - 1];
            pub_f = f;
            pub_c = cin;
        };

        // One column step with every check (lanes starting or finishing, a
        // chunk boundary at any column): the ramp and the tail.
        auto step = [&](const int s) {
            const int j31 = s - (T - 1);
            // Flow control (warp-uniform): wait for the producer's chunk before
            // lane 0 enters it, and for ring space before lane 31 starts writing one.
            if (from_ring && s < Lp && (s % C) == 0) wait_flag(full_in, g_in + 1, abort_flag, a.status);
            if (to_ring && j31 >= 0 && (j31 % C) == 0) wait_flag(empty_out, g_out - D + 1, abort_flag, a.status);

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
                    if (from_global) cp_async_wait1();
                }
                const uint32_t wd = (s3 & 2) ? quad.y : quad.x;
                cin = (s3 & 1) ? (wd >> 16) : (wd & 0xffffu);
                if (from_ring) {
                    const uint2 v = ring_in[(g_in % D) * C + (s % C)];
                    hin = v.x;
                    fin = v.y;
                } else if (from_global) {
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
                } else {                  // H(0,j) = 0, F(1,j) = -o
                    hin = BNEG_O2;
                    fin = BNEG_O2;
                }
            }
            if (act) {
                cells(hin, fin, cin);
                if (k == T - 1) {
                    if (to_ring)
                        ring_out[(g_out % D) * C + (j31 % C)] = make_uint2(pub_h, pub_f);
                    else if (to_global)
                        gbnd2[j31] = make_uint2(pub_h, pub_f);
                }
            }
            // Release a consumed chunk (lane 0 has used its last column) and
            // publish a produced one (lane 31 wrote its last column).
            if (from_ring && s < Lp && ((s % C) == C - 1 || s == Lp - 1)) {
                if (k == 0) st_release(empty_in, g_in + 1);
                ++g_in;
            }
            if (to_ring && j31 >= 0 && j31 < Lp && ((j31 % C) == C - 1 || j31 == Lp - 1)) {
                __syncwarp();
                if (k == T - 1) st_release(full_out, g_out + 1);
                ++g_out;
            }
        };

        // One steady column step (every lane inside the sequence), U = s % 4:
        // lane 0 takes its inputs from the broadcast loads ib[U] (boundary
        // value) and quad (codes); lane 31 writes its bottom row to ob[U].
        auto sstep = [&](const uint2 *ib, uint2 *ob, auto u_c) {
            constexpr int U = decltype(u_c)::value;
            uint32_t hin = __shfl_up_sync(0xffffffffu, pub_h, 1, T);
            uint32_t fin = __shfl_up_sync(0xffffffffu, pub_f, 1, T);
            uint32_t cin = __shfl_up_sync(0xffffffffu, pub_c, 1, T);
            const uint2 v = ib[U];
            const uint32_t wd = (U & 2) ? quad.y : quad.x;
            const uint32_t c0 = (U & 1) ? (wd >> 16) : (wd & 0xffffu);
            const bool lane0 = k == 0;
            hin = lane0 ? v.x : hin;
            fin = lane0 ? v.y : fin;
            cin = lane0 ? c0 : cin;
            cells(hin, fin, cin);
            if (ob != nullptr && k == T - 1) ob[U] = make_uint2(pub_h, pub_f);
        };
        using U0 = std::integral_constant<int, 0>;
        using U1 = std::integral_constant<int, 1>;
        using U2 = std::integral_constant<int, 2>;
        using U3 = std::integral_constant<int, 3>;

        int s = 0;
        for (; s < T && s < steps; ++s) step(s);
        // Steady groups of four columns: s % 4 == 0, s >= 32 (lane 31 started),
        // s + 3 < Lp (lane 0 inside).  A ring chunk starts at s % 64 == 0 (wait
        // for it) and ends at s % 64 == 63 or at the last column (release it);
        // lane 31, 31 columns behind, ends an output chunk at s % 64 == 30
        // (publish it) and starts the next at s % 64 == 31 (wait for space):
        // both fall in the group at s % 64 == 28.  Lane 31's last partial chunk
        // ends at s = Lp + 30, in the tail.
        for (; s + 3 < Lp; s += 4) {
            const int g64 = s & (C - 1);
            const uint2 *ib;
            if (from_ring) {
                if (g64 == 0) wait_flag(full_in, g_in + 1, abort_flag, a.status);
                ib = ring_in + (g_in % D) * C + g64;
            } else if (from_global) {
                cp_async_wait1();                            // the group for columns s..s+3 has landed
                ib = stg + ((s >> 2) & 1) * 4;
            } else {
                ib = top4;
            }
            quad = quad_next;
            if (s + 4 < Lp) quad_next = __ldg(cptr + ((s >> 2) + 1) * kBundlePairs);
            uint2 *ob = nullptr;
            if (to_ring) ob = ring_out + (g_out % D) * C + ((g64 - (T - 1)) & (C - 1));
            else if (to_global) ob = gbnd2 + (s - (T - 1));
            sstep(ib, ob, U0());
            sstep(ib, ob, U1());
            sstep(ib, ob, U2());
            if (to_ring && g64 == 28) {
                __syncwarp();
                if (k == T - 1) st_release(full_out, g_out + 1);
                ++g_out;
                wait_flag(empty_out, g_out - D + 1, abort_flag, a.status);
                ob = ring_out + (g_out % D) * C - 3;         // ob[3]: column 0 of the new chunk
            }
            sstep(ib, ob, U3());
            if (from_global) {
                if (k == 0 && s + 5 < Lp) {
                    const uint4 *g = gsrc + size_t((s >> 2) + 2) * 2;
                    cp_async16(stg + ((s >> 2) & 1) * 4, g);
                    cp_async16(stg + ((s >> 2) & 1) * 4 + 2, g + 1);
                }
                cp_async_commit();
            }
            // lane 0 has used the chunk's last column (s % 64 == 63, or the
            // sequence's last column: Lp is a multiple of 4, so the last steady
            // group ends the sequence when Lp >= 36)
            if (from_ring && (g64 == C - 4 || s + 4 == Lp)) {
                if (k == 0) st_release(empty_in, g_in + 1);
                ++g_in;
            }
        }
        for (; s < steps; ++s) step(s);
    }

#pragma unroll
    for (int dd = 16; dd >= 1; dd >>= 1) {
        const uint32_t other = __shfl_xor_sync(0xffffffffu, mx, dd);
        mx = __vimax3_u16x2(mx, other, other);
    }
    if (k == 0) red[warp] = mx;
    __syncthreads();
    if (valid && w == 0 && k == 0) {
#pragma unroll
        for (int i = 1; i < NW; ++i) mx = __vimax3_u16x2(mx, red[pl * NW + i], red[pl * NW + i]);
        const int hA = int(mx & 0xffffu) - 32768;
        const int hB = int(mx >> 16) - 32768;
        const int64_t tA = 2 * pair;
        int mask = 0;
        const int64_t oA = a.db.perm[tA];
        const int64_t oB = a.db.perm[tA + 1];
        if (oA >= 0) {
            if (hA >= a.sat_limit) mask |= 1;
            else scores[oA] = hA;
        }
        if (oB >= 0) {
            if (hB >= a.sat_limit) mask |= 2;
            else scores[oB] = hB;
        }
        if (mask) {
            const int idx = atomicAdd(a.ovf_count + q, 1);
            ovf_list[idx] = int32_t(pair * 4 + mask);
            atomicAdd(a.ovf_seqs + q, __popc(mask));
        }
    }
}

// Self-test of the bounded wait: one warp waits on a shared-memory flag that
// nothing sets, with the given spin limit, and must give up and record
// SW_ERR_TIMEOUT in *status rather than hang.
__global__ void k_wait_probe(long long limit, int32_t *status) {
    __shared__ int flag, abort_flag;
    if (threadIdx.x == 0) {
        flag = 0;
        abort_flag = 0;
    }
    __syncthreads();
    wait_flag(&flag, 1, &abort_flag, status, limit);
}

template <int R, int NW, int P>
size_t intra_smem() {
    return size_t(NW) * kProfRows * 32 * 16 * ((R + 15) / 16) + size_t(P) * NW * kDepth * kChunk * sizeof(uint2) +
           size_t(P) * 8 * sizeof(uint2) + kProfRows * kProfRows + sizeof(int) * (2 * P * NW + 1);
}

template <int R, int NW, int P>
cudaError_t launch_rnp(const IntraArgs &a, cudaStream_t s) {
    const int64_t pairs = a.pair_end - a.pair_begin;
    if (pairs <= 0 || a.n_q <= 0) return cudaSuccess;
    const int64_t groups = (pairs + P - 1) / P;
    const int64_t grid = groups * a.n_q;
    if (grid >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    const size_t smem = intra_smem<R, NW, P>();   // attribute set by prepare_intra_i16x2 at planning
    k_intra_i16x2<R, NW, P><<<unsigned(grid), NW * P * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int R, int NW, int P>
cudaError_t prepare_rnp() {
    return cudaFuncSetAttribute(k_intra_i16x2<R, NW, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(intra_smem<R, NW, P>()));
}

}  // namespace

// Shapes: warps per pipeline (NW) and rows per lane (R); pipelines per CTA (P)
// follow: (4 warps, 8 rows) x 3 pipelines (1,024-row super-passes, the
// shortest column step), (4 warps, 16 rows) x 3 pipelines, (2 warps, 32 rows)
// x 4 pipelines (2,048-row super-passes).
bool intra_config_supported(int warps, int rows) {
    return (warps == 4 && rows == 8) || (warps == 4 && rows == 16) || (warps == 2 && rows == 32);
}

int intra_rows_per_superpass(int warps, int rows) { return warps * 32 * rows; }

cudaError_t launch_wait_probe(long long limit, int32_t *status, cudaStream_t s) {
    if (limit < 1 || limit > kSpinLimit) return cudaErrorInvalidValue;
    k_wait_probe<<<1, 32, 0, s>>>(limit, status);
    return cudaGetLastError();
}

cudaError_t prepare_intra_i16x2(int warps, int rows) {
    if (rows == 8 && warps == 4) return prepare_rnp<8, 4, 3>();
    if (rows == 16 && warps == 4) return prepare_rnp<16, 4, 3>();
    if (rows == 32 && warps == 2) return prepare_rnp<32, 2, 4>();
    return cudaErrorInvalidValue;
}

cudaError_t launch_intra_i16x2(const IntraArgs &a, int warps, int rows, cudaStream_t s) {
    if (rows == 8 && warps == 4) return launch_rnp<8, 4, 3>(a, s);
    if (rows == 16 && warps == 4) return launch_rnp<16, 4, 3>(a, s);
    if (rows == 32 && warps == 2) return launch_rnp<32, 2, 4>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace swdb
