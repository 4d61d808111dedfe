// Exact int32 Smith-Waterman/Gotoh scoring of selected database sequences.
//
// Same recurrences as the int16x2 kernel (Section 2.2; affine gaps as in
// Section 4.1), one database sequence per subwarp, in 32-bit DPX
// arithmetic.  It serves two roles:
//   * rescoring the sequences whose int16 maximum reached the saturation
//     limit (their int16 result may have overflowed), and
//   * the int32-throughout path, when the matrix or penalties do not fit
//     the int16 kernel's ranges.
// Subwarps work independently: each takes the next (pair, mask) item from
// an atomic counter and scores the masked halves one after another.  The
// query profile is a global int32 table [residue][row] built once per
// query (it stays in L2); lane k reads its R rows for the current column's
// residue with 128-bit loads.
#include "swdb_internal.cuh"

namespace swdb {
namespace {

struct Prof32Args {
    const uint8_t *query;
    int32_t m, m_pad, A, gap_open;
    int32_t matrix[kProfRows * kProfRows];
    int32_t *prof32;
};

// prof32[a*m_pad + i] = S(q_i, a) + o for i < m and a < A; a large negative
// value elsewhere (query padding rows, residue codes outside the alphabet,
// the padding code).
__global__ void k_profile32(const __grid_constant__ Prof32Args p) {
    const int64_t total = int64_t(kProfRows) * p.m_pad;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int res = int(idx / p.m_pad);
        const int i = int(idx % p.m_pad);
        int v = -(1 << 28);
        if (i < p.m && res < p.A) {
            const int qc = p.query[i];
            if (qc < p.A) v = p.matrix[qc * kProfRows + res] + p.gap_open;
        }
        p.prof32[idx] = v;
    }
}

template <int T, int R>
__device__ void score_one(const I32Args &a, int64_t pair, int h, int k, uint32_t submask) {
    constexpr int TR = T * R;
    const int64_t t = 2 * pair + h;
    const int64_t orig = a.db.perm[t];
    if (orig < 0) return;                       // padding slot
    const int n = a.db.len[t];
    const int o = a.gap_open;
    const int ge = a.gap_extend;
    const int gmin = ge < o ? ge : o;
    if (n == 0 || a.m == 0) {
        if (k == 0) a.scores[orig] = 0;
        return;
    }
    const int64_t b = pair / kBundlePairs;
    const int slot = int(pair % kBundlePairs);
    const int64_t off = a.db.bundle_off[b];
    const uint2 *cptr = reinterpret_cast<const uint2 *>(a.db.codes + off) + slot;
    uint2 *bnd = a.boundary + off / 2 + slot;
    const int npass = (a.m + TR - 1) / TR;
    int mx = -o;

    for (int pass = 0; pass < npass; ++pass) {
        int E[R], Ho[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { E[r] = -o; Ho[r] = -o; }
        int hd = -o;
        int pub_h = -o, pub_f = -o, pub_c = 0;
        uint2 quad = make_uint2(0, 0);
        const bool last_pass = (pass + 1 == npass);
        const int32_t *prow = a.prof32 + pass * TR + k * R;
        const int steps = n + T - 1;
        for (int s = 0; s < steps; ++s) {
            int hin = __shfl_up_sync(submask, pub_h, 1, T);
            int fin = __shfl_up_sync(submask, pub_f, 1, T);
            int cin = __shfl_up_sync(submask, pub_c, 1, T);
            const int j = s - k;
            const bool act = (j >= 0) && (j < n);
            if (k == 0 && act) {
                if ((s & 3) == 0) quad = __ldg(cptr + (s >> 2) * kBundlePairs);
                const uint32_t w = (s & 2) ? quad.y : quad.x;
                cin = int((w >> (16 * (s & 1) + 8 * h)) & 0xffu);
                if (pass == 0) {
                    hin = -o;
                    fin = -o;
                } else {
                    const uint2 bv = bnd[size_t(s) * kBundlePairs];
                    hin = int(bv.x);
                    fin = int(bv.y);
                }
            }
            if (act) {
                const int4 *pp = reinterpret_cast<const int4 *>(prow + size_t(cin) * a.m_pad);
                int P[R];
#pragma unroll
                for (int v = 0; v < R / 4; ++v) {
                    const int4 x = __ldg(pp + v);
                    P[4 * v + 0] = x.x; P[4 * v + 1] = x.y; P[4 * v + 2] = x.z; P[4 * v + 3] = x.w;
                }
                int f = __viaddmax_s32(fin, -ge, hin);
                int d = hd;
                int xo_prev = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e_r = __viaddmax_s32(E[r], -ge, Ho[r]);
                    const int x = __viaddmax_s32_relu(d, P[r], e_r);
                    if (r > 0) f = __viaddmax_s32(f, -gmin, xo_prev);
                    const int xo = x - o;
                    const int ho = __viaddmax_s32(f, -o, xo);
                    d = Ho[r];
                    E[r] = e_r;
                    Ho[r] = ho;
                    xo_prev = xo;
                }
#pragma unroll
                for (int r = 0; r < R; r += 2) mx = __vimax3_s32(mx, Ho[r], Ho[r + 1]);
                hd = hin;
                pub_h = Ho[R - 1];
                pub_f = f;
                pub_c = cin;
                if (k == T - 1 && !last_pass)
                    bnd[size_t(j) * kBundlePairs] = make_uint2(uint32_t(Ho[R - 1]), uint32_t(f));
            }
        }
        // Lane T-1's boundary writes must be visible to lane 0 in the next pass.
        __syncwarp(submask);
    }
#pragma unroll
    for (int dd = T / 2; dd >= 1; dd >>= 1) mx = max(mx, __shfl_xor_sync(submask, mx, dd, T));
    if (k == 0) a.scores[orig] = mx + o;
}

template <int T, int R>
__global__ void __launch_bounds__(kCtaThreads) k_i32(const __grid_constant__ I32Args a) {
    const int tid = threadIdx.x;
    const int k = tid % T;
    const int lane = tid & 31;
    const uint32_t submask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane - k));
    const int64_t count = a.list ? int64_t(*a.list_count) : (a.pair_end - a.pair_begin);
    if (count <= 0) return;
    for (;;) {
        int item = 0;
        if (k == 0) item = atomicAdd(a.work_counter, 1);
        item = __shfl_sync(submask, item, 0, T);
        if (item >= count) break;
        int64_t pair;
        int mask;
        if (a.list) {
            const int32_t e = a.list[item];
            pair = e >> 2;
            mask = e & 3;
        } else {
            pair = a.pair_begin + item;
            mask = 3;
        }
        if (mask & 1) score_one<T, R>(a, pair, 0, k, submask);
        if (mask & 2) score_one<T, R>(a, pair, 1, k, submask);
    }
}

template <int T, int R>
cudaError_t launch_tr(const I32Args &a, int grid, cudaStream_t s) {
    k_i32<T, R><<<grid, kCtaThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool i32_config_supported(int lanes, int rows) {
    switch (lanes * 100 + rows) {
        case 816: case 1616: case 3216: case 3232: return true;
        default: return false;
    }
}

cudaError_t launch_i32(const I32Args &a, int lanes, int rows, int grid, cudaStream_t s) {
    switch (lanes * 100 + rows) {
        case 816: return launch_tr<8, 16>(a, grid, s);
        case 1616: return launch_tr<16, 16>(a, grid, s);
        case 3216: return launch_tr<32, 16>(a, grid, s);
        case 3232: return launch_tr<32, 32>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_profile32(const uint8_t *query, int32_t m, int32_t m_pad, const int32_t *matrix_host,
                             int32_t A, int32_t gap_open, int32_t *prof32, cudaStream_t s) {
    Prof32Args p;
    p.query = query;
    p.m = m;
    p.m_pad = m_pad;
    p.A = A;
    p.gap_open = gap_open;
    for (int i = 0; i < kProfRows * kProfRows; ++i) p.matrix[i] = 0;
    for (int x = 0; x < A; ++x)
        for (int y = 0; y < A; ++y) p.matrix[x * kProfRows + y] = matrix_host[x * A + y];
    p.prof32 = prof32;
    const int64_t total = int64_t(kProfRows) * m_pad;
    int grid = int((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    k_profile32<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace swdb
