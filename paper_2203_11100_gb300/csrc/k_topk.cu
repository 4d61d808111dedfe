// Per-query top-k of a score row: the k best database entries, ordered by
// score descending and then database index ascending (the paper does not
// say how ties are ordered; this order is the library's convention).
//
// Scores are signed (the non-local alignment modes give negative ones); the
// kernel orders the keys v = score XOR 0x80000000 as unsigned, which keeps
// the order of signed values.
//
// One CTA per row.  (1) A radix select over the 32-bit keys, 8 bits per
// round, finds the k-th largest score tau and how many ties with tau are
// needed.  (2) One ordered sweep over the row collects every score > tau
// (any order) and the first `need` entries equal to tau in index order
// (a block-wide prefix count keeps the index order).  (3) A bitonic sort of
// 64-bit keys (score << 32 | ~index) in shared memory puts them in order.
#include "swdb_internal.cuh"

namespace swdb {
namespace {

constexpr int kTopkThreads = 1024;
constexpr int kTopkMax = 4096;

struct Hit {
    int32_t score;
    int32_t reserved;
    int64_t db_index;
};

__global__ void __launch_bounds__(kTopkThreads) k_topk(const int32_t *scores, int64_t n_cols, int32_t k,
                                                     Hit *hits) {
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long keys[kTopkMax];
    __shared__ uint32_t warp_cnt[kTopkThreads / 32];
    __shared__ uint32_t sh_sel, sh_above;
    __shared__ uint32_t cnt_gt;
    __shared__ uint32_t eq_taken;

    const int tid = threadIdx.x;
    const int64_t row = blockIdx.x;
    const int32_t *s = scores + row * n_cols;
    Hit *out = hits + row * int64_t(k);
    const int kk = int(n_cols < int64_t(k) ? n_cols : int64_t(k));  // entries that exist

    int P = 1;
    while (P < kk) P <<= 1;
    for (int i = tid; i < P; i += kTopkThreads) keys[i] = 0ull;

    // (1) radix select of the kk-th largest key.
    uint32_t prefix = 0, pmask = 0;
    uint32_t remaining = uint32_t(kk);
    bool take_all = (int64_t(kk) == n_cols);
    if (!take_all && kk > 0) {
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += kTopkThreads) hist[i] = 0;
            __syncthreads();
            for (int64_t i = tid; i < n_cols; i += kTopkThreads) {
                const uint32_t v = uint32_t(s[i]) ^ 0x80000000u;
                if ((v & pmask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t cum = 0;
                int sel = 0;
                for (int bin = 255; bin >= 0; --bin) {
                    if (cum + hist[bin] >= remaining) { sel = bin; break; }
                    cum += hist[bin];
                }
                sh_sel = uint32_t(sel);
                sh_above = cum;
            }
            __syncthreads();
            remaining -= sh_above;
            prefix |= sh_sel << shift;
            pmask |= 255u << shift;
            __syncthreads();
        }
    }
    const uint32_t tau = prefix;
    const uint32_t need = remaining;          // ties with tau to take
    const uint32_t n_gt = uint32_t(kk) - need;

    if (tid == 0) { cnt_gt = 0; eq_taken = 0; }
    __syncthreads();

    // (2) ordered collection.
    if (kk > 0) {
        for (int64_t base = 0; base < n_cols; base += kTopkThreads) {
            const int64_t i = base + tid;
            uint32_t v = 0;
            bool in = i < n_cols;
            if (in) v = uint32_t(s[i]) ^ 0x80000000u;
            const unsigned long long key =
                (static_cast<unsigned long long>(v) << 32) | (0xffffffffull - uint64_t(i));
            bool is_eq = false;
            if (in) {
                if (take_all) {
                    keys[i] = key;
                } else if (v > tau) {
                    const uint32_t pos = atomicAdd(&cnt_gt, 1u);
                    keys[pos] = key;
                } else if (v == tau) {
                    is_eq = true;
                }
            }
            if (take_all) continue;
            const unsigned ballot = __ballot_sync(0xffffffffu, is_eq);
            if ((tid & 31) == 0) warp_cnt[tid >> 5] = __popc(ballot);
            __syncthreads();
            uint32_t before = 0;
            for (int w = 0; w < (tid >> 5); ++w) before += warp_cnt[w];
            before += __popc(ballot & ((1u << (tid & 31)) - 1u));
            const uint32_t taken = eq_taken;
            if (is_eq && taken + before < need) keys[n_gt + taken + before] = key;
            __syncthreads();
            if (tid == 0) {
                uint32_t tot = 0;
                for (int w = 0; w < kTopkThreads / 32; ++w) tot += warp_cnt[w];
                eq_taken = taken + tot;
            }
            __syncthreads();
        }
    }
    __syncthreads();

    // (3) bitonic sort, descending.
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P; i += kTopkThreads) {
                const int partner = i ^ stride;
                if (partner > i) {
                    const bool desc = ((i & size) == 0);
                    const unsigned long long x = keys[i], y = keys[partner];
                    if (desc ? (x < y) : (x > y)) { keys[i] = y; keys[partner] = x; }
                }
            }
            __syncthreads();
        }
    }

    for (int i = tid; i < k; i += kTopkThreads) {
        Hit h;
        h.reserved = 0;
        if (i < kk) {
            const unsigned long long key = keys[i];
            h.score = int32_t(uint32_t(key >> 32) ^ 0x80000000u);
            h.db_index = int64_t(0xffffffffull - (key & 0xffffffffull));
        } else {
            h.score = -1;
            h.db_index = -1;
        }
        out[i] = h;
    }
}

}  // namespace

cudaError_t launch_topk(const int32_t *scores, int64_t n_rows, int64_t n_cols, int32_t k, void *hits,
                        cudaStream_t s) {
    if (n_rows <= 0 || k <= 0) return cudaSuccess;
    if (k > kTopkMax) return cudaErrorInvalidValue;
    k_topk<<<unsigned(n_rows), kTopkThreads, 0, s>>>(scores, n_cols, k, static_cast<Hit *>(hits));
    return cudaGetLastError();
}

}  // namespace swdb
