// sw_search_no_alloc: one query against a loaded database with no device
// allocation at call time.
//
// Some callers cannot allocate device memory when they search: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc and
// cudaFree are not allowed to appear there), serving loops that must not
// touch the allocator after start-up (an allocation can synchronise the
// device and stall every stream, and its latency is unbounded), and hosts
// whose device memory is all handed out by a framework's own pool.  For
// them this entry point runs the same kernels as sw_search (the int16x2
// inter-task kernel, then an exact int32 rescore of saturated sequences),
// but takes its scratch (overflow list and counters, the int32 query
// profile, and the strip-boundary rows of multi-pass queries) from one
// fixed array in device memory that the library owns.  The caller passes
// the query and the score row as device buffers.
//
// The array is a file-scope __device__ variable of SW_NO_ALLOC_SCRATCH_BYTES
// bytes: every GPU that loads this part of the library holds it until the
// process exits.  Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the first call on each
// device looks the address up with cudaGetSymbolAddress while that device is
// current, checks the result and caches it; that first call should come
// before any stream capture.  The cached address belongs to the CUDA context
// it was looked up in: if that context is destroyed and another one created
// (cudaDeviceReset, say), the module is loaded again and the array may move,
// so the cache is keyed by the context's unique id as well and the lookup is
// repeated in a new context.  All calls share the array and it keeps the
// previous call's contents: the counters that must start at zero are cleared
// on the stream at the start of every call, and calls whose work overlaps on
// the GPU (on different streams, or from several threads) race on it.
#include <mutex>

#include "../../include/swdb.h"
#include "swdb_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(SW_NO_ALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;
constexpr int kLanes = 8, kRows = 16;   // launch shape of both kernels here

static __device__ __align__(256) unsigned char g_no_alloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context id the address was looked up in

// Unique id of the calling thread's current CUDA context (driver entry points
// fetched through the runtime, so the library needs no link to the driver
// library); 0 when there is no current context or the driver lacks the call.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx) return 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

bool device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int sw_search_no_alloc(const sw_db *db, const uint8_t *query, int32_t m, const int32_t *matrix,
                                  int32_t gap_open, int32_t gap_extend, int32_t *scores, void *stream) {
    using namespace swdb;
    DbView view;
    int device = 0;
    int32_t A = 0;
    int64_t codes_bytes = 0;
    if (!db_describe(db, &view, &device, &A, &codes_bytes)) return set_error(SW_ERR_INVALID_ARG, "db is NULL");
    if (m < 0) return set_error(SW_ERR_INVALID_ARG, "m < 0");
    if (!matrix) return set_error(SW_ERR_INVALID_ARG, "matrix is NULL");
    if (gap_open < 0 || gap_extend < 0) return set_error(SW_ERR_INVALID_ARG, "gap penalties must be >= 0");
    if (view.n_seqs == 0) return SW_OK;
    if (!scores || !device_ptr(scores)) return set_error(SW_ERR_INVALID_ARG, "scores must be a device pointer");
    if (m > 0 && (!query || !device_ptr(query))) return set_error(SW_ERR_INVALID_ARG, "query must be a device pointer");
    if (device < 0 || device >= kMaxDevices) return set_error(SW_ERR_UNSUPPORTED, "device ordinal too large");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return set_error(SW_ERR_CUDA, "cudaSetDevice failed");
    struct Restore {
        int dev;
        ~Restore() {
            if (dev >= 0) cudaSetDevice(dev);
        }
    } restore{prev};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Device address of the scratch array, looked up once per device (and
    // again only if the device's context has changed since).
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_ptr[device] || (ctx != 0 && ctx != g_scratch_ctx[device])) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_no_alloc_scratch);
            if (e != cudaSuccess || !p) return set_error(SW_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            g_scratch_ptr[device] = static_cast<unsigned char *>(p);
            g_scratch_ctx[device] = current_context_id();
        }
        scratch = g_scratch_ptr[device];
    }

    if (m == 0) {
        if (cudaMemsetAsync(scores, 0, sizeof(int32_t) * size_t(view.n_seqs), st) != cudaSuccess)
            return set_error(SW_ERR_CUDA, "cudaMemsetAsync failed");
        return SW_OK;
    }

    // Arithmetic: the same limits as sw_search (int8 profile S+o, int16 range).
    int smax = matrix[0], smin = matrix[0];
    for (int i = 0; i < A * A; ++i) {
        smax = matrix[i] > smax ? matrix[i] : smax;
        smin = matrix[i] < smin ? matrix[i] : smin;
    }
    const long long absmax = smax > -smin ? smax : -smin;
    const long long span = (long long)m * (smax > 0 ? smax : 0);
    if (absmax > (1 << 20) || (long long)gap_open + gap_extend > (1 << 28) ||
        span + gap_open + gap_extend + absmax > (1ll << 30))
        return set_error(SW_ERR_OVERFLOW, "matrix entries, penalties or lengths too large for exact int32 scores");
    const bool fits16 = (smax + (long long)gap_open <= 127) && (smin + (long long)gap_open >= -127) &&
                        gap_open <= 16384 && (long long)gap_open + gap_extend <= 32768;

    // Scratch layout: counters | overflow list | int32 profile | boundary rows.
    const int TR = kLanes * kRows;
    const int64_t n_pairs = view.n_sorted / 2;
    const int32_t m_pad = int32_t((int64_t(m) + TR - 1) / TR * TR);
    const size_t off_list = 256;
    const size_t off_prof = off_list + align256(sizeof(int32_t) * size_t(n_pairs));
    const size_t off_bnd = off_prof + align256(sizeof(int32_t) * size_t(kProfRows) * size_t(m_pad));
    const bool multipass = m > TR;
    const size_t need = off_bnd + (multipass ? size_t(codes_bytes) * 4 + 64 : 0);
    if (need > kScratchBytes)
        return set_error(SW_ERR_INVALID_ARG,
                         "query and database need more scratch than the fixed no-allocation array holds "
                         "(SW_NO_ALLOC_SCRATCH_BYTES); use sw_search with a workspace instead");
    int32_t *counters = reinterpret_cast<int32_t *>(scratch);   // list length, work counter, flagged, status
    int32_t *list = reinterpret_cast<int32_t *>(scratch + off_list);
    int32_t *prof32 = reinterpret_cast<int32_t *>(scratch + off_prof);
    uint2 *boundary = multipass ? reinterpret_cast<uint2 *>(scratch + off_bnd) : nullptr;

    if (cudaMemsetAsync(counters, 0, 4 * sizeof(int32_t), st) != cudaSuccess)
        return set_error(SW_ERR_CUDA, "cudaMemsetAsync failed");
    if (launch_profile32(query, m, m_pad, matrix, A, gap_open, prof32, st) != cudaSuccess)
        return set_error(SW_ERR_CUDA, "profile launch failed");

    I32Args ja = {};
    ja.db = view;
    ja.gap_open = gap_open;
    ja.gap_extend = gap_extend;
    ja.boundary = boundary;
    ja.prof32 = prof32;
    ja.m = m;
    ja.m_pad = m_pad;
    ja.scores = scores;
    ja.work_counter = counters + 1;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid32 = (sms > 0 ? sms : 1) * 8;

    if (fits16) {
        InterArgs ia = {};
        for (int x = 0; x < kProfRows; ++x)
            for (int y = 0; y < kProfRows; ++y) {
                int v = -128;
                if (x < A && y < A) v = matrix[x * A + y] + gap_open;
                ia.prof8[x][y] = int8_t(v < -128 ? -128 : (v > 127 ? 127 : v));
            }
        ia.db = view;
        ia.pair_begin = 0;
        ia.pair_end = n_pairs;
        ia.query = query;
        ia.m = m;
        ia.gap_open = gap_open;
        ia.gap_extend = gap_extend;
        ia.sat_limit = 32767 - (smax > 0 ? smax : 0);
        ia.boundary = boundary;        // per-pair layout, one CTA per chunk
        ia.slot_stride = 0;
        ia.chunk_counter = nullptr;
        ia.scores = scores;
        ia.ovf_list = list;
        ia.ovf_count = counters;
        ia.ovf_seqs = counters + 2;
        ia.status = counters + 3;
        if (launch_inter_i16x2(ia, kLanes, kRows, st) != cudaSuccess)
            return set_error(SW_ERR_CUDA, "inter-task launch failed");
        ja.list = list;
        ja.list_count = counters;
    } else {
        ja.pair_begin = 0;
        ja.pair_end = n_pairs;
    }
    if (launch_i32(ja, kLanes, kRows, grid32, st) != cudaSuccess) return set_error(SW_ERR_CUDA, "int32 launch failed");
    return SW_OK;
}
