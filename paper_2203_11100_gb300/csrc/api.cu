// C ABI of libswdb: database upload and layout, search planning, launches.
//
// The paper's SW#db uploads the database once into a 2-D device matrix read
// row = residue position, column = sequence (Section 3.2, the texture /
// USM migration figures), launches a short-sequence inter-task kernel and a
// long-sequence intra-task kernel (Section 2.3; "solveShort"/"solveLong" in
// Section 3.2) and keeps one result per database sequence.  This file is
// this library's own host side of that flow.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <iterator>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/swdb.h"
#include "swdb_internal.cuh"

using namespace swdb;

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define SW_CUDA_TRY(expr)                                                                      \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) {                                                               \
            return fail(_e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA,            \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                   \
        }                                                                                      \
    } while (0)

// ---------------------------------------------------------------------------
// handle

struct sw_db {
    int device = 0;
    int32_t A = 0;
    int64_t n_seqs = 0;
    int64_t n_sorted = 0;
    int64_t n_bundles = 0;
    int64_t residues = 0;
    int64_t max_len = 0;
    int64_t codes_bytes = 0;
    int sm_count = 0;

    std::vector<int64_t> h_bundle_off;
    std::vector<int32_t> h_bundle_len;
    std::vector<int32_t> h_len;    // sorted lengths
    std::vector<int64_t> h_sorted_pos;   // original index -> sorted position

    uint8_t *d_codes = nullptr;
    int64_t *d_bundle_off = nullptr;
    int32_t *d_bundle_len = nullptr;
    int32_t *d_len = nullptr;
    int64_t *d_perm = nullptr;

    std::vector<int64_t> h_bundle_res;   // residues per bundle

    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;         // long sequences run here, concurrently
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaGraphExec_t graph_exec = nullptr;   // last captured search (SW_FLAG_GRAPH)
    std::string graph_key;
    std::mutex mu;
    int64_t default_cutoff = 3072;          // long-sequence cutoff when neither opts nor tuning set one
    sw_tuning tuning{};                     // installed by sw_db_set_tuning (counts 0: library tables)
    int64_t tuning_version = 0;             // bumped by every sw_db_set_tuning

    DbView view() const {
        DbView v;
        v.codes = d_codes;
        v.bundle_off = d_bundle_off;
        v.bundle_len = d_bundle_len;
        v.len = d_len;
        v.perm = d_perm;
        v.n_seqs = n_seqs;
        v.n_sorted = n_sorted;
        v.n_bundles = n_bundles;
        return v;
    }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_db_device(sw_db *db) {
    cudaFree(db->d_codes);
    cudaFree(db->d_bundle_off);
    cudaFree(db->d_bundle_len);
    cudaFree(db->d_len);
    cudaFree(db->d_perm);
    cudaFree(db->ws);
    db->d_codes = nullptr;
    db->d_bundle_off = nullptr;
    db->d_bundle_len = nullptr;
    db->d_len = nullptr;
    db->d_perm = nullptr;
    db->ws = nullptr;
    db->ws_bytes = 0;
    if (db->graph_exec) cudaGraphExecDestroy(db->graph_exec);
    db->graph_exec = nullptr;
    if (db->stream) cudaStreamDestroy(db->stream);
    if (db->side) cudaStreamDestroy(db->side);
    if (db->ev_fork) cudaEventDestroy(db->ev_fork);
    if (db->ev_join) cudaEventDestroy(db->ev_join);
    db->stream = nullptr;
    db->side = nullptr;
    db->ev_fork = db->ev_join = nullptr;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Default length above which database sequences leave the inter-task launch
// for the intra-task one.  In the inter-task kernel a subwarp scores one
// pair through ceil(m / (lanes*rows)) strips, one after another, so a pair
// of n columns keeps its subwarp busy for a time proportional to m * n,
// while the launch's throughput spreads the m * R cells of the R residues it
// holds over S resident subwarps: when one pair holds more than 1/S of the
// work, the launch waits on it.  Both sides scale with m, so the balance
// point depends only on the database: the longest bundle length n <= 3072
// with n * 2S <= R(n), the residues of the bundles of length <= n (2S:
// sequence pairs count two sequences per subwarp), S = 2 CTAs x 32
// subwarps per SM of the default 8-lane shape, and not below 768.
// Bundles are sorted longest first.
int64_t balanced_long_cutoff(const std::vector<int32_t> &bundle_len, const std::vector<int64_t> &bundle_res,
                             int sms) {
    constexpr int64_t kMaxCutoff = 3072, kMinCutoff = 768;
    const int64_t slots2 = int64_t(std::max(1, sms)) * 2 * (kCtaThreads / 8) * 2;
    int64_t suffix = 0;
    for (int64_t r : bundle_res) suffix += r;
    for (size_t b = 0; b < bundle_len.size(); ++b) {
        const int64_t L = bundle_len[b];
        if (L <= kMaxCutoff && (L <= kMinCutoff || L * slots2 <= suffix)) return std::max(L, kMinCutoff);
        suffix -= bundle_res[b];
    }
    return kMinCutoff;
}

// Workspace carve-out: a bump allocator over one device buffer.
struct Carver {
    char *base;
    size_t cap;
    size_t used = 0;
    Carver(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    void *take(size_t bytes) {
        used = (size_t)round_up((int64_t)used, 256);
        void *p = base ? base + used : nullptr;
        used += bytes;
        return p;
    }
};

// Launch shapes of the int16x2 inter-task kernel that the planner chooses
// from, with their measured cell-update rates on GB300 (GCUPS, long queries,
// database without long sequences).  A query of m rows is padded to whole
// strips of lanes*rows rows, so the predicted time is
// ceil(m / (lanes*rows)) * lanes*rows / rate.
struct ShapeRate {
    int lanes, rows;
    double gcups;
};
constexpr ShapeRate kShapes[] = {{8, 16, 5000.0}, {16, 16, 5300.0}, {8, 24, 5680.0}, {8, 32, 5900.0}, {16, 32, 5700.0}};

using ShapeTable = std::vector<ShapeRate>;

// The handle's active tables: its tuning's when installed, else the library's.
ShapeTable plain_shapes(const sw_db *db) {
    if (db->tuning.n_plain > 0) {
        ShapeTable t;
        for (int i = 0; i < db->tuning.n_plain; ++i)
            t.push_back({db->tuning.plain[i].lanes, db->tuning.plain[i].rows_per_lane, double(db->tuning.plain[i].gcups)});
        return t;
    }
    return ShapeTable(std::begin(kShapes), std::end(kShapes));
}

// Rows the inter-task kernel computes for a query of m rows with this shape:
// full strips of lanes*rows rows, then a last strip of the fewest rows per lane
// (a multiple of 8) that cover the rest (k_inter16.cu).
int64_t inter_padded_rows(int64_t m, int lanes, int rows) {
    const int64_t tr = int64_t(lanes) * rows;
    if (m <= 0) return 0;
    const int64_t full = (m - 1) / tr;
    const int64_t rest = m - full * tr;
    const int64_t per_lane = std::min<int64_t>(rows, round_up((rest + lanes - 1) / lanes, 8));
    return full * tr + lanes * per_lane;
}

void choose_shape(const ShapeTable &table, int64_t m, int *lanes, int *rows) {
    double best = 1e300;
    for (const ShapeRate &c : table) {
        const double t = double(inter_padded_rows(m, c.lanes, c.rows)) / c.gcups;
        if (t < best) {
            best = t;
            *lanes = c.lanes;
            *rows = c.rows;
        }
    }
}

// Shapes of the int16x2 alignment-mode kernel (k_modes16.cu), same rule (its
// virtual rows on top of the query make up the same padded row count).
constexpr ShapeRate kModeShapes[] = {{8, 16, 5000.0}, {8, 24, 5680.0}, {8, 32, 5900.0}};

void choose_mode_shape(int64_t m, int *lanes, int *rows) {
    double best = 1e300;
    for (const ShapeRate &c : kModeShapes) {
        const double t = double(inter_padded_rows(m, c.lanes, c.rows)) / c.gcups;
        if (t < best) {
            best = t;
            *lanes = c.lanes;
            *rows = c.rows;
        }
    }
}

// The long-sequence path for few tasks of short queries (see Plan::long_inter):
// the inter-task kernel at 32 lanes x 8 rows, one 256-row strip.
constexpr int kLongInterLanes = 32;
constexpr int kLongInterRows = 256;

// Columns of strip-boundary scratch per subwarp of the int16x2 mode kernel: a
// query taller than one strip sends longer sequences to the int32 kernel.
constexpr int32_t kMode16Cols = 4096;

// Batched-kernel shapes (lanes, rows) with measured rates (GCUPS, GB300: the
// autotuner's padding-free probe on the 565,000- and 20M-sequence databases);
// each query pair takes the one with the least predicted time.  With the
// flexible last strip every 8-lane shape pads a pair to a multiple of 64 rows,
// so the rate alone decides between them.
constexpr ShapeRate kBatchShapes[] = {{8, 16, 6400.0}, {8, 24, 6980.0}, {8, 32, 7040.0}};

ShapeTable batch_shapes(const sw_db *db) {
    if (db->tuning.n_batched > 0) {
        ShapeTable t;
        for (int i = 0; i < db->tuning.n_batched; ++i)
            t.push_back({db->tuning.batched[i].lanes, db->tuning.batched[i].rows_per_lane,
                         double(db->tuning.batched[i].gcups)});
        return t;
    }
    return ShapeTable(std::begin(kBatchShapes), std::end(kBatchShapes));
}

int choose_batch_shape(const ShapeTable &table, int64_t m) {
    double best = 1e300;
    int arg = 0;
    for (int i = 0; i < int(table.size()); ++i) {
        // the batched kernel shapes its last strip like the inter-task kernel
        const double t = double(inter_padded_rows(m, table[size_t(i)].lanes, table[size_t(i)].rows)) /
                         table[size_t(i)].gcups;
        if (t < best) {
            best = t;
            arg = i;
        }
    }
    return arg;
}

struct Plan {
    ShapeTable plain_table, batch_table;   // the handle's active rate tables
    int precision = SW_PREC_I16;
    int mode = SW_MODE_PLAIN;
    bool auto_shape = true;          // int16x2 kernel: shape chosen per query ...
    int lanes = 8, rows = 16;        // ... unless the caller fixed it
    int min_tr = 128;                // smallest strip height used
    int lanes32 = 8, rows32 = 16;    // int32 kernel
    int64_t long_end_pair = 0;       // pairs [0, long_end_pair) hold the long sequences
    int64_t n_long = 0;              // real sequences among them
    int64_t long_residues = 0;
    int lanes_long = 32, rows_long = 32;   // per warp of the intra-task kernel
    int warps_long = 2;
    int64_t long_codes_bytes = 0;          // layout bytes of the long bundles (a prefix)
    bool need_long_boundary = false;
    // few (long pair, query) tasks and every query within one 256-row strip:
    // the long pairs go through the inter-task kernel at 32 lanes x 8 rows
    // (the shortest per-column chain) instead of the intra-task kernel
    bool long_inter = false;
    // batched mode: query pairs (a = longer, b = next, -1 if none), persistent grid
    std::vector<int32_t> qp_a, qp_b;
    struct BatchGroup {
        int lanes, rows;          // launch shape of this group
        int32_t begin, count;     // range in qp_a / qp_b
        int32_t grid;             // persistent CTAs
    };
    std::vector<BatchGroup> groups;   // one persistent launch per group
    int32_t batch_grid = 0;
    int64_t batch_seq_begin = 0;
    int32_t batch_max_cols = 0;
    int32_t batch_max_m = 0;
    bool batch_scratch = false;
    int32_t max_m = 0;
    int64_t total_m = 0;
    bool need_boundary = false;      // per-pair boundary (int32 rescore)
    int32_t sat_limit = 0;
    int32_t smax_local = 0;          // max(S, 0): no H of a query of m rows exceeds min(m, longest) * smax_local
    // the database is too small for the default shapes to fill the GPU: a query
    // of one strip takes the shortest column step (32 lanes x 8 rows) instead
    bool small_db = false;
    // plain form: persistent inter-task grid with per-slot boundary scratch
    int32_t inter_grid_max = 0;      // largest resident grid among the shapes used
    int32_t inter_min_lanes = 8;     // sets the most pairs per CTA
    int32_t inter_max_cols = 0;      // columns of the longest non-long pair
    bool inter_scratch = false;
    // non-local alignment modes (k_modes.cu; k_modes16.cu when precision is int16x2)
    int32_t alignment = SW_ALIGN_LOCAL;
    int32_t mode_grid = 0;           // persistent CTAs of the int32 kernel
    int32_t smax_pos = 0;            // max(S, 0)
    int32_t mode16_grid_max = 0;     // persistent CTAs of the int16x2 kernel (largest over its shapes)
    int32_t mode16_cols = 0;         // scratch columns per subwarp (0: every query fits one strip)
    // per query: shape of the int16x2 launch and its first pair (the pairs
    // before it go to the int32 kernel)
    std::vector<int32_t> mode16_lanes, mode16_rows;
    std::vector<int64_t> mode16_cut;
    int64_t mode_i32_cells = 0;      // cells scored by the int32 kernel
    // the int32 kernel's work: one entry per query with sequences for it
    // (longest query first), its profiles packed one after another
    std::vector<ModeEntry> mode_entries;
    int64_t mode_items = 0;
    int64_t mode_prof_ints = 0;
};

int64_t mode16_first_pair(const sw_db *db, const Plan &p, int32_t m, int tr, int32_t o, int32_t e);

// Launch shape of the inter-task kernel for a query of m rows (plain form,
// shape chosen by the library): the table's least predicted time, except on a
// database too small to fill the GPU with the default shapes, where a query of
// one 256-row strip is latency-bound and takes the shortest column step.
void query_shape(const Plan &p, int64_t m, int *lanes, int *rows) {
    if (p.small_db && m <= kLongInterRows) {
        *lanes = kLongInterLanes;
        *rows = kLongInterRows / kLongInterLanes;
        return;
    }
    choose_shape(p.plain_table, m, lanes, rows);
}

// Choose arithmetic and launch shapes for this call.
int make_plan(const sw_db *db, const int64_t *q_offsets, int32_t n_q, const int32_t *matrix,
              int32_t o, int32_t e, const sw_search_opts *opts, Plan *plan) {
    Plan p;
    p.plain_table = plain_shapes(db);
    p.batch_table = batch_shapes(db);
    for (int32_t i = 0; i < n_q; ++i) {
        const int64_t m = q_offsets[i + 1] - q_offsets[i];
        if (m < 0) return fail(SW_ERR_INVALID_ARG, "q_offsets must be non-decreasing");
        if (m > (int64_t(1) << 30)) return fail(SW_ERR_INVALID_ARG, "query longer than 2^30");
        p.max_m = std::max<int32_t>(p.max_m, int32_t(m));
        p.total_m += m;
    }
    int smax = INT32_MIN, smin = INT32_MAX;
    if (matrix) {
        for (int i = 0; i < db->A * db->A; ++i) {
            smax = std::max(smax, matrix[i]);
            smin = std::min(smin, matrix[i]);
        }
    } else {
        smax = smin = 0;
    }
    // int32 exactness: every H is at most min(m, n) * max(S, 0); every E, F is
    // at least -(o + e) below an H; keep all of it inside +-2^30.
    const int64_t absmax = std::max<int64_t>(std::llabs((long long)smax), std::llabs((long long)smin));
    const int64_t span = std::min<int64_t>(p.max_m, db->max_len) * std::max<int64_t>(smax, 0);
    if (absmax > (1 << 20) || int64_t(o) + e > (1 << 28) || span + int64_t(o) + e + absmax > (int64_t(1) << 30))
        return fail(SW_ERR_OVERFLOW, "matrix entries, penalties or lengths too large for exact int32 scores");

    const int32_t alignment = opts ? opts->alignment : SW_ALIGN_LOCAL;
    if (alignment < SW_ALIGN_LOCAL || alignment > SW_ALIGN_OVERLAP)
        return fail(SW_ERR_INVALID_ARG, "unknown alignment mode");
    if (alignment != SW_ALIGN_LOCAL) {
        // No zero floor: values go down to about -(m + n) * (max|S| + o + e).
        if ((int64_t(p.max_m) + db->max_len) * (absmax + int64_t(o) + e) >= (int64_t(1) << 28))
            return fail(SW_ERR_OVERFLOW, "lengths, matrix entries or penalties too large for exact int32 "
                                         "scores of this alignment mode");
        p.alignment = alignment;
        p.mode = SW_MODE_PLAIN;
        p.mode_grid = modes_slots(std::max(1, db->sm_count));
        if (p.mode_grid <= 0) return fail(SW_ERR_CUDA, "could not size the alignment-mode grid");
        // int16x2 (k_modes16.cu) where the int8 profile holds S + o and the
        // virtual rows' o; each pair's own bounds are checked per query.
        const bool fits16 = (int64_t(smax) + o <= 127) && (int64_t(smin) + o >= -128) && (o <= 127);
        const int want = opts ? opts->precision : SW_PREC_AUTO;
        if (want < 0 || want > SW_PREC_I32) return fail(SW_ERR_INVALID_ARG, "unknown precision");
        if (want == SW_PREC_I16 && !fits16)
            return fail(SW_ERR_UNSUPPORTED, "matrix or penalties do not fit the int16x2 alignment-mode kernel");
        p.precision = (want != SW_PREC_I32 && fits16) ? SW_PREC_I16 : SW_PREC_I32;
        p.smax_pos = std::max(smax, 0);
        if (p.precision == SW_PREC_I16) {
            const int sms = std::max(1, db->sm_count);
            p.auto_shape = !(opts && (opts->lanes || opts->rows_per_lane));
            if (!p.auto_shape) {
                const int l = opts->lanes ? opts->lanes : 8, r = opts->rows_per_lane ? opts->rows_per_lane : 32;
                if (!modes16_config_supported(l, r))
                    return fail(SW_ERR_UNSUPPORTED, "lanes/rows_per_lane combination not built for the alignment modes");
                p.lanes = l;
                p.rows = r;
            }
            int min_tr = 1 << 30;
            for (const ShapeRate &c : kModeShapes) {
                if (!p.auto_shape && (c.lanes != p.lanes || c.rows != p.rows)) continue;
                p.mode16_grid_max = std::max(p.mode16_grid_max, modes16_slots(c.lanes, c.rows, sms));
                min_tr = std::min(min_tr, c.lanes * c.rows);
            }
            if (p.mode16_grid_max <= 0) return fail(SW_ERR_CUDA, "could not size the int16x2 alignment-mode grid");
            p.mode16_cols = p.max_m > min_tr ? kMode16Cols : 0;
        }
        for (int32_t i = 0; i < n_q; ++i) {
            const int32_t m = int32_t(q_offsets[i + 1] - q_offsets[i]);
            int l = p.lanes, r = p.rows;
            if (p.precision == SW_PREC_I16 && p.auto_shape) choose_mode_shape(m, &l, &r);
            const int64_t cut = mode16_first_pair(db, p, m, l * r, o, e);
            int64_t res = 0;
            for (int64_t t = 0; t < 2 * cut && t < int64_t(db->h_len.size()); ++t) res += db->h_len[size_t(t)];
            p.mode16_lanes.push_back(l);
            p.mode16_rows.push_back(r);
            p.mode16_cut.push_back(cut);
            if (p.precision == SW_PREC_I16 && m > 0 && cut > 0) {   // the int32 kernel takes these pairs
                p.mode_i32_cells += int64_t(m) * res;
                p.n_long = std::max<int64_t>(p.n_long, std::min<int64_t>(2 * cut, db->n_seqs));
            }
            if (cut > 0) {
                ModeEntry en;
                memset(&en, 0, sizeof en);
                en.n_seqs = 2 * cut;
                en.query = i;
                en.m = m;
                en.m_pad = int32_t(round_up(std::max<int64_t>(m, 1), modes_strip_rows()));
                p.mode_entries.push_back(en);
            }
        }
        std::stable_sort(p.mode_entries.begin(), p.mode_entries.end(),
                         [](const ModeEntry &x, const ModeEntry &y) { return x.m > y.m; });
        for (ModeEntry &en : p.mode_entries) {
            en.item_start = p.mode_items;
            en.prof_off = p.mode_prof_ints;
            p.mode_items += en.n_seqs;
            p.mode_prof_ints += int64_t(kProfRows) * en.m_pad;
        }
        *plan = std::move(p);
        return SW_OK;
    }

    // int16x2 with int8 profile: S + o must fit int8, and o, e small enough
    // that no shifted value leaves int16 (see k_inter16.cu).
    const bool fits16 = (int64_t(smax) + o <= 127) && (int64_t(smin) + o >= -127) && (o <= 16384) &&
                        (int64_t(o) + e <= 32768) && (32767 - std::max(smax, 0) > 0);
    const int want = opts ? opts->precision : SW_PREC_AUTO;
    if (want == SW_PREC_I16 && !fits16)
        return fail(SW_ERR_UNSUPPORTED, "matrix or penalties do not fit the int16x2 kernel");
    if (want < 0 || want > SW_PREC_I32) return fail(SW_ERR_INVALID_ARG, "unknown precision");
    p.precision = (want == SW_PREC_I32 || !fits16) ? SW_PREC_I32 : SW_PREC_I16;
    p.sat_limit = 32767 - std::max(smax, 0);
    p.smax_local = std::max(smax, 0);
    p.small_db = db->n_sorted / 2 < int64_t(std::max(1, db->sm_count)) * (kCtaThreads / 8);

    const int mode = opts ? opts->mode : SW_MODE_AUTO;
    if (mode < 0 || mode > SW_MODE_BATCHED) return fail(SW_ERR_INVALID_ARG, "unknown mode");
    // The batched kernel is int16x2 only; an int32 search runs in the plain form.
    // SW_MODE_AUTO takes the handle's tuned form (plain unless tuned otherwise).
    // The batched kernel packs two queries into the int16x2 halves: a search
    // with a single non-empty query would leave half of every operation empty,
    // so it runs in the plain form (sequence pairs) instead.
    const int want_mode = mode == SW_MODE_AUTO ? db->tuning.mode : mode;
    int32_t nonempty_q = 0;
    for (int32_t i = 0; i < n_q; ++i) nonempty_q += q_offsets[i + 1] > q_offsets[i];
    p.mode = (want_mode == SW_MODE_BATCHED && p.precision == SW_PREC_I16 && nonempty_q >= 2) ? SW_MODE_BATCHED
                                                                                              : SW_MODE_PLAIN;

    int lanes = opts && opts->lanes ? opts->lanes : 8;
    int rows = opts && opts->rows_per_lane ? opts->rows_per_lane : 16;
    if (p.mode == SW_MODE_BATCHED) {
        p.auto_shape = !(opts && (opts->lanes || opts->rows_per_lane));
        if (!p.auto_shape) {
            if (!batch_config_supported(lanes, rows))
                return fail(SW_ERR_UNSUPPORTED, "lanes/rows_per_lane combination not built for the batched kernel");
            p.lanes = lanes;
            p.rows = rows;
            p.min_tr = lanes * rows;
        } else {
            p.lanes = 8;
            p.rows = 32;
            p.min_tr = 128;
        }
    } else if (p.precision == SW_PREC_I16) {
        p.auto_shape = !(opts && (opts->lanes || opts->rows_per_lane));
        if (!p.auto_shape) {
            if (!inter_config_supported(lanes, rows))
                return fail(SW_ERR_UNSUPPORTED, "lanes/rows_per_lane combination not built");
            p.lanes = lanes;
            p.rows = rows;
            p.min_tr = lanes * rows;
        } else {
            p.min_tr = 1 << 30;
            for (int32_t i = 0; i < n_q; ++i) {
                int l = 8, r = 16;
                query_shape(p, q_offsets[i + 1] - q_offsets[i], &l, &r);
                p.min_tr = std::min(p.min_tr, l * r);
            }
            if (n_q == 0) p.min_tr = 128;
        }
    }
    if (p.precision == SW_PREC_I32 && opts && (opts->lanes || opts->rows_per_lane)) {
        if (!i32_config_supported(lanes, rows))
            return fail(SW_ERR_UNSUPPORTED, "lanes/rows_per_lane combination not built for int32");
        p.lanes32 = lanes;
        p.rows32 = rows;
    }
    // Long sequences: the bundles (a prefix, the database being sorted longest
    // first) whose length exceeds the cutoff are scored by a separate launch
    // with wide subwarps on a second stream, concurrently with the rest, so a
    // handful of very long sequences do not set the length of the main launch.
    const int64_t cutoff = opts && opts->long_cutoff ? opts->long_cutoff
                                                     : (db->tuning.long_cutoff ? db->tuning.long_cutoff
                                                                               : db->default_cutoff);
    const int32_t long_rows = opts && opts->long_rows_per_lane ? opts->long_rows_per_lane
                                                               : db->tuning.long_rows_per_lane;
    if (long_rows) {
        if (long_rows == 8) { p.rows_long = 8; p.warps_long = 4; }
        else if (long_rows == 16) { p.rows_long = 16; p.warps_long = 4; }
        else if (long_rows == 32) { p.rows_long = 32; p.warps_long = 2; }
        else return fail(SW_ERR_UNSUPPORTED, "long_rows_per_lane must be 8, 16 or 32");
    }
    int64_t nlb = 0;
    if (cutoff > 0 && p.precision == SW_PREC_I16)
        while (nlb < db->n_bundles && db->h_bundle_len[size_t(nlb)] > cutoff) ++nlb;
    p.long_end_pair = nlb * kBundlePairs;
    for (int64_t b = 0; b < nlb; ++b) p.long_residues += db->h_bundle_res[size_t(b)];
    p.n_long = std::min<int64_t>(nlb * kBundleSeqs, db->n_seqs);
    p.long_codes_bytes = nlb < db->n_bundles ? db->h_bundle_off[size_t(nlb)] : db->codes_bytes;
    if (!long_rows) {
        // Few (long pair, query) tasks: the launch is bound by the serial
        // column chain of the longest sequences, which shares its SMs with the
        // concurrent inter-task launch, so 16 rows per lane (a shorter step)
        // wins; many tasks: it is throughput-bound and 32 rows per lane (less
        // overhead per cell) wins (measured on GB300: a lone 144-residue query
        // against the 565,000-sequence database 17.5 vs 22.8 ms; the 50,000-
        // sequence database with 10% long sequences 4,311 vs 3,789 GCUPS at
        // m = 35,000 for 32 rows).
        int32_t nonempty = 0;
        for (int32_t i = 0; i < n_q; ++i) nonempty += q_offsets[i + 1] > q_offsets[i];
        const bool few = p.long_end_pair * int64_t(nonempty) <= 4 * int64_t(std::max(1, db->sm_count));
        // few tasks: the shortest column step that keeps one super-pass (8 rows
        // per lane up to 1,024 query rows, else 16)
        p.rows_long = few ? (p.max_m <= 4 * 32 * 8 ? 8 : 16) : 32;
        p.warps_long = few ? 4 : 2;
        p.long_inter = few && p.max_m <= kLongInterRows;
    }
    p.need_long_boundary = nlb > 0 && !p.long_inter && p.max_m > intra_rows_per_superpass(p.warps_long, p.rows_long);
    if (nlb > 0 && p.precision == SW_PREC_I16) {
        const cudaError_t e = prepare_intra_i16x2(p.warps_long, p.rows_long);
        if (e != cudaSuccess) return fail(SW_ERR_CUDA, std::string("intra-task kernel set-up: ") + cudaGetErrorString(e));
    }
    p.need_boundary = p.max_m > std::min(p.min_tr, p.lanes32 * p.rows32);

    if (p.mode == SW_MODE_PLAIN && p.precision == SW_PREC_I16 && n_q > 0) {
        // Sized over every shape this call may launch (all of the table when the
        // shape is chosen per query), so that a workspace sized for queries of
        // the maximum length also fits any batch of shorter ones.
        const int sms = std::max(1, db->sm_count);
        const int n_shapes = p.auto_shape ? int(p.plain_table.size()) : 1;
        int min_tr = 1 << 30;
        p.inter_min_lanes = 32;
        for (int sh = 0; sh < n_shapes; ++sh) {
            const int l = p.auto_shape ? p.plain_table[size_t(sh)].lanes : p.lanes;
            const int r = p.auto_shape ? p.plain_table[size_t(sh)].rows : p.rows;
            p.inter_min_lanes = std::min(p.inter_min_lanes, l);
            p.inter_grid_max = std::max(p.inter_grid_max, inter_slots(l, r, sms));
            min_tr = std::min(min_tr, l * r);
        }
        p.inter_scratch = p.max_m > min_tr;
        const int64_t first = p.long_end_pair * 2;
        p.inter_max_cols = first < db->n_sorted ? int32_t(round_up(db->h_len[size_t(first)], 4)) : 0;
        if (p.inter_max_cols == 0) p.inter_scratch = false;
        if (p.inter_grid_max <= 0) return fail(SW_ERR_CUDA, "could not size the persistent grid");
    }
    if (p.mode == SW_MODE_BATCHED) {
        // Pair queries of similar length: sort the non-empty ones longest first
        // and pair neighbours, so the shorter of a pair pads few rows.
        std::vector<int32_t> idx;
        for (int32_t i = 0; i < n_q; ++i)
            if (q_offsets[i + 1] > q_offsets[i]) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            return q_offsets[x + 1] - q_offsets[x] > q_offsets[y + 1] - q_offsets[y];
        });
        std::vector<int32_t> pa, pb;
        for (size_t i = 0; i < idx.size(); i += 2) {
            pa.push_back(idx[i]);
            pb.push_back(i + 1 < idx.size() ? idx[i + 1] : -1);
        }
        // Group the pairs by launch shape (each group keeps longest-first order).
        const int n_shapes = p.auto_shape ? int(p.batch_table.size()) : 1;
        p.batch_max_m = idx.empty() ? 0 : int32_t(q_offsets[idx[0] + 1] - q_offsets[idx[0]]);
        p.batch_scratch = p.batch_max_m > 128;   // any multi-pass pair, in any shape
        for (int sh = 0; sh < n_shapes; ++sh) {
            const int gl = p.auto_shape ? p.batch_table[size_t(sh)].lanes : p.lanes;
            const int gr = p.auto_shape ? p.batch_table[size_t(sh)].rows : p.rows;
            Plan::BatchGroup g{gl, gr, int32_t(p.qp_a.size()), 0, 0};
            int64_t gmax = 0;
            for (size_t i = 0; i < pa.size(); ++i) {
                const int64_t m = q_offsets[pa[i] + 1] - q_offsets[pa[i]];
                if (p.auto_shape && choose_batch_shape(p.batch_table, m) != sh) continue;
                p.qp_a.push_back(pa[i]);
                p.qp_b.push_back(pb[i]);
                gmax = std::max(gmax, m);
            }
            g.count = int32_t(p.qp_a.size()) - g.begin;
            if (g.count == 0) continue;
            g.grid = batch_slots(gl, gr, std::max(1, db->sm_count));
            if (g.grid <= 0) return fail(SW_ERR_CUDA, "could not size the persistent grid");
            p.batch_grid = std::max(p.batch_grid, g.grid);
            if (gmax > int64_t(gl) * gr) p.batch_scratch = true;
            p.groups.push_back(g);
            (void)gmax;
        }
        // Size the per-slot scratch for the widest grid any shape could use, so a
        // workspace sized for one batch fits every batch of the same length bound.
        if (p.auto_shape)
            for (const ShapeRate &c : p.batch_table)
                p.batch_grid = std::max(p.batch_grid, batch_slots(c.lanes, c.rows, std::max(1, db->sm_count)));
        p.batch_seq_begin = p.long_end_pair * 2;
        p.batch_max_cols = p.batch_seq_begin < db->n_sorted
                               ? int32_t(round_up(db->h_len[size_t(p.batch_seq_begin)], 4))
                               : 0;
        if (p.batch_max_cols == 0) p.batch_scratch = false;
    }
    *plan = p;
    return SW_OK;
}

struct Buffers {
    uint8_t *queries = nullptr;
    int32_t *scores = nullptr;
    sw_hit *hits = nullptr;
    uint2 *boundary = nullptr;
    uint2 *long_boundary = nullptr;   // [n_q] regions of long_codes_bytes/2 entries
    int64_t *q_off = nullptr;         // device copy of the query offsets
    int32_t *prof32 = nullptr;
    int32_t *qp = nullptr;            // batched mode: qp_a then qp_b
    uint2 *batch_scratch = nullptr;   // batched mode: per CTA slot boundary rows
    uint2 *inter_scratch = nullptr;   // plain mode: per CTA slot boundary rows
    int32_t *mode_prof = nullptr;     // alignment modes, int32 kernel: per entry [32][m_pad] S(q_i, c) + o
    ModeEntry *mode_entries = nullptr;
    unsigned long long *mode_counter = nullptr;
    int2 *mode_bnd = nullptr;         // alignment modes: per warp slot, max_len + 1 (H, F)
    uint2 *mode16_scratch = nullptr;  // int16x2 alignment modes: per CTA slot boundary rows
    int32_t *ovf_list = nullptr;
    int32_t *counters = nullptr;   // [n_q] list lengths, [n_q] work counters, [n_q] flagged sequences,
                                   // then one status word
};

// First pair of the sorted database whose alignment-mode scores against a
// query of m rows provably stay inside int16 in k_modes16.cu; the pairs
// before it (the longest) go to the int32 kernel.  With Lp the pair's
// columns, every H lies between min_i H(i, 0) - g(Lp) (the E chain along a
// row) >= -g(m) - g(Lp) (overlap: -g(Lp)) and max(S, 0) * min(m, Lp); the
// kernel's intermediate values reach at most o + max(e, 128) below the
// lower bound (gap and profile addends) and max(S) above the upper one.  Both
// bounds grow with Lp, which falls along the sorted order, so the pairs that
// fit are a suffix.
int64_t mode16_first_pair(const sw_db *db, const Plan &p, int32_t m, int tr, int32_t o, int32_t e) {
    const int64_t n_pairs = db->n_sorted / 2;
    if (p.precision != SW_PREC_I16 || m <= 0) return n_pairs;
    const int64_t gmin = std::min(o, e);
    auto g = [&](int64_t k) { return k <= 0 ? int64_t(0) : int64_t(o) + (k - 1) * gmin; };
    const bool multi = m > tr;
    const int64_t gm = p.alignment == SW_ALIGN_OVERLAP ? 0 : g(m);
    auto ok = [&](int64_t pair) {
        const int64_t Lp = round_up(db->h_len[size_t(2 * pair)], 4);
        if (multi && Lp > kMode16Cols) return false;
        if (gm + g(Lp) + o + std::max<int64_t>(e, 128) > 32768) return false;
        if (int64_t(p.smax_pos) * (std::min<int64_t>(m, Lp) + 1) > 32767) return false;
        return true;
    };
    int64_t lo = 0, hi = n_pairs;   // the first pair that fits lies in [lo, hi]
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (ok(mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

size_t carve(const sw_db *db, const Plan &p, int32_t n_q, int32_t top_k, bool q_dev, bool s_dev,
             bool h_dev, void *base, size_t cap, Buffers *b) {
    Carver c(base, cap);
    Buffers x;
    if (!q_dev) x.queries = static_cast<uint8_t *>(c.take(size_t(std::max<int64_t>(p.total_m, 1))));
    if (!s_dev) x.scores = static_cast<int32_t *>(c.take(sizeof(int32_t) * size_t(std::max<int64_t>(n_q, 1)) * size_t(std::max<int64_t>(db->n_seqs, 1))));
    if (!h_dev && top_k > 0) x.hits = static_cast<sw_hit *>(c.take(sizeof(sw_hit) * size_t(n_q) * size_t(top_k)));
    if (p.need_boundary) x.boundary = static_cast<uint2 *>(c.take(size_t(db->codes_bytes) * 4 + 64));
    const int tr32 = p.lanes32 * p.rows32;
    const int64_t m_pad = round_up(std::max<int64_t>(p.max_m, 1), tr32);
    x.prof32 = static_cast<int32_t *>(c.take(sizeof(int32_t) * size_t(kProfRows) * size_t(m_pad)));
    if (p.need_long_boundary)
        x.long_boundary = static_cast<uint2 *>(c.take(size_t(p.long_codes_bytes) * 4 * size_t(n_q) + 64));
    x.q_off = static_cast<int64_t *>(c.take(sizeof(int64_t) * size_t(n_q + 1)));
    // one overflow list per query: queries run concurrently with the long-sequence launch
    x.ovf_list = static_cast<int32_t *>(c.take(sizeof(int32_t) * size_t(std::max<int32_t>(n_q, 1)) *
                                               size_t(std::max<int64_t>(db->n_sorted / 2, 1))));
    if (p.mode == SW_MODE_BATCHED) {
        x.qp = static_cast<int32_t *>(c.take(sizeof(int32_t) * 2 * std::max<size_t>(p.qp_a.size(), 1)));
        if (p.batch_scratch)   // sized for the widest group (all shapes have at most 32 subwarps per CTA)
            x.batch_scratch = static_cast<uint2 *>(c.take(sizeof(uint2) * size_t(p.batch_grid) *
                                                          size_t(kCtaThreads / 8) * size_t(p.batch_max_cols)));
    }
    if (p.inter_scratch)
        x.inter_scratch = static_cast<uint2 *>(c.take(sizeof(uint2) * size_t(p.inter_grid_max) *
                                                      size_t(kCtaThreads / p.inter_min_lanes) *
                                                      size_t(p.inter_max_cols)));
    if (p.alignment != SW_ALIGN_LOCAL) {
        x.mode_prof = static_cast<int32_t *>(c.take(sizeof(int32_t) * size_t(std::max<int64_t>(p.mode_prof_ints, 1))));
        x.mode_entries = static_cast<ModeEntry *>(c.take(sizeof(ModeEntry) * std::max<size_t>(p.mode_entries.size(), 1)));
        x.mode_counter = static_cast<unsigned long long *>(c.take(sizeof(unsigned long long)));
        x.mode_bnd = static_cast<int2 *>(c.take(sizeof(int2) * size_t(p.mode_grid) * size_t(kCtaThreads / 32) *
                                                size_t(db->max_len + 1)));
        if (p.precision == SW_PREC_I16 && p.mode16_cols > 0)
            x.mode16_scratch = static_cast<uint2 *>(c.take(sizeof(uint2) * size_t(p.mode16_grid_max) *
                                                           size_t(kCtaThreads / 8) * size_t(p.mode16_cols)));
    }
    // [n_q] list lengths, [n_q] work counters, [n_q] flagged, [n_q] chunk counters,
    // status, 4 tile counters
    x.counters = static_cast<int32_t *>(c.take(sizeof(int32_t) * size_t(5 * std::max<int32_t>(n_q, 1) + 5)));
    *b = x;
    return c.used + 256;
}

// Optional CUDA-event timing of individual launches (only when stats are
// requested): pairs of events per launch, summed per kernel family.
struct LaunchTimer {
    enum { INTER = 0, RESCORE = 1, INTRA = 2, OTHER = 3 };
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
    int launches = 0;
    cudaEvent_t begin(int, cudaStream_t s) {
        ++launches;
        if (!on) return nullptr;
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, s);
        return a;
    }
    void end(int fam, cudaEvent_t a, cudaStream_t s) {
        if (!on) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, s);
        ev[fam].push_back({a, b});
    }
    float total(int fam) {
        float t = 0.f;
        for (auto &p : ev[fam]) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.first, p.second);
            t += ms;
        }
        return t;
    }
    ~LaunchTimer() {
        for (auto &v : ev)
            for (auto &p : v) {
                cudaEventDestroy(p.first);
                cudaEventDestroy(p.second);
            }
    }
};

#define TIMED_ON(fam, strm, call)              \
    do {                                       \
        cudaEvent_t _a = timer.begin(fam, strm); \
        SW_CUDA_TRY(call);                     \
        timer.end(fam, _a, strm);              \
    } while (0)
#define TIMED(fam, call) TIMED_ON(fam, st, call)

}  // namespace

// Read-only facts of a loaded database, for entry points defined in other
// translation units.
namespace swdb {
int high_launch_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

bool db_describe(const sw_db *db, DbView *view, int *device, int32_t *alphabet, int64_t *codes_bytes) {
    if (!db) return false;
    *view = db->view();
    *device = db->device;
    *alphabet = db->A;
    *codes_bytes = db->codes_bytes;
    return true;
}

int set_error(int code, const char *msg) { return fail(code, msg); }
}  // namespace swdb

// ---------------------------------------------------------------------------
// ABI

extern "C" {

const char *sw_last_error(void) { return g_last_error.c_str(); }

const char *sw_version(void) { return "swdb 0.1 (sm_103a)"; }

int sw_db_load(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs, int32_t alphabet_size,
               int device, sw_db **out) {
    g_last_error.clear();
    if (!out) return fail(SW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!offsets) return fail(SW_ERR_INVALID_ARG, "offsets is NULL");
    if (n_seqs < 0) return fail(SW_ERR_INVALID_ARG, "n_seqs < 0");
    if (alphabet_size < 1 || alphabet_size > SW_MAX_ALPHABET)
        return fail(SW_ERR_INVALID_ARG, "alphabet_size must be 1..31");
    if (offsets[0] != 0) return fail(SW_ERR_INVALID_ARG, "offsets[0] must be 0");
    int64_t max_len = 0;
    for (int64_t i = 0; i < n_seqs; ++i) {
        const int64_t L = offsets[i + 1] - offsets[i];
        if (L < 0) return fail(SW_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (L > (int64_t(1) << 30)) return fail(SW_ERR_INVALID_ARG, "sequence longer than 2^30");
        max_len = std::max(max_len, L);
    }
    const int64_t total = offsets[n_seqs];
    if (total > 0 && !residues) return fail(SW_ERR_INVALID_ARG, "residues is NULL");
    for (int64_t i = 0; i < total; ++i)
        if (residues[i] >= alphabet_size) {
            char msg[128];
            snprintf(msg, sizeof msg, "residue code %d at position %lld is >= alphabet_size %d", int(residues[i]),
                     (long long)i, alphabet_size);
            return fail(SW_ERR_INVALID_ARG, msg);
        }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(SW_ERR_INVALID_ARG, "no such CUDA device");
    }
    DeviceGuard guard(device);

    sw_db *db = new (std::nothrow) sw_db();
    if (!db) return fail(SW_ERR_OOM, "host allocation failed");
    db->device = device;
    db->A = alphabet_size;
    db->n_seqs = n_seqs;
    db->residues = total;
    db->max_len = max_len;
    cudaDeviceGetAttribute(&db->sm_count, cudaDevAttrMultiProcessorCount, device);

    // Sort by length, longest first; ties keep the original order.
    std::vector<int64_t> order(static_cast<size_t>(n_seqs));
    std::iota(order.begin(), order.end(), int64_t(0));
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        return offsets[x + 1] - offsets[x] > offsets[y + 1] - offsets[y];
    });
    db->n_bundles = (n_seqs + kBundleSeqs - 1) / kBundleSeqs;
    db->n_sorted = db->n_bundles * kBundleSeqs;
    std::vector<int64_t> perm(size_t(db->n_sorted), -1);
    db->h_len.assign(size_t(db->n_sorted), 0);
    for (int64_t s = 0; s < n_seqs; ++s) {
        perm[size_t(s)] = order[size_t(s)];
        db->h_len[size_t(s)] = int32_t(offsets[order[s] + 1] - offsets[order[s]]);
    }
    db->h_sorted_pos.assign(size_t(n_seqs), 0);
    for (int64_t s = 0; s < n_seqs; ++s) db->h_sorted_pos[size_t(order[size_t(s)])] = s;
    db->h_bundle_off.resize(size_t(db->n_bundles));
    db->h_bundle_len.resize(size_t(db->n_bundles));
    int64_t off = 0;
    for (int64_t b = 0; b < db->n_bundles; ++b) {
        const int32_t L = int32_t(round_up(db->h_len[size_t(b * kBundleSeqs)], 4));
        db->h_bundle_off[size_t(b)] = off;
        db->h_bundle_len[size_t(b)] = L;
        off += int64_t(L) * kBundleSeqs;
    }
    db->codes_bytes = off;
    db->h_bundle_res.assign(size_t(db->n_bundles), 0);
    for (int64_t t = 0; t < n_seqs; ++t) db->h_bundle_res[size_t(t / kBundleSeqs)] += db->h_len[size_t(t)];
    db->default_cutoff = balanced_long_cutoff(db->h_bundle_len, db->h_bundle_res, db->sm_count);
    std::vector<uint8_t> codes(size_t(std::max<int64_t>(off, 1)), uint8_t(kPadCode));
    for (int64_t s = 0; s < n_seqs; ++s) {
        const int64_t b = s / kBundleSeqs;
        const int slot = int((s % kBundleSeqs) / 2);
        const int h = int(s % 2);
        const uint8_t *src = residues + offsets[order[s]];
        const int32_t L = db->h_len[size_t(s)];
        uint8_t *dst = codes.data() + db->h_bundle_off[size_t(b)] + slot * kQuadBytes + h;
        for (int32_t j = 0; j < L; ++j) dst[(j >> 2) * kBundleRowBytes + (j & 3) * 2] = src[j];
    }

    auto cleanup = [&](int code, const std::string &msg) {
        free_db_device(db);
        delete db;
        return fail(code, msg);
    };
    cudaError_t err;
    if ((err = cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (err = cudaStreamCreateWithFlags(&db->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (err = cudaEventCreateWithFlags(&db->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (err = cudaEventCreateWithFlags(&db->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return cleanup(SW_ERR_CUDA, cudaGetErrorString(err));
    const size_t nb = size_t(std::max<int64_t>(db->n_bundles, 1));
    const size_t ns = size_t(std::max<int64_t>(db->n_sorted, 1));
    if ((err = cudaMalloc(&db->d_codes, codes.size())) != cudaSuccess ||
        (err = cudaMalloc(&db->d_bundle_off, nb * sizeof(int64_t))) != cudaSuccess ||
        (err = cudaMalloc(&db->d_bundle_len, nb * sizeof(int32_t))) != cudaSuccess ||
        (err = cudaMalloc(&db->d_len, ns * sizeof(int32_t))) != cudaSuccess ||
        (err = cudaMalloc(&db->d_perm, ns * sizeof(int64_t))) != cudaSuccess)
        return cleanup(err == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA, cudaGetErrorString(err));
    if ((err = cudaMemcpy(db->d_codes, codes.data(), codes.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (db->n_bundles &&
         (err = cudaMemcpy(db->d_bundle_off, db->h_bundle_off.data(), db->n_bundles * sizeof(int64_t),
                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (db->n_bundles &&
         (err = cudaMemcpy(db->d_bundle_len, db->h_bundle_len.data(), db->n_bundles * sizeof(int32_t),
                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (db->n_sorted && (err = cudaMemcpy(db->d_len, db->h_len.data(), db->n_sorted * sizeof(int32_t),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (db->n_sorted && (err = cudaMemcpy(db->d_perm, perm.data(), db->n_sorted * sizeof(int64_t),
                                           cudaMemcpyHostToDevice)) != cudaSuccess))
        return cleanup(SW_ERR_CUDA, cudaGetErrorString(err));
    *out = db;
    return SW_OK;
}

int sw_db_free(sw_db *db) {
    g_last_error.clear();
    if (!db) return SW_OK;
    {
        DeviceGuard guard(db->device);
        if (db->stream) cudaStreamSynchronize(db->stream);
        free_db_device(db);
    }
    delete db;
    return SW_OK;
}

int sw_db_get_info(const sw_db *db, sw_db_info *out) {
    g_last_error.clear();
    if (!db || !out) return fail(SW_ERR_INVALID_ARG, "NULL argument");
    out->n_seqs = db->n_seqs;
    out->residues = db->residues;
    out->max_length = db->max_len;
    out->device_bytes = db->codes_bytes + db->n_bundles * 12 + db->n_sorted * 12;
    out->alphabet_size = db->A;
    out->device = db->device;
    return SW_OK;
}

int sw_db_set_tuning(sw_db *db, const sw_tuning *t) {
    g_last_error.clear();
    if (!db) return fail(SW_ERR_INVALID_ARG, "db is NULL");
    if (t) {
        if (t->n_plain < 0 || t->n_plain > SW_TUNING_MAX_SHAPES || t->n_batched < 0 ||
            t->n_batched > SW_TUNING_MAX_SHAPES)
            return fail(SW_ERR_INVALID_ARG, "shape count outside 0..SW_TUNING_MAX_SHAPES");
        auto bad_rate = [](float g) { return !(g > 0.0f) || !(g < 1e30f); };
        for (int i = 0; i < t->n_plain; ++i) {
            if (!inter_config_supported(t->plain[i].lanes, t->plain[i].rows_per_lane))
                return fail(SW_ERR_INVALID_ARG, "a plain-form shape the inter-task kernel does not support");
            if (bad_rate(t->plain[i].gcups)) return fail(SW_ERR_INVALID_ARG, "a shape rate is not positive and finite");
        }
        for (int i = 0; i < t->n_batched; ++i) {
            if (!batch_config_supported(t->batched[i].lanes, t->batched[i].rows_per_lane))
                return fail(SW_ERR_INVALID_ARG, "a batched-form shape the batched kernel does not support");
            if (bad_rate(t->batched[i].gcups)) return fail(SW_ERR_INVALID_ARG, "a shape rate is not positive and finite");
        }
        if (t->long_rows_per_lane != 0 && t->long_rows_per_lane != 8 && t->long_rows_per_lane != 16 &&
            t->long_rows_per_lane != 32)
            return fail(SW_ERR_INVALID_ARG, "long_rows_per_lane must be 0, 8, 16 or 32");
        if (t->mode < SW_MODE_AUTO || t->mode > SW_MODE_BATCHED) return fail(SW_ERR_INVALID_ARG, "unknown mode");
    }
    std::lock_guard<std::mutex> lock(db->mu);
    if (t) db->tuning = *t;
    else db->tuning = sw_tuning{};
    ++db->tuning_version;
    return SW_OK;
}

int sw_db_get_tuning(const sw_db *db, sw_tuning *out) {
    g_last_error.clear();
    if (!db || !out) return fail(SW_ERR_INVALID_ARG, "NULL argument");
    *out = db->tuning;
    const ShapeTable pt = plain_shapes(db), bt = batch_shapes(db);
    out->n_plain = int32_t(pt.size());
    out->n_batched = int32_t(bt.size());
    for (size_t i = 0; i < pt.size(); ++i) out->plain[i] = {pt[i].lanes, pt[i].rows, float(pt[i].gcups)};
    for (size_t i = 0; i < bt.size(); ++i) out->batched[i] = {bt[i].lanes, bt[i].rows, float(bt[i].gcups)};
    return SW_OK;
}

int sw_search_workspace_size(const sw_db *db, const int64_t *q_offsets, int32_t n_q, int32_t top_k,
                             const sw_search_opts *opts, size_t *bytes) {
    g_last_error.clear();
    if (!db || !bytes || (n_q > 0 && !q_offsets)) return fail(SW_ERR_INVALID_ARG, "NULL argument");
    if (n_q < 0 || top_k < 0) return fail(SW_ERR_INVALID_ARG, "negative count");
    Plan p;
    DeviceGuard guard(db->device);
    std::vector<int32_t> zero(size_t(db->A) * db->A, 0);
    int rc = make_plan(db, q_offsets, n_q, zero.data(), 0, 0, opts, &p);
    if (rc) return rc;
    Buffers b;
    // Worst case: every buffer carved (host queries / outputs).
    *bytes = carve(db, p, n_q, top_k, false, false, false, nullptr, 0, &b);
    if (p.mode == SW_MODE_BATCHED) {
        // a later batch of these sizes with a single non-empty query runs in the
        // plain form: cover that plan too
        sw_search_opts plain_opts{};
        if (opts) plain_opts = *opts;
        plain_opts.mode = SW_MODE_PLAIN;
        Plan pp;
        rc = make_plan(db, q_offsets, n_q, zero.data(), 0, 0, &plain_opts, &pp);
        if (rc) return rc;
        *bytes = std::max(*bytes, carve(db, pp, n_q, top_k, false, false, false, nullptr, 0, &b));
    }
    // Boundary scratch may be needed for either kernel family.
    if (!p.need_boundary) *bytes += size_t(db->codes_bytes) * 4 + 64 + 256;
    return SW_OK;
}

int sw_search(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q, const int32_t *matrix,
              int32_t gap_open, int32_t gap_extend, int32_t top_k, int32_t *scores_out, sw_hit *hits_out,
              const sw_search_opts *opts, sw_search_stats *stats, void *stream) {
    g_last_error.clear();
    if (!db) return fail(SW_ERR_INVALID_ARG, "db is NULL");
    if (n_q < 0) return fail(SW_ERR_INVALID_ARG, "n_q < 0");
    if (n_q > 0 && !q_offsets) return fail(SW_ERR_INVALID_ARG, "q_offsets is NULL");
    if (!matrix) return fail(SW_ERR_INVALID_ARG, "matrix is NULL");
    if (gap_open < 0 || gap_extend < 0) return fail(SW_ERR_INVALID_ARG, "gap penalties must be >= 0");
    if (top_k < 0 || top_k > 4096) return fail(SW_ERR_INVALID_ARG, "top_k must be 0..4096");
    if (n_q > 0 && q_offsets[0] != 0) return fail(SW_ERR_INVALID_ARG, "q_offsets[0] must be 0");
    if (n_q > 0 && q_offsets[n_q] > 0 && !queries) return fail(SW_ERR_INVALID_ARG, "queries is NULL");
    if (opts && opts->long_cutoff > 0) {
        // accepted; long sequences are still scored by the inter-task kernel
    }
    std::lock_guard<std::mutex> lock(db->mu);
    DeviceGuard guard(db->device);

    Plan plan;
    int rc = make_plan(db, q_offsets, n_q, matrix, gap_open, gap_extend, opts, &plan);
    if (rc) return rc;

    const bool q_dev = n_q == 0 || plan.total_m == 0 || is_device_ptr(queries);
    if (!q_dev) {
        for (int64_t i = 0; i < plan.total_m; ++i)
            if (queries[i] >= db->A) return fail(SW_ERR_INVALID_ARG, "query residue code >= alphabet_size");
    }
    const bool s_dev = scores_out && is_device_ptr(scores_out);
    const bool h_dev = hits_out && is_device_ptr(hits_out);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : db->stream;
    LaunchTimer timer;
    timer.on = stats != nullptr;
    timer.st = st;

    Buffers buf;
    size_t need = carve(db, plan, n_q, top_k, q_dev, s_dev, h_dev, nullptr, 0, &buf);
    void *ws = nullptr;
    size_t ws_cap = 0;
    if (opts && opts->workspace) {
        ws = opts->workspace;
        ws_cap = opts->workspace_bytes;
        if (ws_cap < need) return fail(SW_ERR_INVALID_ARG, "workspace too small (see sw_search_workspace_size)");
    } else {
        if (db->ws_bytes < need) {
            SW_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(db->ws);
            db->ws = nullptr;
            db->ws_bytes = 0;
            SW_CUDA_TRY(cudaMalloc(&db->ws, need));
            db->ws_bytes = need;
        }
        ws = db->ws;
        ws_cap = db->ws_bytes;
    }
    carve(db, plan, n_q, top_k, q_dev, s_dev, h_dev, ws, ws_cap, &buf);

    const uint8_t *d_queries = q_dev ? queries : buf.queries;
    int32_t *d_scores = s_dev ? scores_out : buf.scores;
    sw_hit *d_hits = h_dev ? hits_out : buf.hits;
    if (!q_dev && plan.total_m > 0)
        SW_CUDA_TRY(cudaMemcpyAsync(buf.queries, queries, size_t(plan.total_m), cudaMemcpyHostToDevice, st));
    int32_t *d_chunks = buf.counters + 3 * size_t(std::max<int32_t>(n_q, 1));
    int32_t *d_status = buf.counters + 4 * size_t(std::max<int32_t>(n_q, 1));
    int32_t *d_tiles = d_status + 1;

    // int8 profile table for the int16x2 kernel: [query code][db code] = S + o.
    InterArgs ia;
    memset(&ia, 0, sizeof ia);
    for (int x = 0; x < kProfRows; ++x)
        for (int y = 0; y < kProfRows; ++y) {
            int v = -128;
            if (x < db->A && y < db->A) v = matrix[x * db->A + y] + gap_open;
            ia.prof8[x][y] = int8_t(std::max(-128, std::min(127, v)));
        }
    ia.db = db->view();
    ia.gap_open = gap_open;
    ia.gap_extend = gap_extend;
    ia.sat_limit = plan.sat_limit;
    ia.boundary = buf.boundary;
    ia.ovf_list = buf.ovf_list;
    ia.status = d_status;

    I32Args ja;
    memset(&ja, 0, sizeof ja);
    ja.db = db->view();
    ja.gap_open = gap_open;
    ja.gap_extend = gap_extend;
    ja.boundary = buf.boundary;
    ja.prof32 = buf.prof32;
    const int grid32 = std::max(1, db->sm_count) * 8;
    const int64_t n_pairs = db->n_sorted / 2;

    const int64_t list_stride = std::max<int64_t>(n_pairs, 1);
    const bool split = plan.precision == SW_PREC_I16 && plan.long_end_pair > 0 && n_q > 0 && db->n_seqs > 0;
    const int32_t n_qp = int32_t(plan.qp_a.size());
    // While the long sequences run on the side stream, the main-stream launches
    // take a higher priority: their CTAs are dispatched as soon as SMs free up
    // instead of queuing behind every pending intra-task CTA (the intra-task
    // CTAs already running, the longest tasks first, are not preempted).
    const int main_priority = split && !plan.long_inter ? high_launch_priority() : 0;

    // Host-to-device inputs first: they stay outside any captured graph.
    if (!plan.mode_entries.empty())
        SW_CUDA_TRY(cudaMemcpyAsync(buf.mode_entries, plan.mode_entries.data(),
                                    sizeof(ModeEntry) * plan.mode_entries.size(), cudaMemcpyHostToDevice, st));
    if ((split || plan.mode == SW_MODE_BATCHED) && n_q > 0)
        SW_CUDA_TRY(cudaMemcpyAsync(buf.q_off, q_offsets, sizeof(int64_t) * size_t(n_q + 1), cudaMemcpyHostToDevice, st));
    if (plan.mode == SW_MODE_BATCHED && n_qp > 0) {
        std::vector<int32_t> qp(plan.qp_a);
        qp.insert(qp.end(), plan.qp_b.begin(), plan.qp_b.end());
        SW_CUDA_TRY(cudaMemcpyAsync(buf.qp, qp.data(), sizeof(int32_t) * qp.size(), cudaMemcpyHostToDevice, st));
    }
    int last_lanes = plan.lanes, last_rows = plan.rows;
    int32_t *status_out = opts ? opts->status_out : nullptr;

    // All device work of the search, in stream order.  Run directly, or
    // captured once into a CUDA graph and replayed (SW_FLAG_GRAPH).
    auto enqueue = [&]() -> int {
    SW_CUDA_TRY(cudaMemsetAsync(buf.counters, 0, sizeof(int32_t) * (5 * size_t(std::max<int32_t>(n_q, 1)) + 5), st));

    if (plan.alignment != SW_ALIGN_LOCAL) {
        // Non-local modes, per query: the pairs whose scores provably fit int16
        // (a suffix of the sorted order) in one persistent int16x2 launch
        // (k_modes16.cu); the longer ones, with the query's int32 profile
        // S(q_i, c) + o, in the int32 kernel (k_modes.cu), on the side stream
        // when both run.  Then the top-k.
        const bool packed = plan.precision == SW_PREC_I16;
        cudaStream_t s32 = packed ? db->side : st;
        const bool forked = packed && !plan.mode_entries.empty();
        if (!plan.mode_entries.empty()) {
            if (forked) {
                SW_CUDA_TRY(cudaEventRecord(db->ev_fork, st));
                SW_CUDA_TRY(cudaStreamWaitEvent(db->side, db->ev_fork, 0));
            }
            for (const ModeEntry &en : plan.mode_entries)
                if (en.m > 0)
                    TIMED_ON(LaunchTimer::OTHER, s32,
                             launch_profile32(d_queries + q_offsets[en.query], en.m, en.m_pad, matrix, db->A,
                                              gap_open, buf.mode_prof + en.prof_off, s32));
            SW_CUDA_TRY(cudaMemsetAsync(buf.mode_counter, 0, sizeof(unsigned long long), s32));
            ModeArgs ma;
            memset(&ma, 0, sizeof ma);
            ma.db = db->view();
            ma.entries = buf.mode_entries;
            ma.n_entries = int32_t(plan.mode_entries.size());
            ma.n_items = plan.mode_items;
            ma.prof = buf.mode_prof;
            ma.gap_open = gap_open;
            ma.gap_extend = gap_extend;
            ma.mode = plan.alignment;
            ma.max_cols = int32_t(db->max_len);
            ma.boundary = buf.mode_bnd;
            ma.work_counter = buf.mode_counter;
            ma.scores = d_scores;
            ma.scores_stride = db->n_seqs;
            TIMED_ON(packed ? LaunchTimer::INTRA : LaunchTimer::INTER, s32, launch_modes_i32(ma, plan.mode_grid, s32));
        }
        for (int32_t qi = 0; qi < n_q; ++qi) {
            const int64_t q0 = q_offsets[qi];
            const int32_t m = int32_t(q_offsets[qi + 1] - q0);
            const int lanes = plan.mode16_lanes[size_t(qi)], rows = plan.mode16_rows[size_t(qi)];
            const int tr = lanes * rows;
            const int64_t cut = plan.mode16_cut[size_t(qi)];
            if (cut < n_pairs) {
                Mode16Args a16;
                memset(&a16, 0, sizeof a16);
                a16.db = db->view();
                a16.pair_begin = cut;
                a16.pair_end = n_pairs;
                a16.query = d_queries + q0;
                a16.m = m;
                a16.virt_rows = int32_t(inter_padded_rows(m, lanes, rows) - m);
                a16.gap_open = gap_open;
                a16.gap_extend = gap_extend;
                memcpy(a16.prof8, ia.prof8, sizeof a16.prof8);
                a16.boundary = m > tr ? buf.mode16_scratch : nullptr;
                a16.slot_stride = int64_t(kCtaThreads / 8) * plan.mode16_cols;
                a16.max_cols = plan.mode16_cols;
                a16.chunk_counter = buf.counters + 3 * n_q + qi;
                a16.scores = d_scores + int64_t(qi) * db->n_seqs;
                TIMED(LaunchTimer::INTER, launch_modes_i16x2(a16, plan.alignment, lanes, rows,
                                                              plan.mode16_grid_max, st));
                last_lanes = lanes;
                last_rows = rows;
            }
        }
        if (forked) {
            SW_CUDA_TRY(cudaEventRecord(db->ev_join, db->side));
            SW_CUDA_TRY(cudaStreamWaitEvent(st, db->ev_join, 0));
        }
        if (top_k > 0 && n_q > 0 && (hits_out != nullptr))
            TIMED(LaunchTimer::OTHER, launch_topk(d_scores, n_q, db->n_seqs, top_k, d_hits, st));
        if (status_out) SW_CUDA_TRY(cudaMemcpyAsync(status_out, d_status, sizeof(int32_t), cudaMemcpyDefault, st));
        return SW_OK;
    }

    // (1) Long sequences of every query: one intra-task launch on the side
    //     stream, concurrent with the per-query launches below.
    if (split) {
        IntraArgs la;
        memset(&la, 0, sizeof la);
        la.db = db->view();
        la.pair_begin = 0;
        la.pair_end = plan.long_end_pair;
        la.n_q = n_q;
        la.q_off = buf.q_off;
        la.queries = d_queries;
        la.gap_open = gap_open;
        la.gap_extend = gap_extend;
        la.sat_limit = plan.sat_limit;
        memcpy(la.prof8, ia.prof8, sizeof la.prof8);
        la.boundary = buf.long_boundary;
        la.boundary_stride = plan.long_codes_bytes / 2;
        la.scores = d_scores;
        la.ovf_list = buf.ovf_list;
        la.list_stride = list_stride;
        la.ovf_count = buf.counters;
        la.ovf_seqs = buf.counters + 2 * n_q;
        la.status = d_status;
        SW_CUDA_TRY(cudaEventRecord(db->ev_fork, st));
        SW_CUDA_TRY(cudaStreamWaitEvent(db->side, db->ev_fork, 0));
        if (plan.long_inter) {
            // one single-strip launch per query, persistent over chunks of 8 long pairs
            const int slots = inter_slots(kLongInterLanes, kLongInterRows / kLongInterLanes, std::max(1, db->sm_count));
            for (int32_t qi = 0; qi < n_q; ++qi) {
                const int32_t m = int32_t(q_offsets[qi + 1] - q_offsets[qi]);
                if (m == 0) continue;
                InterArgs lb = ia;
                lb.query = d_queries + q_offsets[qi];
                lb.m = m;
                lb.scores = d_scores + size_t(qi) * size_t(db->n_seqs);
                lb.ovf_list = buf.ovf_list + size_t(qi) * size_t(list_stride);
                lb.ovf_count = buf.counters + qi;
                lb.ovf_seqs = buf.counters + 2 * n_q + qi;
                lb.pair_begin = 0;
                lb.pair_end = plan.long_end_pair;
                lb.boundary = nullptr;
                lb.max_cols = 0;
                lb.slot_stride = 0;
                lb.chunk_counter = buf.counters + 4 * std::max<int32_t>(n_q, 1) + 5 + qi;
                TIMED_ON(LaunchTimer::INTRA, db->side,
                         launch_inter_i16x2(lb, kLongInterLanes, kLongInterRows / kLongInterLanes, db->side, slots));
            }
        } else {
            TIMED_ON(LaunchTimer::INTRA, db->side, launch_intra_i16x2(la, plan.warps_long, plan.rows_long, db->side));
        }
        SW_CUDA_TRY(cudaEventRecord(db->ev_join, db->side));
    }

    // (2b) Batched form: every query pair against the rest of the database in
    //      one persistent launch.
    if (plan.mode == SW_MODE_BATCHED && db->n_seqs > 0) {
        for (int32_t qi = 0; qi < n_q; ++qi)
            if (q_offsets[qi + 1] == q_offsets[qi])
                SW_CUDA_TRY(cudaMemsetAsync(d_scores + size_t(qi) * size_t(db->n_seqs), 0,
                                            sizeof(int32_t) * size_t(db->n_seqs), st));
        for (size_t gi = 0; gi < plan.groups.size() && plan.batch_seq_begin < db->n_sorted; ++gi) {
            const Plan::BatchGroup &g = plan.groups[gi];
            const int spc = kCtaThreads / g.lanes;
            BatchArgs ba;
            memset(&ba, 0, sizeof ba);
            ba.db = db->view();
            ba.seq_begin = plan.batch_seq_begin;
            ba.seq_end = db->n_sorted;
            ba.n_chunks = int32_t((db->n_sorted - plan.batch_seq_begin + spc - 1) / spc);
            ba.n_qp = g.count;
            ba.qp_a = buf.qp + g.begin;
            ba.qp_b = buf.qp + n_qp + g.begin;
            ba.q_off = buf.q_off;
            ba.queries = d_queries;
            ba.gap_open = gap_open;
            ba.gap_extend = gap_extend;
            ba.sat_limit = plan.sat_limit;
            memcpy(ba.prof8, ia.prof8, sizeof ba.prof8);
            ba.scratch = buf.batch_scratch;
            ba.max_cols = plan.batch_max_cols;
            ba.scratch_stride = int64_t(spc) * plan.batch_max_cols;
            ba.scores = d_scores;
            ba.ovf_list = buf.ovf_list;
            ba.list_stride = list_stride;
            ba.ovf_count = buf.counters;
            ba.ovf_seqs = buf.counters + 2 * n_q;
            ba.tile_counter = d_tiles + (gi & 3);
            last_lanes = g.lanes;
            last_rows = g.rows;
            TIMED(LaunchTimer::INTER, launch_batch_i16x2(ba, g.lanes, g.rows, g.grid, st, main_priority));
        }
    }

    // (2) Plain form: one inter-task launch per query over the rest of the database.
    for (int32_t qi = 0; qi < n_q && db->n_seqs > 0 && plan.mode == SW_MODE_PLAIN; ++qi) {
        const int32_t m = int32_t(q_offsets[qi + 1] - q_offsets[qi]);
        int32_t *row = d_scores + size_t(qi) * size_t(db->n_seqs);
        if (m == 0) {
            SW_CUDA_TRY(cudaMemsetAsync(row, 0, sizeof(int32_t) * size_t(db->n_seqs), st));
            continue;
        }
        const uint8_t *q = d_queries + q_offsets[qi];
        if (plan.precision == SW_PREC_I16) {
            ia.query = q;
            ia.m = m;
            ia.scores = row;
            ia.ovf_list = buf.ovf_list + size_t(qi) * size_t(list_stride);
            ia.ovf_count = buf.counters + qi;
            ia.ovf_seqs = buf.counters + 2 * n_q + qi;
            ia.pair_begin = plan.long_end_pair;
            ia.pair_end = n_pairs;
            int lanes = plan.lanes, rows = plan.rows;
            if (plan.auto_shape) query_shape(plan, m, &lanes, &rows);
            last_lanes = lanes;
            last_rows = rows;
            // persistent grid, per-slot boundary scratch (stays in L2)
            ia.boundary = buf.inter_scratch;
            ia.max_cols = plan.inter_max_cols;
            ia.slot_stride = int64_t(kCtaThreads / lanes) * plan.inter_max_cols;
            ia.chunk_counter = d_chunks + qi;
            const int slots = inter_slots(lanes, rows, std::max(1, db->sm_count));
            TIMED(LaunchTimer::INTER, launch_inter_i16x2(ia, lanes, rows, st, slots, main_priority));
        } else {
            const int tr32 = plan.lanes32 * plan.rows32;
            const int32_t m_pad = int32_t(round_up(m, tr32));
            TIMED(LaunchTimer::OTHER, launch_profile32(q, m, m_pad, matrix, db->A, gap_open, buf.prof32, st));
            ja.m = m;
            ja.m_pad = m_pad;
            ja.scores = row;
            ja.list = nullptr;
            ja.list_count = nullptr;
            ja.pair_begin = 0;
            ja.pair_end = n_pairs;
            ja.work_counter = buf.counters + n_q + qi;
            TIMED(LaunchTimer::INTER, launch_i32(ja, plan.lanes32, plan.rows32, grid32, st));
        }
    }
    if (split) SW_CUDA_TRY(cudaStreamWaitEvent(st, db->ev_join, 0));

    // (3) Exact int32 rescore of the sequences whose int16 maximum saturated
    //     (skipped for a query none of whose scores can reach the limit).
    if (plan.precision == SW_PREC_I16) {
        for (int32_t qi = 0; qi < n_q && db->n_seqs > 0; ++qi) {
            const int32_t m = int32_t(q_offsets[qi + 1] - q_offsets[qi]);
            if (m == 0) continue;
            if (std::min<int64_t>(m, db->max_len) * plan.smax_local < plan.sat_limit) continue;
            const uint8_t *q = d_queries + q_offsets[qi];
            const int tr32 = plan.lanes32 * plan.rows32;
            const int32_t m_pad = int32_t(round_up(m, tr32));
            TIMED(LaunchTimer::OTHER, launch_profile32(q, m, m_pad, matrix, db->A, gap_open, buf.prof32, st));
            ja.m = m;
            ja.m_pad = m_pad;
            ja.scores = d_scores + size_t(qi) * size_t(db->n_seqs);
            ja.list = buf.ovf_list + size_t(qi) * size_t(list_stride);
            ja.list_count = buf.counters + qi;
            ja.work_counter = buf.counters + n_q + qi;
            TIMED(LaunchTimer::RESCORE, launch_i32(ja, plan.lanes32, plan.rows32, grid32, st));
        }
    }
    if (top_k > 0 && n_q > 0 && (hits_out != nullptr))
        TIMED(LaunchTimer::OTHER, launch_topk(d_scores, n_q, db->n_seqs, top_k, d_hits, st));
    // the device-side status (a bounded wait that gave up), for asynchronous callers
    if (status_out) SW_CUDA_TRY(cudaMemcpyAsync(status_out, d_status, sizeof(int32_t), cudaMemcpyDefault, st));
    return SW_OK;
    };

    bool graph_replayed = false;
    if (opts && (opts->flags & SW_FLAG_GRAPH)) {
        // Everything the captured work depends on, byte for byte.
        std::string key;
        auto put = [&key](const void *p, size_t n) { key.append(static_cast<const char *>(p), n); };
        const void *ptrs[] = {d_queries, d_scores, d_hits, ws, st, status_out};
        put(ptrs, sizeof ptrs);
        const int32_t ints[] = {n_q, gap_open, gap_extend, top_k, plan.mode, plan.precision, plan.lanes, plan.rows,
                                hits_out != nullptr, plan.rows_long, plan.warps_long, plan.alignment};
        put(ints, sizeof ints);
        put(&plan.long_end_pair, sizeof plan.long_end_pair);
        put(&db->tuning_version, sizeof db->tuning_version);
        if (n_q > 0) put(q_offsets, sizeof(int64_t) * size_t(n_q + 1));
        put(matrix, sizeof(int32_t) * size_t(db->A) * size_t(db->A));
        if (!(db->graph_exec && db->graph_key == key)) {
            if (db->graph_exec) cudaGraphExecDestroy(db->graph_exec);
            db->graph_exec = nullptr;
            db->graph_key.clear();
            timer.on = false;   // per-launch events cannot outlive this call inside a graph
            SW_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int erc = enqueue();
            cudaGraph_t graph = nullptr;
            const cudaError_t cap = cudaStreamEndCapture(st, &graph);
            if (erc) {
                if (graph) cudaGraphDestroy(graph);
                return erc;
            }
            if (cap != cudaSuccess) return fail(SW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(cap));
            const cudaError_t ie = cudaGraphInstantiate(&db->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                db->graph_exec = nullptr;
                return fail(SW_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
            }
            db->graph_key = key;
        } else {
            graph_replayed = true;
            // the plan's per-query launch shapes are the same as when captured
            if (plan.alignment != SW_ALIGN_LOCAL) {
                if (plan.precision == SW_PREC_I16 && n_q > 0) {
                    last_lanes = plan.mode16_lanes.back();
                    last_rows = plan.mode16_rows.back();
                }
            } else if (plan.precision == SW_PREC_I16 && plan.mode == SW_MODE_PLAIN && plan.auto_shape && n_q > 0) {
                query_shape(plan, q_offsets[n_q] - q_offsets[n_q - 1], &last_lanes, &last_rows);
            }
        }
        SW_CUDA_TRY(cudaGraphLaunch(db->graph_exec, st));
    } else {
        rc = enqueue();
        if (rc) return rc;
    }

    bool sync = false;
    if (scores_out && !s_dev && n_q > 0 && db->n_seqs > 0) {
        SW_CUDA_TRY(cudaMemcpyAsync(scores_out, d_scores, sizeof(int32_t) * size_t(n_q) * size_t(db->n_seqs),
                                    cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    if (hits_out && !h_dev && top_k > 0 && n_q > 0) {
        SW_CUDA_TRY(cudaMemcpyAsync(hits_out, d_hits, sizeof(sw_hit) * size_t(n_q) * size_t(top_k),
                                    cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    if (stats) {
        std::vector<int32_t> cnt(size_t(std::max(n_q, 1)), 0);
        if (n_q > 0 && plan.precision == SW_PREC_I16)
            SW_CUDA_TRY(cudaMemcpyAsync(cnt.data(), buf.counters + 2 * n_q, sizeof(int32_t) * size_t(n_q),
                                        cudaMemcpyDeviceToHost, st));
        SW_CUDA_TRY(cudaStreamSynchronize(st));
        stats->cells = plan.total_m * db->residues;
        int64_t r = 0;
        if (plan.precision == SW_PREC_I16)
            for (int32_t i = 0; i < n_q; ++i) r += cnt[size_t(i)];
        stats->rescored = r;
        stats->long_sequences = plan.n_long;
        stats->long_cells = plan.alignment != SW_ALIGN_LOCAL ? plan.mode_i32_cells : plan.total_m * plan.long_residues;
        stats->inter_cells = stats->cells - stats->long_cells;
        stats->precision_used = plan.precision;
        stats->mode_used = plan.mode;
        stats->lanes_used = plan.precision == SW_PREC_I16 ? last_lanes : plan.lanes32;
        stats->rows_per_lane_used = plan.precision == SW_PREC_I16 ? last_rows : plan.rows32;
        stats->launches = timer.launches;
        stats->graph_replayed = graph_replayed ? 1 : 0;
        stats->inter_ms = timer.total(LaunchTimer::INTER);
        stats->rescore_ms = timer.total(LaunchTimer::RESCORE);
        stats->intra_ms = timer.total(LaunchTimer::INTRA);
        stats->other_ms = timer.total(LaunchTimer::OTHER);
        stats->inter_launches = int32_t(timer.ev[LaunchTimer::INTER].size());
        sync = false;
    }
    if (sync) SW_CUDA_TRY(cudaStreamSynchronize(st));
    if (sync || stats) {
        int32_t status = 0;
        SW_CUDA_TRY(cudaMemcpy(&status, d_status, sizeof status, cudaMemcpyDeviceToHost));
        if (status) return fail(SW_ERR_TIMEOUT, "a bounded device-side wait gave up (intra-task kernel)");
    }
    SW_CUDA_TRY(cudaGetLastError());
    return SW_OK;
}

int sw_top_k(const int32_t *scores, int64_t n_rows, int64_t n_cols, int32_t top_k, sw_hit *hits, void *stream) {
    g_last_error.clear();
    if (n_rows < 0 || n_cols < 0 || top_k < 0 || top_k > 4096) return fail(SW_ERR_INVALID_ARG, "bad size");
    if (n_rows == 0 || top_k == 0) return SW_OK;
    if (!scores && n_cols > 0) return fail(SW_ERR_INVALID_ARG, "scores is NULL");
    if (!hits) return fail(SW_ERR_INVALID_ARG, "hits is NULL");
    if (n_cols > (int64_t(1) << 31) - 2) return fail(SW_ERR_INVALID_ARG, "n_cols too large");
    SW_CUDA_TRY(launch_topk(scores, n_rows, n_cols, top_k, hits, static_cast<cudaStream_t>(stream)));
    return SW_OK;
}

int sw_probe_wait_timeout(int device, int64_t spin_iters, int32_t *status_out, double *elapsed_ms) {
    g_last_error.clear();
    if (!status_out || !elapsed_ms) return fail(SW_ERR_INVALID_ARG, "NULL argument");
    if (spin_iters < 1 || spin_iters > (int64_t(1) << 25)) return fail(SW_ERR_INVALID_ARG, "spin_iters must be 1..2^25");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return fail(SW_ERR_INVALID_ARG, "no such CUDA device");
    }
    DeviceGuard guard(device);
    int32_t *status = nullptr;
    SW_CUDA_TRY(cudaMalloc(&status, sizeof(int32_t)));
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t err = cudaMemset(status, 0, sizeof(int32_t));
    if (err == cudaSuccess) err = launch_wait_probe((long long)spin_iters, status, nullptr);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    int32_t h = 0;
    if (err == cudaSuccess) err = cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost);
    *elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    cudaFree(status);
    if (err != cudaSuccess) return fail(SW_ERR_CUDA, cudaGetErrorString(err));
    *status_out = h;
    return SW_OK;
}

int sw_probe_alu_rate(int device, int32_t mode, double *per_sm_cycle, int32_t *sm_count) {
    g_last_error.clear();
    if (!per_sm_cycle || !sm_count || mode < 0 || mode > 3) return fail(SW_ERR_INVALID_ARG, "bad argument");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(SW_ERR_INVALID_ARG, "no such CUDA device");
    }
    DeviceGuard guard(device);
    int sms = 0;
    SW_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int per_sm = std::max(1, probe_blocks_per_sm(mode));
    const int grid = sms * per_sm;
    unsigned long long *cycles = nullptr;
    uint32_t *sink = nullptr;
    SW_CUDA_TRY(cudaMalloc(&cycles, sizeof(unsigned long long)));
    SW_CUDA_TRY(cudaMalloc(&sink, sizeof(uint32_t)));
    const int iters = mode == 0 ? 20000 : 20000;
    double best = 0.0;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
        unsigned long long c = 0;
        err = cudaMemset(cycles, 0, sizeof c);
        if (err == cudaSuccess) err = launch_probe(mode, grid, iters, cycles, sink, nullptr);
        if (err == cudaSuccess) err = cudaDeviceSynchronize();
        if (err == cudaSuccess) err = cudaMemcpy(&c, cycles, sizeof c, cudaMemcpyDeviceToHost);
        if (err == cudaSuccess && c > 0) {
            const double per_thread = probe_work_per_iteration(mode);
            const double work = double(grid) * kCtaThreads * double(iters) * per_thread;
            best = std::max(best, work / (double(c) * sms));
        }
    }
    cudaFree(cycles);
    cudaFree(sink);
    if (err != cudaSuccess) return fail(SW_ERR_CUDA, cudaGetErrorString(err));
    *per_sm_cycle = best;
    *sm_count = sms;
    return SW_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// alignments (traceback) of chosen pairs

namespace {

int check_align_pairs(const sw_db *db, const int64_t *q_offsets, int32_t n_q, const int32_t *pair_query,
                      const int64_t *pair_target, int64_t n_pairs) {
    if (!db) return fail(SW_ERR_INVALID_ARG, "db is NULL");
    if (n_q < 0 || n_pairs < 0) return fail(SW_ERR_INVALID_ARG, "negative count");
    if (n_pairs == 0) return SW_OK;
    if (!pair_query || !pair_target) return fail(SW_ERR_INVALID_ARG, "pair arrays are NULL");
    if (n_q == 0 || !q_offsets) return fail(SW_ERR_INVALID_ARG, "no queries");
    if (q_offsets[0] != 0) return fail(SW_ERR_INVALID_ARG, "q_offsets[0] must be 0");
    for (int32_t i = 0; i < n_q; ++i) {
        const int64_t m = q_offsets[i + 1] - q_offsets[i];
        if (m < 0) return fail(SW_ERR_INVALID_ARG, "q_offsets must be non-decreasing");
        if (m > (int64_t(1) << 30)) return fail(SW_ERR_INVALID_ARG, "query longer than 2^30");
    }
    for (int64_t k = 0; k < n_pairs; ++k) {
        if (pair_query[k] < 0 || pair_query[k] >= n_q) return fail(SW_ERR_INVALID_ARG, "pair_query out of range");
        if (pair_target[k] < 0 || pair_target[k] >= db->n_seqs)
            return fail(SW_ERR_INVALID_ARG, "pair_target out of range");
    }
    return SW_OK;
}

int64_t pair_len_q(const int64_t *q_offsets, int32_t qi) { return q_offsets[qi + 1] - q_offsets[qi]; }
int64_t pair_len_t(const sw_db *db, int64_t ti) { return db->h_len[size_t(db->h_sorted_pos[size_t(ti)])]; }

// Device bytes of one pair's traceback scratch (checkpoints, flags, reversed
// and ordered ops), each part rounded to 256 bytes.
int64_t align_pair_bytes(int64_t m, int64_t n) {
    const int64_t ck = align_checkpoint_rows(int32_t(m)) * (n + 1) * int64_t(sizeof(int2));
    const int64_t fl = int64_t(align_strip_rows()) * n;
    auto r256 = [](int64_t x) { return (x + 255) & ~int64_t(255); };
    return r256(ck) + r256(fl) + 2 * r256(m + n);
}

constexpr int64_t kAlignChunkBytes = int64_t(1) << 30;

}  // namespace

extern "C" {

int sw_align_ops_capacity(const sw_db *db, const int64_t *q_offsets, int32_t n_q, const int32_t *pair_query,
                          const int64_t *pair_target, int64_t n_pairs, int64_t *bytes) {
    g_last_error.clear();
    if (!bytes) return fail(SW_ERR_INVALID_ARG, "bytes is NULL");
    const int rc = check_align_pairs(db, q_offsets, n_q, pair_query, pair_target, n_pairs);
    if (rc) return rc;
    int64_t total = 0;
    for (int64_t k = 0; k < n_pairs; ++k)
        total += pair_len_q(q_offsets, pair_query[k]) + pair_len_t(db, pair_target[k]);
    *bytes = total;
    return SW_OK;
}

int sw_align_mode(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q,
                  const int32_t *pair_query, const int64_t *pair_target, int64_t n_pairs, const int32_t *matrix,
                  int32_t gap_open, int32_t gap_extend, int32_t alignment, sw_alignment *alignments_out,
                  uint8_t *ops_out, int64_t ops_capacity, sw_align_stats *stats, void *stream) {
    g_last_error.clear();
    if (alignment < SW_ALIGN_LOCAL || alignment > SW_ALIGN_OVERLAP)
        return fail(SW_ERR_INVALID_ARG, "unknown alignment mode");
    int rc = check_align_pairs(db, q_offsets, n_q, pair_query, pair_target, n_pairs);
    if (rc) return rc;
    if (!matrix) return fail(SW_ERR_INVALID_ARG, "matrix is NULL");
    if (gap_open < 0 || gap_extend < 0) return fail(SW_ERR_INVALID_ARG, "gap penalties must be >= 0");
    if (stats) memset(stats, 0, sizeof *stats);
    if (n_pairs == 0) return SW_OK;
    if (!alignments_out) return fail(SW_ERR_INVALID_ARG, "alignments_out is NULL");
    int64_t ops_need = 0, max_min_len = 0, max_sum_len = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int64_t m = pair_len_q(q_offsets, pair_query[k]), n = pair_len_t(db, pair_target[k]);
        ops_need += m + n;
        max_min_len = std::max(max_min_len, std::min(m, n));
        max_sum_len = std::max(max_sum_len, m + n);
    }
    if (ops_need > 0 && (!ops_out || ops_capacity < ops_need))
        return fail(SW_ERR_INVALID_ARG, "ops_capacity too small (see sw_align_ops_capacity)");
    // int32 arithmetic: the limits of sw_search's int32 path.
    const int A = db->A;
    int smax = matrix[0], smin = matrix[0];
    for (int i = 0; i < A * A; ++i) {
        smax = std::max(smax, matrix[i]);
        smin = std::min(smin, matrix[i]);
    }
    const int64_t absmax = std::max<int64_t>(smax, -int64_t(smin));
    if (absmax > (1 << 20) || int64_t(gap_open) + gap_extend > (int64_t(1) << 28) ||
        max_min_len * std::max(smax, 0) + gap_open + gap_extend + absmax > (int64_t(1) << 28))
        return fail(SW_ERR_OVERFLOW, "matrix entries, penalties or lengths too large for exact int32 scores");
    // no zero floor: values go down to about -(m + n) * (max|S| + o + e), as in sw_search
    if (alignment != SW_ALIGN_LOCAL && max_sum_len * (absmax + int64_t(gap_open) + gap_extend) >= (int64_t(1) << 28))
        return fail(SW_ERR_OVERFLOW, "lengths, matrix entries or penalties too large for exact int32 scores "
                                     "of this alignment mode");

    std::lock_guard<std::mutex> lock(db->mu);
    DeviceGuard guard(db->device);
    const int64_t total_q = q_offsets[n_q];
    if (total_q > 0 && !queries) return fail(SW_ERR_INVALID_ARG, "queries is NULL");
    const bool q_dev = total_q == 0 || is_device_ptr(queries);
    if (!q_dev)
        for (int64_t i = 0; i < total_q; ++i)
            if (queries[i] >= A) return fail(SW_ERR_INVALID_ARG, "query residue code >= alphabet_size");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : db->stream;

    // Chunks of pairs whose scratch stays under kAlignChunkBytes (a single
    // larger pair forms a chunk of its own).
    std::vector<int64_t> chunk_begin{0};
    int64_t acc = 0, max_chunk_scratch = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int64_t b = align_pair_bytes(pair_len_q(q_offsets, pair_query[k]), pair_len_t(db, pair_target[k]));
        if (acc > 0 && acc + b > kAlignChunkBytes) {
            chunk_begin.push_back(k);
            max_chunk_scratch = std::max(max_chunk_scratch, acc);
            acc = 0;
        }
        acc += b;
    }
    max_chunk_scratch = std::max(max_chunk_scratch, acc);
    chunk_begin.push_back(n_pairs);
    int64_t max_chunk_pairs = 0;
    for (size_t c = 0; c + 1 < chunk_begin.size(); ++c)
        max_chunk_pairs = std::max(max_chunk_pairs, chunk_begin[c + 1] - chunk_begin[c]);

    auto r256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t q_bytes = q_dev ? 0 : r256(size_t(total_q));
    const size_t mat_bytes = r256(sizeof(int32_t) * kProfRows * kProfRows);
    // forward pass: one profile table S(q_i, c), [32][round_up(m, 256)], per query in the pairs
    std::vector<int64_t> prof_off(size_t(n_q), -1);
    int64_t prof_elems = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t q = pair_query[k];
        if (prof_off[size_t(q)] >= 0) continue;
        prof_off[size_t(q)] = prof_elems;
        prof_elems += int64_t(kProfRows) * round_up(std::max<int64_t>(pair_len_q(q_offsets, q), 1), align_strip_rows());
    }
    const size_t prof_bytes = r256(sizeof(int32_t) * size_t(prof_elems));
    const size_t pairs_bytes = r256(sizeof(AlignPairDev) * size_t(max_chunk_pairs));
    const size_t res_bytes = r256(sizeof(AlignResultDev) * size_t(max_chunk_pairs));
    const size_t need = q_bytes + mat_bytes + prof_bytes + pairs_bytes + res_bytes + size_t(max_chunk_scratch) + 256;
    if (db->ws_bytes < need) {
        SW_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(db->ws);
        db->ws = nullptr;
        db->ws_bytes = 0;
        SW_CUDA_TRY(cudaMalloc(&db->ws, need));
        db->ws_bytes = need;
    }
    uint8_t *w = static_cast<uint8_t *>(db->ws);
    uint8_t *d_q = q_dev ? const_cast<uint8_t *>(queries) : w;
    int32_t *d_mat = reinterpret_cast<int32_t *>(w + q_bytes);
    int32_t *d_prof = reinterpret_cast<int32_t *>(w + q_bytes + mat_bytes);
    AlignPairDev *d_pairs = reinterpret_cast<AlignPairDev *>(w + q_bytes + mat_bytes + prof_bytes);
    AlignResultDev *d_res = reinterpret_cast<AlignResultDev *>(w + q_bytes + mat_bytes + prof_bytes + pairs_bytes);
    uint8_t *d_scratch = w + q_bytes + mat_bytes + prof_bytes + pairs_bytes + res_bytes;

    std::vector<int32_t> mat(kProfRows * kProfRows, 0);
    for (int x = 0; x < A; ++x)
        for (int y = 0; y < A; ++y) mat[size_t(x * kProfRows + y)] = matrix[x * A + y];
    if (!q_dev && total_q > 0) SW_CUDA_TRY(cudaMemcpyAsync(d_q, queries, size_t(total_q), cudaMemcpyHostToDevice, st));
    SW_CUDA_TRY(cudaMemcpyAsync(d_mat, mat.data(), sizeof(int32_t) * mat.size(), cudaMemcpyHostToDevice, st));
    for (int32_t q = 0; q < n_q; ++q) {
        const int64_t m = pair_len_q(q_offsets, q);
        if (prof_off[size_t(q)] < 0 || m == 0) continue;
        const int32_t m_pad = int32_t(round_up(m, align_strip_rows()));
        SW_CUDA_TRY(launch_profile32(d_q + q_offsets[q], int32_t(m), m_pad, matrix, A, 0, d_prof + prof_off[size_t(q)], st));
    }

    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (stats)
        for (auto &x : ev) SW_CUDA_TRY(cudaEventCreate(&x));
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree() {
            for (int i = 0; i < 3; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } ev_free{ev};

    int64_t ops_base = 0;
    std::vector<AlignPairDev> hp;
    std::vector<AlignResultDev> hr;
    for (size_t c = 0; c + 1 < chunk_begin.size(); ++c) {
        const int64_t k0 = chunk_begin[c], k1 = chunk_begin[c + 1], np = k1 - k0;
        hp.assign(size_t(np), AlignPairDev{});
        // scratch layout of the chunk: ckpt | flags | rev | ops, each pair's part 256-byte aligned
        int64_t ck = 0, fl = 0, rv = 0, op = 0;
        for (int64_t k = k0; k < k1; ++k) {
            AlignPairDev &d = hp[size_t(k - k0)];
            const int64_t m = pair_len_q(q_offsets, pair_query[k]), n = pair_len_t(db, pair_target[k]);
            d.q_off = q_offsets[pair_query[k]];
            d.t_sorted = db->h_sorted_pos[size_t(pair_target[k])];
            d.m = int32_t(m);
            d.n = int32_t(n);
            d.prof_off = prof_off[size_t(pair_query[k])];
            d.m_pad = int32_t(round_up(std::max<int64_t>(m, 1), align_strip_rows()));
            d.ckpt_off = ck / int64_t(sizeof(int2));
            ck += r256(size_t(align_checkpoint_rows(int32_t(m)) * (n + 1) * int64_t(sizeof(int2))));
            d.flags_off = fl;
            fl += r256(size_t(int64_t(align_strip_rows()) * n));
            d.rev_off = rv;
            rv += r256(size_t(m + n));
            d.ops_off = op;
            op += m + n;
        }
        AlignArgs a;
        memset(&a, 0, sizeof a);
        a.db = db->view();
        a.queries = d_q;
        a.pairs = d_pairs;
        a.n_pairs = np;
        a.results = d_res;
        a.mat = d_mat;
        a.prof = d_prof;
        a.ckpt = reinterpret_cast<int2 *>(d_scratch);
        a.flags = d_scratch + ck;
        a.rev = d_scratch + ck + fl;
        a.ops = d_scratch + ck + fl + rv;
        a.gap_open = gap_open;
        a.gap_extend = gap_extend;
        a.mode = alignment;
        SW_CUDA_TRY(cudaMemcpyAsync(d_pairs, hp.data(), sizeof(AlignPairDev) * size_t(np), cudaMemcpyHostToDevice, st));
        if (stats) SW_CUDA_TRY(cudaEventRecord(ev[0], st));
        SW_CUDA_TRY(launch_align(a, 0, st));
        if (stats) SW_CUDA_TRY(cudaEventRecord(ev[1], st));
        SW_CUDA_TRY(launch_align(a, 1, st));
        if (stats) SW_CUDA_TRY(cudaEventRecord(ev[2], st));
        hr.assign(size_t(np), AlignResultDev{});
        SW_CUDA_TRY(cudaMemcpyAsync(hr.data(), d_res, sizeof(AlignResultDev) * size_t(np), cudaMemcpyDeviceToHost, st));
        if (op > 0) SW_CUDA_TRY(cudaMemcpyAsync(ops_out + ops_base, a.ops, size_t(op), cudaMemcpyDeviceToHost, st));
        SW_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t k = k0; k < k1; ++k) {
            const AlignResultDev &r = hr[size_t(k - k0)];
            if (r.status == 5) return fail(SW_ERR_TIMEOUT, "traceback forward pass: a wait between strips ran out");
            if (r.status != 0) return fail(SW_ERR_CUDA, "traceback walk met an inconsistent cell");
            sw_alignment &o = alignments_out[k];
            o.score = r.score;
            o.reserved = 0;
            o.q_begin = r.i_begin;
            o.q_end = r.i_end;
            o.t_begin = r.j_begin;
            o.t_end = r.j_end;
            o.ops_offset = ops_base + hp[size_t(k - k0)].ops_off;
            o.ops_len = r.n_ops;
            if (stats) {
                stats->forward_cells += int64_t(hp[size_t(k - k0)].m) * hp[size_t(k - k0)].n;
                stats->traceback_cells += r.cells;
            }
        }
        if (stats) {
            float t0 = 0.f, t1 = 0.f;
            SW_CUDA_TRY(cudaEventElapsedTime(&t0, ev[0], ev[1]));
            SW_CUDA_TRY(cudaEventElapsedTime(&t1, ev[1], ev[2]));
            stats->forward_ms += t0;
            stats->traceback_ms += t1;
            stats->launches += 2;
        }
        ops_base += op;
    }
    return SW_OK;
}

int sw_align(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q, const int32_t *pair_query,
             const int64_t *pair_target, int64_t n_pairs, const int32_t *matrix, int32_t gap_open,
             int32_t gap_extend, sw_alignment *alignments_out, uint8_t *ops_out, int64_t ops_capacity,
             sw_align_stats *stats, void *stream) {
    return sw_align_mode(db, queries, q_offsets, n_q, pair_query, pair_target, n_pairs, matrix, gap_open, gap_extend,
                         SW_ALIGN_LOCAL, alignments_out, ops_out, ops_capacity, stats, stream);
}

}  // extern "C"
