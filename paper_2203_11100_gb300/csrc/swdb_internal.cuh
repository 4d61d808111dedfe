// Internal declarations shared by the translation units of libswdb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace swdb {

// Residue code used for padding past the end of a sequence.  Its profile
// entries are negative, which never raises a local-alignment maximum when
// the padding sits after the last real row/column (all dependencies in the
// recurrences run up and left).
constexpr int kPadCode = 31;
constexpr int kProfRows = 32;           // profile rows: 31 codes + padding
constexpr int kBundleSeqs = 16;         // sequences per interleaved bundle
constexpr int kBundlePairs = kBundleSeqs / 2;
constexpr int kQuadBytes = 8;           // 4 columns x (code A, code B)
constexpr int kBundleRowBytes = kBundlePairs * kQuadBytes;  // 64 bytes per 4 columns
constexpr int kCtaThreads = 256;

// Device view of the resident database.
//
// Sequences are sorted by length, longest first (stable), and cut into
// bundles of 16.  Sequence 2p and 2p+1 of the sorted order form pair p;
// bundle b holds pairs 8b..8b+7.  Bundle b occupies bundle_len[b] columns
// (its longest length rounded up to 4) starting at byte bundle_off[b]:
//   byte bundle_off[b] + (j/4)*64 + slot*8 + (j%4)*2 + h
// is column j of sequence 2*(8b+slot)+h.  Neighbouring pairs therefore read
// neighbouring 8-byte words for the same 4 columns (a coalesced, position-
// major interleave).
struct DbView {
    const uint8_t *codes;
    const int64_t *bundle_off;  // [n_bundles]
    const int32_t *bundle_len;  // [n_bundles]
    const int32_t *len;         // [n_sorted] sorted lengths (0 for padding slots)
    const int64_t *perm;        // [n_sorted] sorted -> original index (-1 for padding)
    int64_t n_seqs;
    int64_t n_sorted;           // n_bundles * 16
    int64_t n_bundles;
};

// Arguments of the packed int16x2 inter-task kernel: one query against the
// pairs [pair_begin, pair_end) of the sorted database.
struct InterArgs {
    DbView db;
    int64_t pair_begin, pair_end;
    const uint8_t *query;       // device, m codes
    int32_t m;
    int32_t gap_open, gap_extend;
    int32_t sat_limit;          // flag a sequence when its int16 maximum H >= sat_limit
    int8_t prof8[kProfRows][kProfRows];  // [query code][db code] = S + o, pads = -128
    // Strip-boundary scratch for multi-pass queries, one of two layouts:
    //  slot_stride == 0: per database pair, 4 bytes per layout byte (grid: one
    //                    CTA per chunk of pairs);
    //  slot_stride  > 0: per resident CTA slot, slot_stride uint2 entries each,
    //                    max_cols per subwarp (persistent grid pulling chunks
    //                    from *chunk_counter; the scratch is reused and stays in L2).
    uint2 *boundary;
    int64_t slot_stride;
    int32_t max_cols;
    int32_t *chunk_counter;     // persistent grid only; zeroed before launch
    int32_t *scores;            // row of this query, original database order
    int32_t *ovf_list;          // entries pair*4 + mask of saturated halves
    int32_t *ovf_count;
    int32_t *ovf_seqs;          // sequences flagged (one or two per list entry)
    int32_t *status;            // nonzero after a bounded wait gave up (intra-task kernel)
};

// Arguments of the intra-task kernel: every query against the long pairs
// [pair_begin, pair_end) in one launch, one CTA per (pair, query).
struct IntraArgs {
    DbView db;
    int64_t pair_begin, pair_end;
    int32_t n_q;
    const int64_t *q_off;       // device, n_q+1 query offsets
    const uint8_t *queries;     // device, all query codes
    int32_t gap_open, gap_extend;
    int32_t sat_limit;
    int8_t prof8[kProfRows][kProfRows];
    uint2 *boundary;            // per-query scratch regions (null when no query needs one)
    int64_t boundary_stride;    // uint2 entries per query
    int32_t *scores;            // [n_q][n_seqs]
    int32_t *ovf_list;          // [n_q][list_stride]
    int64_t list_stride;
    int32_t *ovf_count;         // [n_q]
    int32_t *ovf_seqs;          // [n_q]
    int32_t *status;
};

// Arguments of the batched persistent kernel: query pairs (qp_a[i], qp_b[i];
// qp_b = -1 for a lone query) against the sorted sequences
// [seq_begin, seq_end), tiles = chunks of 256/T sequences x query pairs.
struct BatchArgs {
    DbView db;
    int64_t seq_begin, seq_end;
    int32_t n_chunks;
    int32_t n_qp;
    const int32_t *qp_a;
    const int32_t *qp_b;
    const int64_t *q_off;       // device, n_q+1
    const uint8_t *queries;     // device
    int32_t gap_open, gap_extend;
    int32_t sat_limit;
    int8_t prof8[kProfRows][kProfRows];
    uint2 *scratch;             // per CTA slot, per subwarp boundary rows (null: single pass)
    int64_t scratch_stride;     // uint2 entries per CTA slot
    int32_t max_cols;           // uint2 entries per subwarp (>= any chunk's columns)
    int32_t *scores;            // [n_q][n_seqs]
    int32_t *ovf_list;          // [n_q][list_stride]
    int64_t list_stride;
    int32_t *ovf_count;         // [n_q]
    int32_t *ovf_seqs;          // [n_q]
    int32_t *tile_counter;      // zeroed before launch
};

// Arguments of the int32 kernel.  Work items are pairs with a mask of the
// halves to score; either an explicit list (ovf_list/ovf_count) or, when
// list is null, every pair in [pair_begin, pair_end) with mask 3.
struct I32Args {
    DbView db;
    int64_t pair_begin, pair_end;
    const int32_t *list;
    const int32_t *list_count;
    int32_t *work_counter;      // zeroed before launch
    const int32_t *prof32;      // [kProfRows][m_pad] = S + o, pads large negative
    int32_t m, m_pad;
    int32_t gap_open, gap_extend;
    uint2 *boundary;
    int32_t *scores;
    int32_t *status;            // set to nonzero on an internal error
};

// Traceback of chosen pairs (k_align.cu).  One descriptor per pair; every
// offset is into the buffer named beside it.
struct AlignPairDev {
    int64_t q_off;        // queries: first residue of the query
    int64_t t_sorted;     // sorted database position of the target
    int64_t ckpt_off;     // ckpt (int2 units): ceil(m/256) rows of n+1 (H, F)
    int64_t flags_off;    // flags (bytes): one strip, 256 x n
    int64_t rev_off;      // rev (bytes): m + n reversed ops
    int64_t ops_off;      // ops (bytes): m + n ops in order
    int64_t prof_off;     // prof (int32 units): the query's [32][m_pad] table S(q_i, c)
    int32_t m, n;
    int32_t m_pad;        // m rounded up to the 256-row strip
    int32_t pad;
};
struct AlignResultDev {
    int32_t score;
    int32_t i_end, j_end;      // 1-based end cell (0 when the score is 0)
    int32_t i_begin, j_begin;  // rows / columns before the alignment's first column
    int32_t n_ops;
    int32_t status;            // 0; 1-4 the walk found an inconsistent flag; 5 a forward-pass wait ran out
    int32_t pad;
    int64_t cells;             // cells recomputed by the traceback pass
};
struct AlignArgs {
    DbView db;
    const uint8_t *queries;
    const AlignPairDev *pairs;
    int64_t n_pairs;
    AlignResultDev *results;
    const int32_t *mat;        // [32][32] int32, entries outside the alphabet unused
    const int32_t *prof;       // per-query profiles (forward pass), see AlignPairDev::prof_off
    int2 *ckpt;
    uint8_t *flags;
    uint8_t *rev;
    uint8_t *ops;
    int32_t gap_open, gap_extend;
    int32_t mode;              // SW_ALIGN_LOCAL / GLOBAL / SEMIGLOBAL / OVERLAP
};

// Non-local alignment modes in int32 (k_modes.cu): several queries, each
// against a prefix [0, n_seqs) of the sorted database, in one launch, one warp
// per (query, sequence) item.  Items are numbered entry by entry (entry e
// owns items [item_start[e], item_start[e] + n_seqs)), and within an entry
// longest sequence first.
struct ModeEntry {
    int64_t item_start;         // first item of this entry
    int64_t n_seqs;             // sorted sequences [0, n_seqs)
    int64_t prof_off;           // the query's profile in prof (int32 units)
    int32_t query;              // score row
    int32_t m;                  // query length
    int32_t m_pad;              // m rounded up to the 256-row strip (profile row stride)
    int32_t pad;
};
struct ModeArgs {
    DbView db;
    const ModeEntry *entries;   // device, n_entries, item_start increasing
    int32_t n_entries;
    int64_t n_items;            // items of all entries
    const int32_t *prof;        // per entry [kProfRows][m_pad] = S(q_i, c) + o, pads -2^28
    int32_t gap_open, gap_extend;
    int32_t mode;               // SW_ALIGN_GLOBAL / SEMIGLOBAL / OVERLAP
    int32_t max_cols;           // longest sequence; each warp slot owns max_cols + 1 int2
    int2 *boundary;             // grid * 8 warp slots
    unsigned long long *work_counter;   // zeroed before launch
    int32_t *scores;            // [n_q][n_seqs], original database order
    int64_t scores_stride;      // n_seqs
};

// Non-local alignment modes in packed int16x2 (k_modes16.cu): one query
// against the pairs [pair_begin, pair_end) of the sorted database, every one
// of which the host has shown to stay inside int16 (no saturation check on
// the device).  The query is padded at the TOP with virt_rows rows so that
// m + virt_rows is a whole number of strips and row m is the last row of the
// last lane.
struct Mode16Args {
    DbView db;
    int64_t pair_begin, pair_end;
    const uint8_t *query;       // device, m codes
    int32_t m, virt_rows;
    int32_t gap_open, gap_extend;
    int8_t prof8[kProfRows][kProfRows];  // [query code][db code] = S + o, pads = -128
    uint2 *boundary;            // per CTA slot, max_cols entries per subwarp (null: one strip)
    int64_t slot_stride;        // uint2 entries per CTA slot
    int32_t max_cols;           // >= every pair's columns (a multiple of 4)
    int32_t *chunk_counter;     // zeroed before launch
    int32_t *scores;            // row of this query, original database order
};

// Launch a kernel with an execution priority (cudaLaunchAttributePriority;
// 0 = the stream's own).  Among CTAs waiting for an SM, the GPU dispatches
// those of higher-priority launches first; CTAs already running are not
// preempted.
template <typename... KArgs, typename... Args>
cudaError_t launch_with_priority(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 int priority, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = priority != 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The highest launch priority of the current device (numerically smallest).
int high_launch_priority();

// Launchers (return cudaGetLastError() after the launch).
// grid_slots > 0 launches a persistent grid of that many CTAs (slot-layout
// scratch); 0 launches one CTA per chunk of pairs (per-pair scratch).
cudaError_t launch_inter_i16x2(const InterArgs &a, int lanes, int rows, cudaStream_t s, int grid_slots = 0,
                               int priority = 0);
bool inter_config_supported(int lanes, int rows);
int inter_slots(int lanes, int rows, int sms);   // resident CTAs of a persistent grid
cudaError_t launch_intra_i16x2(const IntraArgs &a, int warps, int rows, cudaStream_t s);
int intra_rows_per_superpass(int warps, int rows);
cudaError_t prepare_intra_i16x2(int warps, int rows);   // kernel attributes; call before any capture
bool intra_config_supported(int warps, int rows);
cudaError_t launch_batch_i16x2(const BatchArgs &a, int lanes, int rows, int grid, cudaStream_t s, int priority = 0);
bool batch_config_supported(int lanes, int rows);
int batch_slots(int lanes, int rows, int sms);   // resident CTAs of the persistent grid (sets attributes)
cudaError_t launch_profile32(const uint8_t *query, int32_t m, int32_t m_pad, const int32_t *matrix_host,
                             int32_t A, int32_t gap_open, int32_t *prof32, cudaStream_t s);
cudaError_t launch_i32(const I32Args &a, int lanes, int rows, int grid, cudaStream_t s);
bool i32_config_supported(int lanes, int rows);
cudaError_t launch_probe(int mode, int grid, int iters, unsigned long long *cycles, uint32_t *sink,
                         cudaStream_t s);
int probe_blocks_per_sm(int mode);
double probe_work_per_iteration(int mode);
cudaError_t launch_modes_i32(const ModeArgs &a, int grid, cudaStream_t s);   // grid capped by the items
int modes_slots(int sms);            // resident CTAs of the modes kernel
int32_t modes_strip_rows();
cudaError_t launch_modes_i16x2(const Mode16Args &a, int mode, int lanes, int rows, int grid, cudaStream_t s);
bool modes16_config_supported(int lanes, int rows);
int modes16_slots(int lanes, int rows, int sms);   // resident CTAs (the largest over the three modes)
cudaError_t launch_wait_probe(long long limit, int32_t *status, cudaStream_t s);   // limit 1 .. 2^25
cudaError_t launch_align(const AlignArgs &a, int which, cudaStream_t s);   // 0 forward, 1 traceback
int64_t align_checkpoint_rows(int32_t m);
int32_t align_strip_rows();
cudaError_t launch_topk(const int32_t *scores, int64_t n_rows, int64_t n_cols, int32_t k,
                        void *hits, cudaStream_t s);

// Facts of a loaded database (defined with the handle, in api.cu).
}  // namespace swdb
struct sw_db;
namespace swdb {
bool db_describe(const sw_db *db, DbView *view, int *device, int32_t *alphabet, int64_t *codes_bytes);
// Record a thread-local error message and return code.
int set_error(int code, const char *msg);
}  // namespace swdb
