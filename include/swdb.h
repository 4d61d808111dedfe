/*
 * swdb: exhaustive Smith-Waterman/Gotoh protein database search on one GPU.
 *
 * C ABI of libswdb.so.  Plain pointers and sizes only; no C++ or framework
 * types cross this boundary and no exception escapes it: every entry point
 * returns an sw_status code and, on failure, sets a thread-local message
 * readable with sw_last_error().
 *
 * The operation (Section 2.2 of the paper, "Smith-Waterman Algorithm":
 * optimal local alignment score by dynamic programming; case (b) there,
 * one query against every sequence of a database, computed with
 * inter-task parallelism for many sequences at once and intra-task
 * parallelism for long ones, Section 2.3).  Scores use an integer
 * substitution matrix and affine gap penalties (Section 4.1: BLOSUM62,
 * gap open/extend).  For query q[1..m], database sequence t[1..n]:
 *
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)
 *   H(i,j) = max(0, H(i-1,j-1) + S[q_i][t_j], E(i,j), F(i,j))
 *   score  = max_{i,j} H(i,j),  H(i,0) = H(0,j) = 0,  E(i,0) = F(0,j) = -inf
 *
 * so a gap of length k costs o + (k-1)*e.  (The convention o' + k*e' is the
 * same with o = o' + e'.)  Scores are exact int32 values.
 */
#ifndef SWDB_H
#define SWDB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every entry point. */
typedef enum {
    SW_OK = 0,
    SW_ERR_INVALID_ARG = 1, /* bad pointer, size, code or parameter */
    SW_ERR_OOM = 2,         /* device or host allocation failed */
    SW_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed */
    SW_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    SW_ERR_OVERFLOW = 5,    /* parameters too large for exact int32 scores */
    SW_ERR_UNSUPPORTED = 6  /* option combination not available */
} sw_status;

/* Largest alphabet: residue codes are 0 .. SW_MAX_ALPHABET-1.  (One more
 * code is reserved internally for padding.) */
#define SW_MAX_ALPHABET 31

/* Opaque database handle.  It owns a device copy of the database in the
 * length-sorted, interleaved layout the kernels read, plus a reusable
 * device workspace and a CUDA stream. */
typedef struct sw_db sw_db;

/* One top-k hit: the score and the database index in the caller's original
 * order.  Unused slots (top_k larger than the database) hold {-1, -1}. */
typedef struct {
    int32_t score;
    int32_t reserved; /* always 0 */
    int64_t db_index;
} sw_hit;

/* Arithmetic of the inter-task kernel. */
typedef enum {
    SW_PREC_AUTO = 0, /* int16x2 with saturation flags + exact int32 rescore when
                         the matrix and penalties fit, int32 otherwise */
    SW_PREC_I16 = 1,  /* int16x2 + rescore; SW_ERR_UNSUPPORTED if they do not fit */
    SW_PREC_I32 = 2   /* int32 throughout */
} sw_precision;

/* How a multi-query search is launched. */
typedef enum {
    SW_MODE_AUTO = 0,    /* library choice */
    SW_MODE_PLAIN = 1,   /* one kernel launch per query (the paper's form) */
    SW_MODE_BATCHED = 2  /* all queries in one persistent launch (two queries per int16x2
                            word; a search with a single non-empty query, which has nothing
                            to pair with, runs in the plain form) */
} sw_mode;

/* Which alignment score sw_search computes.  Section 2.2 defines the local
 * (Smith-Waterman) score, the paper's subject; SW# also offers global and
 * semi-global modes (Section 2.3) and the paper leaves other alignment
 * operations to future work (Section 5).  The other modes use the same
 * Gotoh recurrences without the zero floor of H; with g(k) = o +
 * (k-1)*min(o, e) (the first column's own recurrence, o + (k-1)e when
 * o >= e):
 *   GLOBAL      H(i,0) = -g(i), H(0,j) = -g(j); score H(m,n)
 *   SEMIGLOBAL  the whole query against any part of the target:
 *               H(i,0) = -g(i), H(0,j) = 0; score max over j of H(m,j)
 *   OVERLAP     end gaps free on both: H(i,0) = H(0,j) = 0;
 *               score max(max_j H(m,j), max_i H(i,n))
 * Their scores can be negative and are exact.  They require
 * (m + n) * (max|S| + o + e) < 2^28 for every pair (else SW_ERR_OVERFLOW).
 * precision: with SW_PREC_AUTO or SW_PREC_I16, when S + o fits int8 and
 * o <= 127, each query's pairs that provably stay inside int16 run in packed
 * int16x2 (two database sequences per operation, no saturation check needed:
 * with Lp the pair's longer length rounded up to 4, the host requires
 * g(m) + g(Lp) + o + max(e, 128) <= 32768, g(m) counted as 0 for OVERLAP, and
 * max(S, 0) * (min(m, Lp) + 1) <= 32767, and for a query taller than one strip
 * Lp <= 4096); the other pairs (the longest) run in int32, concurrently.
 * SW_PREC_I16 returns SW_ERR_UNSUPPORTED when S + o does not fit; SW_PREC_I32
 * runs every pair in int32.  lanes / rows_per_lane: 8 and 16, 24 or 32 for
 * the packed kernel (0 = chosen per query); stats->long_cells counts the
 * cells scored in int32 and long_sequences the sequences sent there (largest
 * over the queries).  The mode option does not apply. */
typedef enum {
    SW_ALIGN_LOCAL = 0,
    SW_ALIGN_GLOBAL = 1,
    SW_ALIGN_SEMIGLOBAL = 2,
    SW_ALIGN_OVERLAP = 3
} sw_alignment_mode;

/* Optional knobs for sw_search (pass NULL for defaults).  Zero-initialise
 * and set the fields you need. */
typedef struct {
    int32_t precision;        /* sw_precision */
    int32_t mode;             /* sw_mode */
    int64_t long_cutoff;      /* database sequences longer than this are scored by the
                                 intra-task kernel; <0 = never; 0 = the handle's tuning, else
                                 the library default: the longest length n <= 3072 (at
                                 least 768) at which one sequence pair holds no more than
                                 1/S of the residues of the sequences up to n, S the
                                 resident subwarps of the default launch shape (a pair
                                 scored by one subwarp then never outlasts the launch) */
    int32_t lanes;            /* lanes per database-sequence pair in the inter-task kernel
                                 (4, 8, 16 or 32); 0 = chosen per query by the library */
    int32_t rows_per_lane;    /* query rows held per lane (16, 24 or 32; 8 with 32 lanes; the
                                 batched kernel: 16, 24 or 32 with 8 or 16 lanes);
                                 0 = chosen per query */
    void *workspace;          /* caller-owned device scratch, or NULL for the handle's own */
    size_t workspace_bytes;   /* size of workspace */
    int32_t flags;            /* SW_FLAG_* bits */
    int32_t long_rows_per_lane; /* query rows per lane of the intra-task kernel: 8 or 16 (4-warp
                                   pipelines) or 32 (2-warp pipelines); 0 = library choice */
    int32_t alignment;        /* sw_alignment_mode; 0 = local */
    int32_t reserved;
    int32_t *status_out;      /* NULL, or a device (or pinned host) int32 that receives the search's
                                 device-side status on the stream, after all of its kernels: 0, or
                                 SW_ERR_TIMEOUT when a bounded wait of the intra-task kernel gave up
                                 (the long sequences' scores and the hits are then not valid).  For
                                 callers whose call returns before the device finishes (device-only
                                 outputs, stats NULL): read it once the stream has synchronised. */
} sw_search_opts;             /* 64 bytes */

/* Capture the device work of the search into a CUDA graph on first use and
 * replay it while the call's signature (buffers, query lengths, matrix,
 * penalties, options, stream) stays the same.  Query contents may change
 * between replays.  One graph is cached per handle.  Per-kernel times in
 * sw_search_stats are not measured for captured work. */
#define SW_FLAG_GRAPH 1

/* Counters of one search, filled when the caller passes a non-NULL pointer
 * (which makes sw_search wait for the device before returning). */
typedef struct {
    int64_t cells;          /* sum over all (query, sequence) pairs of m*n */
    int64_t rescored;       /* sequences rescored in int32 after int16 saturation */
    int64_t long_sequences; /* database sequences sent to the intra-task kernel */
    int32_t precision_used; /* sw_precision actually used (1 or 2) */
    int32_t mode_used;      /* sw_mode actually used (1 or 2) */
    int32_t lanes_used;     /* inter-task launch shape of the last query */
    int32_t rows_per_lane_used;
    int32_t launches;       /* kernels this call launched */
    float inter_ms;         /* CUDA-event time of the inter-task kernel launches */
    float rescore_ms;       /* CUDA-event time of the int32 kernel launches */
    float intra_ms;         /* CUDA-event time of the long-sequence launches */
    float other_ms;         /* CUDA-event time of profile and top-k kernels */
    int32_t inter_launches; /* launches of the inter-task kernel */
    int64_t inter_cells;    /* cells scored by the inter-task kernel launches */
    int64_t long_cells;     /* cells of the long sequences (intra_ms launches) */
    int32_t graph_replayed; /* 1 if a cached CUDA graph ran the work */
    int32_t reserved0;
} sw_search_stats;

/*
 * Load a database.
 *   residues  host pointer, concatenated residue codes (each < alphabet_size)
 *   offsets   host pointer, n_seqs+1 non-decreasing offsets into residues;
 *             sequence i is residues[offsets[i] .. offsets[i+1]); offsets[0] = 0
 *   n_seqs    number of sequences (>= 0; 0-length sequences are allowed)
 *   alphabet_size  1 .. SW_MAX_ALPHABET
 *   device    CUDA device ordinal
 *   out       receives the handle (set to NULL on failure)
 * The caller keeps ownership of its buffers; the library copies them.
 * Mirrors the database upload the paper describes (Section 3.2, the 2-D
 * sequence matrix read row = position, column = sequence), in an HBM layout
 * of this library's own.
 * Errors: SW_ERR_INVALID_ARG (NULL pointers, bad offsets, codes out of range),
 * SW_ERR_OOM, SW_ERR_CUDA.
 */
int sw_db_load(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs,
               int32_t alphabet_size, int device, sw_db **out);

/* Release a handle and all device memory it owns.  NULL is accepted. */
int sw_db_free(sw_db *db);

/* Database facts. */
typedef struct {
    int64_t n_seqs;
    int64_t residues;        /* sum of lengths */
    int64_t max_length;
    int64_t device_bytes;    /* bytes of the resident database layout */
    int32_t alphabet_size;
    int32_t device;
} sw_db_info;

int sw_db_get_info(const sw_db *db, sw_db_info *out);

/*
 * Launch tuning of one database handle (no counterpart in the paper, whose
 * SW#db picks blocks and threads from fixed per-architecture tables,
 * Section 3.2, and whose results depend on the work-group size, Section
 * 4.2).  sw_search picks, per query, the launch shape of the inter-task
 * kernel (plain form) or of the batched kernel (batched form: per query
 * pair) with the least predicted time, padded rows / gcups, from a table of
 * shapes and their cell rates; the padded rows of a query of m rows are its
 * full strips of lanes*rows rows plus a last strip of lanes x (the fewest
 * rows per lane, a multiple of 8, that cover the rest).  The library's
 * tables hold rates measured on GB300.  An autotuner that measures the rates
 * on the caller's own GPU and database installs its tables here, with the
 * inter/intra-task length cutoff, the intra-task rows per lane and the form
 * that SW_MODE_AUTO takes; sw_search options that are set explicitly still
 * override them.  Tuning never changes scores, only launch shapes.
 */
typedef struct {
    int32_t lanes;            /* lanes per subwarp: with rows_per_lane, a shape sw_search
                                 accepts in opts for that form */
    int32_t rows_per_lane;
    float gcups;              /* measured cell updates per second / 1e9, > 0 */
} sw_shape_rate;              /* 12 bytes */

#define SW_TUNING_MAX_SHAPES 16
typedef struct {
    int32_t n_plain;          /* entries of plain[] in use (0: the library's table) */
    int32_t n_batched;        /* entries of batched[] in use (0: the library's table) */
    sw_shape_rate plain[SW_TUNING_MAX_SHAPES];    /* inter-task kernel, plain form */
    sw_shape_rate batched[SW_TUNING_MAX_SHAPES];  /* batched kernel */
    int64_t long_cutoff;      /* default of opts->long_cutoff (0: the library's, 3072) */
    int32_t long_rows_per_lane; /* default of opts->long_rows_per_lane (0: library choice) */
    int32_t mode;             /* what SW_MODE_AUTO means: 0 or SW_MODE_PLAIN = plain,
                                 SW_MODE_BATCHED = batched */
} sw_tuning;                  /* 408 bytes */

/* Install a tuning on the handle (copied), or NULL to go back to the
 * library's tables.  Do not call it while a search on the handle is in
 * flight or being captured.  Errors: SW_ERR_INVALID_ARG (NULL handle, a
 * count outside 0..SW_TUNING_MAX_SHAPES, a shape the form does not support,
 * a rate that is not a positive finite number, long_rows_per_lane other
 * than 0, 8, 16 or 32, an unknown mode). */
int sw_db_set_tuning(sw_db *db, const sw_tuning *tuning);

/* The handle's tuning, the library's tables when none is installed (with
 * n_plain and n_batched giving their sizes). */
int sw_db_get_tuning(const sw_db *db, sw_tuning *out);

/* Device workspace (bytes) sw_search needs for these queries and options,
 * written to *bytes.  q_offsets is a host pointer (n_q+1 entries). */
int sw_search_workspace_size(const sw_db *db, const int64_t *q_offsets, int32_t n_q,
                             int32_t top_k, const sw_search_opts *opts, size_t *bytes);

/*
 * Score every query against every database sequence.
 *   queries    residue codes of all queries concatenated: host OR device pointer
 *   q_offsets  HOST pointer, n_q+1 offsets into queries (query lengths are
 *              needed on the host to plan the launches)
 *   n_q        number of queries (>= 0)
 *   matrix     HOST pointer, alphabet_size x alphabet_size int32, row-major,
 *              matrix[a*A + b] = score of query residue a against database
 *              residue b (it need not be symmetric)
 *   gap_open, gap_extend   penalties o, e >= 0 (a gap of length k costs o + (k-1)e)
 *   top_k      hits kept per query (>= 0)
 *   scores_out n_q x n_seqs int32, row-major, database in original order:
 *              host or device pointer, or NULL to skip
 *   hits_out   n_q x top_k sw_hit, best first (score descending, then database
 *              index ascending); host or device pointer, or NULL to skip
 *   opts       NULL or options
 *   stats      NULL or counters (non-NULL makes the call synchronous)
 *   stream     cudaStream_t to run on, or NULL for the handle's stream
 * Work is queued on the stream.  The call returns after the device finished
 * when any output is a host pointer or stats is non-NULL; otherwise it may
 * return before the device is done (device outputs are then valid after the
 * stream synchronises).  Calls that share a workspace (the handle's own
 * workspace when opts->workspace is NULL) must not overlap in time.
 * Errors: SW_ERR_INVALID_ARG, SW_ERR_OVERFLOW (|matrix|, o, e or lengths
 * too large for exact int32), SW_ERR_UNSUPPORTED, SW_ERR_OOM, SW_ERR_CUDA,
 * SW_ERR_TIMEOUT (a bounded device-side wait of the intra-task kernel gave
 * up; reported by the return code only when the call waits for the device,
 * i.e. a host output or stats; an asynchronous call reports it through
 * opts->status_out).  A NULL stream means the handle's own stream here,
 * whereas sw_search_no_alloc reads NULL as the legacy default stream.
 */
int sw_search(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q,
              const int32_t *matrix, int32_t gap_open, int32_t gap_extend, int32_t top_k,
              int32_t *scores_out, sw_hit *hits_out, const sw_search_opts *opts,
              sw_search_stats *stats, void *stream);

/*
 * Top-k of score rows already on the device (the last step of sw_search,
 * exposed on its own).  scores: device pointer, n_rows x n_cols int32 (any
 * value); hits: device pointer, n_rows x top_k; order score descending, then
 * column ascending; missing entries (top_k > n_cols) have db_index -1 and
 * score -1.  top_k <= 4096.
 */
int sw_top_k(const int32_t *scores, int64_t n_rows, int64_t n_cols, int32_t top_k,
             sw_hit *hits, void *stream);

/*
 * Measured integer throughput of one device, the denominator of the
 * integer roofline (not a search step).  A register-only kernel fills every
 * SM and counts SM cycles with clock64.
 *   mode 0: packed int16x2 DPX add-max operations per SM cycle
 *   mode 1: cell updates per SM cycle of the inter-task kernel's own
 *           instruction sequence as it ships (32 rows per lane; operands in
 *           registers, profile words from shared memory, no global traffic)
 *   mode 2: cell updates per SM cycle of the same recurrence in unsigned
 *           saturating byte SIMD, four sequences per 32-bit word (the
 *           int8x4 lane packing, measured rather than built)
 *   mode 3: cell updates per SM cycle of the mode-1 sequence with two
 *           columns per step (two F chains in flight per lane)
 * Writes the rate to *per_sm_cycle and the SM count to *sm_count.
 */
int sw_probe_alu_rate(int device, int32_t mode, double *per_sm_cycle, int32_t *sm_count);

/*
 * Self-test of failure detection (no counterpart in the paper, which has no
 * error handling beyond CUDA_SAFE_CALL, Section 3.2).  The intra-task
 * kernel's warps wait on each other through shared-memory flags; every such
 * wait is bounded, and when its limit runs out the kernel records
 * SW_ERR_TIMEOUT in a status word, stops waiting and finishes, so the
 * search returns an error instead of hanging and the CUDA context stays
 * usable.  This entry point runs that same wait routine on a flag that
 * nothing sets, with spin_iters iterations of about 32 ns each (1 ..
 * 2^25, about a second at most), and returns the status the kernel recorded
 * in *status_out (SW_ERR_TIMEOUT when the mechanism works) and the elapsed
 * host time in *elapsed_ms.  Errors: SW_ERR_INVALID_ARG, SW_ERR_CUDA.
 */
int sw_probe_wait_timeout(int device, int64_t spin_iters, int32_t *status_out, double *elapsed_ms);

/*
 * Alignments (traceback) of chosen (query, database sequence) pairs, for
 * instance the hits of sw_search.  Section 2.2 defines the optimal local
 * alignment score by the Smith-Waterman recurrences (here in the affine-gap
 * form of Gotoh with the penalties of Section 4.1, as in sw_search); an
 * alignment reaching that score is read back from the same matrices.  SW#,
 * the tool the paper measures (Section 2.3), reports such alignments; the
 * paper itself times only the scores.  Several alignments can reach the
 * optimum; sw_align returns the one fixed by these rules:
 *   - it ends at the first cell (i, j) in row-major order (smallest query
 *     position i, then smallest target position j) whose H is the maximum;
 *   - walking back from there, a diagonal step is taken before ending a gap
 *     along the target (E), and that before ending a gap along the query
 *     (F); inside a gap, the step at which the gap can open is taken before
 *     extending it; the walk stops at the first cell whose H is 0.
 * A pair scoring 0 has the empty alignment (all coordinates 0, no ops).
 */
#define SW_OP_M 0   /* query residue aligned with target residue */
#define SW_OP_I 1   /* query residue opposite a gap */
#define SW_OP_D 2   /* target residue opposite a gap */

typedef struct {
    int32_t score;
    int32_t reserved;
    int64_t q_begin, q_end;   /* query residues [q_begin, q_end), 0-based */
    int64_t t_begin, t_end;   /* target residues [t_begin, t_end) */
    int64_t ops_offset;       /* index of the first op in ops_out */
    int64_t ops_len;          /* number of ops, from the start of the alignment */
} sw_alignment;               /* 56 bytes */

typedef struct {
    int64_t forward_cells;    /* cells of the forward pass (sum of m * n) */
    int64_t traceback_cells;  /* cells recomputed by the traceback pass */
    float forward_ms;         /* device time of the forward pass */
    float traceback_ms;       /* device time of the traceback pass */
    int32_t launches;
    int32_t reserved;
} sw_align_stats;             /* 32 bytes */

/*
 * Ops capacity sw_align needs for these pairs, in bytes: the sum over pairs
 * of (query length + target length).  Arguments as for sw_align.
 */
int sw_align_ops_capacity(const sw_db *db, const int64_t *q_offsets, int32_t n_q,
                          const int32_t *pair_query, const int64_t *pair_target, int64_t n_pairs,
                          int64_t *bytes);

/*
 * Align n_pairs pairs: query pair_query[k] (index into q_offsets) against
 * database sequence pair_target[k] (caller's original order).
 *   queries, q_offsets, n_q   as for sw_search (queries host or device)
 *   pair_query, pair_target   host arrays of n_pairs entries
 *   matrix, gap_open, gap_extend   as for sw_search (int32 arithmetic)
 *   alignments_out  host array of n_pairs sw_alignment
 *   ops_out         host buffer of ops_capacity bytes (sw_align_ops_capacity);
 *                   pair k's ops are ops_out[ops_offset .. ops_offset + ops_len),
 *                   each SW_OP_M, SW_OP_I or SW_OP_D
 *   stats           NULL or counters
 *   stream          cudaStream_t, or NULL for the handle's stream
 * The call is synchronous.  Device scratch comes from the handle's own
 * workspace (grown as needed): for each pair about 8 * ceil(m/256) * (n+1)
 * bytes of strip checkpoints plus 256 * n bytes of traceback flags, and for
 * each query that appears 128 * round_up(m, 256) bytes of profile.
 * Errors: SW_ERR_INVALID_ARG (NULL or out-of-range argument, ops_capacity too
 * small), SW_ERR_OVERFLOW (as sw_search's int32 limits), SW_ERR_TIMEOUT (a
 * bounded wait between the strips of a pair ran out), SW_ERR_OOM,
 * SW_ERR_CUDA.
 */
int sw_align(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q,
             const int32_t *pair_query, const int64_t *pair_target, int64_t n_pairs,
             const int32_t *matrix, int32_t gap_open, int32_t gap_extend,
             sw_alignment *alignments_out, uint8_t *ops_out, int64_t ops_capacity,
             sw_align_stats *stats, void *stream);

/*
 * sw_align in any sw_alignment_mode (SW_ALIGN_LOCAL gives sw_align).  The
 * non-local modes (global, semi-global, overlap, as defined for sw_search's
 * alignment option; SW# offers them besides local alignment, Section 2.3)
 * read one optimal alignment off their own matrices with the same tie rules,
 * except that:
 *   - the end cell is global (m, n); semi-global the first cell (m, j) of the
 *     last row in row-major order whose H is the row's maximum; overlap the
 *     first cell in row-major order, among the last column (i, n), i = 0..m,
 *     and the last row (m, j), whose H is their maximum;
 *   - the walk does not stop at H = 0; on reaching the first row or column it
 *     emits the leading gap the mode prices there (global: the first row's
 *     D ops or the first column's I ops; semi-global: the first column's I
 *     ops) and stops.
 * So global covers both sequences (score H(m, n), possibly negative),
 * semi-global the whole query, and overlap starts on the first row or column
 * and ends on the last row or column; an empty alignment may sit at a
 * non-zero target position (overlap: q_begin = q_end = 0, t_begin = t_end = n
 * when H(0, n) = 0 is the first maximum).  Arguments, ops capacity and
 * scratch as for sw_align.  Errors: as sw_align, plus SW_ERR_INVALID_ARG for
 * an unknown mode and SW_ERR_OVERFLOW when (m + n) * (max|S| + o + e) >= 2^28
 * for some pair.
 */
int sw_align_mode(sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int32_t n_q,
                  const int32_t *pair_query, const int64_t *pair_target, int64_t n_pairs,
                  const int32_t *matrix, int32_t gap_open, int32_t gap_extend, int32_t alignment,
                  sw_alignment *alignments_out, uint8_t *ops_out, int64_t ops_capacity,
                  sw_align_stats *stats, void *stream);

/*
 * Score one query against a loaded database without allocating any device
 * memory during the call.  (The paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate at search time.)
 *
 * Who needs it: code that searches while a CUDA stream is being captured
 * into a graph (allocation calls may not appear inside a capture), serving
 * loops that must not call the allocator after start-up (an allocation can
 * synchronise the device and has unbounded latency), and processes whose
 * device memory is owned by another framework's pool.  sw_search allocates
 * a workspace unless the caller passes one; this call never does.
 *
 *   db          a handle from sw_db_load (loading allocates; do it at set-up)
 *   query       DEVICE pointer, m residue codes (codes >= alphabet_size
 *               score as padding and are not checked)
 *   m           query length (>= 0)
 *   matrix      HOST pointer, alphabet_size^2 int32, as for sw_search
 *   gap_open, gap_extend   as for sw_search
 *   scores      DEVICE pointer, n_seqs int32, database in original order
 *   stream      cudaStream_t, or NULL for the legacy default stream (unlike
 *               sw_search, where NULL means the handle's own stream)
 * Results equal sw_search's for the same arguments.  The work is queued on
 * the stream and the call returns without waiting.
 *
 * Scratch comes from one array of SW_NO_ALLOC_SCRATCH_BYTES in device
 * memory that the library defines; every GPU that loads the library holds
 * it until the process exits.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is cached per device and CUDA
 * context: after the context is destroyed and a new one created, the next
 * call looks it up again (so make that call, too, outside any capture).  Calls share the array: calls whose work
 * overlaps on the GPU race.  A query/database combination that needs more
 * scratch than the array holds (multi-pass queries, m > 128, need about 4
 * bytes per byte of the database layout) is rejected with
 * SW_ERR_INVALID_ARG and a message; use sw_search with a workspace then.
 * Errors: SW_ERR_INVALID_ARG, SW_ERR_OVERFLOW, SW_ERR_CUDA.
 */
#define SW_NO_ALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int sw_search_no_alloc(const sw_db *db, const uint8_t *query, int32_t m, const int32_t *matrix,
                       int32_t gap_open, int32_t gap_extend, int32_t *scores, void *stream);

/*
 * Database sharding over several GPUs (host-side steps; no device memory).
 * The paper leaves multi-GPU execution to future work (Section 5), and SW#db
 * spreads its search over GPU(s) (Section 2.3).  Every (query, sequence)
 * score is independent, so the database splits into shards that separate
 * GPUs search with the full query batch (one sw_db_load per shard, on its
 * own device), each keeping its own top-k; the one exchange step is a
 * gather of the shards' k best per query and the merge below.
 *
 * sw_shard_plan: partition n_seqs sequences (offsets as for sw_db_load, host
 * pointer, n_seqs + 1 entries) into n_shards shards of balanced residue
 * counts, each with sequences of every length range: sequences are dealt
 * longest first (ties in the caller's order), each to the shard with the
 * fewest residues so far (ties to the lower shard).  The largest and the
 * smallest shard then differ by at most the longest sequence's residues.
 * Outputs (host, caller-allocated): members[n_seqs] lists shard 0's
 * sequences (the caller's indices) in increasing order, then shard 1's, and
 * so on; member_offsets[n_shards + 1] delimits them.  Shard s's local
 * sequence j is the caller's sequence members[member_offsets[s] + j], so a
 * shard's local order is the caller's order.
 * Errors: SW_ERR_INVALID_ARG (NULL pointer, n_shards < 1, bad offsets).
 */
int sw_shard_plan(const int64_t *offsets, int64_t n_seqs, int32_t n_shards, int64_t *members,
                  int64_t *member_offsets);

/*
 * sw_hits_merge: the top-k of an unsharded search from the shards' top-k.
 *   shard_hits  host, [n_shards][n_q][top_k]: shard s's hits as sw_search
 *               returned them for its own database (db_index local to the
 *               shard, {-1, -1} padding when the shard holds fewer than
 *               top_k sequences)
 *   members, member_offsets   the partition from sw_shard_plan
 *   hits_out    host, [n_q][top_k]: score descending, then the caller's
 *               database index ascending; {-1, -1} padding
 * Exact: a sequence outside its shard's k best has k better sequences in
 * that shard, so the merged list equals the unsharded search's top-k, ties
 * included.  Errors: SW_ERR_INVALID_ARG (NULL pointer, bad count, a shard
 * index outside its shard; nothing is written then).
 */
int sw_hits_merge(const sw_hit *shard_hits, const int64_t *members, const int64_t *member_offsets,
                  int32_t n_shards, int32_t n_q, int32_t top_k, sw_hit *hits_out);

/*
 * sw_scores_scatter: one shard's score rows into the unsharded table.
 *   shard_scores  host, [n_q][n_members] as sw_search returned them for the shard
 *   members       host, the shard's n_members caller indices (its slice of
 *                 sw_shard_plan's members)
 *   scores_out    host, [n_q][n_seqs]; row q, column members[j] receives
 *                 shard_scores[q][j]; other columns are left as they are
 * Errors: SW_ERR_INVALID_ARG (NULL pointer, bad count, index >= n_seqs).
 */
int sw_scores_scatter(const int32_t *shard_scores, const int64_t *members, int64_t n_members, int32_t n_q,
                      int64_t n_seqs, int32_t *scores_out);

/* Message of the last failure on the calling thread ("" if none). */
const char *sw_last_error(void);

/* Library version string. */
const char *sw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWDB_H */
