/*
 * ck.h -- C ABI of libck, the GB300 (sm_103a) hot path of the compressed key
 * sort of Kwon et al., "Compressed Key Sort and Fast Index Reconstruction"
 * (arXiv 2009.11543).
 *
 * The library turns a column of index keys into a bulk-loaded index tree:
 *
 *   ck_variant_bits      variant bitmap of the keys              (Sec. 4.2, 4.3)
 *   ck_distinction_bits  D-bitmap of sorted keys                 (Sec. 3.1, Theorem 1)
 *   ck_extract           Compress(key) for every row             (Sec. 3.2, 5.1)
 *   ck_extract_hist      the same, counting the sort's digits    (Sec. 3.2, 5.1)
 *   ck_sort              stable LSD radix sort of (ck, row id)   (Sec. 3.2, 5.2)
 *   ck_sort_static       the same without a caller workspace
 *   ck_build_index       bottom-up bulk load + D refinement      (Sec. 4.3, 5.3)
 *   ck_build_index_keys  the same from the key column and row ids
 *
 * and around that path:
 *
 *   ck_build_batched, ck_graph_*, ck_autotune_sort   all indexes of a table at once
 *   ck_sort_learned, ck_mlp_loss_grad, ck_model_separators   learned CDF partition
 *   ck_insert_batch      DS-metadata under inserts               (Sec. 4.3)
 *   ck_encode_key        index keys of several columns           (Sec. 4.1)
 *   ck_partial_key_mask, ck_partial_keys, ck_search   partial keys and search (Sec. 4.2, 4.3)
 *
 * Conventions shared by every call:
 *   - Bit position p of a key (0 = most significant bit of byte 0) is bit
 *     (7 - p % 8) of byte p / 8 (Sec. 3.1).  Unsigned integer columns
 *     (CK_KIND_U32 / CK_KIND_U64, native little-endian values) compare like
 *     their big-endian bytes, so position 0 is the value's most significant bit.
 *   - A bitmap over key positions (D-bitmap, variant bitmap) is an array of
 *     ceil(key_bits / 64) uint64 words, most significant first: position p is
 *     bit (63 - p % 64) of word p / 64.
 *   - A compressed key of nbits bits is the unsigned integer whose most
 *     significant bit is the key's bit at the first set position (Sec. 3.2),
 *     right-aligned in ck_words uint32 words.  Compressed key columns are
 *     word-major ("structure of arrays") with a padded leading dimension:
 *     word k (k = 0 least significant) of row i is at ck[k * CK_LD(n) + i],
 *     so a column occupies ck_words * CK_LD(n) uint32 and every word array
 *     starts 256-byte aligned.  The padding entries are never read as keys.
 *   - Row ids are uint32; n <= CK_MAX_ROWS.
 *   - Every call is asynchronous on the given stream (NULL = the legacy default
 *     stream) and allocates no device memory, except where its comment says
 *     otherwise (ck_autotune_sort synchronises the stream; ck_btree_plan and
 *     ck_partial_key_mask touch no device).  The caller owns
 *     every buffer.
 *     Device pointers must come from cudaMalloc (or torch) on the current
 *     device; HOST pointers are read before the call returns.
 *   - Argument errors are returned synchronously.  Device-side failures (a
 *     bounded wait that ran out) are recorded in a device status word that
 *     ck_device_status() reads; no call ever traps the GPU.
 */
#ifndef CK_H_
#define CK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ck_stream; /* a cudaStream_t */

typedef enum ck_status {
    CK_OK = 0,
    CK_EINVAL = 1,     /* an argument is out of range or a required pointer is NULL */
    CK_ENOMEM = 2,     /* the caller's workspace is smaller than the size query says */
    CK_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    CK_EOVERFLOW = 4,  /* the D-bitmap has more set positions than ck_words words hold */
    CK_ETIMEOUT = 5,   /* a bounded device-side wait ran out (see ck_device_status) */
    CK_EVERIFY = 6     /* a verification pass failed; the exact fallback produced the result */
} ck_status;

enum {
    CK_KIND_BYTES = 0,
    CK_KIND_U32 = 1,
    CK_KIND_U64 = 2,
    CK_KIND_I32 = 3, /* two's-complement signed integers */
    CK_KIND_I64 = 4,
    CK_KIND_F32 = 5, /* IEEE 754 binary32 / binary64 */
    CK_KIND_F64 = 6,
    CK_KIND_DECIMAL = 7 /* ck_encode_key parts only: scaled int64 values (Sec. 4.1 A) */
};

#define CK_MAX_ROWS ((1ull << 30) - 1) /* look-back words pack a 30-bit count */
#define CK_MAX_KEY_BYTES 512u          /* 4096 key positions; D-bits fit uint16 */
#define CK_NO_DBIT 0xFFFFu             /* "no distinction bit": first key or equal keys */
#define CK_MAX_LEVELS 32u
#define CK_LD(n) ((((uint64_t)(n)) + 63u) & ~(uint64_t)63u) /* leading dimension of ck columns */
#define CK_SORT_TILE 4096u /* default pairs per radix pass tile (one look-back word per tile and digit) */
#define CK_SORT_TILE_MIN 2048u /* the tile sizes a sort takes: 2048, 4096, 8192 */
#define CK_SORT_TILE_MAX 8192u

/* A key column in device memory.  CK_KIND_BYTES: binary-comparable byte
 * strings (fixed-size strings as they are, varchar with its terminating NUL and
 * zero padding, Sec. 4.1).  The numeric kinds hold native little-endian values
 * (key_bytes 4 for U32 / I32 / F32, 8 for U64 / I64 / F64) and are read through
 * the order-preserving index key format Sec. 4.1 refers to ([LKN]): the key is
 * the big-endian bytes of the value, with the sign bit flipped for a signed
 * integer, and for a float all bits inverted if its sign bit is set, else the
 * sign bit flipped.  So -0.0 sorts just before +0.0, and NaNs past the
 * infinities of their sign.  Bit positions, bitmaps and compressed keys refer
 * to that key. */
typedef struct ck_column {
    const void* keys;    /* device, n * row_stride readable bytes; row r starts at
                            (const char*)keys + r * row_stride */
    uint64_t n;          /* number of rows, <= CK_MAX_ROWS */
    uint32_t key_bytes;  /* W, 1 .. CK_MAX_KEY_BYTES */
    uint32_t row_stride; /* bytes between rows, >= key_bytes */
    uint32_t kind;       /* CK_KIND_* */
} ck_column;

/* ---------------------------------------------------------------------------
 * ck_encode_key -- index keys from several columns (Sec. 4.1, "Index Key
 * Format"): row r of `out` is the concatenation, in part order, of each
 * part's index key for row r, so comparing two rows byte by byte compares the
 * tuples of column values lexicographically.  The result is a CK_KIND_BYTES
 * column of width = the sum of the part widths, for every other call here.
 * A part (ck_key_part) is one column, row r at values + r * stride:
 *   CK_KIND_BYTES    a fixed-size string, or a varchar zero-padded to `width`
 *                    bytes (its terminating NUL included, Sec. 4.1 C): copied.
 *   CK_KIND_U32 .. CK_KIND_F64   a native numeric value (width 4 or 8): its
 *                    big-endian order-preserving form (see ck_column).
 *   CK_KIND_DECIMAL  decimal(m, s) as an int64 value * 10^s, with an optional
 *                    null flag per row (nulls[r] != 0: NULL): a header byte
 *                    (bit 1: not null, bit 0: sign, 1 for negative) and the
 *                    magnitude in width - 1 big-endian bytes (Sec. 4.1 A); then
 *                    the sign bit is toggled and, for a negative value, every
 *                    magnitude bit, so NULL < negatives < non-negatives in value
 *                    order.  A NULL's sign and magnitude are 0.  width 2 .. 9.
 *   out        device, n rows of out_stride >= total width bytes.
 * Errors: CK_EINVAL (kind, width or stride); a decimal whose magnitude does not
 * fit width - 1 bytes is recorded as CK_EOVERFLOW in the device status word
 * (its low bytes are written). */
typedef struct ck_key_part {
    const void* values;   /* device */
    const uint8_t* nulls; /* device, n flags, or NULL (decimals only) */
    uint32_t kind;        /* CK_KIND_* */
    uint32_t width;       /* bytes of the part in the key */
    uint32_t stride;      /* bytes between rows of values */
} ck_key_part;
#define CK_MAX_KEY_PARTS 16u

ck_status ck_encode_key(const ck_key_part* parts, uint32_t nparts, uint64_t n, uint8_t* out, uint32_t out_stride,
                        ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_variant_bits -- the variant bitmap of Sec. 4.2: position p is set iff some
 * row differs from the reference row at p (computed as in Sec. 4.3, DS-metadata
 * recompute step 3: OR over all keys of key XOR reference key).
 *   col       key column (device).
 *   ref_row   row used as the reference key value (any row works, Sec. 4.2).
 *   mask_out  device, ceil(8 * key_bytes / 64) words; overwritten.
 * Errors: CK_EINVAL for a bad column or ref_row >= n (n > 0).  n == 0 zeroes
 * the mask. */
ck_status ck_variant_bits(const ck_column* col, uint64_t ref_row, uint64_t* mask_out, ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_distinction_bits -- the D-bitmap of Sec. 3.1 / Theorem 1:
 * D = { D-bit(key_{i-1}, key_i) : 1 <= i < n, key_{i-1} != key_i } over the
 * rows in sorted order, each D-bit the most significant differing position of
 * an adjacent pair.
 *   col       key column (device), rows in ascending key order unless order
 *             is given.
 *   order     device, n uint32 row ids listing the rows in ascending order, or
 *             NULL when the rows are already stored in order.
 *   mask_out  device, ceil(8 * key_bytes / 64) words; overwritten.
 * The result is exact only for sorted input; on unsorted input it is the set
 * of adjacent-pair D-bits of the given order.  Errors: CK_EINVAL.  An order
 * entry >= n is skipped and recorded as CK_EINVAL in the device status word. */
ck_status ck_distinction_bits(const ck_column* col, const uint32_t* order, uint64_t* mask_out,
                              ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_extract -- Compress(key) of Sec. 3.2 for every row: the concatenation of
 * the key's bits at the set positions of the (extended) D-bitmap, in position
 * order (the paper extracts with 8-byte masks and PEXT, Sec. 5.1; any gather
 * with the same bits is equivalent).
 *   col       key column (device).
 *   dmask     HOST, ceil(8 * key_bytes / 64) words: the D-bitmap, or any
 *             superset of it (Sec. 3.2, extended distinction bit positions).
 *   ck_words  uint32 words per compressed key, >= ceil(popcount(dmask) / 32).
 *   ck_out    device, ck_words * n uint32, word-major; fully overwritten.
 * Errors: CK_EINVAL; CK_EOVERFLOW when popcount(dmask) > 32 * ck_words. */
ck_status ck_extract(const ck_column* col, const uint64_t* dmask, uint32_t ck_words, uint32_t* ck_out,
                     ck_stream stream);

/* ck_extract_hist -- ck_extract that also counts, in the same pass over the
 * keys, the radix digits of the compressed keys: hist[q][v] = the number of
 * keys whose digit q (bits [q * digit_bits, (q + 1) * digit_bits) of the
 * compressed value) is v, for q < passes = ceil(popcount(dmask) / digit_bits).
 * Passing hist to ck_sort (ck_sort_opts.hist, same digit_bits) spares the sort
 * a read of all compressed keys.
 *   digit_bits  4 .. 11 (0 = 8), as the sort will use.
 *   hist        device, passes * 2^digit_bits uint32; zeroed and written.
 * Other arguments and errors as ck_extract (CK_EINVAL also for a bad
 * digit_bits, or hist NULL with passes > 0).  With more than 16 KB of
 * counters the digits are counted by a second kernel over ck_out. */
ck_status ck_extract_hist(const ck_column* col, const uint64_t* dmask, uint32_t ck_words, uint32_t* ck_out,
                          uint32_t digit_bits, uint32_t* hist, ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_sort -- stable least-significant-digit radix sort of the pairs
 * (compressed key, row id) by compressed key (the sort step of Sec. 5, done
 * here as a radix sort rather than the paper's comparison sort).  Equal keys
 * keep their input order, so with rid_in = NULL (row ids 0..n-1) ties break by
 * row id, and by Theorem 2 the output order is the sorted order of the full
 * keys.  One onesweep pass per digit of the low nbits bits.
 *   ck_in     device, ck_words * n, word-major; read only.
 *   rid_in    device, n row ids, or NULL for 0..n-1; read only.
 *   ck_out    device, ck_words * n; may equal ck_in (an extra copy may run).
 *   rid_out   device, n; may equal rid_in.
 *   nbits     significant low bits of the keys, <= 32 * ck_words; higher bits
 *             must be zero.  nbits == 0 copies the input.
 *   opts      NULL for defaults.
 *   ws        device workspace of at least ck_sort_workspace_bytes() bytes,
 *             256-byte aligned; its contents on entry do not matter.
 * Errors: CK_EINVAL, CK_ENOMEM (ws too small).  A look-back wait that runs
 * out records CK_ETIMEOUT in the device status word; the output is then
 * undefined but every access stays in bounds. */
typedef struct ck_sort_opts {
    uint32_t digit_bits; /* radix digit width, 4 .. 11; 0 = 8 */
    uint32_t spin_limit; /* polls per look-back wait before giving up; 0 = default (~1 s) */
    uint32_t inject;     /* test-only fault injection (CK_INJECT_*); 0 in production */
    uint32_t flags;      /* CK_SORT_* bits; 0 = default */
    void* pass_events;   /* optional profiling hook: cudaEvent_t[passes + 1]; event 0 is
                            recorded on the stream before the first digit pass and event
                            p + 1 after pass p (passes = ceil(nbits / digit_bits)).  NULL
                            records nothing. */
    const uint32_t* hist; /* optional, device [passes][2^digit_bits]: the digit counts of
                            ck_in as ck_extract_hist writes them (same digit_bits); the
                            sort then skips its own counting pass over the keys.  NULL:
                            counted here. */
    uint32_t tile;       /* pairs per radix pass tile: 0 = CK_SORT_TILE (4096), or 2048 /
                            8192 (see ck_autotune_sort).  The workspace depends on it:
                            size it with the same opts. */
    uint32_t reserved;   /* 0 */
} ck_sort_opts;

/* Only the permutation is wanted: ck_out is used as scratch and its contents
 * are unspecified on return (rid_out is the result).  Each pass then stops
 * carrying the key words whose digits have all been consumed, which cuts the
 * bytes moved per key. */
#define CK_SORT_PERM_ONLY 1u
#define CK_SORT_FLAGS_ALL 1u

/* The first tile of the first pass never publishes its look-back entries, so
 * the waits of the tiles after it run out: exercises the CK_ETIMEOUT path
 * without any GPU fault. */
#define CK_INJECT_STALL_FIRST_TILE 1u

size_t ck_sort_workspace_bytes(uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_sort_opts* opts);

ck_status ck_sort(const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out, uint32_t* rid_out,
                  uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_sort_opts* opts, void* ws,
                  size_t ws_bytes, ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_sort_static -- the same sort as ck_sort, for callers that cannot allocate
 * device memory: its scratch lives in one fixed device array inside the
 * library instead of a caller workspace.  The paper has no counterpart; it
 * exists because some hosts of this library own all device memory through
 * their own memory manager and forbid their components to call cudaMalloc,
 * and because cudaMalloc / cudaFree can synchronise the whole device, which a
 * latency-bound rebuild path cannot afford.
 *   Arguments, outputs and errors are those of ck_sort without ws / ws_bytes.
 *   Limit: the call is accepted only if ck_sort_workspace_bytes(n, ck_words,
 *   nbits, opts) <= CK_SORT_STATIC_SCRATCH_BYTES (32 MiB: up to 1,396,736
 *   pairs of 128-bit keys with 8-bit digits); larger sorts return CK_ENOMEM
 *   without launching anything and should use ck_sort with a workspace.
 *   The array belongs to the library's device code and is held until the
 *   process exits.  CUDA loads that code on a device lazily by default (unless
 *   CUDA_MODULE_LOADING=EAGER), so the 32 MiB are committed on each device at
 *   the latest by the first ck_sort_static call there, which also looks up the
 *   array's device address (with that device current).  A caller whose path
 *   must see no device allocation makes one call at start-up (a warm-up), and
 *   makes it before any stream capture; when the device has no room left for
 *   the array that first call returns CK_ENOMEM.  Every call on a device uses
 *   the same array: calls whose execution overlaps on the GPU (other streams,
 *   other threads) race and give wrong results, so serialise them.  After the
 *   first call on a device nothing is allocated or freed. */
#define CK_SORT_STATIC_SCRATCH_BYTES (32u << 20)

ck_status ck_sort_static(const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out, uint32_t* rid_out,
                         uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_sort_opts* opts, ck_stream stream);

/* ---------------------------------------------------------------------------
 * Learned partition (not in the paper; it replaces most radix passes for wide
 * compressed keys).  A tiny fp32 CDF model
 *   y(x) = b2 + sum_j w2_j * relu(w1_j * x + b1_j),  j < CK_MLP_HIDDEN,
 * parameters packed [w1, b1, w2, b2] (CK_MLP_PARAMS floats), on the feature
 * x = (top 24 bits of the nbits-bit compressed key) / 2^24, is trained on the
 * GPU by full-batch Adam to the empirical CDF (rank + 0.5) / S of a sorted
 * stride sample of S = n / sample_div keys (fitted on at most 2048 of its
 * points, taken at a fixed stride; one block, fixed-order sums, so the same
 * input trains the same bits).
 *
 * The model proposes the bucket boundaries: over the sorted sample, the
 * running maximum of y crosses b / B (B = 2^bucket_bits model buckets) at
 * sample position c_b, and the boundary is the sample key there (moved to the
 * start of its run of equal keys).  A key value with at least h sample copies
 * gets a bucket of its own, [v, v + 1).  Where a model bucket holds more
 * sample keys than a shared-memory sort can take (u, with a margin for
 * sampling noise), sample quantiles cut it into pieces of t = S / B sample
 * keys, or of t = 2u / 3 when S / B > u (few model buckets); h = t / 2, so
 * that such a piece, whose cut may move back over a run of fewer than h
 * equal keys, stays within u.
 * stats.model_boundary_frac is the share of boundaries the model set.  Every
 * key's bucket lies in the range of splitters sharing its top 16 bits (a
 * prefix table), where a short search finds it, started from the model's
 * guess when that range is wide (exact).  Two radix passes on the bucket id
 * partition the pairs
 * stably; each bucket (a contiguous key range in row-id order) is then sorted
 * in shared memory and checked: adjacent keys ascend, the keys lie inside the
 * bucket's range, equal keys keep row-id order, and a sum of 64-bit hashes of
 * all (key, row id) pairs equals the input's (every row once, with its own
 * key).
 *
 * ck_sort_learned gives exactly the output of ck_sort (stable, ties by row id,
 * sorted ck and rid).  Everything is decided on the device: if a check fails,
 * a bucket exceeds the shared-memory capacity, or the boundaries exceed the
 * bucket id space, the plain radix sort (launched gated by the call, idle
 * otherwise) recomputes the result from ck_in and the device status word
 * records CK_EVERIFY (the output is still exact).  The call does not wait for
 * the device and can be captured in a CUDA graph (the library looks up its
 * device status word on the first call of any entry point on a device: make
 * one call before capturing).
 *   ck_in      device, ck_words * CK_LD(n), word-major; read only.
 *   ck_out, rid_out  device outputs as ck_sort (ck_out != ck_in).
 *   ck_words   1 .. 8.
 *   opts       NULL for defaults.
 *   stats      DEVICE, optional: one ck_learned_stats, written by the call's
 *              last kernel (read it after the stream has reached it).
 *   params_out DEVICE, optional: CK_MLP_PARAMS floats, the trained model.
 *   ws         device, >= ck_sort_learned_workspace_bytes(), 256-byte aligned.
 * Errors (synchronous): CK_EINVAL, CK_ENOMEM, CK_ECUDA. */
#define CK_MLP_HIDDEN 16
#define CK_MLP_PARAMS (3 * CK_MLP_HIDDEN + 1)

typedef struct ck_learned_opts {
    uint32_t bucket_bits; /* log2 of the model's bucket count B, 1 .. 15; 0 = chosen from n (an average
                             bucket about half of what one block sorts in shared memory) */
    uint32_t sample_div;  /* one sample per sample_div keys; 0 = 100 (1%) */
    uint32_t epochs;      /* Adam epochs; 0 = 100 */
    float lr;             /* Adam learning rate; 0 = 1e-3 */
    uint32_t flags;       /* CK_LEARNED_* bits */
    uint32_t reserved;    /* must be 0 */
    void* phase_events;   /* NULL, or CK_LEARNED_PHASES + 1 cudaEvent_t recorded on the stream at the start
                             and after each phase: sample + model + boundaries, bucket ids, partition,
                             bucket sorts + checks, verdict + gated fallback */
} ck_learned_opts;

#define CK_LEARNED_PHASES 5

/* No model: the boundaries are sample quantiles and every key's bucket is
 * found by binary search (the method without the network). */
#define CK_LEARNED_NO_MODEL 1u
/* Test-only: the final check reports a failure, forcing the fallback. */
#define CK_LEARNED_INJECT_VERIFY_FAIL 2u
/* Test-only: the local sort exchanges the row ids of the first two pairs of
 * every bucket it sorts, which the checks must catch (fallback). */
#define CK_LEARNED_INJECT_RID_SWAP 4u

typedef struct ck_learned_stats {
    float train_loss;           /* mean squared error of the model on its training points */
    float mean_search_steps;    /* splitter comparisons per key to reach the exact bucket: from the model's
                                   guess (galloping search), or a binary search without the model */
    uint32_t max_search_steps;  /* most comparisons for one key */
    uint32_t buckets;           /* buckets after the boundaries were placed (splitters + 1) */
    uint32_t sample_size;       /* S */
    uint32_t max_bucket;        /* largest bucket (pairs) */
    uint32_t sorted_segments;   /* buckets sorted in shared memory */
    uint32_t constant_buckets;  /* buckets of one key value, left as partitioned */
    uint32_t oversize_buckets;  /* buckets over the shared-memory capacity (they force the fallback) */
    uint32_t fell_back;         /* 1 if the plain radix sort produced the result */
    uint32_t model_buckets;     /* B */
    uint32_t model_boundaries;  /* boundaries placed at a model crossing */
    float model_boundary_frac;  /* model_boundaries / (buckets - 1) */
    uint32_t heavy_keys;        /* key values given a bucket of their own */
    uint32_t capacity;          /* pairs one block sorts in shared memory */
    uint32_t reserved;
} ck_learned_stats;

size_t ck_sort_learned_workspace_bytes(uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_learned_opts* opts);

ck_status ck_sort_learned(const uint32_t* ck_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n, uint32_t ck_words,
                          uint32_t nbits, const ck_learned_opts* opts, ck_learned_stats* stats, float* params_out,
                          void* ws, size_t ws_bytes, ck_stream stream);

/* ck_mlp_loss_grad -- one forward + backward pass of the CDF model over S
 * samples: the mean squared error against t (or against (i + 0.5) / S when t
 * is NULL) and its gradient with respect to the 49 parameters, summed in a
 * fixed order (deterministic).  All pointers are device memory: params [49],
 * x [S], t [S] or NULL, grad_out [49], loss_out [1].
 * ws >= ck_mlp_workspace_bytes() bytes.  Errors: CK_EINVAL, CK_ENOMEM. */
size_t ck_mlp_workspace_bytes(void);
ck_status ck_mlp_loss_grad(const float* params, const float* x, const float* t, uint64_t S, float* grad_out,
                           float* loss_out, void* ws, size_t ws_bytes, ck_stream stream);

/* ---------------------------------------------------------------------------
 * Index tree (Sec. 4.2 structure, Sec. 5.3 bottom-up build).  Canonical
 * layout: each node holds f = max(1, floor(fanout * fill)) consecutive entries
 * (the last node of a level may hold fewer).  Level 0 has one entry per key in
 * sorted order; level l+1 has one entry per node of level l; the first level
 * with at most f entries is the root.  Node j of any level holds entries
 * [j*f, min((j+1)*f, m)), m the level's entry count.
 *
 * ck_btree_plan fills the shape (host only) so that the caller can allocate
 * the arrays of ck_btree.  Errors: CK_EINVAL for fanout * fill < 2 with n > 1,
 * n > CK_MAX_ROWS, or a height above CK_MAX_LEVELS. */
typedef struct ck_btree_shape {
    uint32_t levels;           /* 0 when n == 0 */
    uint32_t entries_per_node; /* f */
    uint64_t n;
    uint64_t level_entries[CK_MAX_LEVELS]; /* entries at level l; [0] = n */
    uint64_t level_nodes[CK_MAX_LEVELS];   /* ceil(level_entries[l] / f) */
    uint64_t inner_offset[CK_MAX_LEVELS];  /* start of level l (l >= 1) in the inner arrays */
    uint64_t inner_entries;                /* sum of level_entries[1 .. levels-1] */
} ck_btree_shape;

ck_status ck_btree_plan(uint64_t n, uint32_t fanout, float fill, ck_btree_shape* shape);

/* Caller-allocated device arrays (sizes from ck_btree_plan).  Leaf entry i:
 * the record id and the full-key D-bit against the previous key (Sec. 4.2;
 * computed through D-offset, Sec. 5.3).  Leaf header j: the sorted index of
 * the node's highest key.  Inner entry (levels >= 1, concatenated level 1
 * first): the child node, the sorted index, record id and compressed key of
 * the highest key under the child, and that key's D-bit against the previous
 * entry's highest key at the same level (CK_NO_DBIT for the level's first
 * entry or equal keys). */
typedef struct ck_btree {
    ck_btree_shape shape;     /* written by ck_build_index */
    uint32_t* leaf_rid;       /* [n] */
    uint16_t* leaf_dbit;      /* [n] */
    uint32_t* leaf_high;      /* [level_nodes[0]] */
    uint32_t* inner_child;    /* [inner_entries] */
    uint32_t* inner_high;     /* [inner_entries] */
    uint32_t* inner_high_rid; /* [inner_entries] */
    uint32_t* inner_high_ck;  /* [inner_entries * ck_words], entry-major, least significant word first */
    uint16_t* inner_dbit;     /* [inner_entries] */
} ck_btree;

/* ---------------------------------------------------------------------------
 * ck_build_index -- bulk-loads the tree from the sorted pairs and, in the same
 * pass over the leaves, recomputes the D-bitmap (Sec. 4.3 rebuild, step 1):
 * refined = { D-offset[D-bit(Compress(key_{i-1}), Compress(key_i))] }, where
 * D-offset[q] is the position of the (q+1)-st set bit of dmask (Sec. 5.3).
 *   sorted_ck, sorted_rid  device, as produced by ck_sort (word-major ck);
 *             sorted_rid may be tree->leaf_rid itself (nothing is copied).
 *   dmask     HOST, ceil(key_bits / 64) words: the bitmap used by ck_extract.
 *   key_bits  8 * key_bytes of the column.
 *   tree      its shape is recomputed and written; its arrays are written.
 *   refined_mask  device, ceil(key_bits / 64) words, or NULL to skip.
 * Errors: CK_EINVAL, CK_EOVERFLOW (popcount(dmask) > 32 * ck_words). */
ck_status ck_build_index(const uint32_t* sorted_ck, const uint32_t* sorted_rid, uint64_t n, uint32_t ck_words,
                         const uint64_t* dmask, uint32_t key_bits, uint32_t fanout, float fill, ck_btree* tree,
                         uint64_t* refined_mask, ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_build_index_keys -- the same tree as ck_build_index, built from the key
 * column and the sorted row ids only (for instance after ck_sort with
 * CK_SORT_PERM_ONLY).  A leaf's D-bit is computed on the two full keys it
 * compares (gathered by row id); by Sec. 5.3 this is the value D-offset maps
 * the compressed D-bit to, so the tree and the refined D-bitmap are
 * identical.  Inner entries' compressed highest keys are extracted with dmask.
 *   col         the key column (device) the row ids refer to.
 *   sorted_rid  device, n row ids in ascending key order (ties by row id);
 *               may be tree->leaf_rid itself (nothing is copied).
 *   dmask       HOST, ceil(8 * key_bytes / 64) words (as given to ck_extract).
 *   ck_words, fanout, fill, tree, refined_mask: as ck_build_index.
 * Errors: CK_EINVAL, CK_EOVERFLOW; a row id >= n is skipped and recorded as
 * CK_EINVAL in the device status word. */
ck_status ck_build_index_keys(const ck_column* col, const uint32_t* sorted_rid, const uint64_t* dmask,
                              uint32_t ck_words, uint32_t fanout, float fill, ck_btree* tree, uint64_t* refined_mask,
                              ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_insert_batch -- DS-metadata under inserts (Sec. 4.3, "Search and Update
 * Operations", Insert).  A batch of new keys joins an index's sorted keys:
 * for every new key K with neighbours A and B in the merged sorted order, the
 * D-bits of (A, K) and (K, B) are set in the D-bitmap (the paper sets the
 * larger of the two per insert; the smaller is D-bit(A, B) by Lemma 1, already
 * set, or itself the D-bit of such a pair), and (K xor reference key) is ORed
 * into the variant bitmap.  The result equals inserting the keys one by one,
 * in any order; with inserts only it is the D-bitmap of the grown key set.
 * Deletes need no call: the bitmaps are left as they are (Sec. 4.3).
 *   keys       the indexed column (device), n >= 1 rows; not modified.
 *   order      device, n uint32: the keys' sorted order (for instance the
 *              tree's leaf_rid, or ck_sort's rid_out).
 *   batch      the new keys (device), same key_bytes and kind as keys, m rows
 *              (m = 0: nothing to do); not modified.
 *   ref_row    row of keys holding the variant bitmap's reference key.
 *   dmask, vmask  device bitmaps of ceil(8 * key_bytes / 64) words (the
 *              layout of ck_distinction_bits), updated in place.
 *   ws         device workspace of ck_insert_workspace_bytes(m, key_bytes)
 *              bytes, 256-byte aligned (sorts the batch).
 * The batch is sorted by its full keys (a superset of its D-bitmap, known
 * without reading the device), so the call never waits for the GPU and can
 * be captured in a CUDA graph.  Errors: CK_EINVAL (shape or kind mismatch,
 * n = 0, ref_row >= n, an
 * order entry >= n is skipped and recorded in the device status word),
 * CK_ENOMEM (ws too small), CK_ECUDA. */
size_t ck_insert_workspace_bytes(uint64_t m, uint32_t key_bytes);
ck_status ck_insert_batch(const ck_column* keys, const uint32_t* order, const ck_column* batch, uint64_t ref_row,
                          uint64_t* dmask, uint64_t* vmask, void* ws, size_t ws_bytes, ck_stream stream);

/* ---------------------------------------------------------------------------
 * Partial keys (Sec. 4.2, after Bohannon, McIlroy and Rastogi's partial-key
 * B+-tree) and search (Sec. 4.3, Search).
 *
 * The partial key of a tree entry is the pk bits (1 <= pk <= 32) of its key
 * that follow the entry's D-bit position (its offset): key positions
 * offset + 1 .. offset + pk, the first of them the most significant of the
 * pk low bits of a uint32; positions past the key's end read 0.  An entry
 * without an offset (CK_NO_DBIT: the first entry of its level, or a key equal
 * to the previous one) takes positions 0 .. pk - 1.  Leaf entry i holds sorted
 * key i; an inner entry holds the highest key under its child.
 *
 * Sec. 5.3 names the source of each bit: (A) a position of the extraction
 * mask is read from the compressed key; (B) an invariant position (0 in the
 * variant bitmap) from the reference key; (C) any other position either from
 * bits added to the compressed key (option a, ck_partial_key_mask) or from
 * the record itself (option b: the key column, by row id). */
#define CK_MAX_PARTIAL_KEY_BITS 32u
#define CK_NO_ROW 0xFFFFFFFFu

/* ck_partial_key_mask -- host only (Sec. 5.3, C a).  out = dmask plus every
 * variant position among 0 .. pk - 1 and among d + 1 .. d + pk for each set
 * position d of dmask.  A superset of D (Theorem 2 keeps the order), with
 * which every partial-key bit is a case A or B bit.  dmask, vmask, out: HOST,
 * ceil(key_bits / 64) words (out may alias neither).  Errors: CK_EINVAL
 * (key_bits = 0 or above 8 * CK_MAX_KEY_BYTES, pk outside 1 .. 32). */
ck_status ck_partial_key_mask(const uint64_t* dmask, const uint64_t* vmask, uint32_t key_bits, uint32_t pk,
                              uint64_t* out);

/* ck_partial_keys -- the partial keys of every leaf and inner entry of a tree
 * built by ck_build_index or ck_build_index_keys.
 *   tree       HOST struct holding the built tree's device arrays.
 *   sorted_ck  device, the word-major sorted compressed keys the tree was
 *              built from (as given to ck_build_index), or NULL: the leaves'
 *              case A bits then come from col.
 *   ck_words   words of sorted_ck and of tree->inner_high_ck.
 *   emask      HOST, the extraction mask of those compressed keys.
 *   vmask      HOST, the variant bitmap (DS-metadata).
 *   ref_key    HOST, key_bytes bytes: the reference key value in index-key
 *              byte order (Sec. 4.1; for a numeric column its mapped
 *              big-endian form).
 *   col        the key column the tree's row ids refer to, or NULL when no
 *              case C bit can occur (emask from ck_partial_key_mask over the
 *              tree's D-bitmap) and sorted_ck is set.
 *   key_bytes  W of the keys (col->key_bytes when col is given).
 *   pk         1 .. 32.
 *   leaf_pk    device [n] uint32;  inner_pk  device [inner_entries] uint32
 *              (NULL allowed when the tree has no inner entries).
 * Errors: CK_EINVAL (sizes; popcount(emask) > 32 * ck_words; sorted_ck and
 * col both NULL).  A case C bit met without a column, or a row id >= col->n,
 * reads as 0 and is recorded as CK_EINVAL in the device status word (detail:
 * the row id). */
ck_status ck_partial_keys(const ck_btree* tree, const uint32_t* sorted_ck, uint32_t ck_words, const uint64_t* emask,
                          const uint64_t* vmask, const uint8_t* ref_key, const ck_column* col, uint32_t key_bytes,
                          uint32_t pk, uint32_t* leaf_pk, uint32_t* inner_pk, ck_stream stream);

/* ck_search -- lower-bound search of a batch of query keys (Sec. 4.3,
 * Search).  In a leaf the entries are scanned in order with their offsets and
 * partial keys (Bohannon et al.): with d the D-bit of the query against the
 * previous key (which the query exceeds), an entry whose offset is below d is
 * above the query, one whose offset is above d is below it, and at offset = d
 * the partial key decides unless it equals the query's bits at the same
 * positions; only then is the entry's full key read.  Inner nodes either
 * compare the query with the entries' highest keys as full keys (inner_pk
 * NULL: the paper's search; binary search over the node, each comparison also
 * giving the D-bit that starts the leaf scan), or are scanned the same way
 * as leaves with the inner entries' partial keys (inner_pk given; the D-bit
 * state carries from a node to its child, whose first key follows the highest
 * key of the entry before).  Both give the same result.
 *   tree, col  the built tree and the key column its row ids refer to.
 *   leaf_pk    device [n], from ck_partial_keys with the same pk.
 *   inner_pk   device [inner_entries] from the same call, or NULL.
 *   queries    column of q keys with col's kind and key_bytes.
 *   pos_out    device [q]: the first sorted position whose key is >= the
 *              query (n if there is none).
 *   rid_out    device [q] or NULL: the row id at pos_out when that key equals
 *              the query (the smallest row id among equal keys), else
 *              CK_NO_ROW.
 *   derefs_out device [q] or NULL: full keys read per query.
 * Errors: CK_EINVAL (kind or width mismatch, pk outside 1 .. 32, a tree
 * whose n is not col->n; a row id >= n in the tree is recorded in the device
 * status word and ends that query's search with pos_out = n). */
ck_status ck_search(const ck_btree* tree, const ck_column* col, const uint32_t* leaf_pk, const uint32_t* inner_pk,
                    uint32_t pk, const ck_column* queries, uint32_t* pos_out, uint32_t* rid_out,
                    uint32_t* derefs_out, ck_stream stream);

/* ---------------------------------------------------------------------------
 * ck_model_separators -- model-proposed inner separators (not in the paper).
 * For every inner entry of a built tree the CDF model (parameters as trained
 * by ck_sort_learned, device [CK_MLP_PARAMS]) proposes the top 24 bits of the
 * entry's separator -- the key of sorted rank min((e + 1) f^l, n) - 1 -- as the
 * smallest 24-bit feature value where the model reaches (rank + 0.5) / n.
 * Each proposal is checked against the tree's canonical separator; the tree
 * is never changed (a wrong proposal is replaced by the canonical key), so it
 * stays bit-identical to ck_build_index's.
 *   proposals  device [inner_entries]: the proposed 24-bit prefixes.
 *   hits       device [1]: the number of proposals equal to the canonical
 *              separator's top 24 bits (zeroed by the call).
 * Errors: CK_EINVAL. */
ck_status ck_model_separators(const float* params, const ck_btree* tree, uint32_t ck_words, uint32_t nbits,
                              uint32_t* proposals, uint32_t* hits, ck_stream stream);

/* ---------------------------------------------------------------------------
 * Batched rebuild of all the indexes of one table (not in the paper, which
 * motivates it: a table can carry many indexes, all rebuilt after a restart).
 * Each job is one index: extract -> sort -> bulk load (+ refined D-bitmap),
 * exactly the calls above.  ck_build_batched records every job on its own
 * internal stream, forked from and joined back to `stream` by events, so the
 * jobs run concurrently and the call is asynchronous; it can be captured into
 * a CUDA graph (ck_graph_capture_batched does that and instantiates it).
 * Every buffer of a job is the caller's; jobs must not share buffers.
 * The internal streams and the fork event are shared by every call on a
 * device, so the library serialises batched calls and captures: a call holds
 * an internal lock from its fork through its last join while it queues its
 * work (a capture from its begin to its end), and the work of two calls runs
 * one after the other on the GPU.
 *   digit_bits  radix digit width of the job's sort, 4 .. 11 (0 = 8); see
 *               ck_autotune_sort.
 *   ws          the job's sort workspace (ck_sort_workspace_bytes); when it
 *               holds, after that size rounded up to 256 bytes, a further
 *               ceil(nbits / digit_bits) * 2^digit_bits uint32, the digit
 *               counts are taken there while extracting (ck_extract_hist).
 * Errors: those of the underlying calls; CK_EINVAL for njobs == 0 or
 * njobs > CK_MAX_JOBS. */
#define CK_MAX_JOBS 64u

typedef struct ck_index_job {
    ck_column col;          /* key column (device) */
    const uint64_t* dmask;  /* HOST, the stored D-bitmap of the column */
    uint32_t ck_words;      /* words per compressed key */
    uint32_t digit_bits;    /* 0 = 8 */
    uint32_t tile;          /* radix pass tile, 0 = CK_SORT_TILE; see ck_autotune_sort */
    uint32_t fanout;
    float fill;
    uint32_t* ck;           /* device, ck_words * CK_LD(n): extracted keys */
    uint32_t* ck_sorted;    /* device, ck_words * CK_LD(n) */
    uint32_t* rid_sorted;   /* device, n */
    ck_btree* tree;         /* HOST struct with device arrays (shape written) */
    uint64_t* refined_mask; /* device or NULL */
    void* ws;
    size_t ws_bytes;
} ck_index_job;

ck_status ck_build_batched(const ck_index_job* jobs, uint32_t njobs, ck_stream stream);

/* A captured, instantiated CUDA graph of one ck_build_batched call (opaque). */
typedef struct ck_graph_st* ck_graph;
ck_status ck_graph_capture_batched(const ck_index_job* jobs, uint32_t njobs, ck_graph* graph_out);
ck_status ck_graph_launch(ck_graph graph, ck_stream stream);
ck_status ck_graph_destroy(ck_graph graph);

/* ---------------------------------------------------------------------------
 * ck_autotune_sort -- picks the radix digit width (4 .. 11, hence the pass
 * count) and the pass tile (2048, 4096 or 8192 pairs) for one index by timing
 * ck_sort on its own extracted keys: every (width, tile) whose workspace fits
 * ws runs once untimed and `reps` times timed with CUDA events on `stream`;
 * the fastest median wins.  best_tile == NULL keeps the default tile and
 * tunes the width alone.  The result is kept in a text cache file (one line
 * per GPU name, n rounded up to a power of two, ck_words, nbits and whether
 * the tile was tuned) when cache_path is not NULL, and read from it when
 * present, in which case nothing runs.  Synchronises `stream`.
 *   ck_in, n, ck_words, nbits  as ck_sort (ck_in is read only).
 *   ck_out, rid_out            scratch outputs of the trial sorts.
 *   best_digit_bits, best_tile, best_ms   HOST outputs (best_tile and best_ms
 *                              may be NULL; best_ms is 0 from the cache).
 * Errors: CK_EINVAL, CK_ENOMEM (no candidate fits ws), CK_ECUDA. */
ck_status ck_autotune_sort(const uint32_t* ck_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n, uint32_t ck_words,
                           uint32_t nbits, void* ws, size_t ws_bytes, uint32_t reps, const char* cache_path,
                           uint32_t* best_digit_bits, uint32_t* best_tile, float* best_ms, ck_stream stream);

/* ---------------------------------------------------------------------------
 * Device status.  ck_device_status synchronises the device, returns the first
 * device-side error recorded since the last clear (CK_OK if none) and, if
 * detail is not NULL, a call-specific detail word (for CK_ETIMEOUT: the pass
 * in bits 0..15 and, in bits 16..47, the waiting tile whose wait ran out
 * first).  The status is one word per device shared by all streams. */
ck_status ck_device_status(uint64_t* detail);
ck_status ck_clear_device_status(void);

/* Static name of a status code. */
const char* ck_status_string(ck_status status);

/* Number of kernels this library launched in the calling process (all calls,
 * all devices), for launch accounting in benchmarks. */
uint64_t ck_launch_count(void);

/* Host-side evaluation of the per-word bit gather that ck_extract runs on the
 * GPU: the bits of x at the set bits of mask, in order, packed into the low
 * popcount(mask) bits (the PEXT of Sec. 5.1 on one 32-bit big-endian word).
 * For host tests of the extraction plan; touches no device. */
uint32_t ck_compress_word_host(uint32_t x, uint32_t mask);

/* The same gather in the form ck_extract's kernel runs for a key word with
 * this mask: two shift-and-mask terms when the mask has at most two contiguous
 * runs, else only the compress-network rounds whose move masks are non-zero.
 * For host tests of the extraction plan; touches no device. */
uint32_t ck_compress_word_program_host(uint32_t x, uint32_t mask);

#ifdef __cplusplus
}
#endif

#endif /* CK_H_ */
