/*
 * rs.h -- C ABI of librs.so: stable ascending LSD radix sort of 32-bit
 * unsigned keys, optionally carrying 32-bit values, on one NVIDIA GB300
 * (sm_103a); also signed and IEEE-float 32-bit keys (rs_sort_typed_ex),
 * 64-bit keys and 64-bit values (rs_sort_kv_ex, rs_sort64_ex), segmented
 * batches and captured graphs.
 *
 * The operation is the one stated by Wassenberg & Sanders, "Faster Radix
 * Sort via Virtual Memory and Write-Combining" (2010): 32-bit integer keys,
 * optionally paired with a 32-bit value (Abstract; Sec. 1), sorted by an LSD
 * radix sort whose every pass is a stable counting sort -- digit histogram,
 * prefix sum over buckets, scatter in input order (Sec. 3; Sec. 4, Alg. 2
 * with K = 32 and D = 8, i.e. four byte-wide passes).  Keys are unsigned and
 * sorted ascending; equal keys keep their input order (stability, Sec. 4), so
 * the result is unique: item i goes to position
 *     #{j : k_j < k_i} + #{j < i : k_j = k_i}.
 * A value is an opaque payload that moves with its key and is never compared.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* are DEVICE pointers (cudaMalloc'd, managed or
 *    otherwise GPU-addressable), owned by the caller and never freed here.
 *    Pointers named h_* are HOST pointers (pinned memory gives full link
 *    bandwidth; pageable memory works but is slower).
 *  - Arrays are dense uint32_t, 4-byte aligned (64-bit keys and values:
 *    uint64_t, 8-byte aligned); no other alignment is needed.
 *    Keys and values must not overlap each other or the workspace.
 *  - Sorting is in place: the sorted keys (and values) replace the input.
 *  - n counts items (keys), 0 <= n < 2^32.  n = 0 is a no-op returning RS_OK.
 *  - Argument errors are detected on the host before anything is enqueued and
 *    returned synchronously (RS_ERR_INVALID_ARG / RS_ERR_UNSUPPORTED).
 *  - Errors found on the device (a look-back wait that ran out, a position
 *    outside the array, a malformed segment table) are recorded in a sticky
 *    device status word.  The plain entry points synchronise and report it;
 *    the _ex entry points are asynchronous and the caller collects it with
 *    rs_stream_status().  After a device-side error the contents of the
 *    caller's arrays are unspecified, but the CUDA context stays usable.
 *  - The plain entry points use the current device, the legacy default
 *    stream and a workspace cached inside the library (allocated on first
 *    use, grown when needed, kept until exit); they serialise on an internal
 *    lock and return after the sort has completed.
 *  - The _ex entry points take a stream (cudaStream_t passed as void*, NULL =
 *    legacy default stream) and a caller-owned device workspace of at least
 *    rs_workspace_bytes(...) bytes, 256-byte aligned.  They allocate nothing,
 *    do not synchronise, and return once the work is enqueued.  Two calls in
 *    flight at the same time must not share a workspace.
 */
#ifndef RS_H_
#define RS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rs_status {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = 1,   /* null pointer with n > 0, n >= 2^32, bad table, ... */
    RS_ERR_OUT_OF_MEMORY = 2, /* device allocation failed (plain calls only) */
    RS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    RS_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
    RS_ERR_UNSUPPORTED = 5,   /* no sm_103a device, or a size this build rejects */
    RS_ERR_BOUNDS = 6,        /* a kernel's own bounds check refused a write */
    RS_ERR_BAD_SEGMENTS = 7   /* segment table not monotone or not ending at n */
} rs_status;

/* Sort n keys in place, ascending (Sec. 4 LSD radix sort, keys only, V = 0
 * in Table 1).  Synchronous. */
rs_status rs_sort_keys(uint32_t* d_keys, size_t n);

/* Sort n (key, value) pairs in place by key, ascending and stable (Sec. 4;
 * K = 32, V = 32 in Table 1).  d_vals[i] travels with d_keys[i].
 * Synchronous. */
rs_status rs_sort_pairs(uint32_t* d_keys, uint32_t* d_vals, size_t n);

/* Asynchronous forms on a caller stream with a caller workspace.
 * workspace_bytes must be >= rs_workspace_bytes(n, with_values, 0). */
rs_status rs_sort_keys_ex(uint32_t* d_keys, size_t n,
                          void* cuda_stream, void* d_workspace, size_t workspace_bytes);
rs_status rs_sort_pairs_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                           void* cuda_stream, void* d_workspace, size_t workspace_bytes);

/* The same sort with wider digits: three stable counting-sort passes of
 * 11, 11 and 10 bits (Sec. 4 with D = 11, so ceil(32 / D) = 3 passes instead
 * of four), keys only (d_vals == NULL) or pairs.  The result is the same as
 * rs_sort_pairs_ex / rs_sort_keys_ex: ascending, stable, in place.
 * Every pass is a reduce-then-scan over 2048 buckets: per-chunk digit counts,
 * their prefix over chunks, then a tile-by-tile scatter of every chunk.
 * Arguments as rs_sort_pairs_ex; workspace (256-byte aligned) of at least
 * rs_workspace_bytes_digits11(n, d_vals != NULL) bytes -- two alternate
 * buffers, since an odd pass count ends in the caller's arrays only by
 * rotating through three.  Asynchronous; a bounds-check failure inside a
 * kernel is reported by rs_stream_status as RS_ERR_BOUNDS. */
rs_status rs_sort_digits11_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n, void* cuda_stream,
                              void* d_workspace, size_t workspace_bytes);
/* Workspace bytes of rs_sort_digits11_ex; 0 for n == 0 or n >= 2^32.  Pure
 * host arithmetic. */
size_t rs_workspace_bytes_digits11(size_t n, int with_values);

/* Segmented sorts: every segment [d_offsets[s], d_offsets[s+1]) of the n-item
 * array, s = 0..num_segments-1, is sorted on its own, stably and ascending,
 * exactly as if it were a separate array (the paper has no segmented case;
 * this is its sort applied per segment).  d_offsets is a device array of
 * num_segments + 1 nondecreasing uint32 entries with d_offsets[num_segments]
 * <= n; segments may be empty; items outside [d_offsets[0],
 * d_offsets[num_segments]) are left as they are; a single segment must hold
 * fewer than 2^30 items.  A table that breaks these rules is detected on the
 * device: nothing is written and the status is RS_ERR_BAD_SEGMENTS.
 * Segments of at most 512 items (the RS_TUNE_WARP_MAX setting) are sorted
 * by one warp each, segments of at most 4096 items (or the RS_TUNE_SMALL_MAX
 * setting, up to 8192) by one CTA each, both in shared memory; larger ones by
 * the four scatter passes of the unsegmented sort, all large segments
 * together.
 * Plain forms are synchronous; _ex forms as above, with
 * workspace_bytes >= rs_workspace_bytes(n, with_values, num_segments). */
rs_status rs_sort_keys_segmented(uint32_t* d_keys, size_t n, const uint32_t* d_offsets,
                                 uint32_t num_segments);
rs_status rs_sort_pairs_segmented(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                  const uint32_t* d_offsets, uint32_t num_segments);
rs_status rs_sort_keys_segmented_ex(uint32_t* d_keys, size_t n, const uint32_t* d_offsets,
                                    uint32_t num_segments, void* cuda_stream,
                                    void* d_workspace, size_t workspace_bytes);
rs_status rs_sort_pairs_segmented_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                     const uint32_t* d_offsets, uint32_t num_segments,
                                     void* cuda_stream, void* d_workspace,
                                     size_t workspace_bytes);

/* Typed keys (the paper's keys are unsigned; this is its sort applied to an
 * order-preserving encoding).  The 32-bit words of d_keys are read as:
 *   RS_KEY_U32  unsigned integers (the calls above);
 *   RS_KEY_I32  two's-complement integers, ascending by value;
 *   RS_KEY_F32  IEEE-754 binary32, ascending by the totalOrder predicate of
 *               IEEE 754-2008 Sec. 5.10: -NaN < -inf < ... < -0 < +0 < ...
 *               < +inf < +NaN, NaNs by payload.
 * Every word is mapped onto an unsigned word with the same order as it is
 * first read and mapped back as it is last written, so the result holds the
 * caller's own bit patterns, stably sorted (equal keys keep their order).
 * d_vals may be NULL (keys only).  Otherwise as the _ex calls above, with the
 * same workspace size; the scatter passes of typed sorts always use tile
 * shape 3.  These two calls take the 32-bit key types only; any other
 * key_type is RS_ERR_INVALID_ARG.  The 64-bit types (RS_KEY_U64, RS_KEY_I64,
 * RS_KEY_F64: unsigned, two's-complement and IEEE-754 binary64, by the same
 * rules) are sorted by rs_sort_kv_ex below. */
typedef enum rs_key_type {
    RS_KEY_U32 = 0,
    RS_KEY_I32 = 1,
    RS_KEY_F32 = 2,
    RS_KEY_U64 = 3,
    RS_KEY_I64 = 4,
    RS_KEY_F64 = 5
} rs_key_type;

rs_status rs_sort_typed_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n, int key_type,
                           void* cuda_stream, void* d_workspace, size_t workspace_bytes);
rs_status rs_sort_segmented_typed_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                     const uint32_t* d_offsets, uint32_t num_segments,
                                     int key_type, void* cuda_stream, void* d_workspace,
                                     size_t workspace_bytes);

/* Bytes of device workspace an _ex call needs.  n = total items; with_values
 * = 0 for keys only, 1 for pairs; num_segments = 0 for the unsegmented calls,
 * else the number of segments of a segmented call.  Pure host arithmetic.
 * For an unsegmented sort whose size class has RS_TUNE_DIGITS = 11 it
 * includes the buffers of the 11-bit order; a smaller workspace (down to the
 * 8-bit order's) is still accepted and then takes the 8-bit order. */
size_t rs_workspace_bytes(size_t n, int with_values, uint32_t num_segments);

/* 64-bit keys: the same LSD radix sort with K = 64 and D = 8 (Sec. 4 leaves
 * the key width general), i.e. eight stable counting-sort passes, unsigned
 * keys ascending, optionally carrying 32-bit values (d_vals may be NULL).
 * Passes whose digit is the same for every key are skipped as for 32-bit
 * keys (keys below 2^32 take four passes).  In place; asynchronous on
 * cuda_stream; d_keys 8-byte aligned, d_vals 4-byte aligned, not overlapping;
 * n < 2^32; workspace_bytes >= rs_workspace_bytes64(n, d_vals != NULL), the
 * workspace 256-byte aligned.  Whole arrays only (no segmented form). */
rs_status rs_sort64_ex(uint64_t* d_keys, uint32_t* d_vals, size_t n, void* cuda_stream,
                       void* d_workspace, size_t workspace_bytes);
size_t rs_workspace_bytes64(size_t n, int with_values);

/* Keys and values of every width this library sorts, in one call: keys of
 * any rs_key_type (32-bit or 64-bit words, unsigned, signed or IEEE float,
 * ordered as stated above), carrying values of value_bits = 0 (keys only;
 * d_vals NULL), 32 or 64 bits (d_vals not NULL).  Sec. 1 fixes the paper's
 * items at 32-bit keys with optional 32-bit values and notes that larger
 * ones work the same way; Sec. 4 leaves K general.  64-bit keys take eight
 * passes (K = 64, D = 8) and a value of any width moves with its key.
 * 32-bit keys with no or 32-bit values take the calls above (same workspace
 * size, same kernels); every other combination takes the scatter passes for
 * every array size (no on-chip sort of small arrays, no MSD-first order).
 * d_keys is aligned to its key width, d_vals to its value width; keys and
 * values do not overlap; n < 2^32; workspace_bytes >=
 * rs_workspace_bytes_kv(n, key_type, value_bits), the workspace 256-byte
 * aligned.  Asynchronous on cuda_stream, in place, stable.  An unknown
 * key_type or value_bits is RS_ERR_INVALID_ARG, and so are d_vals NULL with
 * value_bits != 0 and d_vals not NULL with value_bits = 0.
 * rs_sort64_ex(k, v, ...) is
 * rs_sort_kv_ex(k, v, ..., RS_KEY_U64, v ? 32 : 0, ...).
 * rs_workspace_bytes_kv returns 0 for n = 0 or unknown types. */
rs_status rs_sort_kv_ex(void* d_keys, void* d_vals, size_t n, int key_type, int value_bits,
                        void* cuda_stream, void* d_workspace, size_t workspace_bytes);
size_t rs_workspace_bytes_kv(size_t n, int key_type, int value_bits);

/* The segmented form of rs_sort_kv_ex: items of every width, each segment
 * [d_offsets[s], d_offsets[s+1]) sorted on its own (the plain definition of
 * the sort applied per segment; the paper has no segmented case), for
 * s = 0..num_segments-1.  The table follows the rules of
 * rs_sort_pairs_segmented (nondecreasing, last entry <= n, each segment
 * < 2^30 items; a bad table is reported as RS_ERR_BAD_SEGMENTS and nothing
 * is written).  32-bit keys with no or 32-bit values take the 32-bit
 * segmented sorts; every other combination sorts segments of up to 256
 * items in one warp each (in shared memory) and every longer one with the
 * scatter passes (eight for 64-bit keys).  Pointer, alignment, overlap and
 * type rules as for rs_sort_kv_ex; workspace_bytes >=
 * rs_workspace_bytes_kv_segmented(n, key_type, value_bits, num_segments),
 * 256-byte aligned.  Asynchronous on cuda_stream, in place, stable;
 * allocates nothing.  rs_workspace_bytes_kv_segmented returns 0 for n = 0,
 * num_segments = 0 or unknown types. */
rs_status rs_sort_kv_segmented_ex(void* d_keys, void* d_vals, size_t n, const uint32_t* d_offsets,
                                  uint32_t num_segments, int key_type, int value_bits,
                                  void* cuda_stream, void* d_workspace, size_t workspace_bytes);
size_t rs_workspace_bytes_kv_segmented(size_t n, int key_type, int value_bits,
                                       uint32_t num_segments);

/* Synchronise cuda_stream (NULL = legacy default stream), then return and
 * clear the sticky device status word of the current device: RS_OK, or the
 * first device-side error recorded since the last call (RS_ERR_TIMEOUT,
 * RS_ERR_BOUNDS, RS_ERR_BAD_SEGMENTS), or RS_ERR_CUDA if the synchronisation
 * itself failed.  The word is shared by every stream of the device. */
rs_status rs_stream_status(void* cuda_stream);

/* Static, human-readable name of a status code.  Never NULL. */
const char* rs_status_string(rs_status status);

/* Alg. 2's local step (Sec. 4, "reverse sorting"): one stable counting-sort
 * pass by the most significant digit (bits 24..31) of n keys, with their
 * values when d_vals != NULL, from (d_keys, d_vals) into (d_out_keys,
 * d_out_vals), and the bucket offsets d_bucket_offsets[b] = the first output
 * slot of digit value b (b = 0..255), d_bucket_offsets[256] = n.  Items of
 * one bucket keep their input order.  This is the partition a rank performs
 * before the exchange of the multi-GPU sort: each rank's output is grouped by
 * bucket, so the items bound for a range of buckets are one contiguous slice.
 *  - All pointers are device pointers; outputs must not overlap inputs;
 *    d_out_vals is NULL exactly when d_vals is.  d_bucket_offsets holds 257
 *    uint32_t and is overwritten.  The inputs are read, never written.
 *  - Workspace: d_workspace of at least rs_workspace_bytes(n, d_vals != NULL,
 *    0) bytes, 256-byte aligned.  Asynchronous on cuda_stream; allocates
 *    nothing; device-side errors via rs_stream_status(). */
rs_status rs_msd_partition_ex(const uint32_t* d_keys, const uint32_t* d_vals, size_t n,
                              uint32_t* d_out_keys, uint32_t* d_out_vals,
                              uint32_t* d_bucket_offsets, void* cuda_stream, void* d_workspace,
                              size_t workspace_bytes);

/* Digit histograms of n keys (counting step of Sec. 3 for all four digits at
 * once): d_hist[p*256 + b] = #{i : byte p of d_keys[i] == b}, p = 0..3,
 * b = 0..255.  d_hist is caller-owned device memory of 1024 uint32_t; it is
 * overwritten.  Asynchronous on cuda_stream; allocates nothing. */
rs_status rs_digit_histograms_ex(const uint32_t* d_keys, size_t n, uint32_t* d_hist,
                                 void* cuda_stream);

/* End-to-end sort of HOST arrays: copies h_keys_in (and h_vals_in, if not
 * NULL) to the device, sorts, and copies the result to h_keys_out (and
 * h_vals_out).  Inputs are not modified; output and input may be the same
 * array.  Device buffers are cached inside the library.  Synchronous. */
rs_status rs_sort_pairs_host(const uint32_t* h_keys_in, const uint32_t* h_vals_in,
                             uint32_t* h_keys_out, uint32_t* h_vals_out, size_t n);

/* Pipelined end-to-end sorts of `count` independent HOST arrays: array i
 * (h_keys_in[i] and, if h_vals_in is not NULL, h_vals_in[i]; n[i] items) is
 * copied to the device, sorted as by rs_sort_pairs (or rs_sort_keys when
 * h_vals_in is NULL), and copied back to h_keys_out[i] (h_vals_out[i]).
 * Three device buffer sets rotate, so that array i+1's upload and array
 * i-1's download run while array i is sorted: the host link carries both
 * directions at once.  Every array's copies are still complete copies; the
 * call returns when all arrays are back.  Inputs are not modified; an output
 * may be its own input; arrays with n[i] = 0 are skipped.  Pinned host
 * memory gives full link bandwidth.  Device buffers are cached inside the
 * library.  Synchronous.  n[i] >= 2^32 is RS_ERR_UNSUPPORTED; NULL tables or
 * entries are RS_ERR_INVALID_ARG. */
rs_status rs_sort_pairs_host_batch(const uint32_t* const* h_keys_in,
                                   const uint32_t* const* h_vals_in, uint32_t* const* h_keys_out,
                                   uint32_t* const* h_vals_out, const size_t* n, uint32_t count);

/* ---- captured sorts (CUDA graphs) -----------------------------------------
 * A sort of fixed device buffers captured once into a CUDA graph and then
 * replayed with one launch: the batched form for serving loops that refill
 * the same buffers with new data.  Not in the paper. */
typedef struct rs_graph_s* rs_graph;

/* Capture the sort of d_keys (and d_vals, if not NULL) -- segmented when
 * num_segments > 0 (d_offsets as for rs_sort_*_segmented), whole otherwise --
 * with the caller's workspace (>= rs_workspace_bytes(n, d_vals != NULL,
 * num_segments)) into a new graph, and instantiate it.  Nothing is sorted by
 * this call; the graph reads the buffers' contents when it is launched.  The
 * tuning knobs in force now are baked in.  n > 0. */
rs_status rs_graph_create(rs_graph* out, uint32_t* d_keys, uint32_t* d_vals, size_t n,
                          const uint32_t* d_offsets, uint32_t num_segments,
                          void* d_workspace, size_t workspace_bytes);

/* Enqueue one replay of the captured sort on cuda_stream (NULL = legacy
 * default stream).  Asynchronous; errors via rs_stream_status(). */
rs_status rs_graph_launch(rs_graph graph, void* cuda_stream);

/* Release the graph.  The buffers and workspace stay the caller's. */
rs_status rs_graph_destroy(rs_graph graph);

/* ---- sorting without allocating ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory when they sort: code on a
 * latency-critical path (cudaMalloc and cudaFree can synchronise the whole
 * device and stall every stream in flight), and processes that hand all of
 * the device memory to their own pool or arena, where an extra cudaMalloc
 * may fail.  rs_sort_keys / rs_sort_pairs allocate a cached workspace on
 * first use, and the _ex calls need a caller-provided one; this call needs
 * neither. */

/* Largest n accepted by rs_sort_pairs_noalloc (2^20 items). */
#define RS_NOALLOC_MAX_ITEMS (1u << 20)

/* Sort n keys (d_vals == NULL) or n (key, value) pairs in place, exactly as
 * rs_sort_pairs does, enqueued on cuda_stream (NULL = legacy default stream)
 * without allocating anything: no cudaMalloc, cudaFree or allocating library
 * call is made.  The scratch is a fixed 9 MiB array inside librs.so that
 * every GPU loading the library holds until the process exits.
 *  - n > RS_NOALLOC_MAX_ITEMS returns RS_ERR_UNSUPPORTED before any work.
 *  - Asynchronous: the caller collects device-side errors with
 *    rs_stream_status().
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    process; make that first call before any stream capture.  If the
 *    lookup fails the call returns RS_ERR_CUDA and the next call tries
 *    again.  cudaDeviceReset invalidates the kept address: do not call this
 *    entry point on a device after resetting it.
 *  - Every call on a device shares the one array (each call clears what must
 *    start at zero), so calls whose work overlaps on the GPU -- two streams,
 *    or two host threads -- race and corrupt each other's results; order
 *    them on one stream or synchronise in between. */
rs_status rs_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                void* cuda_stream);

/* ---- instrumentation (used by the benchmark; off by default) ---------- */

/* Number of kernels this library has launched on any device since it was
 * loaded (cudaMemset and copies are not counted). */
uint64_t rs_launch_count(void);

/* on = 1: from now on, bracket every kernel launch with CUDA events on the
 * launching stream; on = 0: stop and discard recorded events. */
rs_status rs_profile_enable(int on);

/* Synchronise the recorded events and return, per kernel kind k =
 * 0..max_kinds-1, the number of launches and their summed device time in
 * milliseconds since rs_profile_enable(1) or the last rs_profile_read.
 * Returns the number of kinds (see rs_kernel_kind_name); resets the tallies. */
int rs_profile_read(uint64_t* launches, double* total_ms, int max_kinds);

/* Name of kernel kind k, or NULL past the last kind. */
const char* rs_kernel_kind_name(int kind);

/* ---- tuning (used by the autotuner and the benchmarks) ------------------
 * Process-wide host settings read at every launch; change them only while no
 * other thread is enqueueing a sort.  Results never depend on them, only
 * speed does. */
typedef enum rs_tune_knob {
    RS_TUNE_TILE_PAIRS = 0,       /* tile shape index (rs_tile_shape) of key-value passes */
    RS_TUNE_TILE_KEYS = 1,        /* tile shape index of keys-only passes */
    RS_TUNE_HIST_CTAS_PER_SM = 2, /* CTAs per SM of the histogram kernel, 1..16 */
    RS_TUNE_HIST_MODE = 3,        /* 0: lane atomics, 1: lane-0 group + atomics, 2: ballot groups,
                                     3: one private shared column per lane (default) */
    RS_TUNE_SMALL_MAX = 4,        /* arrays and segments up to this size (<= 8192) take the
                                     one-CTA shared-memory sort; segments up to 4096 always
                                     take an on-chip sort */
    RS_TUNE_TILE_SEG = 5,         /* tile shape index of the segmented scatter passes */
    RS_TUNE_WARP_MAX = 6,         /* segments (and MSD-first buckets) up to this size (<= 512)
                                     take the one-warp shared-memory sort; 0 turns it off */
    RS_TUNE_SMALL_BITS = 7,       /* digit width of the one-warp and one-CTA sorts: 8 (four
                                     passes, the default) or 4 (eight passes) */
    RS_TUNE_MSD = 8,              /* 1: unsigned whole arrays of up to 2^21 items may take the
                                     MSD-first order of Alg. 2 (one pass by the top digit, then
                                     every bucket sorted on chip) when no top-digit bucket holds
                                     more than 8192 keys; 0: always the four LSD passes */
    RS_TUNE_TYPED_SPLIT = 9       /* signed and float keys: sorts of at least this many items
                                     launch two instances of every scatter pass (the passes that
                                     need no key map run without it, at the unsigned speed);
                                     smaller sorts launch one instance per pass, which maps where
                                     needed (half the launches) */,
    RS_TUNE_D11_SHAPE = 10,       /* tile shape of rs_sort_digits11_ex's scatter kernel: 0: 256
                                     threads x 32 items, two CTAs per SM; 1: 512 x 32, one CTA
                                     (the default); 2: 512 x 16, one CTA; 3: 256 x 24, two CTAs */
    RS_TUNE_DIGITS = 11,          /* 8 (the default): unsigned whole-array sorts run four 8-bit
                                     passes; 11: three 11/11/10-bit passes (as
                                     rs_sort_digits11_ex), taken when the caller's workspace holds
                                     their buffers -- rs_workspace_bytes then includes them */
    RS_TUNE_PDL = 13              /* 1 (the default): the plan and scatter-pass kernels launch as
                                     programmatic dependents of the kernel before them (resident
                                     while it finishes, waiting on the device for its results);
                                     0: plain stream order */
} rs_tune_knob;

/* Knobs 0, 1, 4..8 and 11 are kept per size class of the item count -- the
 * whole array's, or for a segmented sort the average segment's: class 0 up
 * to 2^13 items, 1 up to 2^16, 2 up to 2^20, 3 up to 2^24, 4 up to 2^28,
 * 5 above.  Knobs 2, 3, 9, 10 and 13 are global. */
#define RS_NUM_SIZE_CLASSES 6

/* Set a knob (a per-class knob in every class); RS_ERR_INVALID_ARG for an
 * unknown knob or out-of-range value. */
rs_status rs_tune_set(int knob, int value);

/* Current value of a knob (a per-class knob: its value in class 4), or -1
 * for an unknown knob. */
int rs_tune_get(int knob);

/* Set / read a per-class knob in one size class (0 .. RS_NUM_SIZE_CLASSES-1);
 * -1 / RS_ERR_INVALID_ARG for an unknown class or knob. */
rs_status rs_tune_set_class(int size_class_index, int knob, int value);
int rs_tune_get_class(int size_class_index, int knob);

/* Size class of an item count. */
int rs_size_class(size_t items);

/* Number of tile shapes of the scatter pass compiled into this build. */
int rs_tile_shape_count(void);

/* Shape `index`: CUDA threads per CTA and items per thread (a tile holds
 * threads * items_per_thread items).  RS_ERR_INVALID_ARG past the end. */
rs_status rs_tile_shape(int index, int* threads, int* items_per_thread);

/* ---- fault-injection knobs for tests (host-side settings) ------------- */

/* Iteration limit of every look-back wait (0 restores the default). */
rs_status rs_debug_set_spin_limit(uint32_t iterations);

/* withhold = 1: the first tile of every scatter pass never publishes its
 * counts, so the waits of the tiles after it run out and the call reports
 * RS_ERR_TIMEOUT.  0 restores normal operation. */
rs_status rs_debug_withhold_first_tile(int withhold);

#ifdef __cplusplus
}
#endif

#endif /* RS_H_ */
