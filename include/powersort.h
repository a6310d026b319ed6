/*
 * powersort.h -- C ABI of the GB300 (sm_103a) powersort library, libpowersort.so.
 *
 * The library sorts keys (with an optional 32-bit payload) stably and in place, as natural
 * mergesort in the merge order of powersort: J. I. Munro and S. Wild, "Nearly-Optimal
 * Mergesorts: Fast, Practical Sorting Methods That Optimally Adapt to Existing Runs",
 * arXiv 1805.04154 (the problem statement is a stable sort, Sec. 1; the method is Alg. 2).
 * All sorting work runs in the library's own CUDA kernels on one GPU:
 *   1. run detection  -- maximal weakly ascending / strictly descending runs (Sec. 2),
 *   2. node powers    -- Definition "Node Power", one integer computation per run boundary,
 *   3. merge tree     -- the Cartesian tree of the powers (Corollary "Cartesian tree"),
 *   4. merges         -- the tree's stable merges, scheduled level by level.
 * The result equals the stable sort of the (key, payload) pairs, bit for bit, including the
 * order of equal keys.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or documented as "device" are CUDA device pointers owned by the caller;
 *     the library never frees caller memory.  "host" pointers are ordinary host memory.
 *   - keys and vals need their natural alignment (key size, 4 bytes); sub-arrays at any element
 *     offset are fine.  Bulk copies work on whole 16-byte blocks, so a kernel may read, but never
 *     write, up to 15 bytes before the first or after the last element of an array, inside the
 *     16-byte blocks that hold its first and last elements.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).  Sorting calls
 *     are stream-ordered: they return once all work is enqueued; argument errors are returned
 *     synchronously.  Each sort synchronizes the stream once, after planning, to size its
 *     launches.  Errors posted later by the device are reported by ps_stream_status.
 *   - Limits: one call sorts fewer than 2^32 elements in total, in fewer than 2^31 - 1 runs (only
 *     segments of one element can come close); PS_ERR_UNSUPPORTED otherwise.  Node powers are then
 *     at most 32 and every element position fits 64 bits (Appendix B's node-power note: the
 *     31-bit form of the Java listing is only exact for int-sized arrays).
 *   - Thread safety: calls on different streams may run concurrently; a workspace must not be
 *     shared by calls in flight at the same time.
 */
#ifndef POWERSORT_H_
#define POWERSORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ps_status {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,    /* bad pointer, size, key type, alignment or segment offsets */
  PS_ERR_UNSUPPORTED = 2,    /* n >= 2^32, or 2^31 - 1 runs or more */
  PS_ERR_OUT_OF_MEMORY = 3,  /* workspace allocation failed or workspace too small */
  PS_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  PS_ERR_TIMEOUT = 5,        /* a bounded device wait gave up (results are not valid) */
  PS_ERR_INTERNAL = 6        /* an internal consistency check failed */
} ps_status;

typedef enum ps_key_type {
  PS_KEY_I32 = 0, /* int32, signed order */
  PS_KEY_U32 = 1, /* uint32 */
  PS_KEY_U64 = 2, /* uint64 */
  PS_KEY_F32 = 3  /* binary32 in IEEE 754 totalOrder: -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN;
                     the keys are moved as bit patterns and never altered */
} ps_key_type;

/* Statistics of the powersort plan of an array (Sec. 2.3 merge cost; Sec. 2 entropy). */
typedef struct ps_stats {
  int64_t n;             /* elements */
  int64_t runs;          /* r, detected runs (all segments) */
  uint64_t merge_cost;   /* M = sum over runs of (leaf depth x run length) */
  double entropy_bits;   /* H(L_1/n, ..., L_r/n) of a single array (float accumulation) */
  int32_t max_depth;     /* deepest leaf of the merge tree */
  int32_t merge_passes;  /* level passes over HBM */
  int64_t small_tasks;   /* subtrees merged entirely in shared memory */
} ps_stats;

/* Bytes of device workspace the *_ws entry points need for n elements (segmented != 0 for the
 * segmented entry points).  Depends only on the arguments. */
size_t ps_workspace_size(int key_type, int has_vals, int64_t n, int segmented);

/* Stable in-place sort of keys[0..n) (device, key_type elements) carrying vals[0..n) (device
 * uint32 payload, or NULL), powersort merge order (Alg. 2).  workspace: device memory of at least
 * ps_workspace_size(key_type, vals != NULL, n, 0) bytes, 256-byte aligned, caller-owned.
 * n = 0 or 1 is a no-op.  Errors: PS_ERR_INVALID_ARG (null or misaligned pointers, n < 0, unknown
 * key type), PS_ERR_OUT_OF_MEMORY (workspace too small), PS_ERR_UNSUPPORTED (n >= 2^32, or too
 * many runs), PS_ERR_CUDA, PS_ERR_TIMEOUT. */
ps_status ps_sort_ws(int key_type, void* keys, uint32_t* vals, int64_t n, void* workspace,
                     size_t workspace_bytes, void* stream);

/* As ps_sort_ws, with the workspace taken from a library-owned, stream-ordered device memory pool
 * (allocated and released on `stream`; the pool keeps freed memory for reuse). */
ps_status ps_sort(int key_type, void* keys, uint32_t* vals, int64_t n, void* stream);

/* Typed conveniences: ps_sort with the key type fixed. */
ps_status ps_sort_i32(int32_t* keys, uint32_t* vals, int64_t n, void* stream);
ps_status ps_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, void* stream);
ps_status ps_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, void* stream);
ps_status ps_sort_f32(float* keys, uint32_t* vals, int64_t n, void* stream);

/* Segmented sort: every segment [offsets[k], offsets[k+1]) of keys/vals is sorted on its own by
 * powersort (segment-relative positions in the node powers), all segments in the same launches.
 * d_offsets: device int64[count+1], offsets[0] = 0, non-decreasing, offsets[count] = n; empty
 * segments are allowed.  Offsets that break these rules are detected on the device and
 * reported as PS_ERR_INVALID_ARG (nothing is moved).  workspace as for ps_sort_ws with
 * segmented = 1. */
ps_status ps_sort_segmented_ws(int key_type, void* keys, uint32_t* vals, int64_t n,
                               const int64_t* d_offsets, int64_t count, void* workspace,
                               size_t workspace_bytes, void* stream);

/* As ps_sort_segmented_ws; n is read from d_offsets[count] (one small device-to-host copy) and
 * the workspace comes from the library's pool. */
ps_status ps_sort_segmented(int key_type, void* keys, uint32_t* vals, const int64_t* d_offsets,
                            int64_t count, void* stream);

/* Merge cost M of powersort's merge tree for runs of the given lengths (host int64[r], each
 * > 0, sum < 2^62): M = sum_i d_i L_i with d_i the depth of run i in the Cartesian tree of the
 * node powers (Sec. 2.3, Definition "Node Power", Corollary "Cartesian tree").  Host-only
 * computation.  Errors: PS_ERR_INVALID_ARG for null pointers, r <= 0, a length <= 0 or overflow. */
ps_status ps_merge_cost(const int64_t* run_lengths, int64_t r, uint64_t* out_cost);

/* Stages 1-3 on the device without moving any element: run detection, node powers, merge tree.
 * keys: device array (not modified); d_offsets/count as for ps_sort_segmented_ws, or NULL / 1
 * for one array; workspace as for ps_sort_ws (segmented = d_offsets != NULL).  Host outputs,
 * each optional (NULL to skip), capacity n + 1 entries; r = *out_runs:
 *   starts[r+1]     run starts (int64; starts[r] = n)
 *   desc[r]         1 if the run was strictly descending
 *   power[r+1]      node power of boundary j between runs j-1 and j (0 at j = 0, j = r and at
 *                   segment boundaries)
 *   leaf_depth[r]   depth of run i in the merge tree
 *   node_left[r+1], node_right[r+1]  for boundary j with power >= 1, its merge joins runs
 *                   [node_left[j], j) and [j, node_right[j]) (undefined elsewhere)
 *   node_depth[r+1] depth of boundary j's node (undefined where power is 0)
 * *out_cost receives M.  Synchronizes the stream. */
ps_status ps_analyze(int key_type, const void* keys, int64_t n, const int64_t* d_offsets,
                     int64_t count, void* workspace, size_t workspace_bytes, int64_t* out_runs,
                     uint64_t* out_cost, int64_t* starts, uint8_t* desc, uint8_t* power,
                     uint8_t* leaf_depth, int32_t* node_left, int32_t* node_right,
                     uint8_t* node_depth, void* stream);

/* Merge tree.  PS_TREE_POWERSORT: Alg. 2's tree, the Cartesian tree of the node powers (the
 * default of every other entry point).  PS_TREE_PEEKSORT: Alg. 1's tree, Mehlhorn's Method 1 on
 * the run lengths (Peeksort theorem): a range of runs is split at the run boundary nearest its
 * middle position (after its first run if the middle lies in it, before its last run if the
 * middle lies in that, else at the nearer end of the run holding the middle), applied to the
 * same greedy runs.  Both produce the same (unique stable) output; they differ in the merges
 * and hence the merge cost M. */
typedef enum { PS_TREE_POWERSORT = 0, PS_TREE_PEEKSORT = 1 } ps_tree;

/* ps_workspace_size for the given merge tree (PS_TREE_PEEKSORT needs 8 (n + 2) bytes more for
 * the level-by-level tree construction).  0 for an unknown key type or tree. */
size_t ps_workspace_size_tree(int key_type, int has_vals, int64_t n, int segmented, int tree);

/* ps_sort_ws (d_offsets NULL, count 1) or ps_sort_segmented_ws (d_offsets non-NULL) with the
 * merge tree chosen by `tree`; workspace of ps_workspace_size_tree(..., tree) bytes.  Errors as
 * for those entry points, plus PS_ERR_INVALID_ARG for an unknown tree and PS_ERR_INTERNAL if a
 * peeksort tree were deeper than the plan's 32 levels. */
ps_status ps_sort_tree_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                          int64_t count, int tree, void* workspace, size_t workspace_bytes, void* stream);

/* Failure-path self-test (no fault, trap or hang): queues one warp that waits on a
 * shared-memory mbarrier nothing completes, polling it at most `polls` times with the same
 * bounded loop the merge kernels use; when the polls run out it posts the timeout bit to the
 * library's status word and returns.  ps_stream_status(stream) then reports PS_ERR_TIMEOUT (and
 * clears it), and the device stays usable. */
ps_status ps_selftest_wait_timeout(uint32_t polls, void* stream);

/* Failure-path self-test through the production merge kernel (no fault, trap or hang): sorts
 * keys[0..n) (and vals) as ps_sort_ws does, except that every wait of the level passes polls at
 * most `polls` times and, in the deepest level pass, CTA 0 never issues the copies of its first
 * tile, so the consumers' wait on that stage runs out: they post the timeout bit, the CTA's other
 * waits give up within `polls` polls each, no copy is left in flight, and the kernel returns.
 * ps_stream_status(stream) then reports PS_ERR_TIMEOUT; the array's contents are unspecified
 * afterwards and the device stays usable.  workspace as for ps_sort_ws.  PS_ERR_UNSUPPORTED if the
 * array has no merge large enough for a level pass; PS_ERR_INVALID_ARG for polls = 0; other
 * errors as for ps_sort_ws. */
ps_status ps_selftest_level_pass_timeout(int key_type, void* keys, uint32_t* vals, int64_t n, uint32_t polls,
                                         void* workspace, size_t workspace_bytes, void* stream);

/* Level-pass configuration and its autotuner.  A level pass splits its merges into tiles of
 * items_per_thread x 256 outputs (the merge-path granularity) staged through a ring of `stages`
 * shared-memory buffers; the library carries the configurations (12, 2), (12, 3), (12, 4),
 * (8, 2), (8, 3), (16, 2), (6, 2) and (10, 2).  The configuration a sort uses is looked up by key
 * type, payload choice, plain or segmented call, and the size bucket of its n (n < 2^20, < 2^24,
 * < 2^28, larger):
 * the tuned entry of that bucket if an autotune call set one, else the default of the key type
 * and payload choice (ps_tune_set), else (8, 2) for 4-byte keys and (6, 2) for 8-byte keys.
 * Process-wide. */
typedef struct {
  int items_per_thread;    /* the chosen configuration */
  int stages;
  int n_variants;          /* configurations timed below */
  int variant_items[8];
  int variant_stages[8];
  double variant_ms[8];    /* median device time of one whole sort of the given array */
} ps_tune_result;

/* Time every configuration on copies of the caller's device array keys[0..n) (vals may be NULL;
 * neither is modified; scratch from the library's pool), keep the fastest as the tuned entry of
 * plain sorts of this key type, payload choice and n's size bucket, and report all timings.
 * Synchronizes the stream. */
ps_status ps_autotune(int key_type, const void* keys, const uint32_t* vals, int64_t n, ps_tune_result* out,
                      void* stream);

/* As ps_autotune for segmented sorts: times ps_sort_segmented_ws of the caller's batch (d_offsets:
 * device int64[count+1] as for ps_sort_segmented_ws) and keeps the fastest as the tuned entry of
 * segmented sorts of n's size bucket (used by ps_sort_segmented* and by ps_sort_async_ws with
 * offsets). */
ps_status ps_autotune_segmented(int key_type, const void* keys, const uint32_t* vals, int64_t n,
                                const int64_t* d_offsets, int64_t count, ps_tune_result* out, void* stream);

/* Set the default configuration of a key type and payload choice and clear its tuned entries
 * (0, 0: back to the built-in default); PS_ERR_UNSUPPORTED for a configuration the library does not carry. */
ps_status ps_tune_set(int key_type, int has_vals, int items_per_thread, int stages);

/* The default configuration of a key type and payload choice (what sorts use in size buckets
 * without a tuned entry). */
ps_status ps_tune_get(int key_type, int has_vals, int* items_per_thread, int* stages);

/* The configuration a sort of n elements (segmented != 0: a segmented call) of this key type and
 * payload choice uses. */
ps_status ps_tune_get_for(int key_type, int has_vals, int64_t n, int segmented, int* items_per_thread, int* stages);

/* Device-driven sort: as ps_sort_tree_ws (d_offsets NULL, count 1 for one array), but with no
 * host round trip -- every launch after planning takes its work count from the plan on the
 * device (persistent grids; one level-pass launch per depth the tree can have, empty ones return
 * at once), so the call only queues work on `stream` and can be captured into a CUDA graph and
 * replayed on the same buffers.  Binary level passes.  Argument errors are returned at once;
 * errors found on the device (segment offsets, timeouts, internal) are reported by
 * ps_stream_status, and with rejected offsets nothing is moved.  workspace:
 * ps_workspace_size_tree(key_type, vals != NULL, n, d_offsets != NULL, tree) bytes.  The first
 * call on a device allocates the library's status word and sets kernel attributes: make one
 * call before capturing. */
ps_status ps_sort_async_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                           int64_t count, int tree, void* workspace, size_t workspace_bytes, void* stream);

/* ps_sort_async_ws with powersort's tree (Alg. 2) for callers that know the longest segment:
 * every segment (the whole array when d_offsets is NULL) holds at most max_segment elements.
 * The level passes are launched only down to the deepest node a segment of that length can give
 * a level pass (a node of power p spans fewer than 4 n_s / 2^p of its segment's n_s elements, and
 * depth < power; Definition "Node Power"), so a batch of short segments queues fewer launches.
 * The bound is checked on the device with the offsets: a longer segment is reported by
 * ps_stream_status as rejected offsets and nothing is moved.  PS_ERR_INVALID_ARG for
 * max_segment < 1, or without offsets for n > max_segment.  Workspace and capture rules as for
 * ps_sort_async_ws (tree PS_TREE_POWERSORT). */
ps_status ps_sort_async_bounded_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                                   int64_t count, int64_t max_segment, void* workspace, size_t workspace_bytes,
                                   void* stream);

/* ps_analyze with the merge tree chosen by `tree`.  For PS_TREE_PEEKSORT, power[j] receives the
 * node's depth + 1 at every internal boundary (0 at sentinels and segment borders): the order in
 * which the plan finds parents (a leaf's parent is the larger of its two boundaries, a node's
 * parent the larger of its range ends), as node powers do for Alg. 2. */
ps_status ps_analyze_tree(int key_type, const void* keys, int64_t n, const int64_t* d_offsets, int64_t count,
                          int tree, void* workspace, size_t workspace_bytes, int64_t* out_runs, uint64_t* out_cost,
                          int64_t* starts, uint8_t* desc, uint8_t* power, uint8_t* leaf_depth, int32_t* node_left,
                          int32_t* node_right, uint8_t* node_depth, void* stream);

/* Minimal run length (Sec. 5.1: the tuned implementations extend every run shorter than
 * w = 24 by insertion sort to w elements, capped at the end of the array).  Runs are found left
 * to right as in ExtendRunRight of Alg. 2, but a run [s, e) with e - s < min_run becomes
 * [s, min(s + min_run, end)) (end = n, or the end of its segment); the next run starts there.
 * Such an extended run is sorted stably when it is placed (the order of key, then position: the
 * result of reversing a strictly descending prefix and insertion-sorting the rest), and the
 * powersort tree (Alg. 2) is built over the extended runs.  min_run = 1 is the plain greedy
 * partition of every other entry point.
 *   ps_sort_minrun_ws   as ps_sort_tree_ws with PS_TREE_POWERSORT (d_offsets NULL, count 1 for
 *                       one array; workspace of ps_workspace_size bytes).
 *   ps_analyze_minrun   as ps_analyze; desc[i] has bit 0 set if run i's first pair is strictly
 *                       descending and bit 1 set if the run was extended.
 * Errors as for those entry points, plus PS_ERR_INVALID_ARG for min_run outside [1, 32]. */
ps_status ps_sort_minrun_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                            int64_t count, int min_run, void* workspace, size_t workspace_bytes, void* stream);
ps_status ps_analyze_minrun(int key_type, const void* keys, int64_t n, const int64_t* d_offsets, int64_t count,
                            int min_run, void* workspace, size_t workspace_bytes, int64_t* out_runs,
                            uint64_t* out_cost, int64_t* starts, uint8_t* desc, uint8_t* power, uint8_t* leaf_depth,
                            int32_t* node_left, int32_t* node_right, uint8_t* node_depth, void* stream);

/* Bounds-checked builds.  A library compiled with -DPS_DEBUG (libpowersort_debug.so) compares
 * the data-derived indices of its kernels (shared-memory slots of the subtree merges, stage
 * offsets of the level passes, words of the node-power array, tree outputs, transfer-table
 * states) with their extents, skips any access out of range and counts it.  *hits receives the
 * count since the library was loaded (synchronize the sorting streams first).  PS_ERR_UNSUPPORTED
 * from a library built without the checks. */
ps_status ps_debug_bounds(unsigned long long* hits);

/* Plan statistics of one array (keys on the device, not modified; workspace from the pool).
 * Synchronizes the stream. */
ps_status ps_sort_stats(int key_type, const void* keys, int64_t n, ps_stats* out, void* stream);

/* Sort host arrays through the GPU: copies keys_in/vals_in (host, n elements; pinned memory gives
 * the fastest copies) to device buffers from the library's pool, sorts them as ps_sort does, and
 * copies the result to keys_out/vals_out (host; may alias the inputs).  vals_in and vals_out
 * are both NULL or both non-NULL.  Synchronizes the stream before returning. */
ps_status ps_sort_host(int key_type, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                       uint32_t* vals_out, int64_t n, void* stream);

/* Host arrays sorted through caller-owned device memory, queued on `stream` without waiting for
 * anything: copies keys_in/vals_in (host, n elements) into dev_keys/dev_vals (device, n
 * elements, natural alignment), sorts them with the device-driven pipeline of ps_sort_async_ws
 * and `workspace` (ps_workspace_size(key_type, vals_in != NULL, n, 0) bytes), and copies the
 * result to keys_out/vals_out (host; may alias the inputs).  Synchronize `stream` before reading
 * keys_out.  With pinned host memory and one set of device buffers per stream, consecutive calls
 * on different streams overlap the copy-in of one array, the sort of another and the copy-out of
 * a third.  vals_in, vals_out and dev_vals are all NULL or all non-NULL.  Argument errors are
 * returned at once; errors found on the device are reported by ps_stream_status. */
ps_status ps_sort_host_ws(int key_type, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                          uint32_t* vals_out, int64_t n, void* dev_keys, uint32_t* dev_vals, void* workspace,
                          size_t workspace_bytes, void* stream);

/* Measurement.  While enabled, every sort records CUDA events on its stream around its stages
 * (0 run detection, 1 node powers + merge tree + plan, 2 subtrees merged in shared memory,
 * 3 large-leaf placement, 4 unused, 5 level passes of the large merges).
 * ps_profile_read waits for the recorded events and returns, per stage since the last enable,
 * the device milliseconds, kernel launches and algorithmic HBM bytes (every element a stage
 * moves counted once read and once written: 2 x elements x (key bytes + payload bytes); run
 * detection reads the keys once).  ps_profile_enable(on) also clears the accumulators. */
typedef struct ps_profile {
  double ms[8];
  uint64_t launches[8];
  uint64_t bytes[8];
} ps_profile;
ps_status ps_profile_enable(int on);
ps_status ps_profile_read(ps_profile* out);

/* Number of kernels the library has launched in this process (all devices, all calls). */
uint64_t ps_launch_count(void);

/* Allocation-free sort of a small device array.  The paper has no counterpart; this is an
 * integration entry point for callers that must not allocate device memory while they run
 * (cudaMalloc / cudaFree can synchronize the whole device and can fail once a fixed memory
 * budget is used up, and hosts that own all device memory through their own allocator forbid
 * stray allocations).  Same semantics as ps_sort (stable in-place sort of keys[0..n) with
 * optional vals, powersort merge order), but every piece of scratch memory lives in one
 * fixed array inside the library's device image (about 9 MiB, held by every GPU that loads the
 * library until the process exits), so the call never allocates.
 *   - n <= PS_NOALLOC_MAX_N elements; larger n returns PS_ERR_INVALID_ARG and touches nothing.
 *   - The first call on a device looks up the array's device address with that device current
 *     (a one-time set-up per device); make that first call before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents (each call clears
 *     what must start at zero).  Calls that overlap on the GPU -- on different streams or from
 *     different host threads -- race on it and corrupt each other: serialize them.
 *   - Synchronizes the stream before returning and reports device-posted errors itself.
 * Other errors as for ps_sort_ws. */
#define PS_NOALLOC_MAX_N 262144
ps_status ps_sort_noalloc(int key_type, void* keys, uint32_t* vals, int64_t n, void* stream);

/* Synchronizes `stream`, then reports (and clears) errors the device posted on the current
 * device since the last call: PS_ERR_TIMEOUT if a bounded wait gave up, PS_ERR_CUDA if the
 * stream itself failed, else PS_OK. */
ps_status ps_stream_status(void* stream);

/* Static description of a status code (never NULL). */
const char* ps_status_string(ps_status status);

/* Library version: major * 10000 + minor * 100 + patch. */
int ps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POWERSORT_H_ */
