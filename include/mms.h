/*
 * mms.h -- C ABI of the GB300 (sm_103a) GPU Multiway Mergesort library.
 *
 * The library sorts keys that already live in GPU memory, following the
 * method of "An Efficient Multiway Mergesort for GPU Architectures"
 * (Casanova, Iacono, Karsin, Sitchinava, Weichert):
 *   - a base case that sorts fixed-size tiles on chip (Sec. 4.3),
 *   - then ceil(log_K(N / tile)) K-way merge rounds (Sec. 4, Sec. 6.2), each
 *     partitioned by a multi-sequence pivot search (Sec. 4.1) and merged on
 *     chip without shared-memory bank conflicts (Sec. 4.2).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers the caller owns.  Key and value
 *     arrays need only the alignment of their element (4 bytes for u32, f32
 *     and values, 8 bytes for u64), so a tensor slice at any element offset
 *     is accepted; arrays on the 16-byte grid take the vectorised paths.
 *     Workspaces must be 16-byte aligned (the batched sort's 256-byte
 *     aligned).  `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Calls are asynchronous on `stream`: they return once the work is queued,
 *     also when the library allocates the workspace itself (stream-ordered).
 *     Argument errors are reported synchronously by the return value.
 *     Device-side errors (a bounded wait that ran out, a failed consistency
 *     check) are recorded in the status word of the call's workspace, which
 *     every call clears first, and read back by mms_workspace_status(); a
 *     call whose workspace the library allocated forwards its status word to
 *     a per-device word that mms_stream_status() reads.
 *   - Sorting is ascending and stable: equal keys keep their input order and
 *     32-bit values move with their keys.
 *   - Key types: 32- and 64-bit unsigned integers (the paper's 4- and 8-byte
 *     workloads, Sec. 6.3), and IEEE-754 binary32 ordered by totalOrder on bit
 *     patterns (-NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN, NaNs by
 *     payload; the paper sorts integers only, so this ordering is this
 *     library's reading).  Output bits equal input bits.
 *   - No call throws; calls on distinct streams with distinct buffers and
 *     workspaces may run concurrently.
 */
#ifndef MMS_H_
#define MMS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MMS_OK = 0,
  MMS_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, size mismatch, bad fanout */
  MMS_ERR_UNSUPPORTED = 2,  /* key type / entry point combination not provided */
  MMS_ERR_NO_MEMORY = 3,    /* workspace too small, or internal allocation failed */
  MMS_ERR_CUDA = 4,         /* a CUDA runtime call failed; see mms_last_error_detail */
  MMS_ERR_TIMEOUT = 5,      /* a device-side bounded wait ran out */
  MMS_ERR_INTERNAL = 6      /* a device-side consistency check failed */
} mms_status;

typedef enum { MMS_KEY_U32 = 0, MMS_KEY_U64 = 1, MMS_KEY_F32 = 2 } mms_key_type;

/* Planner overrides and a profiling hook; a NULL pointer or zero fields mean
 * "planner's choice, no hook". */
typedef struct {
  int fanout;        /* K of every merge round, 2..32 (Sec. 6.2: K is tuned per platform) */
  int num_events;    /* entries of `events` */
  void** events;     /* cudaEvent_t handles the caller created: events[0] is recorded on
                        `stream` before the first kernel, events[i] after the i-th kernel
                        (base case, then splitter and merge pass of each round), while
                        i < num_events.  Lets a caller time every step of the real call. */
  int tile_items;    /* CTA tile of the base case and of the merge rounds: 0 =
                        mms_tile_items(kt); else 4096 or 8192 for 4-byte keys, 2048 or
                        4096 for 8-byte keys (the base case's runs: base_items) */
  int merge_tile_items; /* output tile of the merge rounds: 0 = tile_items; else a multiple
                        of 1024 from 4096 (2048 for 8-byte keys) up to tile_items */
  int test_flags;    /* test hooks, 0 in normal use.  MMS_TEST_STAGING_TIMEOUT: every merge
                        CTA of mms_sort_keys_ex, once its staged inputs have all arrived,
                        also waits (about a millisecond) on a barrier that no copy
                        completes, then records MMS_ERR_TIMEOUT and stops: the device-side
                        failure path, with nothing left in flight.  The output is then
                        unspecified. */
  int merge_variant; /* how a merge round merges a tile: MMS_MERGE_TREE (0, the default):
                        the CTA's binary tree of block merges, level by level (Sec. 4.2);
                        MMS_MERGE_PARTITION: the heap-free variant of Sec. 7 (future
                        work), each warp finding its 1024-key output block's pieces in
                        the tile's K segments by the partitioning search of Sec. 4.1 and
                        merging them alone; MMS_MERGE_PIPELINED: the pipelining of
                        Sec. 7 (future work), persistent CTAs whose producer warp plans
                        and stages the next tile while the merging warps merge the
                        current one.  Same results; the variants take the default tile
                        geometry only (tile_items and merge_tile_items 0), apply to
                        mms_sort_keys_ex and mms_sort_pairs_ex, and take no test flags. */
  int base_items;    /* length of the sorted runs the base case of mms_sort_keys_ex
                        produces (Sec. 4.3): 0 = the tile (one CTA per tile, the
                        default); for 4-byte keys at the 8192-key tile also 16384,
                        32768 or 65536 = one thread-block cluster of 2, 4 or 8 CTAs per
                        run, which sorts 8192 keys per CTA and merges them across the
                        cluster's shared memory.  Longer runs leave fewer merge levels
                        to the rounds (same results).  A key-value sort takes 0 or its
                        composite tile. */
} mms_options;

#define MMS_TEST_STAGING_TIMEOUT 1
#define MMS_MERGE_TREE 0
#define MMS_MERGE_PARTITION 1
#define MMS_MERGE_PIPELINED 2

/* Bytes of workspace mms_sort_keys / mms_sort_pairs need for n keys: one
 * ping-pong copy of the keys (and values), the pivot table of the largest
 * round, and a status word. */
size_t mms_sort_workspace_bytes(mms_key_type kt, size_t n, int with_values);

/* Sorts n keys of type kt at d_keys in place (from the caller's view).
 * d_ws: workspace of at least mms_sort_workspace_bytes(kt, n, 0) bytes (any
 * contents: its status word is cleared on `stream` first), or NULL to let the
 * library allocate one stream-ordered (cudaMallocAsync) and free it after the
 * sort; the call then still returns without waiting for the GPU, and its
 * device-side status goes to the word mms_stream_status() reads.  n = 0 and
 * n = 1 are no-ops. */
mms_status mms_sort_keys(mms_key_type kt, void* d_keys, size_t n, void* d_ws, size_t ws_bytes,
                         void* stream);
mms_status mms_sort_keys_ex(mms_key_type kt, void* d_keys, size_t n, void* d_ws, size_t ws_bytes,
                            void* stream, const mms_options* opt);

/* Sorts (key, 32-bit value) pairs stably by key (Sec. 4 with the order of
 * Sec. 4.1 read on (key, position)); values move with keys.  n < 2^32.
 * 4-byte keys (u32, f32): the rounds run on unique 64-bit composites
 * (ordered key << 32 | position) and a last kernel gathers the values.
 * 8-byte keys (u64): two stable 4-byte passes, the low key halves first, then
 * the high halves of the items in that order, whose ties keep the first
 * pass's order (the textbook LSD composition of stable sorts); a last kernel
 * applies the resulting permutation to keys and values.
 * Workspace: mms_sort_workspace_bytes(kt, n, 1), or NULL (allocated and freed
 * stream-ordered).  opt: as for mms_sort_keys_ex; its events are recorded
 * before the value copy, after the base case, after each splitter and merge
 * pass, and after the value gather (for 8-byte keys, those of both passes in
 * turn); tile_items may be 0, 2048 or 4096 (composite tiles). */
mms_status mms_sort_pairs(mms_key_type kt, void* d_keys, uint32_t* d_values, size_t n, void* d_ws,
                          size_t ws_bytes, void* stream);
mms_status mms_sort_pairs_ex(mms_key_type kt, void* d_keys, uint32_t* d_values, size_t n,
                             void* d_ws, size_t ws_bytes, void* stream, const mms_options* opt);

/* Reads (synchronising with `stream`) and clears the workspace status word:
 * MMS_OK, MMS_ERR_TIMEOUT or MMS_ERR_INTERNAL. */
mms_status mms_workspace_status(void* d_ws, size_t ws_bytes, void* stream);

/* Status of the sorts that ran without a caller workspace (d_ws == NULL) on
 * the current device: waits for `stream`, then returns and clears the first
 * device-side error any of them recorded since the last call (MMS_OK,
 * MMS_ERR_TIMEOUT or MMS_ERR_INTERNAL).  The word is per device, shared by
 * all streams: wait for the other streams' sorts before relying on it. */
mms_status mms_stream_status(void* stream);

/* ---- the hot-path steps one by one (for parity tests and profiling) -------- */

/* Items per base-case tile and per merge output tile for key type kt
 * (8192 for 4-byte keys, 4096 for 8-byte keys). */
size_t mms_tile_items(mms_key_type kt);

/* Length of the sorted runs the base case of mms_sort_keys_ex produces for n
 * keys of type kt under opt (NULL: defaults): the tile (tile_items, default
 * mms_tile_items(kt)) or opt->base_items.  0 for an invalid kt or opt. */
size_t mms_base_run_items(mms_key_type kt, size_t n, const mms_options* opt);

/* Plan of a sort: number of merge rounds and the fanout of each (up to 16
 * entries written to fanouts).  Returns the number of rounds. */
int mms_plan(mms_key_type kt, size_t n, const mms_options* opt, int* fanouts, int max_rounds);

/* Base case (Sec. 4.3): sorts every tile of mms_tile_items(kt) consecutive
 * keys of d_in into d_out (d_in == d_out allowed).  The last tile may be
 * short.  Float keys are sorted by totalOrder and written back as floats. */
mms_status mms_tile_sort(mms_key_type kt, const void* d_in, void* d_out, size_t n, void* stream);

/* Number of rows of the pivot table of a merge round over n keys in sorted
 * runs of run_len keys merged K at a time: one row per output tile. */
size_t mms_splitter_rows(mms_key_type kt, size_t n, size_t run_len, int K);

/* Parallel partitioning (Sec. 4.1): d_in holds sorted runs of run_len keys
 * (the last one may be short; run_len a multiple of mms_tile_items(kt)).
 * Groups of K consecutive runs are merged into one; for output tile j of a
 * group, row t of d_table (K int64 entries, rows in tile order, group after
 * group) receives, for each run r of the group, the number of its keys among
 * the group's first j * mms_tile_items(kt) outputs under the strict order
 * (key, run, position).  Integer key types only (u32, u64). */
mms_status mms_splitter(mms_key_type kt, const void* d_in, size_t n, size_t run_len, int K,
                        int64_t* d_table, void* stream);

/* One K-way merge round (Sec. 4.2): merges every group of K runs of d_in into
 * one sorted run of d_out, driven by the table mms_splitter wrote for the
 * same (d_in, n, run_len, K).  d_in and d_out must not overlap.  d_ws: NULL,
 * or a sort workspace whose status word records device-side errors.
 * Integer key types only. */
mms_status mms_merge_pass(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                          size_t run_len, int K, const int64_t* d_table, void* d_ws,
                          size_t ws_bytes, void* stream);

/* The same round merged by the heap-free partition variant (Sec. 7, future
 * work; mms_options.merge_variant = MMS_MERGE_PARTITION): every output tile
 * is cut into 1024-key blocks whose pieces in the tile's K segments the
 * warps find with the search of Sec. 4.1 in shared memory, and each warp
 * merges its own pieces.  Arguments, layout, ownership and errors as for
 * mms_merge_pass; the output is identical. */
mms_status mms_merge_pass_partition(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                                    size_t run_len, int K, const int64_t* d_table, void* d_ws,
                                    size_t ws_bytes, void* stream);

/* The same round merged by the pipelined variant (Sec. 7, future work;
 * mms_options.merge_variant = MMS_MERGE_PIPELINED): persistent CTAs, each
 * with a producer warp that plans and stages tile q + 1 into the third of
 * three tile buffers while its merging warps merge tile q.  Arguments,
 * layout, ownership and errors as for mms_merge_pass; the output is
 * identical. */
mms_status mms_merge_pass_pipelined(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                                    size_t run_len, int K, const int64_t* d_table, void* d_ws,
                                    size_t ws_bytes, void* stream);

/* ---- batched (segmented) sorting ------------------------------------------- */

/* Many independent arrays ("segments") of uneven size, back to back in one
 * buffer, each sorted on its own (ascending, stable) by the same method as a
 * whole array: a base case, then K-way merge rounds (Sec. 4).  The paper
 * sorts one array; batching is this library's extension.  Segment s is
 * d_keys[d_offsets[s], d_offsets[s + 1]); d_offsets (device, 8-byte aligned)
 * holds num_segments + 1 non-decreasing entries from 0 to total_n.  Every
 * segment gets the fanout K of its size class ceil(log2 n) and its own number
 * of rounds; the whole launch sequence needs no host synchronisation, so it
 * can be captured into a CUDA graph (mms_segmented_graph_create).  Offsets
 * out of order, or a segment above max_segment_items, set the workspace
 * status word to MMS_ERR_INTERNAL (read it with mms_workspace_status). */
typedef struct {
  int class_fanout[33];       /* K (2..32) for segments of size class c = ceil(log2 n); 0 =
                                 default (4 for 4-byte keys, 8 for 8-byte keys and key-value
                                 batches).  Filled by the package's autotuner. */
  size_t max_segment_items;   /* largest segment (bounds the rounds launched); 0 = total_n */
  int tile_items;             /* 0 = mms_tile_items (key-value batches: 4096); else as for
                                 mms_options.tile_items */
  int num_events;             /* events[0] before the first kernel, events[1] after the
                                 planning kernels (and the value copy), events[2] after the
                                 base case, events[3 + r] after merge round r, the last after
                                 the value gather (key-value batches) */
  void** events;
  int reserved[4];
} mms_segmented_options;

/* Workspace bytes of a batch: one ping-pong copy of the keys (two 8-byte
 * composite buffers and a copy of the values for key-value batches), the
 * per-segment plan, the tile descriptors of every phase, the pivot table of
 * one round, and the status word. */
size_t mms_segmented_workspace_bytes(mms_key_type kt, size_t total_n, size_t num_segments,
                                     int with_values, const mms_segmented_options* opt);

/* Merge rounds a batch launches (segments that need fewer skip the rest). */
int mms_segmented_rounds(mms_key_type kt, size_t max_segment_items, int with_values,
                         const mms_segmented_options* opt);

/* Sorts every segment of d_keys in place; with d_values (total_n < 2^32) the
 * 32-bit values move with their keys (8-byte keys: two stable passes, as for
 * mms_sort_pairs).  d_keys and d_values must be 16-byte aligned (the
 * segments inside may start at any item).  d_ws (256-byte aligned,
 * mms_segmented_workspace_bytes) is required; its status word is cleared
 * first.  Asynchronous on `stream`. */
mms_status mms_segmented_sort(mms_key_type kt, void* d_keys, uint32_t* d_values,
                              const uint64_t* d_offsets, size_t num_segments, size_t total_n,
                              void* d_ws, size_t ws_bytes, void* stream,
                              const mms_segmented_options* opt);

/* A batched sort captured once into a CUDA graph and replayed with one
 * launch per call: the same buffers, offsets and workspace every time (their
 * contents may change between launches).  Creation queues no work; the
 * options' events are ignored. */
typedef struct mms_graph_s* mms_graph;
mms_status mms_segmented_graph_create(mms_key_type kt, void* d_keys, uint32_t* d_values,
                                      const uint64_t* d_offsets, size_t num_segments,
                                      size_t total_n, void* d_ws, size_t ws_bytes,
                                      const mms_segmented_options* opt, mms_graph* out);
mms_status mms_graph_launch(mms_graph g, void* stream);
void mms_graph_destroy(mms_graph g);

/* ---- sorting without allocating -------------------------------------------- */

/* No counterpart in the paper: a convenience for callers that cannot allocate
 * device memory when they sort -- processes whose GPU memory belongs to
 * another allocator that must not be bypassed, services with a fixed memory
 * budget, or code that may not call cudaMalloc because it can synchronise the
 * device.  mms_sort_keys_noalloc sorts n keys at d_keys in place exactly like
 * mms_sort_keys, but its workspace is a fixed array of about 4 MiB that the
 * library declares in device memory; every GPU that loads the library holds
 * that array until the process exits.  The call allocates nothing.
 *   - n must not exceed MMS_NOALLOC_MAX_KEYS_4B (u32, f32) or
 *     MMS_NOALLOC_MAX_KEYS_8B (u64); larger n returns MMS_ERR_INVALID_ARG
 *     and queues no work.
 *   - The first call on a device looks up that device's copy of the array
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - The address is cached per device and per CUDA context: after a
 *     device reset the next call looks it up again in the new context.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (different streams, no ordering between them) race and corrupt each
 *     other's results.  Order them on one stream or with events.
 *   - Every call clears the array's status word first; device-side errors of
 *     the latest call are read back with mms_noalloc_status(). */
#define MMS_NOALLOC_MAX_KEYS_4B ((size_t)1 << 20)
#define MMS_NOALLOC_MAX_KEYS_8B ((size_t)1 << 19)
mms_status mms_sort_keys_noalloc(mms_key_type kt, void* d_keys, size_t n, void* stream);

/* Device-side status of the latest mms_sort_keys_noalloc call on the current
 * device, as mms_workspace_status reports it for a caller's workspace: waits
 * for `stream`, returns MMS_OK, MMS_ERR_TIMEOUT or MMS_ERR_INTERNAL, and
 * clears the word.  Allocates nothing. */
mms_status mms_noalloc_status(void* stream);

/* ---- diagnostics ----------------------------------------------------------- */

const char* mms_status_string(mms_status s);
/* Copies the detail of the last failing call on this host thread into buf. */
mms_status mms_last_error_detail(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* MMS_H_ */
