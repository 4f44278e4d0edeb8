/*
 * ccl.h -- C ABI of the GB300 (sm_103a) union-find connected-components
 * labelling library (libccl.so).
 *
 * Method: "An Optimized Union-Find Algorithm for Connected Components
 * Labeling Using GPUs" (Chen et al., 2017).  Three phases over a tiled image:
 *   1. local merge inside each tile in shared memory (Kernel 1, §II-A),
 *   2. boundary analysis that unions only across tile seams (Kernel 2, §II-B,
 *      Eq. 1-2),
 *   3. link: every pixel receives the root of its component (§II-C).
 *
 * Result (canonical form).  For an H x W uint8 image, pixel i = y*W + x is
 * foreground iff its byte is nonzero.  With 4- (Manhattan-1) or 8-
 * (Chebyshev-1) adjacency on the foreground pixels,
 *     labels[i] = 0                          for background,
 *     labels[i] = 1 + min{ j : j in C(i) }   for foreground,
 * where C(i) is the component of i.  The paper's union-find links by atomicMin
 * so every root is its component's smallest index, and its IDs are raster
 * indices x + y*imgWidth (Kernel 1 ID conversion); "+1, 0 = background" is
 * this library's encoding.  Results are exact integers and identical for any
 * tile shape, batch composition or thread interleaving.
 *
 * Conventions shared by every call below
 *   - Images and labels are dense row-major (pitch = width), in DEVICE memory
 *     owned by the caller, unless a call says "host".
 *   - 1 <= height, 1 <= width, height*width <= 2^31 - 2 (so 1 + the largest
 *     index fits in int32).  connectivity is 4 or 8.
 *   - Calls that take a stream only enqueue work on it and return; a failure
 *     detected before enqueueing returns an error code and enqueues nothing.
 *     Device-side failures (a bounded loop that ran out, which valid inputs
 *     never cause) are recorded in a per-device error word reported by
 *     ccl_sync().
 *   - Workspace: scratch device memory, caller-owned when given.  Its size
 *     comes from the matching *_workspace_bytes() call and it must be 256-byte
 *     aligned.  Passing NULL makes the library use its own per-(device,
 *     stream) buffer (grown on demand with cudaMalloc, which synchronises the
 *     device; released by ccl_shutdown()).  Two calls in flight at once on
 *     different streams must not share one caller workspace.
 *   - No call throws; all report through ccl_status.
 */
#ifndef CCL_H
#define CCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCL_OK = 0,
    CCL_ERR_INVALID_ARG = 1, /* bad size, connectivity, pointer or workspace */
    CCL_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    CCL_ERR_OOM = 3,         /* device or host allocation failed */
    CCL_ERR_TIMEOUT = 4,     /* a bounded wait/loop ran out (device error word) */
    CCL_ERR_REJECTED = 5,    /* server: request larger than the whole budget */
    CCL_ERR_SHUTDOWN = 6,    /* server: destroyed or shutting down */
    CCL_ERR_NOT_FOUND = 7,   /* server: unknown request id */
    CCL_ERR_PENDING = 8      /* server: request not finished yet (poll) */
} ccl_status;

/* Opaque CUDA stream handle (cudaStream_t); NULL = the legacy default stream. */
typedef void *ccl_stream;

/* Human-readable name of a status code; never NULL, static storage. */
const char *ccl_status_string(int status);

/* ------------------------------------------------------------------------ */
/* Single image                                                              */
/* ------------------------------------------------------------------------ */

/* Tile widths the kernels support: 32, 64, 128 or 256 pixels.  A tile always
 * holds 256 strips x words; its height is (8192 / tile_w) rows for
 * 4-connectivity and twice that for 8-connectivity.  The default for an image
 * comes from a process-wide size-class table (below), capped at the smallest
 * power of two >= width.  Returns 0 on invalid arguments. */
int ccl_default_tile_width(int height, int width, int connectivity);

/* Size-class table.  Heights and widths fall in CCL_TILE_CLASSES classes:
 * class 0 = extent <= 64, class c = extent in (64*2^(c-1), 64*2^c], the last
 * class = extent > 2048.  widths[hc * CCL_TILE_CLASSES + wc] is the tile width
 * used for height class hc and width class wc (host array of
 * CCL_TILE_CLASSES^2 ints).  get reports the effective widths at each class's
 * representative size; set validates every entry (32/64/128/256) before
 * installing any.  Results never depend on the table, only speed does. */
#define CCL_TILE_CLASSES 7
ccl_status ccl_get_tile_table(int connectivity, int *widths);
ccl_status ccl_set_tile_table(int connectivity, const int *widths);

/* Autotuner: for every class pair, label a synthetic image of the class's
 * representative size (64*2^c, 4096 for the last class; foreground drawn with
 * probability 1/2 on the device) with each admissible tile width, `reps`
 * timed runs after one warm-up (CUDA events on `stream`), and install the
 * fastest width.  Allocates its own scratch (cudaMalloc, freed before
 * returning) and blocks until done.  CCL_OK, CCL_ERR_INVALID_ARG, CCL_ERR_OOM
 * or CCL_ERR_CUDA. */
ccl_status ccl_autotune(int connectivity, int reps, ccl_stream stream);

/* Bytes of workspace ccl_label needs for this image: the largest need over
 * every tile width, so a workspace sized once stays valid if the size-class
 * table changes.  ccl_workspace_bytes_tiled: the need for one tile width
 * (tile_w 0 = the default: same as ccl_workspace_bytes).  0 on invalid
 * arguments. */
size_t ccl_workspace_bytes(int height, int width, int connectivity);
size_t ccl_workspace_bytes_tiled(int height, int width, int connectivity, int tile_w);

/* Label one image (all three phases: local merge §II-A, boundary analysis
 * §II-B, link §II-C) with the default tile width.
 *   d_img    : device, height*width bytes, nonzero = foreground (read only)
 *   d_labels : device, height*width int32, fully overwritten by the link
 *              phase (it must not alias d_img or the workspace)
 *   d_ws     : device workspace of ws_bytes >= ccl_workspace_bytes(), or NULL
 *   stream   : CUDA stream to enqueue on
 * Returns CCL_OK once the three kernels are enqueued. */
ccl_status ccl_label(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                     int connectivity, void *d_ws, size_t ws_bytes, ccl_stream stream);

/* Flags for ccl_label_tiled. */
#define CCL_FLAG_LOCAL_ONLY 1u /* stop after the local merge: every tile is
                                  labelled as if it were a separate image and
                                  its root index converted to the global raster
                                  index (Kernel 1 output, the paper's "global
                                  label map after local merge", Fig. 4(a)) */

/* As ccl_label with an explicit tile width (32, 64, 128, 256; 0 = default)
 * and flags.  Same arguments, ownership and errors as ccl_label. */
ccl_status ccl_label_tiled(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                           int connectivity, int tile_w, unsigned flags, void *d_ws,
                           size_t ws_bytes, ccl_stream stream);

/* Label every region of a multi-level image: pixels are connected when they
 * are neighbours and hold the same byte value, which is the predicate the
 * paper's kernels test (equal dBuff values in Kernel 1, §II-A; equal image
 * values in Kernel 2, §II-B) before its pseudo-code is specialised to binary
 * images.  Every pixel whose value is in levels[0..nlevels) gets 1 + the
 * smallest raster index of its equal-value component; every other pixel 0.
 * For a binary image, levels = {0, 1} labels background regions too.
 *   d_img, d_labels, d_ws, ws_bytes, stream : as ccl_label (the workspace
 *              need is ccl_workspace_bytes(), independent of nlevels)
 *   levels   : host, nlevels distinct byte values (read during the call only)
 *   nlevels  : 1..256
 * Runs one three-phase pass per level on `stream`; the first pass writes
 * every pixel, later ones only their own.  CCL_ERR_INVALID_ARG on a NULL or
 * empty level list or a repeated level; otherwise as ccl_label. */
ccl_status ccl_label_regions(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                             int connectivity, const uint8_t *levels, int nlevels, void *d_ws,
                             size_t ws_bytes, ccl_stream stream);

/* ---- volumes ---------------------------------------------------------------
 * Label a 3-D volume (the paper's "2D/3D grid", §I) with the three phases one
 * dimension up: a shared-memory local merge per brick (Kernel 1, §II-A),
 * unions across brick faces (Kernel 2, §II-B) and a link pass (§II-C).  A
 * brick is 32 voxels along x by 16 x 16 strips, a strip being 1 row (6), 2 rows
 * along y (18) or 2 x 2 rows (26): 32 x 16 x 16, 32 x 32 x 16 or 32 x 32 x 32
 * voxels.
 *   d_vol    : device, depth*height*width bytes, voxel (x, y, z) at index
 *              (z*height + y)*width + x, nonzero = foreground (read only)
 *   d_labels : device, depth*height*width int32, fully overwritten: 0 for
 *              background, else 1 + the smallest index of the voxel's
 *              component (must not alias d_vol or the workspace)
 *   connectivity : 6 (faces), 18 (faces and edges) or 26 (faces, edges and
 *              corners)
 *   d_ws     : device workspace of ws_bytes >= ccl_workspace_bytes3d(),
 *              256-byte aligned, or NULL (library-owned, as for ccl_label)
 *   stream   : CUDA stream to enqueue on
 * Limits: depth*height*width <= 2^31 - 2 and at most 2^22 bricks
 * (ceil(width/32) * ceil(height/bh) * ceil(depth/bd) for a brick of
 * 32 x bh x bd voxels).  Returns CCL_OK once
 * the three kernels are enqueued; CCL_ERR_INVALID_ARG for NULL pointers, bad
 * sizes or connectivity, or a workspace that is too small or misaligned;
 * CCL_ERR_OOM / CCL_ERR_CUDA otherwise.  Device-side failures are reported by
 * ccl_sync. */
ccl_status ccl_label3d(const uint8_t *d_vol, int32_t *d_labels, int depth, int height, int width,
                       int connectivity, void *d_ws, size_t ws_bytes, ccl_stream stream);

/* Bytes of workspace ccl_label3d needs for this size and connectivity (the
 * brick shape depends on the connectivity); 0 on invalid arguments. */
size_t ccl_workspace_bytes3d(int depth, int height, int width, int connectivity);

/* Number of unordered pairs of neighbouring pixels that lie in different
 * tiles for this size, connectivity and tile (tile_w x tile_h): the cells the
 * boundary analysis inspects (§II-B; Eq. 1-2 count them for a whole-tile grid).
 * Host-only arithmetic; -1 on invalid arguments. */
long long ccl_seam_pair_count(int height, int width, int connectivity, int tile_w,
                              int tile_h);

/* Benchmark hook: when `events` is non-NULL, the next ccl_label /
 * ccl_label_tiled call made by this host thread records events[0] before its
 * local-merge kernel, events[1] after it, events[2] after the seam-union
 * kernel and events[3] after the link kernel, all on that call's stream.
 * `events` points to 4 caller-owned cudaEvent_t handles (created with timing
 * enabled); the hook is consumed by that one call.  NULL clears it. */
void ccl_set_phase_events(void *const *events);

/* Wait for `stream`, then report and clear the device error word of the
 * current device: CCL_OK, CCL_ERR_TIMEOUT, or CCL_ERR_CUDA for an
 * asynchronous CUDA error. */
ccl_status ccl_sync(ccl_stream stream);

/* Free library-owned workspaces and batched-path state on every
 * device, and forget the device addresses the library caches per device (its
 * error word, the scratch array of ccl_label_static).  Call it after a
 * device's context was reset (cudaDeviceReset) and before using the library
 * on that device again: the cached addresses belong to the old context. */
ccl_status ccl_shutdown(void);

/* ---- failure injection (for tests of the failure paths) ------------------
 * The paper has no counterpart.  These calls let a test drive the library's
 * failure detection without faulting a GPU.
 *
 * ccl_set_hop_budget: every union-find walk of the 2-D kernels (ccl_label,
 * ccl_label_tiled, ccl_label_regions, ccl_label_batched and the server) draws
 * on a per-thread budget of pointer hops -- smem_hops for the shared-memory
 * forest of a tile, global_hops for the global forest of border roots.  When
 * a budget runs out the thread sets the device error word and stops walking,
 * so the kernel returns and ccl_sync() reports CCL_ERR_TIMEOUT (the labels of
 * that call are then unspecified).  The defaults (2^20 hops each) are far
 * above what any valid input needs; a test lowers them to make a walk run out
 * on purpose.  0 restores a default.  The setting is process-wide and applies
 * to calls enqueued after it.  CCL_ERR_INVALID_ARG for negative values.
 *
 * ccl_inject_alloc_failures: the next `count` library-owned workspace
 * allocations (the ones made when a call is given d_ws = NULL) fail as if the
 * device were out of memory: the call returns CCL_ERR_OOM and enqueues
 * nothing.  0 clears pending failures.  CCL_ERR_INVALID_ARG if count < 0. */
ccl_status ccl_set_hop_budget(int smem_hops, int global_hops);
ccl_status ccl_inject_alloc_failures(int count);

/* Allocation-free variant of ccl_label (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory: code inside a host
 * framework that owns every device allocation through its own allocator,
 * plug-ins that are handed only input and output pointers, and latency-
 * critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation or an allocation failure mid-stream).
 *
 * Same result, arguments, layout and ownership as ccl_label, but the scratch
 * lives in a fixed device array of CCL_STATIC_SCRATCH_BYTES inside this
 * library (held on every GPU that loads the library until the process
 * exits); the caller passes only the image and the labels.  The call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *   - Limit: ccl_workspace_bytes(height, width, connectivity) must not exceed
 *     CCL_STATIC_SCRATCH_BYTES (this covers every image up to 4096 x 4096 at
 *     either connectivity); larger images return CCL_ERR_INVALID_ARG and
 *     nothing is enqueued.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.  Later calls read the cache
 *     without locking.  ccl_shutdown() forgets it (needed after a context
 *     reset, which moves the array).
 *   - All calls on a device share the one array and it keeps the previous
 *     call's contents (nothing in it needs clearing: every word is written
 *     before it is read).  Calls whose work overlaps on the GPU (different
 *     streams, or different host threads) race on the array and corrupt each
 *     other's results: serialise them, e.g. on one stream.
 * Errors: CCL_ERR_INVALID_ARG (bad arguments or too large), CCL_ERR_CUDA. */
#define CCL_STATIC_SCRATCH_BYTES (64u << 20)
ccl_status ccl_label_static(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                            int connectivity, ccl_stream stream);

/* ------------------------------------------------------------------------ */
/* Component statistics                                                      */
/* ------------------------------------------------------------------------ */

/* Statistics of one component of a canonical label image: the size and
 * location of each region, which the paper's motivating uses need (§I). */
typedef struct {
    int32_t label;        /* 1 + smallest raster index of the component */
    int32_t count;        /* pixels */
    int32_t xmin, ymin;   /* bounding box, inclusive */
    int32_t xmax, ymax;
    int64_t sum_x;        /* sums of the pixels' coordinates: the centroid is */
    int64_t sum_y;        /* (sum_x / count, sum_y / count)                    */
} ccl_component;

/* Bytes of workspace ccl_component_stats needs for a height x width label
 * image and max_comps records: root counts per row segment, the sorted list
 * of component roots (sized for the most components an image can hold) and
 * per-field accumulators for max_comps components.  0 on invalid arguments. */
size_t ccl_stats_workspace_bytes(int height, int width, int max_comps);

/* Statistics of every component of d_labels, a canonical label image as
 * ccl_label writes it (device, height*width int32, read only; any other
 * content gives unspecified statistics but stays in bounds).
 *   d_comps   : device array of max_comps records (max_comps >= 0), written
 *               in increasing label order; components beyond max_comps are
 *               counted but not written
 *   d_ncomps  : device int32, receives the number of components
 *   d_ws      : device workspace of ws_bytes >= ccl_stats_workspace_bytes(),
 *               or NULL (library-owned, as for ccl_label)
 * A component's root is its one pixel whose label is 1 + its own index; the
 * roots are counted per row segment, ranked by a prefix sum, and every tile
 * of 256 x 64 pixels adds its pixels' contributions into the accumulators of
 * their components (shared-memory aggregation, then one atomic update per
 * field, component and tile), packed into the records at the end.  Enqueues
 * seven kernels on `stream`. */
ccl_status ccl_component_stats(const int32_t *d_labels, int height, int width,
                               ccl_component *d_comps, int max_comps, int32_t *d_ncomps,
                               void *d_ws, size_t ws_bytes, ccl_stream stream);

/* Label one image and gather the statistics of every component in the same
 * pass (the size and location of each region, §I): as ccl_label (same
 * labels, arguments and errors), plus
 *   d_comps   : device array of max_comps records (max_comps >= 0; may be NULL
 *               when max_comps == 0).  Record order is unspecified; each holds
 *               its component's label, so sorting by label gives the records
 *               of ccl_component_stats.  When there are more components than
 *               max_comps, max_comps of them (which ones is unspecified) are
 *               written and nothing past the array.
 *   d_ncomps  : device int32, receives the number of components (zeroed by
 *               the call first).
 *   d_ws      : workspace of ws_bytes >= ccl_workspace_bytes_with_stats(), or
 *               NULL (library-owned).
 * Limit beyond ccl_label's: fewer than 2^22 tiles (a tile is 256 x 64 pixels
 * at 8-connectivity and 256 x 32 at 4 for wide images), i.e. every image of
 * at least 512 rows, and narrower ones up to 2^30 pixels wide; larger tile
 * counts return CCL_ERR_INVALID_ARG.
 * The local merge gives every component that stays inside a tile an output
 * record; the link phase adds each segment's count, bounding box and
 * coordinate sums (from its pixels' bits) into a per-tile table, and flushes
 * it once per tile: into the record of a component inside the tile, or into
 * an accumulator of the border root that is a crossing component's global
 * root; a fourth kernel writes those components' records.  Enqueues four
 * kernels and one memset on `stream`. */
ccl_status ccl_label_with_stats(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                                int connectivity, ccl_component *d_comps, int max_comps,
                                int32_t *d_ncomps, void *d_ws, size_t ws_bytes, ccl_stream stream);

/* Workspace bytes of ccl_label_with_stats (the labelling workspace, each
 * segment's component slot and the border-root accumulators), over every tile
 * width; 0 on invalid arguments. */
size_t ccl_workspace_bytes_with_stats(int height, int width, int connectivity);

/* ------------------------------------------------------------------------ */
/* Batched: many images of different sizes in one launch sequence           */
/* ------------------------------------------------------------------------ */

/* One image of a batch: device pointers, caller-owned. */
typedef struct {
    const uint8_t *d_img;
    int32_t *d_labels;
    int height;
    int width;
} ccl_image;

/* Workspace bytes for a batch (descriptor table, tile work list and per-image
 * scratch).  0 on invalid arguments. */
size_t ccl_batched_workspace_bytes(const ccl_image *imgs, int n, int connectivity);

/* Label n images (host array of descriptors; the images themselves are on the
 * device) with one pass of three persistent kernels that pull tiles of all
 * images from a device work queue; each image's tile width comes from the
 * size-class table (ccl_default_tile_width).  The descriptor table is copied
 * to the workspace with one host-to-device copy on `stream`, so `imgs` may be
 * reused as soon as the call returns.  Per-image results equal ccl_label's
 * exactly.  n >= 1; every image obeys the single-image limits. */
ccl_status ccl_label_batched(const ccl_image *imgs, int n, int connectivity, void *d_ws,
                             size_t ws_bytes, ccl_stream stream);

/* ------------------------------------------------------------------------ */
/* Server: continuous batching of host-memory requests                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    size_t hbm_budget_bytes; /* device bytes requests in flight may hold; 0 = 40 GB */
    int max_batch;           /* most images per batched launch; 0 = 256 */
    int max_inflight;        /* batches in flight at once (>= 1); 0 = 2 */
    int connectivity;        /* 4 or 8 */
    int device;              /* CUDA device ordinal */
} ccl_server_config;

typedef struct ccl_server ccl_server;

/* Start a server: worker thread, streams and pinned staging on `device`. */
ccl_status ccl_server_create(const ccl_server_config *cfg, ccl_server **out);

/* Queue one request (non-blocking).  h_img (height*width bytes) and
 * h_labels_out (height*width int32) are HOST buffers owned by the caller that
 * must stay valid until ccl_server_wait/poll reports completion.  A request
 * larger than the whole budget returns CCL_ERR_REJECTED; smaller ones wait
 * until enough budget is free.  Batches take queued requests in FIFO order
 * and may look up to 32 entries past one that does not fit the free budget;
 * a request passed over 8 times is admitted before any request behind it.
 * *req_id_out receives the request id. */
ccl_status ccl_server_submit(ccl_server *srv, const uint8_t *h_img, int height, int width,
                             int32_t *h_labels_out, uint64_t *req_id_out);

/* Block until request `req_id` finished (its labels are in h_labels_out) or
 * timeout_ms passed (CCL_ERR_TIMEOUT; < 0 waits forever).  Returns the
 * request's own status once finished. */
ccl_status ccl_server_wait(ccl_server *srv, uint64_t req_id, int timeout_ms);

/* Non-blocking: CCL_ERR_PENDING while the request is queued or running. */
ccl_status ccl_server_poll(ccl_server *srv, uint64_t req_id);

/* Statistics since creation: latency percentiles in ms (submit -> labels in
 * host memory), Gpixel/s of completed work over the busy interval, counts. */
ccl_status ccl_server_stats(ccl_server *srv, double *p50_ms, double *p99_ms,
                            double *gpix_per_s, uint64_t *completed, uint64_t *rejected);

/* Where a batch's time goes, as means over the batches completed so far:
 * host-to-device copies, the labelling launch and device-to-host copies of
 * one batch, each measured with CUDA events on the batch's stream (batches of
 * different workers overlap, so the three need not add up to the latency).
 * Any output pointer may be NULL. */
ccl_status ccl_server_timing(ccl_server *srv, double *h2d_ms, double *label_ms, double *d2h_ms,
                             uint64_t *batches);

/* Stop accepting, finish every admitted request, release all resources. */
ccl_status ccl_server_destroy(ccl_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* CCL_H */
