/*
 * vg.h -- C ABI of the GB300 voxel-grid library (libvg.so).
 *
 * Implements the method of "GPU Accelerated Voxel Grid Generation for fast
 * MAV Exploration" (Toumieh & Lambert, arXiv 2112.13169): every depth image
 * or dense point cloud becomes a robot-centred local grid of occupied, free
 * and unknown voxels.  Each step runs in a hand-written sm_103a kernel:
 *   K1 transform + voxelize     (Sec. IV-B, Alg. 1, first half)
 *   K2 inflate by vox_inf       (Sec. IV-B, Alg. 1, the three nested loops)
 *   K3 free-space ray-trace     (Sec. IV-C, Alg. 2)
 *   K4 merge into loc_grid      (Sec. IV-D, Alg. 3)
 *   K5 shift (re-centre)        (Sec. IV-E; on the device a move of the
 *                               grid's ring, which K4 and the reads follow)
 * There is no CPU fallback: every call either enqueues device work or fails.
 *
 * Conventions shared by all entry points
 *  - Grid layout (Sec. IV-D): one byte per voxel, idx = x + y*Nx + z*Nx*Ny.
 *    Voxel codes: VG_UNK 0, VG_FREE 1, VG_OCC 2, VG_TRACED 3
 *    ("unknown and traced", Sec. IV-C).  The paper names the states but gives
 *    no numeric codes; these are this library's.
 *  - Frames: the camera optical frame is x right, y down, z forward; a depth
 *    image holds z-depth.  The world and the grid are ENU-aligned (Sec. IV-A).
 *  - T_wc: row-major 4x4 double, camera optical frame -> world (T^w_c of
 *    Table I).  The library composes T^v_c = T^v_w T^w_c on the host in
 *    double and rounds it to float once (Sec. IV-B).  A pose is rejected
 *    (VG_EINVAL) if any entry is not finite, if an entry of its rotation
 *    block lies outside [-1.5, 1.5], or if the camera is 2^22 voxels or
 *    more from the grid's corner voxel.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Calls are asynchronous with respect to the host unless stated; inputs
 *    must stay valid until the enqueued work completes.  Calls on one grid
 *    must be issued from one host thread at a time; work on different grids
 *    may overlap freely.
 *  - Errors: every call returns a status (VG_OK = 0).  Device faults are
 *    asynchronous and surface as VG_ECUDA at a later call.  No call throws,
 *    prints, or exits.
 *  - Numerics: FP32, IEEE round-to-nearest per operation, no FMA
 *    contraction, in the order the oracle states; grids are bit-exact
 *    against the CPU oracle.
 */
#ifndef VG_H
#define VG_H

#include <stdint.h>

#if defined(__GNUC__)
#define VG_API __attribute__((visibility("default")))
#else
#define VG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    VG_OK = 0,
    VG_EINVAL = 1,   /* bad argument: NULL pointer, bad size, non-finite pose ... */
    VG_ENOMEM = 2,   /* device or host allocation failed */
    VG_ECUDA = 3,    /* a CUDA call failed (including an earlier asynchronous fault) */
    VG_ETIMEOUT = 4, /* a bounded device wait ran out */
    VG_EBUSY = 5,    /* resource in use */
    VG_ESCRATCH = 6  /* the request needs more than the library's fixed scratch array */
};

/* Voxel states stored in loc_grid. */
enum { VG_UNK = 0, VG_FREE = 1, VG_OCC = 2, VG_TRACED = 3 };

/* Depth pixel types. */
enum { VG_DEPTH_F32 = 0, VG_DEPTH_U16 = 1 };

/* Where a buffer lives. */
enum { VG_MEM_DEVICE = 0, VG_MEM_HOST = 1 };

/* Grid flags.  The VG_FLAG_LIT_* bits select literal readings of passages
 * the default reading interprets, for comparison with it; each changes
 * results, none is the paper's intent as this library reads it:
 *  VG_FLAG_LIT_INFLATE_AFTER_TRACE
 *      rays test the occupancy before inflation (trace, then inflate: the
 *      order in which the kernel list names the steps); inflated voxels
 *      are still marked occupied.  Default: Alg. 1 inflates first and rays
 *      stop at inflated voxels.
 *  VG_FLAG_LIT_SKIP_START_VOXEL
 *      Alg. 2 moves by a voxel before its first test, so no ray visits the
 *      camera's voxel.  Default: the start voxel is visited.
 *  VG_FLAG_LIT_LOC_OCCUPANCY
 *      Alg. 2 tests loc_grid (the grid before this measurement, after any
 *      pending re-centre) for occupied voxels, and the rays' free/traced
 *      marks replace this measurement's occupied marks: precedence free >
 *      traced > occupied > unknown.  Default: rays test the measurement's
 *      inflated occupancy and occupied wins.  Costs one more bit plane.
 * INFLATE_AFTER_TRACE and LOC_OCCUPANCY exclude each other.  Grids with a
 * LIT flag take the plain path only (not batches, not the server). */
enum {
    VG_FLAG_STATS = 1u << 0,                    /* count in-grid points and ray-voxel visits (vg_stats) */
    VG_FLAG_LIT_INFLATE_AFTER_TRACE = 1u << 1,
    VG_FLAG_LIT_SKIP_START_VOXEL = 1u << 2,
    VG_FLAG_LIT_LOC_OCCUPANCY = 1u << 3
};

/*
 * Table I parameters of one local grid.
 *  grid_size  voxels per axis (x, y, z), each >= 1, total < 2^31, and fewer
 *             than 2^27 plane words (WX * Ny * Nz, WX = ceil(Nx/32) rounded up
 *             to a power of two, at least 4; only Nx far below 32 nears it).  The paper
 *             gives sizes in metres (Sec. V); callers convert with
 *             round(m / vox_size).
 *  vox_size   voxel edge in metres, finite, > 0.
 *  fov_x_deg, fov_y_deg
 *             camera field of view in degrees, in (0, 180).
 *  depth      range in metres to clear by ray-tracing (Sec. IV-C) and the
 *             largest depth accepted from a depth image; finite, > 0.
 *  vox_inf    inflation radius in voxels (Sec. IV-B), 0 <= vox_inf <= 15.
 *  flags      VG_FLAG_* bits.
 */
typedef struct {
    int32_t grid_size[3];
    float vox_size;
    float fov_x_deg;
    float fov_y_deg;
    float depth;
    int32_t vox_inf;
    uint32_t flags;
} vg_params;

typedef struct vg_grid vg_grid;

/* Counters accumulated since creation when VG_FLAG_STATS is set. */
typedef struct {
    uint64_t frames;          /* vg_integrate_* calls */
    uint64_t points_in_grid;  /* valid points that landed inside the grid (K1) */
    uint64_t ray_visits;      /* in-grid voxel visits over all rays (K3) */
    uint64_t wait_timeouts;   /* device waits for a tile copy (K2) that ran out on the grid's
                                 device since the library was loaded, any grid; the tile was
                                 left unwritten (counted with or without VG_FLAG_STATS) */
} vg_stats_t;

/*
 * Voxel grid set-up (Sec. IV-A).  Allocates loc_grid and the measurement
 * planes on the current device (one allocation, owned by the grid) and sets
 * every voxel to VG_UNK.  The origin is placed so that the robot at
 * robot_pos_w (world metres) sits in voxel floor(N/2) of every axis:
 * origin_k = floor(p_k / vox_size) - floor(N_k / 2), computed in double.
 * Synchronises `stream` once before returning.
 * Errors: VG_EINVAL (NULL, out-of-range parameter, robot_pos_w not finite or
 * |robot_pos_w| / vox_size >= 2^30 on an axis), VG_ENOMEM, VG_ECUDA.
 */
VG_API int vg_create(const vg_params *params, const double robot_pos_w[3], void *stream,
              vg_grid **out);

/* Frees the grid (synchronises the device first).  NULL is accepted.  The
 * paper has no counterpart (its grids live for the whole run); this is the
 * library's resource convention. */
VG_API void vg_destroy(vg_grid *grid);

/*
 * One measurement from a depth image (Sec. IV, steps 2-4): K1 voxelizes the
 * valid pixels, K2 inflates, K3 traces the ray bundle of Sec. IV-C, K4
 * merges the measurement into loc_grid (Alg. 3).
 *  depth        W x H pixels, row-major, tightly packed.  dtype VG_DEPTH_F32
 *               (metres) or VG_DEPTH_U16 (metres = raw * depth_scale).
 *  mem          VG_MEM_DEVICE: depth is a device pointer, read in place.
 *               VG_MEM_HOST: depth is host memory.  Page-locked memory
 *               (cudaMallocHost, cudaHostAlloc, cudaHostRegister) is read in
 *               place by K1 over the host link and must stay valid until
 *               the work on stream completes; other host memory is copied
 *               with cudaMemcpyAsync into a staging buffer the grid owns
 *               (grown on first use of a larger frame).
 *  depth_scale  used for VG_DEPTH_U16 only; finite, > 0.
 *  T_wc         camera pose, see above; must be finite.
 * A pixel is valid iff its depth d is finite, > 0 and <= params.depth.  The
 * pinhole model takes fx = (W/2)/tan(fov_x/2), cx = (W-1)/2 (y likewise).
 * Errors: VG_EINVAL, VG_ENOMEM (staging), VG_ECUDA.
 */
VG_API int vg_integrate_depth(vg_grid *grid, const void *depth, int32_t mem, int32_t width,
                       int32_t height, int32_t dtype, float depth_scale,
                       const double T_wc[16], void *stream);

/*
 * One measurement from a dense point cloud (Sec. IV): n points, xyz float
 * triples in the camera optical frame, packed.  A point is valid iff its
 * three coordinates are finite (no range filter).  mem as above.
 * Errors: VG_EINVAL, VG_ENOMEM (staging), VG_ECUDA.
 */
VG_API int vg_integrate_points(vg_grid *grid, const float *xyz, int32_t mem, int64_t n,
                        const double T_wc[16], void *stream);

/*
 * Re-centre the grid on the robot (Sec. IV-E): the new origin o' is computed
 * as in vg_create; with delta = o' - o, loc'[i] = loc[i + delta] where that
 * voxel exists, else VG_UNK.  The origin changes at once (vg_get_origin).
 * The grid is kept ring-addressed on the device, so no byte moves: the
 * re-centre moves the ring, and the voxels it brings in (those whose
 * loc[i + delta] does not exist) are set to VG_UNK by the grid's next merge
 * (vg_integrate_*, or a batch step); vg_read returns them as VG_UNK
 * meanwhile, and another vg_shift first clears them on its own stream.
 * No device work here unless a re-centre was already pending.
 * Errors: VG_EINVAL (also: |robot_pos_w| / vox_size >= 2^30 on an axis),
 * VG_ECUDA.
 */
VG_API int vg_shift(vg_grid *grid, const double robot_pos_w[3], void *stream);

/*
 * The paper has no counterpart: its planner reads loc_grid in place (Sec.
 * IV, Fig. 1); a library whose grids live on the device hands them out with
 * a copy.
 * Copy loc_grid (Nx*Ny*Nz bytes, layout above) to dst, enqueued on stream;
 * dst is valid once that work completes.  dst_mem is VG_MEM_DEVICE or
 * VG_MEM_HOST; dst_bytes must be >= Nx*Ny*Nz.  origin (may be NULL)
 * receives the grid origin (voxel index of voxel (0,0,0) in the world
 * lattice) as of this call, in the layout above, re-centres included.  Once
 * the grid has been re-centred, K5 reads it out of the device's ring
 * addressing on stream, straight into dst when dst is device memory or
 * page-locked host memory and 16-byte aligned, else through the grid's
 * second buffer and a copy; before that, a plain copy.  The grid's own
 * state does not change.
 * Errors: VG_EINVAL, VG_ECUDA.
 */
VG_API int vg_read(vg_grid *grid, uint8_t *dst, int32_t dst_mem, int64_t dst_bytes,
            int32_t origin[3], void *stream);

/*
 * The paper has no counterpart (no checkpointing); this is the library's
 * resume path, and the way to restore a grid after a failed batch step.
 * Restore loc_grid and its origin (checkpoint / resume): src holds
 * Nx*Ny*Nz bytes of voxel codes 0..3 (not checked), src_bytes must equal
 * Nx*Ny*Nz.  A pending re-centre is dropped and the measurement planes are
 * emptied.  Errors: VG_EINVAL, VG_ECUDA.
 */
VG_API int vg_write(vg_grid *grid, const uint8_t *src, int32_t src_mem, int64_t src_bytes,
             const int32_t origin[3], void *stream);

/* Current origin (host-side state; no device work): the voxel index of
 * voxel (0,0,0) in the world lattice, as Sec. IV-A places it. */
VG_API int vg_get_origin(const vg_grid *grid, int32_t origin[3]);

/* Device bytes one grid with these parameters holds (0 if invalid). */
VG_API int64_t vg_grid_bytes(const vg_params *params);

/* Ray bundle of Sec. IV-C: out = {vox_depth, hw, hh}; vox_width = 2hw+1,
 * vox_height = 2hh+1; returns the ray count (0 if invalid). */
VG_API int64_t vg_ray_bundle(const vg_params *params, int32_t out[3]);

/* Counters (VG_FLAG_STATS); synchronises the device. */
VG_API int vg_stats(vg_grid *grid, vg_stats_t *out);

/*
 * Batched form: many measurements, each into its own grid, in one
 * persistent fused launch (the paper processes one frame at a time).  A batch owns a device descriptor table of `capacity` frames and a
 * pinned host copy of it.
 *
 * One frame of a batch: what vg_integrate_depth takes, plus an optional
 * re-centre (vg_shift) after the merge.  depth must be device memory.
 */
typedef struct {
    vg_grid *grid;          /* the frame's grid; at most one frame per grid in a batch */
    const void *depth;      /* device pointer, W x H row-major */
    int32_t width, height;
    int32_t dtype;          /* VG_DEPTH_F32 or VG_DEPTH_U16 */
    float depth_scale;      /* VG_DEPTH_U16 only */
    double T_wc[16];        /* camera pose, as for vg_integrate_depth */
    int32_t recentre;       /* nonzero: re-centre on robot_pos_w after the merge */
    int32_t pad;
    double robot_pos_w[3];
} vg_frame;

typedef struct vg_batch vg_batch;

/*
 * Creates a batch for up to `capacity` frames (1 .. 65536) on the current
 * device: one device allocation and one pinned host allocation.
 * Errors: VG_EINVAL, VG_ENOMEM, VG_ECUDA.
 */
VG_API int vg_batch_create(int32_t capacity, vg_batch **out);

/* Frees the batch (synchronises the device first).  NULL is accepted. */
VG_API void vg_batch_destroy(vg_batch *batch);

/*
 * Host-only half of a step: validates the n frames and writes their
 * descriptors into the batch's pinned table, and applies the grids'
 * host-side state changes: a grid's pending re-centre is taken into this
 * step's merge, and a frame's own re-centre moves its grid's origin and
 * ring and is left pending, as vg_shift leaves it.  Waits for the previous step's table copy, so the table can be
 * rewritten.  Grids must have vox_inf <= 3 and live on the batch's device.
 * Errors: VG_EINVAL (bad frame, two frames for one grid, n > capacity),
 * VG_ECUDA.
 */
VG_API int vg_batch_prepare(vg_batch *batch, const vg_frame *frames, int32_t n);

/*
 * Device half of a step: copies the table to the device and launches the
 * fused kernel on `stream` (cooperative launch: K1, K2, K3 and K4 of
 * every prepared frame, each grid's merge clearing what a pending re-centre
 * brought in,
 * with a grid-wide barrier between phases).  Can be captured in a CUDA graph; replaying the graph runs
 * whatever vg_batch_prepare wrote last.  Errors: VG_EINVAL, VG_ECUDA.
 */
VG_API int vg_batch_enqueue(vg_batch *batch, void *stream);

/* vg_batch_prepare followed by vg_batch_enqueue. */
VG_API int vg_batch_step(vg_batch *batch, const vg_frame *frames, int32_t n, void *stream);

/*
 * Waits for the last enqueued step and reports how it ended: VG_OK, or
 * VG_ETIMEOUT if a grid barrier gave up waiting (the step's grids are then
 * incomplete), or VG_ECUDA.
 */
VG_API int vg_batch_status(vg_batch *batch);

/*
 * Batch knobs:
 *  VG_TUNE_BATCH_CTAS_PER_SM  CTAs per SM of the fused launch, 1 .. the
 *                             occupancy limit, or 0 for the limit (default).
 *  VG_TUNE_BATCH_LANES        lanes per ray for every frame: 8, 16 or 32, or
 *                             0 to use each grid's own setting (default).
 *  VG_TUNE_BATCH_INFLATE_SLICES
 *                             slices of an inflate tile (phase 2): 8 (the
 *                             default; 0 selects it) or 4.
 *  VG_TUNE_BATCH_MERGE_WORDS  plane words per merge unit (phase 4): 512 (the
 *                             default; 0 selects it) or 256.
 *  VG_TUNE_BATCH_SPREAD       how phase 3 (the ray trace) shares its units,
 *                             groups of 256 / LPR rays, among the CTAs' contiguous
 *                             runs.  1 (default): each frame's rays are
 *                             spread over proportionally more units, so that
 *                             the runs hold equal numbers of units.  2: one
 *                             unit per group; the runs split the units' total
 *                             estimated cost evenly (each frame's unit cost
 *                             from 25 of its rays' lengths in the grid), which
 *                             suits batches of frames of unlike cost.  0: one
 *                             unit per group, equal numbers of units.
 *  VG_TUNE_BATCH_BARRIER_US   how long a CTA of the fused launch waits at a
 *                             grid barrier before it gives up, in
 *                             microseconds, 1 .. 60,000,000, or 0 for the
 *                             default (4 s).  A step whose wait ran out
 *                             ends early; vg_batch_status reports
 *                             VG_ETIMEOUT.
 *  VG_TUNE_BATCH_BARRIER_EXTRA
 *                             0 (default) or 1.  With 1 every grid barrier
 *                             waits for one more arrival than the launch has
 *                             CTAs, so every wait runs out after the limit
 *                             above: a fault injection that tests the
 *                             time-out path without hanging the device.
 * Results do not depend on any knob but the last.  After VG_ETIMEOUT the step's
 * grids hold a partial measurement: restore each with vg_write (which also
 * empties its measurement planes) or destroy it.  Errors: VG_EINVAL.
 */
enum {
    VG_TUNE_BATCH_CTAS_PER_SM = 100,
    VG_TUNE_BATCH_LANES = 101,
    VG_TUNE_BATCH_BARRIER_US = 102,
    VG_TUNE_BATCH_BARRIER_EXTRA = 103,
    VG_TUNE_BATCH_INFLATE_SLICES = 104,
    VG_TUNE_BATCH_MERGE_WORDS = 105,
    VG_TUNE_BATCH_SPREAD = 106
};
VG_API int vg_batch_tune(vg_batch *batch, int32_t knob, int32_t value);

/*
 * Autotuner of the batch's schedule: times `reps` steps of the given frames
 * (re-centring switched off, so every timed step merges the same
 * measurements into the grids, which leaves them as one step would) for
 * each candidate value of one schedule knob at a time -- CTAs per SM (1 ..
 * the occupancy limit), lanes per ray (per grid, 8, 16, 32), inflate tile
 * slices (8, 4), merge words per unit (512, 256), phase-3 spread (2, 1, 0)
 * -- with the other knobs at the best values found so far (coordinate
 * descent), keeps the fastest setting in the batch and writes it to best[5]
 * = {ctas_per_sm, lanes, inflate_slices, merge_words, spread} (may be NULL).
 * Synchronises the device.  Errors: as vg_batch_step, VG_ETIMEOUT.
 */
VG_API int vg_batch_autotune(vg_batch *batch, const vg_frame *frames, int32_t n, int32_t reps,
                             void *stream, int32_t best[5]);

/*
 * Served form: a request loop for many cameras with continuous batching.
 * A server owns one grid per admitted camera (all resident on the device)
 * and a device pool for submitted frames.  A server thread forms batches from the queued
 * requests -- oldest first, at most one frame per camera per launch, so the
 * frames of one camera apply in submission order -- and issues each batch
 * in one of two ways.  A batch of at most plain_max frames runs each frame
 * as the per-frame kernel chain of vg_integrate_depth on one of several
 * streams (a camera always on the same one), so the frames of different
 * cameras overlap on the device.  A larger batch runs as one fused launch
 * (as vg_batch_step); fused launches are ordered after all earlier work of
 * the server and before all later work.  Both read the frames from the
 * pool.  Requests that arrive while launches are on the GPU join the next
 * launch as soon as a launch slot frees up.  While launches are in flight
 * the server thread polls their completion events (it keeps one CPU core
 * busy meanwhile) and stamps each frame's completion as it is seen.  Every
 * entry point is thread-safe.
 *
 *  memory_budget  bytes of device memory the server may hold: its frame
 *                 pool (pending_frames frames of max_width x max_height x 4
 *                 bytes, each rounded up to 256) and launch tables plus the
 *                 grids of the cameras it admits.
 *  max_batch      frames per launch (1 .. 4096).
 *  max_width, max_height
 *                 the largest depth frame a camera may submit.
 *  queue_depth    launches on the GPU at once (1 .. 8); 2 or more overlap
 *                 a launch with the next one's kernels.
 *  pending_frames submitted frames the pool holds (queued or in flight)
 *                 before vg_server_submit reports VG_EBUSY.
 *  plain_max      the largest batch issued as per-frame kernel chains
 *                 (0 .. 4096; 0 selects the default, 4); larger batches
 *                 run as one fused launch.  Results do not depend on it.
 */
typedef struct {
    int64_t memory_budget;
    int32_t max_batch;
    int32_t max_width, max_height;
    int32_t queue_depth;
    int32_t pending_frames;
    int32_t plain_max;
} vg_server_params;

typedef struct {
    uint64_t submitted, completed, failed, batches;
    double mean_batch;        /* frames per launch */
    double latency_p50_us;    /* submission to the moment the frame's device work is seen to end */
    double latency_p99_us;
    double latency_max_us;
    int64_t bytes_in_use;     /* device bytes held (frame pool, tables, grids) */
    int32_t cameras;
} vg_server_stats_t;

typedef struct vg_server vg_server;

/* Creates the server on the current device and starts its thread.
 * Errors: VG_EINVAL, VG_ENOMEM (budget below the server's own needs or an
 * allocation failed), VG_ECUDA. */
VG_API int vg_server_create(const vg_server_params *params, vg_server **out);

/* Finishes every queued frame, stops the thread and frees everything. */
VG_API void vg_server_destroy(vg_server *server);

/* Admits a camera with its own grid (see vg_create) if the memory budget
 * allows; *camera receives its id.  Errors: VG_EINVAL, VG_ENOMEM (over
 * budget or out of memory), VG_ECUDA. */
VG_API int vg_server_add_camera(vg_server *server, const vg_params *params, const double robot_pos_w[3],
                                int32_t *camera);

/* Waits for the camera's queued frames, then frees its grid and returns its
 * memory to the budget.  Errors: VG_EINVAL. */
VG_API int vg_server_remove_camera(vg_server *server, int32_t camera);

/*
 * Queues one frame of a camera: depth is host memory, pageable or
 * page-locked (W x H, dtype as for vg_integrate_depth).  It is copied into
 * the server's device pool, and that copy has ended when the call returns,
 * so the caller may reuse the buffer at once.  recentre != 0 re-centres the grid on robot_pos_w after the
 * merge.  *ticket (may be NULL) identifies the request.
 * Errors: VG_EINVAL (bad argument, frame larger than max_width x max_height,
 * unknown or removed camera), VG_EBUSY (the pool is full: retry later),
 * VG_ECUDA (the copy failed; nothing was queued).
 */
VG_API int vg_server_submit(vg_server *server, int32_t camera, const void *depth, int32_t width,
                            int32_t height, int32_t dtype, float depth_scale, const double T_wc[16],
                            int32_t recentre, const double robot_pos_w[3], uint64_t *ticket);

/* Waits up to timeout_us microseconds (negative: no limit) for a request.
 * Returns VG_OK when its frame's device work completed, VG_ETIMEOUT if still
 * pending, VG_ECUDA or VG_EINVAL if it failed or is unknown.  A ticket's
 * status stays queryable for the server's lifetime (one byte per ticket;
 * the latencies behind vg_server_stats are kept until a reset). */
VG_API int vg_server_wait(vg_server *server, uint64_t ticket, int64_t timeout_us);

/* When a request was submitted (the entry of vg_server_submit) and when its
 * frame's device work was seen to end, in seconds of the host's monotonic
 * clock (CLOCK_MONOTONIC on Linux, the clock of std::chrono::steady_clock),
 * so that a caller can measure latency from its own arrival times.  Either
 * pointer may be NULL.  Returns VG_OK once completed (both written),
 * VG_ETIMEOUT while pending (only submitted_s written), VG_ECUDA if the
 * frame failed, VG_EINVAL for an unknown ticket.  Kept for the server's
 * lifetime (16 bytes per ticket). */
VG_API int vg_server_ticket_times(vg_server *server, uint64_t ticket, double *submitted_s, double *completed_s);

/* Waits for every queued frame of the camera, then copies its grid to dst
 * (as vg_read) and synchronises.  Errors: VG_EINVAL, VG_ECUDA. */
VG_API int vg_server_read(vg_server *server, int32_t camera, uint8_t *dst, int32_t dst_mem, int64_t dst_bytes,
                          int32_t origin[3]);

/* Counters and latency percentiles since creation or the last reset. */
VG_API int vg_server_stats(vg_server *server, vg_server_stats_t *out, int32_t reset);

/* Kernels of one measurement, for profiling and launch counts. */
enum {
    VG_K_VOXELIZE = 0, /* K1 */
    VG_K_INFLATE = 1,  /* K2 */
    VG_K_RAYTRACE = 2, /* K3 */
    VG_K_MERGE = 3,    /* K4 */
    VG_K_SHIFT = 4,    /* K5 */
    VG_K_LOC_OCCUPANCY = 5, /* loc_grid's occupied voxels as a bit plane (VG_FLAG_LIT_LOC_OCCUPANCY) */
    VG_NKERNELS = 6
};

/*
 * Per-kernel timing.  While enabled, every kernel launch of this grid is
 * bracketed by two CUDA events recorded on the launch's own stream (up to
 * 65536 launches are kept; later ones are counted but not timed).
 * vg_profile_read synchronises the device, writes the summed event time in
 * milliseconds and the number of timed launches per kernel, and (if reset)
 * forgets them.  launches_total (may be NULL) receives the number of kernel
 * launches this grid has issued since creation, timed or not.
 * Errors: VG_EINVAL, VG_ENOMEM (event pool), VG_ECUDA.
 */
VG_API int vg_profile_enable(vg_grid *grid, int32_t enable);
VG_API int vg_profile_read(vg_grid *grid, double ms[VG_NKERNELS], int64_t timed[VG_NKERNELS],
                           int64_t launches_total[VG_NKERNELS], int32_t reset);

/*
 * Tuning knobs (defaults are set by vg_create):
 *  VG_TUNE_RT_LANES  lanes of a warp that share one ray in K3: 1, 2, 4, 8,
 *                    16 or 32, or 0 for automatic (the default: the fewest
 *                    lanes, at least 8, whose share of the longest ray is
 *                    at most 1.5 times the per-lane buffer of runs of
 *                    visits).  Results do not depend on it.
 *  VG_TUNE_INFLATE_TILE
 *                    K2's tile of plane words: VG_TILE_AUTO (the default:
 *                    8 words x 8 rows x 8 slices, 4 slices when the grid has
 *                    one to four 8-slice tiles per SM, 4 words for rows of 4
 *                    words), or VG_TILE_4x8x4, _4x8x8, _8x8x4, _8x8x8
 *                    (words x rows x slices; 8-word tiles fall back to 4 on
 *                    rows of 4 words).
 *  VG_TUNE_RT_CTAS_PER_SM
 *                    K3's CTAs per SM, 1 .. the occupancy limit (5), or 0
 *                    for the limit (default).
 *  VG_TUNE_MERGE_WORDS
 *                    plane words per CTA of K4: 256 (default, one per
 *                    thread) or 512 (two per thread).
 *  VG_TUNE_INFLATE_TMA
 *                    1 (default): K2 moves each tile's raw words with one
 *                    tensor-memory-accelerator copy (radius 1..3); 0: its
 *                    threads load them.
 *  VG_TUNE_EARLY_INFLATE
 *                    1 (default): K2's CTAs launch while K1 runs, as soon
 *                    as K1 has waited for the work before the frame; 0:
 *                    they launch when K1 completes, which leaves K1's SM
 *                    slots to K3's CTAs (their walk runs before they wait
 *                    for K2).
 * Results do not depend on any of them.  Errors: VG_EINVAL.
 */
enum {
    VG_TUNE_RT_LANES = 0,
    VG_TUNE_INFLATE_TILE = 1,
    VG_TUNE_RT_CTAS_PER_SM = 2,
    VG_TUNE_MERGE_WORDS = 3,
    VG_TUNE_INFLATE_TMA = 4,
    VG_TUNE_EARLY_INFLATE = 5
};
enum { VG_TILE_AUTO = 0, VG_TILE_4x8x4 = 1, VG_TILE_4x8x8 = 2, VG_TILE_8x8x4 = 3, VG_TILE_8x8x8 = 4 };
VG_API int vg_tune(vg_grid *grid, int32_t knob, int32_t value);

/*
 * Autotuner of the per-frame kernels' schedule.  Starting from the grid's
 * schedule as it stands, it takes one knob at a time -- K2's tile (the four
 * shapes), K3's lanes per ray (8, 16, 32), K3's CTAs per SM (1..5), K4's
 * words per CTA (256, 512), K2's staging (tensor copies or threads) and
 * K2's launch (while K1 runs or after it) --
 * and compares each candidate value with the best schedule so far: `reps`
 * (1 .. 1000) measurements of the given depth frame (arguments as for
 * vg_integrate_depth) under each, alternating and each in turn first,
 * every one starting with a
 * cold L2 (a write of twice the L2's size to a scratch buffer the call
 * allocates and frees); the candidate wins only if its median CUDA event
 * time is at least 2 % below the incumbent's.  Keeps the winning schedule in the grid and writes
 * it to best[6] = {tile, lanes, ctas_per_sm, merge_words, inflate_tma,
 * early_inflate}
 * (tile VG_TILE_AUTO and ctas_per_sm 0 where the defaults won; may be
 * NULL).  Each timed measurement merges the frame over
 * a re-centre by zero, so K4 runs the re-centring merge that a moving
 * robot's frames take; merging the same measurement again leaves the grid
 * as one merge leaves it.  A re-centre pending at the call is applied
 * first.  Synchronises the stream.
 * Errors: as vg_integrate_depth; VG_ENOMEM for the scratch buffer.
 */
VG_API int vg_autotune(vg_grid *grid, const void *depth, int32_t mem, int32_t width, int32_t height,
                       int32_t dtype, float depth_scale, const double T_wc[16], int32_t reps, void *stream,
                       int32_t best[6]);

/*
 * One measurement without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code that must never block in the driver's allocator (a
 * real-time control loop), integrations that hand out all device memory
 * themselves, or processes whose allocator belongs to another runtime.
 *
 * It does what vg_integrate_depth does (K1 voxelize, K2 inflate, K3
 * ray-trace, K4 merge) for a grid the caller owns, without a vg_grid:
 *  params     grid parameters, as for vg_create (flags are ignored).
 *  origin     the grid's origin (voxel index of voxel (0,0,0) in the world
 *             lattice), e.g. as vg_read reports it; the caller keeps it.
 *  loc        the caller's loc_grid in device memory of the current
 *             device, Nx*Ny*Nz bytes in the layout above, read and updated
 *             in place; 16-byte aligned.
 *  depth      W x H pixels as for vg_integrate_depth: device memory of the
 *             current device, or page-locked host memory, which K1 reads
 *             in place.
 *  width, height, dtype, depth_scale, T_wc, stream
 *             as for vg_integrate_depth.
 * The kernels run on the current device.  A loc or depth that it cannot
 * reach (another device's memory, pageable host memory, a pointer CUDA
 * does not know) is refused with VG_EINVAL before any device work.
 * The four measurement bit planes live in one array of 16 MiB compiled into
 * the library (every GPU that loads the library holds it until the process
 * exits).  A grid whose plane needs more than 2^20 32-bit words
 * (ceil(Nx/32) rounded up to a power of two, at least 4, times Ny*Nz) is
 * refused with VG_ESCRATCH before any device work.  No cudaMalloc,
 * cudaFree or other allocating call is made.
 * The first call on a device does a one-time set-up there (it looks up the
 * array's device address and configures the kernels); make that first call
 * before any stream capture.  Every call shares the array and clears the
 * part it uses on its stream before using it, so calls whose device work
 * overlaps -- on different streams or from different host threads -- race
 * and corrupt each other's results; serialise them.
 * Errors: VG_EINVAL (NULL, bad size or pose, unaligned loc), VG_ESCRATCH,
 * VG_ECUDA.
 */
VG_API int vg_integrate_depth_noalloc(const vg_params *params, const int32_t origin[3],
                                      uint8_t *loc, const void *depth, int32_t width,
                                      int32_t height, int32_t dtype, float depth_scale,
                                      const double T_wc[16], void *stream);

/* Static description of a status code (a library convention; the paper
 * defines no error handling). */
VG_API const char *vg_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
