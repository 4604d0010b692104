// vg_internal.cuh -- types shared by the kernels and the host library.
//
// Device data layout of one grid (one cudaMalloc, carved in this order):
//   loc      Nx*Ny*Nz bytes, the paper's index order idx = x + y*Nx + z*Nx*Ny,
//            followed by at least 16 bytes of slack
//   loc_alt  the same size; target of the out-of-place shift (ping-pong)
//   occ_raw, occ_inf, fr, tr
//            bit planes of the measurement grid.  Bit b of word
//            (z*Ny + y)*WX + w is voxel x = 32*w + b of row (y, z), i.e.
//            plane bit (z*Ny + y)*32*WX + x.  WX is ceil(Nx/32) rounded up
//            to a power of two, at least 4 words, so every row starts on a
//            16-byte boundary.  Bits with x >= Nx stay 0.
//   stats    three u64 counters (VG_FLAG_STATS)
// The planes are all-zero between frames: K4 clears every word it reads.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace vg {

// Programmatic dependent launch (sm_90 and later).  The one-step kernels
// are launched with programmatic stream serialization allowed, so a kernel
// may start while the kernel before it in the stream still runs.  Each lets
// its successor launch at once (pdl_trigger) and, before it touches any
// memory that earlier work in the stream writes or reads, waits until its
// predecessor has completed and that kernel's writes are visible (pdl_wait).
// Every such kernel waits in every CTA before it ends, so its completion
// implies its predecessor's, and by induction all earlier work's.  Without
// a programmatic predecessor both are no-ops.  K1, the first kernel of a
// frame, triggers only after its own wait (or not at all): the frame's
// later kernels then launch only once all work before the frame has
// completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... P, class... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

constexpr int kMaxInflate = 15;
// Entries (runs of in-grid visits) a K3 lane keeps in shared memory.  36
// entries (36 KB per 256-thread CTA plus 6 KB of box) let five CTAs share an
// SM.  A packed run needs plane bit indices below 2^26, i.e. plane words
// below kRunWords; larger grids walk each slice twice instead.
constexpr int kRtBuf = 36;
constexpr int64_t kRunWords = int64_t(1) << 21;

struct PlaneGeom {
    int32_t nx, ny, nz;
    int32_t wx;        // words per row
    int64_t words;     // wx * ny * nz
    int64_t nvox;      // nx * ny * nz
};

// T^v_c rounded to float: R row-major, t in metres.
struct Pose32 {
    float R[9];
    float t[3];
};

struct Planes {
    uint32_t *occ_raw;
    uint32_t *occ_inf;
    uint32_t *fr;
    uint32_t *tr;
};

// Ring addressing of loc_grid.  Voxel (x, y, z) of the grid in its current
// frame (origin o) is byte (z' * ny + y') * nx + x' of the buffer, with
// x' = (x + r[0]) mod nx, y' = (y + r[1]) mod ny, z' = (z + r[2]) mod nz.
// A re-centre by d (Sec. IV-E) moves r by d instead of moving the bytes;
// the voxels it brings in (x in [elo[0], ehi[0]) or y in [elo[1], ehi[1])
// or z in [elo[2], ehi[2]): those whose x + d (or y, z) lay outside the old
// grid) still hold stale bytes, which the next K4 (or a read) turns into
// unknown.  All zero: the buffer is the grid itself.
struct Ring {
    int32_t r[3];
    int32_t elo[3], ehi[3];
};

struct FrameArgs {
    PlaneGeom g;
    Pose32 T;
    float vs;          // vox_size
    float depth_max;   // params.depth
    // depth image input
    const void *depth;
    int32_t W, H;
    float scale;       // u16 -> metres
    float fx, fy, cx, cy;
    // point cloud input
    const float *xyz;
    int64_t npts;
    // ray bundle
    int32_t vd, hw, hh;
    int32_t r;         // vox_inf
    Planes pl;
    uint8_t *loc;
    Ring ring;                  // loc's ring addressing, with the voxels a re-centre brought in
    unsigned long long *stats;  // NULL unless VG_FLAG_STATS
    uint32_t *rt_next;          // K3's counter of handed-out bundles, zeroed by K1; NULL: static only
    // literal readings (comparison flags; 0 for the default reading)
    const uint32_t *occ_test;   // the plane K3's rays test; NULL: pl.occ_inf
    int32_t lit;                // kLit* bits
};

constexpr int32_t kLitSkipStart = 1;    // rays do not visit their start voxel
constexpr int32_t kLitRaysLast = 2;     // resolve: free > traced > occupied

// One frame of a batch (k_batch.cu): its FrameArgs plus the layout of its
// units in each phase.
struct BatchItem {
    FrameArgs a;
    int64_t off[4];     // first unit of this frame in phases 1..4
    int32_t tiles[3];   // inflate tile grid (x words / txw, y / 8, z / 8)
    int32_t dtype;      // 0 f32, 1 u16
    int32_t vec;        // depth base aligned for 4-pixel loads
    int32_t lpr;        // K3 lanes per ray: 8, 16 or 32
    int32_t txw;        // inflate tile width in words: 4 or 8
    int32_t tz;         // inflate tile height in slices: 4 or 8
    int32_t mwpu;       // plane words per phase-4 unit: 256 or 512
    int32_t buffered;   // packed runs fit (plane words < kRunWords)
    int64_t woff3;      // phase 3: weight of the units before this frame's
    int64_t w3;         // phase 3: weight of each of this frame's units
};

// Plane words per phase-4 unit of a batch frame whose merge applies a
// pending re-centre, unless tuned (other frames' units are 256 words, one
// per thread).
constexpr int kBatchMergeWords = 512;

// Control block of a batch launch, copied to the device with the items.
struct BatchCtl {
    int32_t n;          // frames
    int32_t pad0;
    int64_t total[4];   // units per phase
    unsigned bar_count; // grid barrier: arrivals
    unsigned bar_gen;   // grid barrier: generation
    unsigned error;     // set when a barrier wait ran out
    unsigned bar_extra; // arrivals a barrier waits for beyond the launch's CTAs (0; 1 only to test the time limit)
    int64_t bar_ns;     // how long a CTA waits at a grid barrier before giving up (globaltimer ns)
    int64_t wtotal3;    // phase 3: the units' total weight, split evenly over the CTAs
};

// Default of BatchCtl::bar_ns: four seconds (a phase of any batch that fits
// the device ends far sooner).
constexpr int64_t kBarrierNs = 4000000000LL;

inline __host__ __device__ int64_t plane_word(const PlaneGeom &g, int32_t x, int32_t y, int32_t z) {
    return ((int64_t)z * g.ny + y) * g.wx + (x >> 5);
}

// Schedule of the one-step kernels: tile shapes and launch shapes, none of
// which changes a result (set with vg_tune, chosen by vg_autotune).
enum {
    kTileAuto = 0,   // K2 picks its tile from the grid's size
    kTile4x8x4 = 1,  // K2 tile: words x rows x slices
    kTile4x8x8 = 2,
    kTile8x8x4 = 3,
    kTile8x8x8 = 4
};
struct Sched {
    int32_t inflate_tile = kTileAuto;
    int32_t rt_ctas = 0;        // K3 CTAs per SM; 0: as many as fit
    int32_t merge_words = 256;  // plane words per CTA of K4: 256 (one per thread) or 512 (two)
    int32_t inflate_tma = 1;    // K2 stages its tiles with tensor-memory-accelerator copies (radius 1..3)
    int32_t early_inflate = 1;  // K2 launches while K1 runs (else when K1 completes)
};

// Kernel launchers (one translation unit each).
cudaError_t launch_voxelize_depth(const FrameArgs &a, int32_t dtype, cudaStream_t s, const Sched &sc = Sched());
cudaError_t launch_voxelize_points(const FrameArgs &a, cudaStream_t s, const Sched &sc = Sched());
cudaError_t configure_inflate();   // once per device, before the first launch_inflate
// device waits of K2 that ran out on the current device since the library was loaded
cudaError_t wait_timeouts(unsigned *out);
cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s, const Sched &sc = Sched());
cudaError_t configure_raytrace(int dev);   // once per device, before the first launch_raytrace
int auto_lanes_per_ray(int32_t vd, int32_t hw, int32_t hh);
cudaError_t launch_raytrace(const FrameArgs &a, int lanes_per_ray, cudaStream_t s, const Sched &sc = Sched());
// K4 into the ring-addressed a.loc (a.ring), which also clears the voxels a
// re-centre brought in; with all-zero planes only those
cudaError_t launch_merge(const FrameArgs &a, cudaStream_t s, const Sched &sc = Sched());
// K5: the grid in its own frame, out of the ring-addressed src (ring), into dst
cudaError_t launch_shift(const PlaneGeom &g, const Ring &ring, const uint8_t *src, uint8_t *dst, cudaStream_t s);
// loc_grid's occupied voxels in the grid's own frame, as a bit plane
cudaError_t launch_loc_occupancy(const PlaneGeom &g, const uint8_t *loc, const Ring &ring, uint32_t *out,
                                 cudaStream_t s);
cudaError_t configure_batch(int dev);   // once per device, before the first launch_batch
int batch_max_blocks(int dev);          // CTAs of k_batch resident at once on the device
cudaError_t launch_batch(const BatchItem *items, BatchCtl *ctl, int blocks, cudaStream_t s);

}  // namespace vg
