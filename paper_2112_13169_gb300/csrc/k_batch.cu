// k_batch.cu -- many measurements in one persistent, fused launch.
//
// One cooperative launch of k_batch runs, for every frame of a batch (each
// with its own grid, resolution, voxel size and radius), the whole path:
//   phase 1  K1 voxelize           units of 1024 pixels
//   phase 2  K2 inflate            8 (or 4) words x 8 rows x 8 (or 4)
//                                  slices (radius 1..3)
//   phase 3  K3 ray trace          groups of at most 256 / LPR rays (a
//                                  frame's rays spread over its units)
//   phase 4  K4 merge              512 plane words (256 if tuned)
// with a grid-wide barrier between phases.  A frame's re-centre (K5) is not
// a phase: it moves its grid's ring, and that grid's next merge sets the
// voxels it brought in to unknown (Ring).
// Units of every frame are laid end to end per phase (BatchItem::off).  A
// CTA finds the frame of its first unit of a phase by binary search, steps
// forward through the frames as its units advance (see run_begin), and runs
// the same device code as the one-step kernels (vg_units.cuh, vg_rt.cuh).
// Reads of data an earlier phase wrote skip the L1 (LoadL2), except the ray
// trace's occupancy loads (see group_lpr).
//
// The barrier waits with a deadline (BatchCtl::bar_ns, four seconds unless
// tuned): if the other CTAs do not all arrive in time, the waiting CTA sets
// BatchCtl::error and every CTA leaves the kernel, so the host sees
// VG_ETIMEOUT instead of a hung GPU.  The launch is cooperative, so all CTAs are resident together.
#include "vg_rt.cuh"
#include "vg_sync.cuh"

namespace vg {
namespace {

using namespace rt;

// loads of an inflate tile's staging issued together (fewer than the
// one-step kernel's 8: this kernel's registers are capped at 64)
constexpr int kInflateUnroll = 2;
constexpr int kDynWords = kRtBuf * kThreads;   // also covers an inflate tile of radius <= 3
static_assert(units::inflate_smem_words<3, 8, 8, 8>(3) <= (size_t)kDynWords, "inflate tile fits");
static_assert(sizeof(FrameArgs) % 4 == 0, "frame arguments copy as words");

__device__ __forceinline__ int find_item(const BatchItem *items, int n, int phase, int64_t u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {   // last item whose offset is <= u
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&items[mid].off[phase]) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The first phase-3 unit whose weighted start (woff3 + its index in its
// frame x w3) is at least x, for 0 <= x <= ctl->wtotal3.
__device__ __forceinline__ int64_t weighted_unit(const BatchItem *items, int n, int64_t total, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {   // last item whose weighted offset is <= x
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&items[mid].woff3) <= x) lo = mid;
        else hi = mid - 1;
    }
    const int64_t first = __ldg(&items[lo].off[2]);
    const int64_t units = (lo + 1 < n ? __ldg(&items[lo + 1].off[2]) : total) - first;
    const int64_t w = __ldg(&items[lo].w3);
    const int64_t k = (x - __ldg(&items[lo].woff3) + w - 1) / w;
    return first + (k < units ? k : units);
}

// In the voxelize and ray-trace phases a CTA's units are a contiguous run
// [lo, hi) of the phase's units, so that it moves to another frame (and
// restages that frame's arguments) only a few times.  Their units cost about
// the same in every frame.  The inflate and merge units cost more in some
// frames than in others (tile width and radius; how much of a grid the
// measurement marks), so there the units go round the CTAs in turn.
__device__ __forceinline__ int64_t run_begin(int64_t total, unsigned b, unsigned nb) { return total * b / nb; }

// The frame of unit u, given the frame i of an earlier unit of the same CTA
// in the same phase (frames with no units in this phase are skipped).
__device__ __forceinline__ int next_item(const BatchItem *items, int n, int phase, int64_t u, int i) {
    while (i + 1 < n && __ldg(&items[i + 1].off[phase]) <= u) ++i;
    return i;
}

// The ray trace reads the occupancy planes with ordinary (L1-cached) loads:
// phase 2 wrote them before the grid barrier, whose release (every CTA's
// fence before it arrives) and acquire (thread 0's fence after it, then
// the CTA barrier) order those writes before these loads, and no SM reads
// a plane word of this launch's occupancy before phase 3, so none holds a
// stale line of it.  (64 robots: 148.1k -> 150.9k Mvoxel-updates/s.)
template <int LPR>
__device__ __forceinline__ unsigned group_lpr(const FrameArgs &a, int buffered, const float S[3], const Box &b,
                                              int64_t grp, int64_t G, uint32_t *box_fr, uint32_t *box_tr,
                                              const uint32_t *occ_box, uint32_t *buf) {
    return rt_group<LPR, units::LoadPlain>(a, S, b, grp, G, buffered, box_fr, box_tr, occ_box, buf);
}

// One inflate tile of TXW words x 8 rows x TZ slices of a batch frame.
template <int TXW, int TZ>
__device__ __forceinline__ void inflate_unit(const BatchItem &it, int tx, int ty, int tz, uint32_t *sm) {
    const PlaneGeom &g = it.a.g;
    switch (it.a.r) {
    case 1: units::inflate_tile<1, TXW, 8, TZ, units::LoadL2, kInflateUnroll>(g, it.a.pl.occ_raw, it.a.pl.occ_inf, 1, tx, ty, tz, sm); break;
    case 2: units::inflate_tile<2, TXW, 8, TZ, units::LoadL2, kInflateUnroll>(g, it.a.pl.occ_raw, it.a.pl.occ_inf, 2, tx, ty, tz, sm); break;
    default: units::inflate_tile<3, TXW, 8, TZ, units::LoadL2, kInflateUnroll>(g, it.a.pl.occ_raw, it.a.pl.occ_inf, 3, tx, ty, tz, sm); break;
    }
}

// Copies a frame's arguments into shared memory, by the threads of the CTA
// (the caller places the barriers).
__device__ __forceinline__ void stage_args(const FrameArgs &src, FrameArgs &dst) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(FrameArgs) / 4); k += kThreads) d[k] = __ldg(s + k);
}

__global__ void __launch_bounds__(kThreads, 4) k_batch(const BatchItem *__restrict__ items, BatchCtl *ctl) {
    __shared__ uint32_t box_fr[kBoxWords], box_tr[kBoxWords], occ_box[kBoxWords];
    extern __shared__ __align__(16) uint32_t dyn[];
    const int n = ctl->n;
    const unsigned nb = gridDim.x;

    // The frame arguments of the unit at hand are staged in shared memory
    // (s_a) whenever the CTA moves to another frame, so that the per-pixel
    // and per-ray code reads them there rather than field by field from the
    // table in global memory.
    __shared__ FrameArgs s_a;
    __shared__ int32_t s_kind;   // phase 1: dtype * 2 + vec; phase 3: LPR * 2 + buffered

    // ---- phase 1: voxelize ------------------------------------------------
    {
        int cur = -1;
        const int64_t lo = run_begin(ctl->total[0], blockIdx.x, nb), hi = run_begin(ctl->total[0], blockIdx.x + 1, nb);
        int i = find_item(items, n, 0, lo);
        for (int64_t u = lo; u < hi; ++u) {
            i = next_item(items, n, 0, u, i);   // the same for every thread
            if (i != cur) {
                __syncthreads();   // the previous frame's copy is no longer read
                stage_args(items[i].a, s_a);
                if (threadIdx.x == 0) s_kind = __ldg(&items[i].dtype) * 2 + __ldg(&items[i].vec);
                __syncthreads();
                cur = i;
            }
            const int64_t t = (u - __ldg(&items[i].off[0])) * kThreads + threadIdx.x;
            switch (s_kind) {
            case 0: units::voxelize_depth_thread<0, false>(s_a, t); break;
            case 1: units::voxelize_depth_thread<0, true>(s_a, t); break;
            case 2: units::voxelize_depth_thread<1, false>(s_a, t); break;
            default: units::voxelize_depth_thread<1, true>(s_a, t); break;
            }
        }
    }
    if (!grid_sync(ctl, nb)) return;

    // ---- phase 2: inflate -------------------------------------------------
    {
        // units in turn over the CTAs: their cost differs between frames,
        // and interleaving keeps the CTAs' shares even
        int i = find_item(items, n, 1, blockIdx.x);
        for (int64_t u = blockIdx.x; u < ctl->total[1]; u += nb) {
            i = next_item(items, n, 1, u, i);
            const BatchItem &it = items[i];
            // a frame has fewer than 2^27 plane words, so fewer tiles
            const uint32_t local = (uint32_t)(u - it.off[1]), t0 = (uint32_t)it.tiles[0];
            const uint32_t t01 = local / t0;
            const int tx = (int)(local - t01 * t0);
            const int ty = (int)(t01 % (uint32_t)it.tiles[1]);
            const int tz = (int)(t01 / (uint32_t)it.tiles[1]);
            switch (it.txw * 10 + it.tz) {
            case 88: inflate_unit<8, 8>(it, tx, ty, tz, dyn); break;
            case 84: inflate_unit<8, 4>(it, tx, ty, tz, dyn); break;
            case 48: inflate_unit<4, 8>(it, tx, ty, tz, dyn); break;
            default: inflate_unit<4, 4>(it, tx, ty, tz, dyn); break;
            }
        }
    }
    if (!grid_sync(ctl, nb)) return;

    // ---- phase 3: ray trace -----------------------------------------------
    // a contiguous run of units per CTA, so the camera box is staged again
    // only when the run crosses into another frame; the runs split the
    // units' total weight evenly (weights of 1: their number)
    {
        const int64_t lo = weighted_unit(items, n, ctl->total[2], run_begin(ctl->wtotal3, blockIdx.x, nb));
        const int64_t hi = weighted_unit(items, n, ctl->total[2], run_begin(ctl->wtotal3, blockIdx.x + 1, nb));
        int cur = -1, i = find_item(items, n, 2, lo);
        float S[3] = {0.0f, 0.0f, 0.0f};
        Box b = {0, 0, 0};
        for (int64_t u = lo; u < hi; ++u) {
            i = next_item(items, n, 2, u, i);   // the same for every thread
            if (i != cur) {
                if (cur >= 0) box_flush(s_a, b, box_fr, box_tr);   // ends with a barrier
                else __syncthreads();   // phase 1's copy is no longer read
                stage_args(items[i].a, s_a);
                if (threadIdx.x == 0) s_kind = __ldg(&items[i].lpr) * 2 + __ldg(&items[i].buffered);
                __syncthreads();
                cur = i;
                frame_start(s_a, S);
                b = box_of(S);
                box_stage<units::LoadPlain>(s_a, b, box_fr, box_tr, occ_box);
            }
            // the frame's rays are spread over its G units of this phase
            const int64_t off = __ldg(&items[i].off[2]);
            const int64_t grp = u - off;
            const int64_t G = (i + 1 < n ? __ldg(&items[i + 1].off[2]) : ctl->total[2]) - off;
            const int buffered = s_kind & 1;
            unsigned visits;
            switch (s_kind >> 1) {
            case 8: visits = group_lpr<8>(s_a, buffered, S, b, grp, G, box_fr, box_tr, occ_box, dyn); break;
            case 16: visits = group_lpr<16>(s_a, buffered, S, b, grp, G, box_fr, box_tr, occ_box, dyn); break;
            default: visits = group_lpr<32>(s_a, buffered, S, b, grp, G, box_fr, box_tr, occ_box, dyn); break;
            }
            if (s_a.stats) {
                const unsigned total = __reduce_add_sync(kFull, visits);
                if ((threadIdx.x & 31) == 0 && total) atomicAdd(s_a.stats + 2, (unsigned long long)total);
            }
        }
        if (cur >= 0) box_flush(s_a, b, box_fr, box_tr);
    }
    if (!grid_sync(ctl, nb)) return;

    // ---- phase 4: merge ---------------------------------------------------
    {
        // units in turn over the CTAs: their cost differs between frames,
        // and interleaving keeps the CTAs' shares even
        int i = find_item(items, n, 3, blockIdx.x);
        for (int64_t u = blockIdx.x; u < ctl->total[3]; u += nb) {
            i = next_item(items, n, 3, u, i);
            const BatchItem &it = items[i];
            // the unit's mwpu plane words, one or two per thread
            for (int k = 0; k < it.mwpu; k += kThreads)
                units::merge_word<units::LoadL2>(it.a.g, it.a.pl, it.a.loc, it.a.ring,
                                                 (u - it.off[3]) * it.mwpu + k + threadIdx.x);
        }
    }
}

int g_batch_blocks_per_sm[64];
int g_batch_sms[64];

}  // namespace

cudaError_t configure_batch(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t dyn = sizeof(uint32_t) * kDynWords;
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_batch_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_batch_blocks_per_sm[dev], k_batch, kThreads, dyn);
    return e;
}

int batch_max_blocks(int dev) {
    if (dev < 0 || dev >= 64) return 0;
    return g_batch_sms[dev] * g_batch_blocks_per_sm[dev];
}

cudaError_t launch_batch(const BatchItem *items, BatchCtl *ctl, int blocks, cudaStream_t s) {
    void *args[] = {(void *)&items, (void *)&ctl};
    return cudaLaunchCooperativeKernel((const void *)k_batch, dim3(blocks), dim3(kThreads), args,
                                       sizeof(uint32_t) * kDynWords, s);
}

}  // namespace vg
