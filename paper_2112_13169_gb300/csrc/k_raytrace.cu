// K3 as its own launch: one resident wave of CTAs, each with one group of
// rays of the frame and the camera box staged once; groups past the wave go
// out bundle by bundle.  The work itself is in vg_rt.cuh.
#include "vg_rt.cuh"

namespace vg {
namespace {

using namespace rt;

template <int LPR, bool EXACT>
__global__ void __launch_bounds__(kThreads, 5) k_raytrace(const FrameArgs a, const int buffered) {
    __shared__ uint32_t box_fr[kBoxWords], box_tr[kBoxWords], occ_box[kBoxWords];
    extern __shared__ uint32_t buf[];   // kRtBuf * kThreads, one column per thread
    pdl_trigger();
    float S[3];
    frame_start(a, S);
    const Box b = box_of(S);
    const int64_t groups = rt_groups<LPR>(a);
    // the first group's set-up and walk need only the pose and the grid's
    // shape, so they overlap the end of K2; the occupancy is read and the
    // planes are marked after the wait (every CTA has a first group: the
    // grid is no larger than the group count)
    Lane ln;
    rt_setup<LPR>(a, S, b, blockIdx.x, groups, ln);
    box_clear(box_fr, box_tr);
    const Pass1 p1 = rt_record(a, ln, b, buffered, buf);
    pdl_wait();
    box_stage<units::LoadRO, false>(a, b, box_fr, box_tr, occ_box);
    unsigned visits = rt_resolve<LPR, units::LoadRO, EXACT>(a, ln, b, p1, box_fr, box_tr, occ_box, buf);
    if (a.rt_next && groups > (int64_t)gridDim.x) {
        // the groups past the launch's CTAs go out one bundle at a time, from
        // a counter in device memory (zeroed by this frame's K1), so that the
        // warps whose first bundles were short take more
        constexpr int kWarps = kThreads / 32;
        for (;;) {
            uint32_t t = 0;
            if ((threadIdx.x & 31) == 0) t = atomicAdd(a.rt_next, 1u);
            t = __shfl_sync(kFull, t, 0);
            const int64_t grp = (int64_t)gridDim.x + t / kWarps;
            if (grp >= groups) break;
            visits += rt_bundle<LPR, units::LoadRO, EXACT>(a, S, b, (int64_t)(t % kWarps) * groups + grp, buffered,
                                                           box_fr, box_tr, occ_box, buf);
        }
    } else {
        for (int64_t grp = blockIdx.x + gridDim.x; grp < groups; grp += gridDim.x)
            visits += rt_group<LPR, units::LoadRO, EXACT>(a, S, b, grp, groups, buffered, box_fr, box_tr, occ_box,
                                                          buf);
    }
    box_flush(a, b, box_fr, box_tr);
    if (a.stats) {
        const unsigned total = __reduce_add_sync(kFull, visits);
        if ((threadIdx.x & 31) == 0 && total) atomicAdd(a.stats + 2, (unsigned long long)total);
    }
}

int g_sms[64];
int g_blocks_per_sm[64][6];

template <int LPR>
cudaError_t configure_lpr(int dev, int idx) {
    const size_t dyn = sizeof(uint32_t) * kRtBuf * kThreads;
    cudaError_t e = cudaFuncSetAttribute(k_raytrace<LPR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_raytrace<LPR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    // the exact variant is sized like the default one (same bounds and buffer)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_blocks_per_sm[dev][idx], k_raytrace<LPR, false>,
                                                         kThreads, dyn);
}

template <int LPR>
cudaError_t launch_lpr(const FrameArgs &a, int idx, cudaStream_t s, int ctas_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int64_t nrays = (2 * (int64_t)a.hw + 1) * (2 * (int64_t)a.hh + 1);
    const int64_t need = (nrays * LPR + kThreads - 1) / kThreads;
    int per_sm = g_blocks_per_sm[dev][idx] > 0 ? g_blocks_per_sm[dev][idx] : 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const int64_t resident = (int64_t)g_sms[dev] * per_sm;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    if (blocks == 0) return cudaSuccess;
    // a packed run holds a plane bit index below 2^26
    const int buffered = a.g.words < kRunWords ? 1 : 0;
    const size_t dyn = sizeof(uint32_t) * kRtBuf * kThreads;
    // traced marks must skip tested-occupied voxels only when the tested
    // plane is not covered by occ_inf (the literal loc_grid reading)
    if (a.lit & kLitRaysLast) return launch_pdl(k_raytrace<LPR, true>, blocks, kThreads, dyn, s, a, buffered);
    return launch_pdl(k_raytrace<LPR, false>, blocks, kThreads, dyn, s, a, buffered);
}

}  // namespace

cudaError_t configure_raytrace(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaError_t e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = configure_lpr<1>(dev, 0);
    if (e == cudaSuccess) e = configure_lpr<2>(dev, 1);
    if (e == cudaSuccess) e = configure_lpr<4>(dev, 2);
    if (e == cudaSuccess) e = configure_lpr<8>(dev, 3);
    if (e == cudaSuccess) e = configure_lpr<16>(dev, 4);
    if (e == cudaSuccess) e = configure_lpr<32>(dev, 5);
    return e;
}

int auto_lanes_per_ray(int32_t vd, int32_t hw, int32_t hh) {
    // a slice of 1/LPR of a ray crosses about L1/LPR faces, plus up to three
    // more at its ends; the buffer keeps runs of same-word visits, fewer
    // than the visits (about half of them on the measured frames), so pick
    // the fewest lanes, at least 8, whose slices' visits fit 1.5 buffers (a
    // lane whose runs still overflow walks twice).  A 1280x720 frame at
    // 6 m and 0.05 m (L1 about 313 voxels) then takes 8 lanes: 74 against
    // 77 us a frame with 16.
    const int64_t l1 = (int64_t)vd + hw + hh + 4;
    for (int lpr = 8; lpr < 32; lpr *= 2)
        if ((l1 + lpr - 1) / lpr + 3 <= kRtBuf * 3 / 2) return lpr;
    return 32;
}

cudaError_t launch_raytrace(const FrameArgs &a_in, int lanes_per_ray, cudaStream_t s, const Sched &sc) {
    FrameArgs a = a_in;
    if (!a.occ_test) a.occ_test = a.pl.occ_inf;   // the default reading: rays test the inflated plane
    const int c = sc.rt_ctas;
    switch (lanes_per_ray) {
    case 1: return launch_lpr<1>(a, 0, s, c);
    case 2: return launch_lpr<2>(a, 1, s, c);
    case 4: return launch_lpr<4>(a, 2, s, c);
    case 8: return launch_lpr<8>(a, 3, s, c);
    case 16: return launch_lpr<16>(a, 4, s, c);
    case 32: return launch_lpr<32>(a, 5, s, c);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vg
