// K2 as its own launch: one CTA per 8-word x 8-row x 8-slice tile of the
// occupancy plane (4 slices for grids of one to four such tiles per SM);
// the work itself is in vg_units.cuh.  For r = 1, 2, 3 the
// radius is a compile-time constant; other radii use a runtime radius.
#include "vg_units.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

namespace vg {
namespace {

template <int R, int TXW, int TY, int TZ>
__global__ void __launch_bounds__(256) k_inflate(const PlaneGeom g, const uint32_t *__restrict__ raw,
                                                 uint32_t *__restrict__ out, const int r_rt) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    units::inflate_tile<R, TXW, TY, TZ, units::LoadRO>(g, raw, out, r_rt, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// ---------------------------------------------------------------------------
// The same tile with its raw words moved by the tensor memory accelerator:
// one thread issues a single 3-D tiled copy of the tile and its halo from
// the occ_raw plane into shared memory (cp.async.bulk.tensor, completion
// counted on an mbarrier), and the copy engine fills the parts outside the
// grid with zeros, which is the dilation's clipping.  The box starts four
// words left of the tile, so that its innermost coordinate is a multiple of
// 16 bytes: it is TXW + 8 words wide, rows y0 - R .. y0 + TY + R - 1 and
// slices z0 - R .. z0 + TZ + R - 1.  The CTA waits for the copy with a
// deadline; a wait that runs out is counted in g_wait_timeouts and the tile
// is left unwritten.
// ---------------------------------------------------------------------------
__device__ unsigned g_wait_timeouts;

__device__ __forceinline__ int64_t global_ns_k2() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

constexpr int64_t kTmaWaitNs = 2000000000LL;   // two seconds

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <int R, int TXW, int TY, int TZ>
__host__ __device__ constexpr int tma_box_words() { return (TXW + 8) * (TY + 2 * R) * (TZ + 2 * R); }

template <int R, int TXW, int TY, int TZ>
__global__ void __launch_bounds__(256) k_inflate_tma(const __grid_constant__ CUtensorMap tm, const PlaneGeom g,
                                                     uint32_t *__restrict__ out) {
    constexpr int BW = TXW + 8, HY = TY + 2 * R, HZ = TZ + 2 * R;
    constexpr uint32_t kBytes = (uint32_t)tma_box_words<R, TXW, TY, TZ>() * 4u;
    extern __shared__ __align__(128) uint32_t sm[];   // the box, then the x pass's HZ * HY * TXW words
    __shared__ __align__(8) uint64_t bar;
    pdl_trigger();
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();   // occ_raw is K1's
    if (threadIdx.x == 0) {
        const int x = (int)blockIdx.x * TXW - 4, y = (int)blockIdx.y * TY - R, z = (int)blockIdx.z * TZ - R;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kBytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(smem_addr(sm)), "l"(reinterpret_cast<uint64_t>(&tm)), "r"(x), "r"(y), "r"(z), "r"(b)
            : "memory");
    }
    // every thread waits for phase 0 of the barrier, with a deadline
    uint32_t done = 0;
    const int64_t t0 = global_ns_k2();
    do {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(b) : "memory");
    } while (!done && global_ns_k2() - t0 < kTmaWaitNs);
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }
    // the word w0 - 1 of each staged row is column 3 of the box
    units::inflate_passes<R, TXW, TY, TZ>(g, out, R, blockIdx.x, blockIdx.y, blockIdx.z, sm, BW, 3,
                                          sm + BW * HY * HZ);
}

template <int R, int TXW, int TY, int TZ>
cudaError_t run(const FrameArgs &a, cudaStream_t s) {
    dim3 grid((a.g.wx + TXW - 1) / TXW, (a.g.ny + TY - 1) / TY, (a.g.nz + TZ - 1) / TZ);
    const size_t bytes = sizeof(uint32_t) * units::inflate_smem_words<R, TXW, TY, TZ>(a.r);
    return launch_pdl(k_inflate<R, TXW, TY, TZ>, grid, 256, bytes, s, a.g, (const uint32_t *)a.pl.occ_raw,
                      a.pl.occ_inf, a.r);
}

// The driver's tensor-map encoder, looked up once through the runtime (the
// library does not link the driver library itself); NULL if unavailable,
// and then the tiles are staged by the threads.
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

// The tensor map of a plane (wx x ny x nz 32-bit words at base) with a box
// of bw x hy x hz words; the last few are kept per host thread, since a
// grid's map only changes with its plane and tile.
struct MapKey {
    const void *base;
    int32_t wx, ny, nz, bw, hy, hz;
    bool operator==(const MapKey &o) const {
        return base == o.base && wx == o.wx && ny == o.ny && nz == o.nz && bw == o.bw && hy == o.hy && hz == o.hz;
    }
};

bool plane_map(const void *base, const PlaneGeom &g, int bw, int hy, int hz, CUtensorMap &out) {
    struct Entry {
        MapKey k;
        CUtensorMap m;
        bool valid;
    };
    thread_local Entry cache[4] = {};
    thread_local int next = 0;
    const MapKey k{base, g.wx, g.ny, g.nz, bw, hy, hz};
    for (const Entry &e : cache)
        if (e.valid && e.k == k) {
            out = e.m;
            return true;
        }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.wx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.wx * 4, (cuuint64_t)g.wx * (cuuint64_t)g.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)hy, (cuuint32_t)hz};
    const cuuint32_t es[3] = {1, 1, 1};
    CUtensorMap m;
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    Entry &e = cache[next];
    next = (next + 1) % 4;
    e.k = k;
    e.m = m;
    e.valid = true;
    out = m;
    return true;
}

// The tile with its words moved by the tensor memory accelerator, or by
// the threads where no tensor map can be had.
template <int R, int TXW, int TY, int TZ>
cudaError_t run_tma(const FrameArgs &a, cudaStream_t s) {
    CUtensorMap m;
    if (!plane_map(a.pl.occ_raw, a.g, TXW + 8, TY + 2 * R, TZ + 2 * R, m)) return run<R, TXW, TY, TZ>(a, s);
    dim3 grid((a.g.wx + TXW - 1) / TXW, (a.g.ny + TY - 1) / TY, (a.g.nz + TZ - 1) / TZ);
    const size_t bytes = sizeof(uint32_t) * (tma_box_words<R, TXW, TY, TZ>() + (TZ + 2 * R) * (TY + 2 * R) * TXW);
    return launch_pdl(k_inflate_tma<R, TXW, TY, TZ>, grid, 256, bytes, s, m, a.g, a.pl.occ_inf);
}

template <int TXW, int TZ>
cudaError_t run_r(const FrameArgs &a, cudaStream_t s, bool tma) {
    switch (a.r) {
    case 1: return tma ? run_tma<1, TXW, 8, TZ>(a, s) : run<1, TXW, 8, TZ>(a, s);
    case 2: return tma ? run_tma<2, TXW, 8, TZ>(a, s) : run<2, TXW, 8, TZ>(a, s);
    case 3: return tma ? run_tma<3, TXW, 8, TZ>(a, s) : run<3, TXW, 8, TZ>(a, s);
    default: return run<0, TXW, 8, 8>(a, s);   // other radii: 8-slice tiles, the radius at run time
    }
}

std::atomic<int> g_sms[64];   // SMs per device, read on first use (any thread)

int sms_of_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int n = g_sms[dev].load(std::memory_order_relaxed);
    if (!n) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        g_sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace

cudaError_t configure_inflate() {
    // the runtime-radius tile at vox_inf 15 needs about 104 KB of shared memory
    cudaError_t e = cudaFuncSetAttribute(k_inflate<0, 4, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_inflate<0, 8, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024);
    return e;
}

// Tiles of 8 words (4 for rows of 4 words) by 8 rows by 8 slices, or 4
// slices when a grid has between one and four 8-slice tiles per SM: the
// shorter tiles stage more halo per word, but twice as many CTAs share the
// device and the launch ends sooner.  Measured frame times: a 200x200x100
// grid (325 tiles of 8 slices) fell by about 2.3 us with 650 of 4; an
// 80x80x40 grid (50 tiles, fewer than the SMs) rose by 1.3 us, and a
// 400x400x120 grid (1500 tiles) did better with 8 slices.  sc.inflate_tile
// picks a shape instead (8-word tiles only where rows have a multiple of 8
// words).
cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s, const Sched &sc) {
    // rows are a power of two of words, at least 4
    const bool wide_ok = a.g.wx % 8 == 0;
    int tile = sc.inflate_tile;
    if (tile == kTileAuto) {
        const int txw = wide_ok ? 8 : 4;
        const int64_t tiles8 = (int64_t)((a.g.wx + txw - 1) / txw) * ((a.g.ny + 7) / 8) * ((a.g.nz + 7) / 8);
        const int64_t sms = sms_of_current_device();
        const bool short_tiles = tiles8 >= sms && tiles8 < 4 * sms;
        tile = wide_ok ? (short_tiles ? kTile8x8x4 : kTile8x8x8) : (short_tiles ? kTile4x8x4 : kTile4x8x8);
    }
    if (!wide_ok && tile == kTile8x8x4) tile = kTile4x8x4;
    if (!wide_ok && tile == kTile8x8x8) tile = kTile4x8x8;
    const bool tma = sc.inflate_tma != 0;
    switch (tile) {
    case kTile4x8x4: return run_r<4, 4>(a, s, tma);
    case kTile4x8x8: return run_r<4, 8>(a, s, tma);
    case kTile8x8x4: return run_r<8, 4>(a, s, tma);
    default: return run_r<8, 8>(a, s, tma);
    }
}

cudaError_t wait_timeouts(unsigned *out) {
    return cudaMemcpyFromSymbol(out, g_wait_timeouts, sizeof(unsigned));
}

}  // namespace vg
