// vg_host.h -- host-side set-up arithmetic shared by every entry point of
// the library (vg_api.cu, vg_noalloc.cu, vg_server.cu), so that all of them
// give a frame exactly the same kernel arguments.
//
// Everything here runs in double on the host and is rounded once to float
// or integer (Sec. IV-A..IV-C):
//   origin_k   = floor(p_k / vox_size) - floor(N_k / 2)          (Sec. IV-A)
//   R^v_c      = R^w_c,  t^v_c = t^w_c - origin * vox_size       (Sec. IV-B)
//   vox_depth  = lround(depth / vox_size)                         (Sec. IV-C)
//   hw         = lround(tan(fov_x / 2) * vox_depth), hh likewise
//   fx         = (W / 2) / tan(fov_x / 2), cx = (W - 1) / 2, y likewise
// with fov/2 in radians taken as fov_deg * pi / 360.
#pragma once

#include "vg.h"
#include "vg_internal.cuh"

#include <cmath>
#include <cstring>

namespace vg {
namespace host {

constexpr double kPi = 3.14159265358979323846;

inline int status_of(cudaError_t e) {
    if (e == cudaSuccess) return VG_OK;
    if (e == cudaErrorMemoryAllocation) return VG_ENOMEM;
    return VG_ECUDA;
}

inline double half_fov(float deg) { return (double)deg * kPi / 360.0; }

// Table I parameters that every kind of grid accepts (flags aside): sizes
// >= 1 with fewer than 2^31 voxels and fewer than 2^27 plane words (K3
// indexes plane bits with 32 bits; only Nx far below 32 nears that), a
// finite positive voxel size and range, fields of view in (0, 180) degrees,
// 0 <= vox_inf <= 15, and fewer than 10^6 voxels of range.
inline bool shape_ok(const vg_params *p) {
    if (!p) return false;
    int64_t nv = 1;
    for (int k = 0; k < 3; ++k) {
        if (p->grid_size[k] < 1) return false;
        nv *= p->grid_size[k];
        if (nv >= (int64_t(1) << 31)) return false;
    }
    if (!(std::isfinite(p->vox_size) && p->vox_size > 0.0f)) return false;
    if (!(p->fov_x_deg > 0.0f && p->fov_x_deg < 180.0f)) return false;
    if (!(p->fov_y_deg > 0.0f && p->fov_y_deg < 180.0f)) return false;
    if (!(std::isfinite(p->depth) && p->depth > 0.0f)) return false;
    if (p->vox_inf < 0 || p->vox_inf > kMaxInflate) return false;
    {
        int64_t w = (p->grid_size[0] + 31) / 32, wx = 4;
        while (wx < w) wx *= 2;
        if (wx * (int64_t)p->grid_size[1] * p->grid_size[2] >= (int64_t(1) << 27)) return false;
    }
    const double vd = (double)p->depth / (double)p->vox_size;
    return vd < 1.0e6;
}

inline PlaneGeom geom_of(const vg_params *p) {
    PlaneGeom g;
    g.nx = p->grid_size[0];
    g.ny = p->grid_size[1];
    g.nz = p->grid_size[2];
    const int32_t w = (g.nx + 31) / 32;
    g.wx = 4;
    while (g.wx < w) g.wx *= 2;
    g.words = (int64_t)g.wx * g.ny * g.nz;
    g.nvox = (int64_t)g.nx * g.ny * g.nz;
    return g;
}

// The ray bundle of Sec. IV-C: vox_depth and the half widths.
inline void bundle_of(const vg_params *p, int32_t &vd, int32_t &hw, int32_t &hh) {
    const long d = lround((double)p->depth / (double)p->vox_size);
    vd = (int32_t)d;
    hw = (int32_t)lround(tan(half_fov(p->fov_x_deg)) * (double)d);
    hh = (int32_t)lround(tan(half_fov(p->fov_y_deg)) * (double)d);
}

inline void origin_of(const vg_params *p, const double pos[3], int32_t o[3]) {
    for (int k = 0; k < 3; ++k)
        o[k] = (int32_t)floor(pos[k] / (double)p->vox_size) - p->grid_size[k] / 2;
}

// Composes T^v_c (Sec. IV-B) from T^w_c and the grid origin.  Rejects poses
// that are not finite, whose rotation block has an entry outside
// [-1.5, 1.5] (no rotation does), or whose camera lies 2^22 voxels or more
// from the grid corner: K3's walk length is bounded by the ray's length in
// voxels, and these limits keep it bounded and keep FP32 voxel
// coordinates exact to well below one voxel.
inline bool pose_vc(const double T_wc[16], const int32_t origin[3], float vox_size, Pose32 &T) {
    if (!T_wc) return false;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_wc[i])) return false;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            if (!(std::fabs(T_wc[r * 4 + c]) <= 1.5)) return false;
            T.R[r * 3 + c] = (float)T_wc[r * 4 + c];
        }
        const double t = T_wc[r * 4 + 3] - (double)origin[r] * (double)vox_size;
        if (!(std::fabs(t / (double)vox_size) < 4194304.0)) return false;
        T.t[r] = (float)t;
    }
    return true;
}

// A depth frame's shape and pixel type: 1 <= W, H with fewer than 2^31
// pixels, VG_DEPTH_F32 or VG_DEPTH_U16, and a finite positive scale for u16.
inline bool depth_frame_ok(int32_t width, int32_t height, int32_t dtype, float depth_scale) {
    if (width < 1 || height < 1 || (int64_t)width * height >= (int64_t(1) << 31)) return false;
    if (dtype != VG_DEPTH_F32 && dtype != VG_DEPTH_U16) return false;
    if (dtype == VG_DEPTH_U16 && !(std::isfinite(depth_scale) && depth_scale > 0.0f)) return false;
    return true;
}

// The kernel arguments of one measurement of a grid with parameters p and
// plane geometry g (planes, loc and stats are left for the caller).
inline FrameArgs frame_args(const vg_params *p, const PlaneGeom &g, const Pose32 &T) {
    FrameArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.T = T;
    a.vs = p->vox_size;
    a.depth_max = p->depth;
    bundle_of(p, a.vd, a.hw, a.hh);
    a.r = p->vox_inf;
    return a;
}

// Adds a depth frame's input and pinhole intrinsics to a.
inline void set_depth_frame(FrameArgs &a, const vg_params *p, const void *depth, int32_t width, int32_t height,
                            int32_t dtype, float depth_scale) {
    a.depth = depth;
    a.W = width;
    a.H = height;
    a.scale = (dtype == VG_DEPTH_U16) ? depth_scale : 1.0f;
    a.fx = (float)(((double)width / 2.0) / tan(half_fov(p->fov_x_deg)));
    a.fy = (float)(((double)height / 2.0) / tan(half_fov(p->fov_y_deg)));
    a.cx = (float)(((double)width - 1.0) / 2.0);
    a.cy = (float)(((double)height - 1.0) / 2.0);
}

}  // namespace host
}  // namespace vg
