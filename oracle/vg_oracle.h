/*
 * vg_oracle.h -- CPU oracle for the voxel-grid generation method of
 * "GPU Accelerated Voxel Grid Generation for fast MAV Exploration"
 * (Toumieh & Lambert, arXiv 2112.13169).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded C
 * restatement of the method, written to be checked against the paper by eye.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the CUDA
 * library, and the CUDA library never calls it: there is no CPU fallback.
 *
 * Arithmetic: FP32, every operation rounded to nearest-even, no contraction
 * (built with -ffp-contract=off, FLT_EVAL_METHOD must be 0).  Host-side
 * set-up quantities (intrinsics, ray-bundle sizes, grid origin, T^v_c) are
 * computed in double and rounded once, as stated per function.
 *
 * Voxel state codes (the paper names the four states -- free, occupied,
 * unknown, unknown-and-traced -- in Sec. IV-C and Fig. 2, without numbers):
 *   OR_UNK = 0, OR_FREE = 1, OR_OCC = 2, OR_TRACED = 3.
 *
 * Grid layout (Sec. IV-D): idx = x + y*Nx + z*Nx*Ny, one byte per voxel.
 *
 * Parity status: every function below is pinned by the CPU tests
 * (tests/test_oracle_*.py) against closed forms, brute force or library
 * routines; none is "parity unpinned".
 */
#ifndef VG_ORACLE_H
#define VG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_UNK = 0, OR_FREE = 1, OR_OCC = 2, OR_TRACED = 3 };
enum { OR_DEPTH_F32 = 0, OR_DEPTH_U16 = 1 };

/* Literal readings of passages the default reading interprets (bit flags,
 * for comparison with the default; 0 is the default reading):
 *  OR_LIT_INFLATE_AFTER_TRACE  rays test the occupancy before inflation;
 *                              the inflation still marks its voxels
 *                              occupied (the order in which the kernel
 *                              list names the steps, trace before inflate).
 *  OR_LIT_SKIP_START           Alg. 2 moves by a voxel before its first
 *                              test, so a ray's start voxel is not visited.
 *  OR_LIT_LOC_OCCUPANCY        Alg. 2 tests loc_grid (the grid before this
 *                              measurement) for occupied voxels, and its
 *                              writes of the ray state replace the
 *                              measurement grid's occupied mark.
 * INFLATE_AFTER_TRACE and LOC_OCCUPANCY both choose the tested grid; when
 * both are set LOC_OCCUPANCY decides. */
enum { OR_LIT_INFLATE_AFTER_TRACE = 1, OR_LIT_SKIP_START = 2, OR_LIT_LOC_OCCUPANCY = 4 };

/* Table I parameters.  n = grid_size in voxels (x, y, z). */
typedef struct {
    int32_t n[3];
    float vox_size;
    float fov_x_deg;
    float fov_y_deg;
    float depth;
    int32_t vox_inf;
    uint32_t literal;   /* OR_LIT_* flags, 0 for the default reading */
} or_params;

/* T^v_c rounded to float: R row-major (3x3), t in metres. */
typedef struct {
    float R[9];
    float t[3];
} or_pose;

/* Sec. IV-A, Fig. 1: origin (voxel index of the grid's corner voxel) that
 * puts the robot in voxel floor(N/2) of every axis.  Computed in double:
 * o_k = floor(p_k / vox_size) - floor(N_k / 2). */
void or_origin(const or_params *p, const double robot_pos_w[3], int32_t o[3]);

/* Sec. IV-B: T^v_c = T^v_w * T^w_c, with T^v_w the pure translation by
 * -o*vox_size (the grid is ENU-aligned, Sec. IV-A).  T_wc is row-major 4x4,
 * camera optical frame (x right, y down, z forward) to world.  Composed in
 * double, then R and t are rounded to float. */
void or_pose_vc(const or_params *p, const double T_wc[16], const int32_t o[3],
                or_pose *out);

/* Pinhole intrinsics of a W x H depth image (the paper gives no formula):
 * fx = (W/2)/tan(fov_x/2), fy = (H/2)/tan(fov_y/2), cx = (W-1)/2,
 * cy = (H-1)/2, in double, rounded to float.  K = {fx, fy, cx, cy}. */
void or_intrinsics(const or_params *p, int32_t W, int32_t H, float K[4]);

/* Sec. IV-C ray bundle: out = {vox_depth, hw, hh} with
 * vox_depth = lround(depth/vox_size), hw = lround(tan(fov_x/2)*vox_depth),
 * hh = lround(tan(fov_y/2)*vox_depth); vox_width = 2hw+1,
 * vox_height = 2hh+1.  Returns the ray count vox_width*vox_height. */
int64_t or_ray_bundle(const or_params *p, int32_t out[3]);

/* Alg. 1, transform and voxelize, for a depth image.  Pixel (u, v) with
 * depth d is valid iff d is finite, d > 0 and d <= depth; it back-projects
 * to ((u-cx)*d/fx, (v-cy)*d/fy, d) and lands in voxel floor(g) with
 * g = (R p + t)/vox_size, kept iff 0 <= g_k < N_k.  Sets occ_raw[idx] = 1.
 * For OR_DEPTH_U16 the depth is (float)raw * scale.  Returns the number of
 * in-grid points. */
int64_t or_voxelize_depth(const or_params *p, const or_pose *T, const void *depth,
                          int32_t W, int32_t H, int32_t dtype, float scale,
                          uint8_t *occ_raw);

/* Alg. 1 for a point cloud in the camera frame (n x 3 floats).  A point is
 * valid iff its three coordinates are finite; no range filter. */
int64_t or_voxelize_points(const or_params *p, const or_pose *T, const float *xyz,
                           int64_t n, uint8_t *occ_raw);

/* Alg. 1, inflation: for every occupied voxel, set the clipped cube of side
 * 2*vox_inf+1 around it (Chebyshev dilation of occ_raw). */
void or_inflate(const or_params *p, const uint8_t *occ_raw, uint8_t *occ_inf);

/* Alg. 1 taken literally: stamp the cube around each point's voxel, point by
 * point (depth image input).  Used by the tests to show it equals
 * or_voxelize_depth followed by or_inflate. */
int64_t or_add_occ_literal_depth(const or_params *p, const or_pose *T, const void *depth,
                                 int32_t W, int32_t H, int32_t dtype, float scale,
                                 uint8_t *occ_inf);

/* Amanatides-Woo traversal (Alg. 2) of the segment S + tau*D, tau in [0,1],
 * in voxel units.  Writes the in-grid voxels visited, in visit order, as
 * (x, y, z) triples into out (up to cap triples) and returns how many were
 * visited (which may exceed cap; then only cap are written).  literal:
 * OR_LIT_SKIP_START leaves out the start voxel; other bits are ignored. */
int64_t or_dda(const int32_t n[3], const float S[3], const float D[3], uint32_t literal,
               int32_t *out, int64_t cap);

/* Alg. 2 over the whole bundle.  For each ray, voxels before the first
 * occupied voxel of occ_inf (the grid the rays test: the inflated
 * occupancy, or what p->literal chooses) get fr = 1, voxels after it get
 * tr = 1, occupied voxels are never written.  p->literal's
 * OR_LIT_SKIP_START applies to every ray.  ray_order, if not NULL, is a permutation of
 * the ray ids (id = (b+hh)*(2hw+1) + (a+hw)) giving the processing order.
 * Returns the number of in-grid voxel visits. */
int64_t or_raytrace(const or_params *p, const or_pose *T, const uint8_t *occ_inf,
                    const int64_t *ray_order, uint8_t *fr, uint8_t *tr);

/* Measurement-grid state of every voxel: OCC if occ_inf, else FREE if fr,
 * else TRACED if tr, else UNK.  With OR_LIT_LOC_OCCUPANCY in literal the
 * rays' writes come after the occupied marks: FREE if fr, else TRACED if
 * tr, else OCC if occ_inf, else UNK. */
void or_resolve(int64_t nvox, uint32_t literal, const uint8_t *occ_inf, const uint8_t *fr,
                const uint8_t *tr, uint8_t *ms);

/* Alg. 3: loc[idx] = ms[idx] wherever ms[idx] != UNK. */
void or_merge(int64_t nvox, const uint8_t *ms, uint8_t *loc);

/* Sec. IV-E: dst[i] = src[i + delta] where i + delta is inside the grid,
 * else UNK.  src and dst must not overlap. */
void or_shift(const int32_t n[3], const int32_t delta[3], const uint8_t *src,
              uint8_t *dst);

/* One whole measurement (steps 2-4 of Sec. IV) on a depth image: voxelize,
 * inflate, ray-trace, resolve, merge into loc (in place), in the reading
 * p->literal selects.  o is the current
 * grid origin.  ms_out, if not NULL, receives the resolved measurement grid.
 * Returns 0, or -1 if scratch memory could not be allocated. */
int or_integrate_depth(const or_params *p, const int32_t o[3], const double T_wc[16],
                       const void *depth, int32_t W, int32_t H, int32_t dtype,
                       float scale, uint8_t *loc, uint8_t *ms_out);

/* The same for a point cloud. */
int or_integrate_points(const or_params *p, const int32_t o[3], const double T_wc[16],
                        const float *xyz, int64_t n, uint8_t *loc, uint8_t *ms_out);

#ifdef __cplusplus
}
#endif
#endif
