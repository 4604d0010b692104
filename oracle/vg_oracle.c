/*
 * vg_oracle.c -- CPU oracle (test infrastructure only; see vg_oracle.h).
 *
 * Plain single-threaded C11.  Built with -O2 -ffp-contract=off and without
 * -ffast-math, so every float expression below is evaluated left to right
 * with one IEEE round-to-nearest per operation.  Each function cites the
 * passage of the paper it restates; where the paper is silent the reading
 * taken is stated in the comment.
 */
#include "vg_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs FLT_EVAL_METHOD == 0 (one rounding per float operation)"
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int64_t nvox_of(const int32_t n[3]) {
    return (int64_t)n[0] * n[1] * n[2];
}

/* Sec. IV-D: idx = x + y*Nx + z*Nx*Ny. */
static int64_t lin(const int32_t n[3], int32_t x, int32_t y, int32_t z) {
    return (int64_t)x + (int64_t)n[0] * ((int64_t)y + (int64_t)n[1] * z);
}

static int in_grid(const int32_t n[3], int32_t x, int32_t y, int32_t z) {
    return x >= 0 && x < n[0] && y >= 0 && y < n[1] && z >= 0 && z < n[2];
}

/* Half field of view in radians, in double: fov_deg * pi / 360. */
static double half_fov_rad(float fov_deg) {
    return (double)fov_deg * M_PI / 360.0;
}

void or_origin(const or_params *p, const double robot_pos_w[3], int32_t o[3]) {
    /* Sec. IV-A: the robot sits at the centre of the grid; for an even size
     * the "centre" voxel is floor(N/2).  The lattice is world-aligned, so
     * the origin moves in whole voxels (Sec. IV-E). */
    for (int k = 0; k < 3; ++k) {
        double c = floor(robot_pos_w[k] / (double)p->vox_size);
        o[k] = (int32_t)c - p->n[k] / 2;
    }
}

void or_pose_vc(const or_params *p, const double T_wc[16], const int32_t o[3],
                or_pose *out) {
    /* Sec. IV-B: T^v_c = T^v_w T^w_c.  T^v_w has identity rotation (ENU
     * grid) and translation -o*vox_size, so R^v_c = R^w_c and
     * t^v_c = t^w_c - o*vox_size. */
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) out->R[r * 3 + c] = (float)T_wc[r * 4 + c];
        double t = T_wc[r * 4 + 3] - (double)o[r] * (double)p->vox_size;
        out->t[r] = (float)t;
    }
}

void or_intrinsics(const or_params *p, int32_t W, int32_t H, float K[4]) {
    double fx = ((double)W / 2.0) / tan(half_fov_rad(p->fov_x_deg));
    double fy = ((double)H / 2.0) / tan(half_fov_rad(p->fov_y_deg));
    K[0] = (float)fx;
    K[1] = (float)fy;
    K[2] = (float)(((double)W - 1.0) / 2.0);
    K[3] = (float)(((double)H - 1.0) / 2.0);
}

int64_t or_ray_bundle(const or_params *p, int32_t out[3]) {
    /* Sec. IV-C: vox_depth = depth / vox_size, vox_width =
     * 2 tan(fov_x/2) vox_depth + 1 (likewise vox_height), rounded to
     * integers.  The text says both are odd by construction, so the half
     * widths are rounded and doubled. */
    long vd = lround((double)p->depth / (double)p->vox_size);
    long hw = lround(tan(half_fov_rad(p->fov_x_deg)) * (double)vd);
    long hh = lround(tan(half_fov_rad(p->fov_y_deg)) * (double)vd);
    out[0] = (int32_t)vd;
    out[1] = (int32_t)hw;
    out[2] = (int32_t)hh;
    return (int64_t)(2 * hw + 1) * (int64_t)(2 * hh + 1);
}

/* Alg. 1, transform and divide by the voxel size:
 * g_k = ((R_k0 x + R_k1 y) + R_k2 z + t_k) / vox_size, voxel = floor(g).
 * Returns 1 and the voxel iff 0 <= g_k < N_k on every axis (a NaN fails the
 * comparison and is dropped). */
static int point_voxel(const or_params *p, const or_pose *T, float x, float y, float z,
                       int32_t v[3]) {
    for (int k = 0; k < 3; ++k) {
        float g = T->R[k * 3 + 0] * x + T->R[k * 3 + 1] * y;
        g = g + T->R[k * 3 + 2] * z;
        g = g + T->t[k];
        g = g / p->vox_size;
        if (!(g >= 0.0f && g < (float)p->n[k])) return 0;
        v[k] = (int32_t)floorf(g);
    }
    return 1;
}

/* Depth pixel -> camera-frame point (reading of Sec. IV: a depth image is
 * z-depth in the optical frame).  Returns 0 for an invalid pixel. */
static int pixel_point(const or_params *p, const float K[4], const void *depth,
                       int32_t W, int32_t u, int32_t v, int32_t dtype, float scale,
                       float xyz[3]) {
    float d;
    if (dtype == OR_DEPTH_U16) {
        uint16_t raw = ((const uint16_t *)depth)[(int64_t)v * W + u];
        d = (float)raw * scale;
    } else {
        d = ((const float *)depth)[(int64_t)v * W + u];
    }
    if (!(isfinite(d) && d > 0.0f && d <= p->depth)) return 0;
    xyz[0] = ((float)u - K[2]) * d / K[0];
    xyz[1] = ((float)v - K[3]) * d / K[1];
    xyz[2] = d;
    return 1;
}

int64_t or_voxelize_depth(const or_params *p, const or_pose *T, const void *depth,
                          int32_t W, int32_t H, int32_t dtype, float scale,
                          uint8_t *occ_raw) {
    float K[4];
    or_intrinsics(p, W, H, K);
    int64_t kept = 0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            float q[3];
            int32_t g[3];
            if (!pixel_point(p, K, depth, W, u, v, dtype, scale, q)) continue;
            if (!point_voxel(p, T, q[0], q[1], q[2], g)) continue;
            occ_raw[lin(p->n, g[0], g[1], g[2])] = 1;
            ++kept;
        }
    }
    return kept;
}

int64_t or_voxelize_points(const or_params *p, const or_pose *T, const float *xyz,
                           int64_t n, uint8_t *occ_raw) {
    int64_t kept = 0;
    for (int64_t i = 0; i < n; ++i) {
        float x = xyz[3 * i + 0], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        int32_t g[3];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
        if (!point_voxel(p, T, x, y, z, g)) continue;
        occ_raw[lin(p->n, g[0], g[1], g[2])] = 1;
        ++kept;
    }
    return kept;
}

/* Alg. 1, the three nested loops: set every in-grid voxel of the cube of
 * half side r around voxel c. */
static void stamp_cube(const int32_t n[3], const int32_t c[3], int32_t r, uint8_t *grid) {
    for (int32_t i = c[0] - r; i <= c[0] + r; ++i)
        for (int32_t j = c[1] - r; j <= c[1] + r; ++j)
            for (int32_t k = c[2] - r; k <= c[2] + r; ++k)
                if (in_grid(n, i, j, k)) grid[lin(n, i, j, k)] = 1;
}

void or_inflate(const or_params *p, const uint8_t *occ_raw, uint8_t *occ_inf) {
    const int32_t *n = p->n;
    for (int32_t z = 0; z < n[2]; ++z)
        for (int32_t y = 0; y < n[1]; ++y)
            for (int32_t x = 0; x < n[0]; ++x)
                if (occ_raw[lin(n, x, y, z)]) {
                    int32_t c[3] = {x, y, z};
                    stamp_cube(n, c, p->vox_inf, occ_inf);
                }
}

int64_t or_add_occ_literal_depth(const or_params *p, const or_pose *T, const void *depth,
                                 int32_t W, int32_t H, int32_t dtype, float scale,
                                 uint8_t *occ_inf) {
    float K[4];
    or_intrinsics(p, W, H, K);
    int64_t kept = 0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            float q[3];
            int32_t g[3];
            if (!pixel_point(p, K, depth, W, u, v, dtype, scale, q)) continue;
            if (!point_voxel(p, T, q[0], q[1], q[2], g)) continue;
            stamp_cube(p->n, g, p->vox_inf, occ_inf);
            ++kept;
        }
    }
    return kept;
}

/*
 * Amanatides & Woo traversal of S + tau*D, tau in [0, 1] (Alg. 2; the
 * paper cites the method by reference).  Readings taken:
 *  - the start voxel floor(S) is visited (it lies between the camera and any
 *    obstacle);
 *  - an axis takes part iff D_k != 0 and 1/D_k is finite; its next crossing
 *    time is recomputed from the integer boundary at every step,
 *    tMax_k = (b_k - S_k) * (1/D_k), b_k = i_k + 1 if D_k > 0 else i_k;
 *  - the next axis is the one with the smallest tMax, the lowest axis on a
 *    tie; the walk ends when that tMax is >= 1 (the end of the segment,
 *    max_dist in voxel units);
 *  - voxels outside the grid are skipped; once an out-of-range axis can no
 *    longer come back the walk ends (this changes no result).
 * visit(ctx, x, y, z) is called for each in-grid voxel in order.
 */
typedef void (*visit_fn)(void *ctx, int32_t x, int32_t y, int32_t z);

static int64_t dda_walk(const int32_t n[3], const float S[3], const float D[3], int skip_start,
                        visit_fn visit, void *ctx) {
    int32_t i[3], step[3];
    float inv[3], tmax[3];
    for (int k = 0; k < 3; ++k) {
        i[k] = (int32_t)floorf(S[k]);
        step[k] = 0;
        inv[k] = 0.0f;
        tmax[k] = INFINITY;
        if (D[k] != 0.0f) {
            float r = 1.0f / D[k];
            if (isfinite(r)) {
                inv[k] = r;
                step[k] = D[k] > 0.0f ? 1 : -1;
                float b = (float)(step[k] > 0 ? i[k] + 1 : i[k]);
                tmax[k] = (b - S[k]) * inv[k];
            }
        }
    }
    int64_t visits = 0;
    int first = 1;
    for (;;) {
        if (first && skip_start) {
            /* the literal reading moves before its first test */
        } else if (in_grid(n, i[0], i[1], i[2])) {
            visit(ctx, i[0], i[1], i[2]);
            ++visits;
        } else {
            int gone = 0;
            for (int k = 0; k < 3; ++k) {
                if (i[k] < 0 && step[k] <= 0) gone = 1;
                if (i[k] >= n[k] && step[k] >= 0) gone = 1;
            }
            if (gone) break;
        }
        first = 0;
        int m = 0;
        if (tmax[1] < tmax[m]) m = 1;
        if (tmax[2] < tmax[m]) m = 2;
        if (!(tmax[m] < 1.0f)) break;
        i[m] += step[m];
        float b = (float)(step[m] > 0 ? i[m] + 1 : i[m]);
        tmax[m] = (b - S[m]) * inv[m];
    }
    return visits;
}

typedef struct {
    int32_t *out;
    int64_t cap;
    int64_t count;
} list_ctx;

static void list_visit(void *c, int32_t x, int32_t y, int32_t z) {
    list_ctx *L = (list_ctx *)c;
    if (L->count < L->cap) {
        L->out[3 * L->count + 0] = x;
        L->out[3 * L->count + 1] = y;
        L->out[3 * L->count + 2] = z;
    }
    ++L->count;
}

int64_t or_dda(const int32_t n[3], const float S[3], const float D[3], uint32_t literal,
               int32_t *out, int64_t cap) {
    list_ctx L = {out, cap, 0};
    dda_walk(n, S, D, (literal & OR_LIT_SKIP_START) != 0, list_visit, &L);
    return L.count;
}

/* Alg. 2, the body of the loop: vox_val starts as free and becomes
 * unknown-and-traced at the first occupied voxel; occupied voxels are never
 * written.  The occupancy test reads the measurement grid after inflation
 * (the text says "before hitting an occupied voxel"; the listing's loc_grid
 * reference is read as ms_grid).  Free and traced marks go to separate
 * planes so that rays sharing a voxel cannot overwrite each other. */
typedef struct {
    const int32_t *n;
    const uint8_t *occ;
    uint8_t *fr;
    uint8_t *tr;
    int traced;
} ray_ctx;

static void ray_visit(void *c, int32_t x, int32_t y, int32_t z) {
    ray_ctx *R = (ray_ctx *)c;
    int64_t idx = lin(R->n, x, y, z);
    if (R->occ[idx]) {
        R->traced = 1;
    } else if (!R->traced) {
        R->fr[idx] = 1;
    } else {
        R->tr[idx] = 1;
    }
}

int64_t or_raytrace(const or_params *p, const or_pose *T, const uint8_t *occ_inf,
                    const int64_t *ray_order, uint8_t *fr, uint8_t *tr) {
    int32_t b3[3];
    int64_t nrays = or_ray_bundle(p, b3);
    int32_t vd = b3[0], hw = b3[1], hh = b3[2];
    int64_t width = 2 * (int64_t)hw + 1;
    /* Alg. 2: ray_start = T^v_c [0 0 0 1]^t, in voxel units. */
    float S[3];
    for (int k = 0; k < 3; ++k) S[k] = T->t[k] / p->vox_size;
    int64_t visits = 0;
    for (int64_t q = 0; q < nrays; ++q) {
        int64_t id = ray_order ? ray_order[q] : q;
        int32_t a = (int32_t)(id % width) - hw;
        int32_t b = (int32_t)(id / width) - hh;
        /* Alg. 2: ray_dir = R^v_c (x_i, y_i, z_i) with z_i = vox_depth; only
         * the rotation applies to a direction. */
        float D[3];
        for (int k = 0; k < 3; ++k) {
            float d = T->R[k * 3 + 0] * (float)a + T->R[k * 3 + 1] * (float)b;
            d = d + T->R[k * 3 + 2] * (float)vd;
            D[k] = d;
        }
        ray_ctx R = {p->n, occ_inf, fr, tr, 0};
        visits += dda_walk(p->n, S, D, (p->literal & OR_LIT_SKIP_START) != 0, ray_visit, &R);
    }
    return visits;
}

void or_resolve(int64_t nvox, uint32_t literal, const uint8_t *occ_inf, const uint8_t *fr,
                const uint8_t *tr, uint8_t *ms) {
    /* Precedence occupied > free > traced > unknown: a voxel any ray saw
     * free before its obstacle is free (reading of the concurrent-write
     * remark of Sec. IV-C).  In the loc_grid reading the rays do not see
     * this measurement's occupied voxels and Alg. 2's writes replace them:
     * free > traced > occupied > unknown. */
    const int rays_last = (literal & OR_LIT_LOC_OCCUPANCY) != 0;
    for (int64_t i = 0; i < nvox; ++i) {
        if (occ_inf[i] && !rays_last) ms[i] = OR_OCC;
        else if (fr[i]) ms[i] = OR_FREE;
        else if (tr[i]) ms[i] = OR_TRACED;
        else if (occ_inf[i]) ms[i] = OR_OCC;
        else ms[i] = OR_UNK;
    }
}

void or_merge(int64_t nvox, const uint8_t *ms, uint8_t *loc) {
    for (int64_t i = 0; i < nvox; ++i)
        if (ms[i] != OR_UNK) loc[i] = ms[i];
}

void or_shift(const int32_t n[3], const int32_t delta[3], const uint8_t *src,
              uint8_t *dst) {
    for (int32_t z = 0; z < n[2]; ++z)
        for (int32_t y = 0; y < n[1]; ++y)
            for (int32_t x = 0; x < n[0]; ++x) {
                int32_t sx = x + delta[0], sy = y + delta[1], sz = z + delta[2];
                dst[lin(n, x, y, z)] =
                    in_grid(n, sx, sy, sz) ? src[lin(n, sx, sy, sz)] : (uint8_t)OR_UNK;
            }
}

/* Steps 2-4 of Sec. IV after the occupied voxels are in occ_raw. */
static int finish_frame(const or_params *p, const or_pose *T, uint8_t *occ_raw,
                        uint8_t *loc, uint8_t *ms_out) {
    int64_t nv = nvox_of(p->n);
    uint8_t *occ_inf = (uint8_t *)calloc((size_t)nv, 1);
    uint8_t *fr = (uint8_t *)calloc((size_t)nv, 1);
    uint8_t *tr = (uint8_t *)calloc((size_t)nv, 1);
    uint8_t *ms = (uint8_t *)calloc((size_t)nv, 1);
    int rc = -1;
    if (occ_inf && fr && tr && ms) {
        or_inflate(p, occ_raw, occ_inf);
        /* the grid the rays test: Alg. 1's order (inflated), the kernel
         * list's order (raw), or Alg. 2's literal loc_grid (the grid before
         * this measurement; the ms scratch holds it until the resolve) */
        const uint8_t *tested = occ_inf;
        if (p->literal & OR_LIT_INFLATE_AFTER_TRACE) tested = occ_raw;
        if (p->literal & OR_LIT_LOC_OCCUPANCY) {
            for (int64_t i = 0; i < nv; ++i) ms[i] = loc[i] == OR_OCC;
            tested = ms;
        }
        or_raytrace(p, T, tested, NULL, fr, tr);
        or_resolve(nv, p->literal, occ_inf, fr, tr, ms);
        or_merge(nv, ms, loc);
        if (ms_out) memcpy(ms_out, ms, (size_t)nv);
        rc = 0;
    }
    free(occ_inf);
    free(fr);
    free(tr);
    free(ms);
    return rc;
}

int or_integrate_depth(const or_params *p, const int32_t o[3], const double T_wc[16],
                       const void *depth, int32_t W, int32_t H, int32_t dtype,
                       float scale, uint8_t *loc, uint8_t *ms_out) {
    or_pose T;
    or_pose_vc(p, T_wc, o, &T);
    uint8_t *occ_raw = (uint8_t *)calloc((size_t)nvox_of(p->n), 1);
    if (!occ_raw) return -1;
    or_voxelize_depth(p, &T, depth, W, H, dtype, scale, occ_raw);
    int rc = finish_frame(p, &T, occ_raw, loc, ms_out);
    free(occ_raw);
    return rc;
}

int or_integrate_points(const or_params *p, const int32_t o[3], const double T_wc[16],
                        const float *xyz, int64_t n, uint8_t *loc, uint8_t *ms_out) {
    or_pose T;
    or_pose_vc(p, T_wc, o, &T);
    uint8_t *occ_raw = (uint8_t *)calloc((size_t)nvox_of(p->n), 1);
    if (!occ_raw) return -1;
    or_voxelize_points(p, &T, xyz, n, occ_raw);
    int rc = finish_frame(p, &T, occ_raw, loc, ms_out);
    free(occ_raw);
    return rc;
}
