/*
 * render.c -- seeded synthetic depth images for the voxel-grid workloads.
 *
 * Casts one ray per pixel through an analytic scene of axis-aligned boxes,
 * spheres, vertical cylinders and an enclosing room, and writes z-depth in
 * the camera optical frame (x right, y down, z forward), 0 where nothing is
 * hit within max_t.  This is the stand-in for the simulator's depth camera;
 * it holds none of the voxel-grid method's arithmetic and serves the CPU
 * oracle and the CUDA path alike.  Double precision throughout.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

enum { SY_BOX = 0, SY_SPHERE = 1, SY_CYL = 2, SY_ROOM = 3 };

/* box/room: p = lo xyz, hi xyz; sphere: p = c xyz, r;
 * cylinder (axis along z): p = cx, cy, zlo, zhi, r */
typedef struct {
    int32_t type;
    int32_t pad;
    double p[6];
} sy_prim;

#define TILE 16
#define EPS_T 1e-6

static double hit_box(const double o[3], const double d[3], const double lo[3],
                      const double hi[3], int inside_wanted) {
    double tn = -INFINITY, tf = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < lo[k] || o[k] > hi[k]) return INFINITY;
            continue;
        }
        double a = (lo[k] - o[k]) / d[k], b = (hi[k] - o[k]) / d[k];
        if (a > b) { double t = a; a = b; b = t; }
        if (a > tn) tn = a;
        if (b < tf) tf = b;
    }
    if (tn > tf) return INFINITY;
    if (inside_wanted) return tf > EPS_T ? tf : INFINITY;
    return tn > EPS_T ? tn : INFINITY;
}

static double hit_sphere(const double o[3], const double d[3], const double *p) {
    double oc[3] = {o[0] - p[0], o[1] - p[1], o[2] - p[2]};
    double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - p[3] * p[3];
    double disc = b * b - a * c;
    if (disc < 0) return INFINITY;
    double s = sqrt(disc);
    double t = (-b - s) / a;
    if (t > EPS_T) return t;
    return INFINITY;
}

static double hit_cyl(const double o[3], const double d[3], const double *p) {
    double best = INFINITY;
    double ox = o[0] - p[0], oy = o[1] - p[1];
    double a = d[0] * d[0] + d[1] * d[1];
    if (a > 0) {
        double b = ox * d[0] + oy * d[1];
        double c = ox * ox + oy * oy - p[4] * p[4];
        double disc = b * b - a * c;
        if (disc >= 0) {
            double t = (-b - sqrt(disc)) / a;
            double z = o[2] + t * d[2];
            if (t > EPS_T && z >= p[2] && z <= p[3]) best = t;
        }
    }
    if (d[2] != 0) {
        for (int e = 2; e <= 3; ++e) {
            double t = (p[e] - o[2]) / d[2];
            if (t > EPS_T && t < best) {
                double x = ox + t * d[0], y = oy + t * d[1];
                if (x * x + y * y <= p[4] * p[4]) best = t;
            }
        }
    }
    return best;
}

static double hit_prim(const sy_prim *q, const double o[3], const double d[3]) {
    switch (q->type) {
    case SY_BOX: return hit_box(o, d, q->p, q->p + 3, 0);
    case SY_ROOM: return hit_box(o, d, q->p, q->p + 3, 1);
    case SY_SPHERE: return hit_sphere(o, d, q->p);
    case SY_CYL: return hit_cyl(o, d, q->p);
    default: return INFINITY;
    }
}

static void prim_aabb(const sy_prim *q, double lo[3], double hi[3]) {
    if (q->type == SY_BOX || q->type == SY_ROOM) {
        for (int k = 0; k < 3; ++k) { lo[k] = q->p[k]; hi[k] = q->p[3 + k]; }
    } else if (q->type == SY_SPHERE) {
        for (int k = 0; k < 3; ++k) { lo[k] = q->p[k] - q->p[3]; hi[k] = q->p[k] + q->p[3]; }
    } else {
        lo[0] = q->p[0] - q->p[4]; hi[0] = q->p[0] + q->p[4];
        lo[1] = q->p[1] - q->p[4]; hi[1] = q->p[1] + q->p[4];
        lo[2] = q->p[2]; hi[2] = q->p[3];
    }
}

/* Screen rectangle [u0,u1] x [v0,v1] (inclusive) a primitive can cover; the
 * whole image when part of its box is behind the camera. */
static void prim_rect(const sy_prim *q, const double T[16], int W, int H, double fx,
                      double fy, double cx, double cy, int r[4]) {
    double lo[3], hi[3];
    prim_aabb(q, lo, hi);
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int c = 0; c < 8; ++c) {
        double w[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
        double rel[3] = {w[0] - T[3], w[1] - T[7], w[2] - T[11]};
        /* camera coordinates: R^T (w - t), R columns are T[0,4,8], T[1,5,9], T[2,6,10] */
        double xc = T[0] * rel[0] + T[4] * rel[1] + T[8] * rel[2];
        double yc = T[1] * rel[0] + T[5] * rel[1] + T[9] * rel[2];
        double zc = T[2] * rel[0] + T[6] * rel[1] + T[10] * rel[2];
        if (zc <= 1e-3) {
            r[0] = 0; r[1] = W - 1; r[2] = 0; r[3] = H - 1;
            return;
        }
        double u = cx + fx * xc / zc, v = cy + fy * yc / zc;
        if (u < umin) umin = u;
        if (u > umax) umax = u;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
    }
    double u0 = floor(umin) - 1, u1 = ceil(umax) + 1, v0 = floor(vmin) - 1, v1 = ceil(vmax) + 1;
    r[0] = u0 < 0 ? 0 : (u0 > W - 1 ? W : (int)u0);
    r[1] = u1 > W - 1 ? W - 1 : (u1 < 0 ? -1 : (int)u1);
    r[2] = v0 < 0 ? 0 : (v0 > H - 1 ? H : (int)v0);
    r[3] = v1 > H - 1 ? H - 1 : (v1 < 0 ? -1 : (int)v1);
}

/* Render one W x H z-depth image.  T_wc: row-major 4x4 camera-to-world.
 * Returns 0, or -1 if scratch memory could not be allocated. */
int sy_render(const sy_prim *prims, int32_t nprims, const double T_wc[16], int32_t W,
              int32_t H, double fx, double fy, double cx, double cy, double max_t,
              float *out) {
    int tw = (W + TILE - 1) / TILE, th = (H + TILE - 1) / TILE, nt = tw * th;
    int *count = (int *)calloc((size_t)nt + 1, sizeof(int));
    int (*rect)[4] = (int (*)[4])malloc(sizeof(int[4]) * (size_t)(nprims > 0 ? nprims : 1));
    if (!count || !rect) { free(count); free(rect); return -1; }
    for (int i = 0; i < nprims; ++i) {
        prim_rect(&prims[i], T_wc, W, H, fx, fy, cx, cy, rect[i]);
        for (int ty = rect[i][2] / TILE; rect[i][3] >= rect[i][2] && ty <= rect[i][3] / TILE; ++ty)
            for (int tx = rect[i][0] / TILE; rect[i][1] >= rect[i][0] && tx <= rect[i][1] / TILE; ++tx)
                count[ty * tw + tx + 1]++;
    }
    for (int t = 0; t < nt; ++t) count[t + 1] += count[t];
    int *list = (int *)malloc(sizeof(int) * (size_t)(count[nt] > 0 ? count[nt] : 1));
    int *fill = (int *)calloc((size_t)nt, sizeof(int));
    if (!list || !fill) { free(count); free(rect); free(list); free(fill); return -1; }
    for (int i = 0; i < nprims; ++i) {
        for (int ty = rect[i][2] / TILE; rect[i][3] >= rect[i][2] && ty <= rect[i][3] / TILE; ++ty)
            for (int tx = rect[i][0] / TILE; rect[i][1] >= rect[i][0] && tx <= rect[i][1] / TILE; ++tx) {
                int t = ty * tw + tx;
                list[count[t] + fill[t]++] = i;
            }
    }
    const double o[3] = {T_wc[3], T_wc[7], T_wc[11]};
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            double dc[3] = {((double)u - cx) / fx, ((double)v - cy) / fy, 1.0};
            double d[3];
            for (int k = 0; k < 3; ++k)
                d[k] = T_wc[4 * k + 0] * dc[0] + T_wc[4 * k + 1] * dc[1] + T_wc[4 * k + 2] * dc[2];
            int t = (v / TILE) * tw + (u / TILE);
            double best = INFINITY;
            for (int j = count[t]; j < count[t + 1]; ++j) {
                double h = hit_prim(&prims[list[j]], o, d);
                if (h < best) best = h;
            }
            out[(int64_t)v * W + u] = (best <= max_t) ? (float)best : 0.0f;
        }
    }
    free(count); free(rect); free(list); free(fill);
    return 0;
}
