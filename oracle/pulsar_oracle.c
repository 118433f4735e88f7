/*
 * Pulsar reference renderer (the oracle): TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, brute-force CPU statement of what the differentiable sphere
 * renderer of Lassner & Zollhoefer (arXiv 2004.07484) computes.  For every
 * pixel it loops over every sphere.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The CUDA
 * product path never calls it, and the two share no code.
 *
 * Precision.  Values (weights, image, gradients) are computed in IEEE double
 * from the float32 inputs (widened exactly).  The discrete decisions that must
 * match the GPU bit for bit are made by a separate float32 routine:
 *   - the camera-space centre and the effective radius,
 *   - culling, the enclosing rectangle and the sort key,
 *   - the per-pixel hit predicate and the hit depth that orders hits.
 * That routine uses only correctly rounded IEEE operations (+ - * / sqrt and
 * fused multiply-add) in a fixed order.  Compile with -ffp-contract=off so the
 * compiler adds no fusion of its own.
 *
 * Model (Sec. 3.1, Sec. 3.2 with Eq. 1, Appendix A, Appendix B; the readings
 * taken where the paper is silent are listed in the design notes):
 *   scene       S = {(p_i, f_i, r_i, o_i)}, i < M                 (Sec. 3.1)
 *   camera      cam = [t(3), a1(3), a2(3), focal, sensor_width]   (Listing 1 order,
 *               6D rotation of Zhou et al. as Listing 1's text states)
 *   rotation    b1 = a1/|a1|, b2 = unit(a2 - (b1.a2) b1), b3 = b1 x b2;
 *               b1, b2, b3 are the camera's x, y, z axes in world space, so
 *               the camera-space centre is c = (b1.(p-t), b2.(p-t), b3.(p-t)).
 *   pinhole     pixel (u, v) has the ray (rho_x, rho_y, 1) with
 *               rho = ((u + 1/2 - W/2) k, (v + 1/2 - H/2) k), k = s / (W f).
 *   orthographic (option; Sec. 1: "pinhole and orthogonal camera model")
 *               pixel (u, v) has the ray from (rho_x, rho_y, 0) along +z,
 *               with k = s / W (the sensor width in scene units across the
 *               image; the focal length does not enter).  Everything below
 *               then holds for the shifted centre c' = c - (rho_x, rho_y, 0)
 *               and the ray (0, 0, 1); the minimum size is R = max(r, 0.75 k)
 *               and the rectangle is the centre -+ R in pixels (+- 1/8).
 *   min size    every sphere is drawn with at least one pixel (App. B,
 *               Step 0): R = max(r, 0.75 |c| k).
 *   depth       z = (zfar - t_h) / (zfar - znear) in [0, 1], 0 = max depth
 *               (Sec. 3.2), t_h = camera-space z of the front intersection.
 *   distance    d = 1 - min(1, dist/R) by default; d = min(1, dist/R) with
 *               dist_literal set (Sec. 3.2 prints the latter).
 *   blending    w_i = o_i d_i e^{o_i z_i / g} / (e^{eps/g} + sum_k o_k d_k e^{o_k z_k / g})
 *               (Eq. 1); F = sum_i w_i f_i + w_B bg with w_B = e^{eps/g} / D.
 *   tracking    the n_track hits closest to the camera (smallest t_h, ties by
 *               sphere index) are kept for the backward pass (App. B, Step 2
 *               and "Preparing for the Backward Pass"); all hits contribute to
 *               the image; gradients flow through the tracked hits only.
 *   paper       optional gradient normalisations of App. B (end of "The
 *   gradients   Backward Pass") and Sec. 3.2 / Sec. 6: every sphere gradient
 *               is divided by n_i, the number of pixels at which sphere i is
 *               a tracked hit; position and radius gradients are zero unless
 *               the sphere's projected radius R / (c_z k) exceeds 3 pixels
 *               (float32 decision); the camera gradient is the sum over
 *               spheres of the averaged per-sphere terms weighted by the
 *               sphere's area, taken as n_i pixels, times 1e-3 -- that is,
 *               1e-3 times the plain camera gradient.  The background
 *               gradient is unchanged.
 *   paper stop  optional early termination of App. B, Step 2 (the paper's
 *               default, an approximation): a pixel takes its hits in the tile
 *               list's order (sort key c_z - R, then index) and stops before
 *               the first whose largest possible weight e^{o_max z_b / g} /
 *               (D + e^{o_max z_b / g}) is below min_contrib (the paper's
 *               "n percent", 1 % by default), z_b the depth term of its key,
 *               o_max the largest opacity of the scene's visible spheres and D
 *               the denominator of the hits taken so far; blending and
 *               tracking see only the hits taken.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

typedef struct {
  int32_t width, height;
  int32_t n_spheres, n_channels;
  int32_t n_track;       /* number of closest hits kept for the backward pass */
  int32_t tile;          /* edge length of the square screen tiles of the tile lists */
  int32_t min_size;      /* 1: apply the one-pixel minimum size rule */
  int32_t dist_literal;  /* 1: d = min(1, dist/R) instead of 1 - min(1, dist/R) */
  int32_t paper_grad;    /* 1: the paper's gradient normalisations (header) */
  int32_t ortho;         /* 1: orthographic camera (header) */
  int32_t paper_stop;    /* 1: the paper's early termination (header) */
  double gamma, eps, znear, zfar;
  double min_contrib;    /* its threshold as a fraction (the paper's n percent; 0.01 by default) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* float32 decision path                                                      */
/* ------------------------------------------------------------------------ */

/* Gram-Schmidt of the 6D rotation vector in float32, fixed operation order. */
static void rows_f32(const float a[6], float B[9]) {
  float n1 = sqrtf(fmaf(a[0], a[0], fmaf(a[1], a[1], a[2] * a[2])));
  float b1x = a[0] / n1, b1y = a[1] / n1, b1z = a[2] / n1;
  float dt = fmaf(b1x, a[3], fmaf(b1y, a[4], b1z * a[5]));
  float ux = fmaf(-dt, b1x, a[3]);
  float uy = fmaf(-dt, b1y, a[4]);
  float uz = fmaf(-dt, b1z, a[5]);
  float n2 = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  float b2x = ux / n2, b2y = uy / n2, b2z = uz / n2;
  B[0] = b1x; B[1] = b1y; B[2] = b1z;
  B[3] = b2x; B[4] = b2y; B[5] = b2z;
  B[6] = fmaf(b1y, b2z, -(b1z * b2y));
  B[7] = fmaf(b1z, b2x, -(b1x * b2z));
  B[8] = fmaf(b1x, b2y, -(b1y * b2x));
}

typedef struct {
  float cx, cy, cz;   /* camera-space centre */
  float R, R2;        /* effective radius and its square */
  float tmin;         /* c_z - R: no point of the sphere is nearer */
  float key;          /* earliest possible intersection depth, +inf when culled */
  int visible;
  int x0, x1, y0, y1; /* inclusive pixel rectangle, valid when visible */
} proj32;

static float kappa_f32(const float* cam, int width, int ortho) {
  return ortho ? cam[10] / (float)width : cam[10] / ((float)width * cam[9]);
}

/* One axis of the enclosing rectangle.  In the (axis, z) plane the sphere is a
 * disk of radius R about (cx, cz); the tangent lines through the eye have the
 * slopes m = (cx cz -+ R sqrt(cx^2 + cz^2 - R^2)) / (cz^2 - R^2).  The pixels
 * whose centres lie between them, with the bounds widened by 1/8 pixel on
 * each side against rounding (App. B, Step 0: the bounds are made robust to
 * numerical inaccuracy; the float32 hit predicate's boundary lies within
 * ~1e-4 pixel of the exact one), contain every pixel whose ray meets the
 * sphere. */
static void axis_range_f32(float cx, float cz, float R, float R2, float kappa, int n,
                           int* lo, int* hi) {
  float den = fmaf(cz, cz, -R2);
  float disc = fmaf(cx, cx, den);
  float root = sqrtf(disc);
  float base = cx * cz;
  float rs = R * root;
  float mlo = (base - rs) / den;
  float mhi = (base + rs) / den;
  float half = (float)(n - 1) * 0.5f;
  float flo = mlo / kappa + half;
  float fhi = mhi / kappa + half;
  flo = fmaxf(fminf(flo, (float)n + 2.0f), -4.0f);
  fhi = fmaxf(fminf(fhi, (float)n + 2.0f), -4.0f);
  *lo = (int)ceilf(flo - 0.125f);
  *hi = (int)floorf(fhi + 0.125f);
}

/* One axis of the rectangle of the orthographic camera: the centre -+ R in
 * pixels, widened by 1/8 pixel on each side. */
static void axis_range_ortho_f32(float cx, float R, float kappa, int n, int* lo, int* hi) {
  float half = (float)(n - 1) * 0.5f;
  float flo = (cx - R) / kappa + half;
  float fhi = (cx + R) / kappa + half;
  flo = fmaxf(fminf(flo, (float)n + 2.0f), -4.0f);
  fhi = fmaxf(fminf(fhi, (float)n + 2.0f), -4.0f);
  *lo = (int)ceilf(flo - 0.125f);
  *hi = (int)floorf(fhi + 0.125f);
}

static void project_f32(const orc_params* P, const float* cam, const float B[9],
                        const float p[3], float r, proj32* o) {
  float kappa = kappa_f32(cam, P->width, P->ortho);
  float dx = p[0] - cam[0], dy = p[1] - cam[1], dz = p[2] - cam[2];
  o->cx = fmaf(B[0], dx, fmaf(B[1], dy, B[2] * dz));
  o->cy = fmaf(B[3], dx, fmaf(B[4], dy, B[5] * dz));
  o->cz = fmaf(B[6], dx, fmaf(B[7], dy, B[8] * dz));
  float R = r;
  if (P->min_size) {
    float rmin;
    if (P->ortho) {
      rmin = 0.75f * kappa;
    } else {
      float cn = sqrtf(fmaf(o->cx, o->cx, fmaf(o->cy, o->cy, o->cz * o->cz)));
      rmin = 0.75f * (cn * kappa);
    }
    if (rmin > r) R = rmin;
  }
  o->R = R;
  o->R2 = R * R;
  o->key = INFINITY;
  o->visible = 0;
  o->x0 = o->x1 = o->y0 = o->y1 = -1;
  float key = o->cz - R;
  o->tmin = key;
  float znear = (float)P->znear, zfar = (float)P->zfar;
  if (!(R > 0.0f) || !(key > znear) || !(key < zfar)) return;
  int x0, x1, y0, y1;
  if (P->ortho) {
    axis_range_ortho_f32(o->cx, R, kappa, P->width, &x0, &x1);
    axis_range_ortho_f32(o->cy, R, kappa, P->height, &y0, &y1);
  } else {
    axis_range_f32(o->cx, o->cz, R, o->R2, kappa, P->width, &x0, &x1);
    axis_range_f32(o->cy, o->cz, R, o->R2, kappa, P->height, &y0, &y1);
  }
  if (x1 < 0 || x0 > P->width - 1 || y1 < 0 || y0 > P->height - 1) return;
  o->x0 = x0 < 0 ? 0 : x0;
  o->x1 = x1 > P->width - 1 ? P->width - 1 : x1;
  o->y0 = y0 < 0 ? 0 : y0;
  o->y1 = y1 > P->height - 1 ? P->height - 1 : y1;
  o->key = key;
  o->visible = 1;
}

static float ray_coord_f32(int u, int n, float kappa) {
  return ((float)(2 * u + 1 - n) * 0.5f) * kappa;
}

/* Hit predicate and front-hit depth in float32.  Returns 1 and writes t_h
 * when the ray (rx, ry, 1) meets the sphere in front of zfar.  The depth is
 * never taken nearer than c_z - R, which holds exactly in real arithmetic;
 * in float32 the clamp keeps every hit depth at or beyond the sphere's sort
 * key, the property that depth-ordered early termination relies on. */
static int hit_f32(const proj32* s, float rx, float ry, float zfar, float* t_out) {
  float ex = fmaf(s->cz, rx, -s->cx);
  float ey = fmaf(s->cz, ry, -s->cy);
  float ez = fmaf(s->cx, ry, -(s->cy * rx));
  float cr2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
  float rr = fmaf(rx, rx, fmaf(ry, ry, 1.0f));
  float disc = fmaf(rr, s->R2, -cr2);
  if (!(disc > 0.0f)) return 0;
  float off = fmaf(rx, ex, fmaf(ry, ey, sqrtf(disc))) / rr;
  float t = s->cz - off;
  if (t < s->tmin) t = s->tmin;
  if (!(t < zfar)) return 0;
  *t_out = t;
  return 1;
}

/* The hit predicate of either camera: the orthographic ray from
 * (rho_x, rho_y, 0) along +z is the pinhole test of the shifted centre
 * c - (rho_x, rho_y, 0) with the ray (0, 0, 1). */
static int hit_px(const orc_params* P, const proj32* s, float rx, float ry, float zfar, float* t_out) {
  if (!P->ortho) return hit_f32(s, rx, ry, zfar, t_out);
  proj32 q = *s;
  q.cx = s->cx - rx;
  q.cy = s->cy - ry;
  return hit_f32(&q, 0.0f, 0.0f, zfar, t_out);
}

/* ------------------------------------------------------------------------ */
/* double value path                                                          */
/* ------------------------------------------------------------------------ */

static void rows_f64(const double a[6], double B[9]) {
  double n1 = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double b1[3] = {a[0] / n1, a[1] / n1, a[2] / n1};
  double dt = b1[0] * a[3] + b1[1] * a[4] + b1[2] * a[5];
  double u[3] = {a[3] - dt * b1[0], a[4] - dt * b1[1], a[5] - dt * b1[2]};
  double n2 = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double b2[3] = {u[0] / n2, u[1] / n2, u[2] / n2};
  B[0] = b1[0]; B[1] = b1[1]; B[2] = b1[2];
  B[3] = b2[0]; B[4] = b2[1]; B[5] = b2[2];
  B[6] = b1[1] * b2[2] - b1[2] * b2[1];
  B[7] = b1[2] * b2[0] - b1[0] * b2[2];
  B[8] = b1[0] * b2[1] - b1[1] * b2[0];
}

/* The same map over complex numbers, for complex-step derivatives of the
 * rotation rows with respect to the 6D vector. */
static void rows_c(const double complex a[6], double complex B[9]) {
  double complex n1 = csqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double complex b1[3] = {a[0] / n1, a[1] / n1, a[2] / n1};
  double complex dt = b1[0] * a[3] + b1[1] * a[4] + b1[2] * a[5];
  double complex u[3] = {a[3] - dt * b1[0], a[4] - dt * b1[1], a[5] - dt * b1[2]};
  double complex n2 = csqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double complex b2[3] = {u[0] / n2, u[1] / n2, u[2] / n2};
  B[0] = b1[0]; B[1] = b1[1]; B[2] = b1[2];
  B[3] = b2[0]; B[4] = b2[1]; B[5] = b2[2];
  B[6] = b1[1] * b2[2] - b1[2] * b2[1];
  B[7] = b1[2] * b2[0] - b1[0] * b2[2];
  B[8] = b1[0] * b2[1] - b1[1] * b2[0];
}

typedef struct {
  int id;
  float t32;
  float key;      /* the sphere's sort key (tile-list order) */
} hit_rec;

static int hit_cmp(const void* a, const void* b) {
  const hit_rec* x = (const hit_rec*)a;
  const hit_rec* y = (const hit_rec*)b;
  if (x->t32 < y->t32) return -1;
  if (x->t32 > y->t32) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* Per-sphere quantities of the value path. */
typedef struct {
  double c[3];      /* camera-space centre */
  double R;         /* effective radius */
  int clamped;      /* 1 when the minimum-size radius replaced r */
} sph64;

typedef struct {
  /* inputs widened to double */
  const double *pos, *rad, *opa, *feat, *cam, *bg;
  double B[9];
  double kappa;
  float camf[11];
  float Bf[9];
  float kappaf;
  double omax;      /* largest |opacity| of the visible spheres (float32 values) */
  proj32* pj;
  sph64* sv;
} ctx_t;

/* dpos/drad/dcam, when not NULL, are the inputs of the float32 decisions;
 * otherwise the value inputs are used.  Finite differences pass the
 * unperturbed inputs here so that the set of hits stays fixed. */
static void ctx_init(const orc_params* P, const double* pos, const double* rad,
                     const double* cam, const double* dpos, const double* drad,
                     const double* dcam, ctx_t* C) {
  int M = P->n_spheres;
  if (!dpos) dpos = pos;
  if (!drad) drad = rad;
  if (!dcam) dcam = cam;
  for (int k = 0; k < 11; ++k) C->camf[k] = (float)dcam[k];
  rows_f32(C->camf + 3, C->Bf);
  C->kappaf = kappa_f32(C->camf, P->width, P->ortho);
  rows_f64(cam + 3, C->B);
  C->kappa = P->ortho ? cam[10] / (double)P->width : cam[10] / ((double)P->width * cam[9]);
  C->pj = (proj32*)malloc(sizeof(proj32) * (size_t)(M > 0 ? M : 1));
  C->sv = (sph64*)malloc(sizeof(sph64) * (size_t)(M > 0 ? M : 1));
  for (int i = 0; i < M; ++i) {
    float pf[3] = {(float)dpos[3 * i], (float)dpos[3 * i + 1], (float)dpos[3 * i + 2]};
    project_f32(P, C->camf, C->Bf, pf, (float)drad[i], &C->pj[i]);
    double d[3] = {pos[3 * i] - cam[0], pos[3 * i + 1] - cam[1], pos[3 * i + 2] - cam[2]};
    sph64* s = &C->sv[i];
    for (int k = 0; k < 3; ++k)
      s->c[k] = C->B[3 * k] * d[0] + C->B[3 * k + 1] * d[1] + C->B[3 * k + 2] * d[2];
    /* the branch of the minimum-size rule is a decision: take it from float32 */
    s->clamped = P->min_size && (C->pj[i].R != (float)drad[i]);
    double cn = sqrt(s->c[0] * s->c[0] + s->c[1] * s->c[1] + s->c[2] * s->c[2]);
    s->R = s->clamped ? (P->ortho ? 0.75 * C->kappa : 0.75 * cn * C->kappa) : rad[i];
  }
  C->omax = 0.0;
  if (C->opa)
    for (int i = 0; i < M; ++i)
      if (C->pj[i].visible && fabs((double)(float)C->opa[i]) > C->omax) C->omax = fabs((double)(float)C->opa[i]);
}

static void ctx_free(ctx_t* C) {
  free(C->pj);
  free(C->sv);
}

/* Textbook ray/sphere quantities in double for ray r = (rx, ry, 1):
 *   b = r.c, rr = r.r, q = |c|^2 - R^2, disc = b^2 - rr q,
 *   t = (b - sqrt(disc)) / rr (front root), dist^2 = |c|^2 - b^2 / rr. */
typedef struct {
  double r[3], b, rr, q, disc, sq, t, dist, z, d, s, dq;
  double cs[3];   /* the centre the ray meets: c, or c - (rho_x, rho_y, 0) orthographic */
} rayq;

static void ray_values(const orc_params* P, const sph64* s, double rx, double ry, rayq* o) {
  if (P->ortho) {   /* ray from (rx, ry, 0) along +z: shifted centre, ray (0, 0, 1) */
    o->cs[0] = s->c[0] - rx;
    o->cs[1] = s->c[1] - ry;
    rx = ry = 0.0;
  } else {
    o->cs[0] = s->c[0];
    o->cs[1] = s->c[1];
  }
  o->cs[2] = s->c[2];
  o->r[0] = rx; o->r[1] = ry; o->r[2] = 1.0;
  const double* c = o->cs;
  double cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
  o->b = rx * c[0] + ry * c[1] + c[2];
  o->rr = rx * rx + ry * ry + 1.0;
  o->q = cc - s->R * s->R;
  o->disc = o->b * o->b - o->rr * o->q;
  if (o->disc < 0.0) o->disc = 0.0;
  o->sq = sqrt(o->disc);
  o->t = (o->b - o->sq) / o->rr;
  double d2 = cc - o->b * o->b / o->rr;
  o->dist = d2 > 0.0 ? sqrt(d2) : 0.0;
  o->z = (P->zfar - o->t) / (P->zfar - P->znear);
  o->dq = o->dist / s->R;
  if (o->dq > 1.0) o->dq = 1.0;
  o->d = P->dist_literal ? o->dq : 1.0 - o->dq;
}

/* Order of the tile lists: sort key, then index. */
static int hit_key_cmp(const void* a, const void* b) {
  const hit_rec* x = (const hit_rec*)a;
  const hit_rec* y = (const hit_rec*)b;
  float kx = x->key, ky = y->key;
  if (kx < ky) return -1;
  if (kx > ky) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

static void ray_values(const orc_params* P, const sph64* s, double rx, double ry, rayq* o);

/* The paper's early termination: keeps the hits (in tile-list order) before
 * the first whose largest possible weight is below 1 % (header).  The hits
 * come in and go out ordered by (key, index).  With margin != NULL, *margin
 * receives the smallest |ln(a / tau)| over the tests taken, a the tested
 * largest possible weight: how far the pixel's decisions are from the
 * threshold (a renderer that accumulates D in another precision can decide
 * otherwise only where this is small). */
static int paper_stop_filter(const orc_params* P, const ctx_t* C, int u, int v, hit_rec* hits, int n,
                             double* margin) {
  const double tau = P->min_contrib, g = P->gamma, zr = P->zfar - P->znear;
  double rx = (double)(2 * u + 1 - P->width) * 0.5 * C->kappa;
  double ry = (double)(2 * v + 1 - P->height) * 0.5 * C->kappa;
  double m = P->eps / g, den = 1.0;   /* the background term alone, shifted by its own exponent */
  for (int j = 0; j < n; ++j) {
    int i = hits[j].id;
    double zb = (P->zfar - (double)C->pj[i].key) / zr;
    double amax = exp(C->omax * zb / g - m);
    double a = amax / (den + amax);
    if (margin) {
      double mg = fabs(log(a / tau));
      if (mg < *margin) *margin = mg;
    }
    if (a < tau) return j;
    rayq q;
    ray_values(P, &C->sv[i], rx, ry, &q);
    double s = C->opa[i] * q.z / g;
    if (s > m) {
      den *= exp(m - s);
      m = s;
    }
    den += C->opa[i] * q.d * exp(s - m);
  }
  return n;
}

/* Collect and order the hits of one pixel.  Returns the hit count. */
static int pixel_hits_m(const orc_params* P, const ctx_t* C, int u, int v, hit_rec* hits, double* margin) {
  int M = P->n_spheres, n = 0;
  float rx = ray_coord_f32(u, P->width, C->kappaf);
  float ry = ray_coord_f32(v, P->height, C->kappaf);
  for (int i = 0; i < M; ++i) {
    if (!C->pj[i].visible) continue;
    float t;
    if (hit_px(P, &C->pj[i], rx, ry, (float)P->zfar, &t)) {
      hits[n].id = i;
      hits[n].t32 = t;
      hits[n].key = C->pj[i].key;
      ++n;
    }
  }
  if (P->paper_stop && n > 0) {
    qsort(hits, (size_t)n, sizeof(hit_rec), hit_key_cmp);
    n = paper_stop_filter(P, C, u, v, hits, n, margin);
  }
  qsort(hits, (size_t)n, sizeof(hit_rec), hit_cmp);
  return n;
}

static int pixel_hits(const orc_params* P, const ctx_t* C, int u, int v, hit_rec* hits) {
  return pixel_hits_m(P, C, u, v, hits, NULL);
}

/* Blend one pixel by Eq. 1.  Writes F (C values) and returns log D, where
 * D = e^{eps/g} + sum_k o_k d_k e^{o_k z_k / g}.  The common factor e^{-m},
 * m the largest exponent, is divided out of numerator and denominator. */
static double blend_pixel(const orc_params* P, const ctx_t* C, int u, int v,
                          const hit_rec* hits, int n, double* F, double* wsum_out) {
  int Cn = P->n_channels;
  double rx = (double)(2 * u + 1 - P->width) * 0.5 * C->kappa;
  double ry = (double)(2 * v + 1 - P->height) * 0.5 * C->kappa;
  double sB = P->eps / P->gamma, m = sB;
  double* sarr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* darr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) {
    rayq q;
    int i = hits[j].id;
    ray_values(P, &C->sv[i], rx, ry, &q);
    sarr[j] = C->opa[i] * q.z / P->gamma;
    darr[j] = q.d;
    if (sarr[j] > m) m = sarr[j];
  }
  double D = exp(sB - m), wsum = 0.0;
  for (int c = 0; c < Cn; ++c) F[c] = D * C->bg[c];
  for (int j = 0; j < n; ++j) {
    int i = hits[j].id;
    double a = C->opa[i] * darr[j] * exp(sarr[j] - m);
    D += a;
    wsum += a;
    for (int c = 0; c < Cn; ++c) F[c] += a * C->feat[(size_t)i * Cn + c];
  }
  for (int c = 0; c < Cn; ++c) F[c] /= D;
  if (wsum_out) *wsum_out = wsum / D;
  free(sarr);
  free(darr);
  return m + log(D);
}

/* ------------------------------------------------------------------------ */
/* exported entry points                                                      */
/* ------------------------------------------------------------------------ */

/* Step 0 decisions in float32 (App. B, Step 0): per sphere the camera-space
 * centre, effective radius, sort key (+inf when culled) and the inclusive
 * pixel rectangle (-1 when culled). */
void orc_project(const orc_params* P, const double* pos, const double* rad, const double* cam,
                 float* c_out, float* r_out, float* key_out, int32_t* rect_out) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  ctx_init(P, pos, rad, cam, NULL, NULL, NULL, &C);
  for (int i = 0; i < P->n_spheres; ++i) {
    const proj32* s = &C.pj[i];
    c_out[3 * i] = s->cx; c_out[3 * i + 1] = s->cy; c_out[3 * i + 2] = s->cz;
    r_out[i] = s->R;
    key_out[i] = s->key;
    rect_out[4 * i] = s->x0; rect_out[4 * i + 1] = s->x1;
    rect_out[4 * i + 2] = s->y0; rect_out[4 * i + 3] = s->y1;
  }
  ctx_free(&C);
}

/* Per-tile sphere lists by definition: tile (tx, ty) of edge T lists every
 * visible sphere whose rectangle overlaps it, ordered by (key, index).
 * offsets has n_tiles + 1 entries.  Returns the total length, or -1 when it
 * exceeds capacity (offsets are still written). */
static const float* g_sort_keys;
static int key_cmp(const void* a, const void* b) {
  int i = *(const int*)a, j = *(const int*)b;
  float ki = g_sort_keys[i], kj = g_sort_keys[j];
  if (ki < kj) return -1;
  if (ki > kj) return 1;
  return (i > j) - (i < j);
}

int64_t orc_tile_lists(const orc_params* P, const float* key, const int32_t* rect,
                       int64_t* offsets, int32_t* ids, int64_t capacity) {
  int T = P->tile, M = P->n_spheres;
  int ntx = (P->width + T - 1) / T, nty = (P->height + T - 1) / T;
  int nt = ntx * nty;
  int* order = (int*)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
  int nv = 0;
  for (int i = 0; i < M; ++i)
    if (rect[4 * i] >= 0) order[nv++] = i;
  g_sort_keys = key;
  qsort(order, (size_t)nv, sizeof(int), key_cmp);
  /* tiles are independent: first every tile's length, then (after the
   * prefix sum) every tile's entries, both by scanning the sorted spheres */
  int64_t* len = (int64_t*)calloc((size_t)(nt > 0 ? nt : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 4)
  for (int t = 0; t < nt; ++t) {
    int tx = t % ntx, ty = t / ntx;
    int ux0 = tx * T, ux1 = tx * T + T - 1, vy0 = ty * T, vy1 = ty * T + T - 1;
    int64_t n = 0;
    for (int k = 0; k < nv; ++k) {
      const int32_t* q = rect + 4 * order[k];
      if (q[1] < ux0 || q[0] > ux1 || q[3] < vy0 || q[2] > vy1) continue;
      ++n;
    }
    len[t] = n;
  }
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) {
    offsets[t] = total;
    total += len[t];
  }
  offsets[nt] = total;
  if (total <= capacity) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nt; ++t) {
      int tx = t % ntx, ty = t / ntx;
      int ux0 = tx * T, ux1 = tx * T + T - 1, vy0 = ty * T, vy1 = ty * T + T - 1;
      int64_t o = offsets[t];
      for (int k = 0; k < nv; ++k) {
        int i = order[k];
        const int32_t* q = rect + 4 * i;
        if (q[1] < ux0 || q[0] > ux1 || q[3] < vy0 || q[2] > vy1) continue;
        ids[o++] = i;
      }
    }
  }
  free(len);
  free(order);
  return total > capacity ? -1 : total;
}

/* Forward pass (Eq. 1) by brute force.  Outputs: image H x W x C, log D per
 * pixel, the hit count per pixel, and per pixel the n_track tracked sphere
 * indices (-1 padded) with their float32 hit depths, ordered closest first. */
void orc_render_fwd(const orc_params* P, const double* pos, const double* rad,
                    const double* opa, const double* feat, const double* cam, const double* bg,
                    const double* dpos, const double* drad, const double* dcam,
                    double* image, double* log_d, int32_t* n_hits, int32_t* tracked,
                    float* tracked_t, double* wsum) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  C.pos = pos; C.rad = rad; C.opa = opa; C.feat = feat; C.cam = cam; C.bg = bg;
  ctx_init(P, pos, rad, cam, dpos, drad, dcam, &C);
  int W = P->width, H = P->height, K = P->n_track, Cn = P->n_channels;
#pragma omp parallel
  {
    hit_rec* hits = (hit_rec*)malloc(sizeof(hit_rec) * (size_t)(P->n_spheres + 1));
#pragma omp for schedule(dynamic, 1)
    for (int v = 0; v < H; ++v)
      for (int u = 0; u < W; ++u) {
        size_t px = (size_t)v * W + u;
        int n = pixel_hits(P, &C, u, v, hits);
        double ws = 0.0;
        double ld = blend_pixel(P, &C, u, v, hits, n, image + px * Cn, &ws);
        if (log_d) log_d[px] = ld;
        if (wsum) wsum[px] = ws;
        if (n_hits) n_hits[px] = n;
        for (int k = 0; k < K; ++k) {
          if (tracked) tracked[px * K + k] = k < n ? hits[k].id : -1;
          if (tracked_t) tracked_t[px * K + k] = k < n ? hits[k].t32 : INFINITY;
        }
      }
    free(hits);
  }
  ctx_free(&C);
}

/* The decision margin of the early termination (paper_stop set): per pixel
 * the smallest |ln(a / min_contrib)| over the tests the pixel takes, a the largest
 * possible weight tested (see paper_stop_filter); +inf where no test is
 * taken.  margin: H x W. */
void orc_paper_stop_margin(const orc_params* P, const double* pos, const double* rad,
                           const double* opa, const double* cam, double* margin) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  C.pos = pos; C.rad = rad; C.opa = opa; C.cam = cam;
  ctx_init(P, pos, rad, cam, NULL, NULL, NULL, &C);
  int W = P->width, H = P->height, M = P->n_spheres;
#pragma omp parallel
  {
    hit_rec* hits = (hit_rec*)malloc(sizeof(hit_rec) * (size_t)(M + 1));
#pragma omp for schedule(dynamic, 1)
    for (int v = 0; v < H; ++v)
      for (int u = 0; u < W; ++u) {
        double mg = INFINITY;
        pixel_hits_m(P, &C, u, v, hits, &mg);
        margin[(size_t)v * W + u] = mg;
      }
    free(hits);
  }
  ctx_free(&C);
}

/* Backward pass by the chain rule, for an upstream gradient G = dL/dF.
 * Gradients flow through each pixel's tracked hits only (App. B).
 * Outputs (all accumulated from zero here): g_pos M x 3, g_rad M, g_opa M,
 * g_feat M x C, g_cam 11 (same order as cam), g_bg C. */
/* The backward pass over the pixels of the window [u0, u0 + ww) x [v0, v0 + wh);
 * grad holds dL/dF of the window's pixels (row-major, ww x wh x C), and dL/dF
 * is zero everywhere else.  Without the paper's normalisations, pixels with
 * zero dL/dF contribute nothing, so this equals the full-image pass with that
 * dL/dF. */
static void render_bwd_window(const orc_params* P, const double* pos, const double* rad,
                              const double* opa, const double* feat, const double* cam, const double* bg,
                              const double* grad, int u0, int v0, int ww, int wh, double* g_pos,
                              double* g_rad, double* g_opa, double* g_feat, double* g_cam, double* g_bg) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  C.pos = pos; C.rad = rad; C.opa = opa; C.feat = feat; C.cam = cam; C.bg = bg;
  ctx_init(P, pos, rad, cam, NULL, NULL, NULL, &C);
  int W = P->width, H = P->height, K = P->n_track, Cn = P->n_channels, M = P->n_spheres;
  double g = P->gamma, zr = P->zfar - P->znear;
  /* per-sphere accumulators: dL/dc (3), dL/dR (1) */
  double* gc = (double*)calloc((size_t)(M > 0 ? M : 1) * 4, sizeof(double));
  /* paper gradients: pixels at which each sphere is a tracked hit */
  int* n_px = (int*)calloc((size_t)(M > 0 ? M : 1), sizeof(int));
  double g_kappa = 0.0;
  memset(g_pos, 0, sizeof(double) * 3 * (size_t)M);
  memset(g_rad, 0, sizeof(double) * (size_t)M);
  memset(g_opa, 0, sizeof(double) * (size_t)M);
  memset(g_feat, 0, sizeof(double) * (size_t)M * Cn);
  memset(g_cam, 0, sizeof(double) * 11);
  memset(g_bg, 0, sizeof(double) * (size_t)Cn);
#pragma omp parallel
  {
    hit_rec* hits = (hit_rec*)malloc(sizeof(hit_rec) * (size_t)(M + 1));
    double* F = (double*)malloc(sizeof(double) * (size_t)(Cn > 0 ? Cn : 1));
    double gk_local = 0.0;
    double* gbg_local = (double*)calloc((size_t)(Cn > 0 ? Cn : 1), sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int v = v0; v < v0 + wh; ++v)
      for (int u = u0; u < u0 + ww; ++u) {
        size_t px = (size_t)(v - v0) * ww + (u - u0);
        const double* G = grad + px * Cn;
        int nz = 0;
        for (int c = 0; c < Cn; ++c) nz |= G[c] != 0.0;
        /* every contribution of this pixel is a multiple of G; the paper
         * normalisation still counts the pixel's tracked hits */
        if (!nz && !P->paper_grad) continue;
        int n = pixel_hits(P, &C, u, v, hits);
        double logD = blend_pixel(P, &C, u, v, hits, n, F, NULL);
        double wB = exp(P->eps / g - logD);
        for (int c = 0; c < Cn; ++c) gbg_local[c] += wB * G[c];
        double pxo = (double)(2 * u + 1 - W) * 0.5, pyo = (double)(2 * v + 1 - H) * 0.5;
        double rx = pxo * C.kappa, ry = pyo * C.kappa;
        int nt = n < K ? n : K;
        for (int j = 0; j < nt; ++j) {
          int i = hits[j].id;
          if (P->paper_grad) {
#pragma omp atomic
            n_px[i] += 1;
          }
          if (!nz) continue;
          const sph64* s = &C.sv[i];
          rayq q;
          ray_values(P, s, rx, ry, &q);
          double o = opa[i];
          double sx = o * q.z / g;
          double E = exp(sx - logD);          /* e^{s} / D */
          double w = o * q.d * E;             /* Eq. 1 weight */
          const double* f = feat + (size_t)i * Cn;
          double gdot = 0.0;                  /* G . (f_i - F) */
          for (int c = 0; c < Cn; ++c) gdot += G[c] * (f[c] - F[c]);
          for (int c = 0; c < Cn; ++c) {
#pragma omp atomic
            g_feat[(size_t)i * Cn + c] += w * G[c];
          }
          /* a = o d e^{o z / g};  dL/da = gdot / D */
          double dL_do = gdot * q.d * E * (1.0 + sx);
          double dL_dd = gdot * o * E;
          double dL_dz = gdot * w * o / g;
          double dL_dt = -dL_dz / zr;
          /* d from dist: default d = 1 - dist/R, literal d = dist/R (0 slope when clamped) */
          double dL_ddist = 0.0, dL_dR = 0.0;
          if (q.dist < s->R) {
            double sgn = P->dist_literal ? 1.0 : -1.0;
            dL_ddist = sgn * dL_dd / s->R;
            dL_dR = -sgn * dL_dd * q.dist / (s->R * s->R);
          }
          /* derivatives of t = (b - sqrt(disc)) / rr and dist^2 = |c|^2 - b^2/rr
           * (c the centre the ray meets; orthographic: shifted, ray (0, 0, 1)) */
          const double* c = q.cs;
          double dc[3] = {0, 0, 0}, dr[3] = {0, 0, 0};
          if (q.sq > 0.0) {
            for (int k = 0; k < 3; ++k) {
              double dt_dc = (q.r[k] - (q.b * q.r[k] - q.rr * c[k]) / q.sq) / q.rr;
              double dt_dr = (c[k] - (q.b * c[k] - q.q * q.r[k]) / q.sq) / q.rr
                             - 2.0 * q.t * q.r[k] / q.rr;
              dc[k] += dL_dt * dt_dc;
              dr[k] += dL_dt * dt_dr;
            }
            dL_dR += dL_dt * (-s->R / q.sq);
          }
          if (q.dist > 0.0) {
            double tc = q.b / q.rr;
            for (int k = 0; k < 3; ++k) {
              double e = c[k] - tc * q.r[k];
              dc[k] += dL_ddist * e / q.dist;
              dr[k] += dL_ddist * (-tc * e / q.dist);
            }
          }
          /* the pitch k enters through the ray slopes (pinhole) or through the
           * shift c - k (pxo, pyo, 0) of the centre (orthographic) */
          gk_local += P->ortho ? -(dc[0] * pxo + dc[1] * pyo) : dr[0] * pxo + dr[1] * pyo;
#pragma omp atomic
          gc[4 * (size_t)i] += dc[0];
#pragma omp atomic
          gc[4 * (size_t)i + 1] += dc[1];
#pragma omp atomic
          gc[4 * (size_t)i + 2] += dc[2];
#pragma omp atomic
          gc[4 * (size_t)i + 3] += dL_dR;
#pragma omp atomic
          g_opa[i] += dL_do;
        }
      }
#pragma omp critical
    {
      g_kappa += gk_local;
      for (int c = 0; c < Cn; ++c) g_bg[c] += gbg_local[c];
    }
    free(hits);
    free(F);
    free(gbg_local);
  }
  /* per-sphere chain: R -> (r | c, kappa);  c = B (p - t) -> p, t, B */
  double gB[9] = {0};
  for (int i = 0; i < M; ++i) {
    const sph64* s = &C.sv[i];
    double* a = gc + 4 * (size_t)i;
    if (!C.pj[i].visible) continue;
    /* paper gradients: 1 / n_i, and positions and radii only for spheres of
     * more than 3 pixels projected radius (float32 decision) */
    double scale = 1.0, geo_scale = 1.0;
    if (P->paper_grad) {
      scale = 1.0 / (double)(n_px[i] > 1 ? n_px[i] : 1);
      const float px_size = P->ortho ? C.kappaf : C.pj[i].cz * C.kappaf;
      const float rpx = C.pj[i].R / px_size;
      geo_scale = rpx > 3.0f ? scale : 0.0;
      g_opa[i] *= scale;
      for (int c = 0; c < Cn; ++c) g_feat[(size_t)i * Cn + c] *= scale;
    }
    if (s->clamped && P->ortho) {
      g_kappa += a[3] * 0.75;   /* R = 0.75 k */
    } else if (s->clamped) {
      double cn = sqrt(s->c[0] * s->c[0] + s->c[1] * s->c[1] + s->c[2] * s->c[2]);
      for (int k = 0; k < 3; ++k) a[k] += a[3] * 0.75 * C.kappa * s->c[k] / cn;
      g_kappa += a[3] * 0.75 * cn;
    } else {
      g_rad[i] = geo_scale * a[3];
    }
    double d[3] = {pos[3 * i] - cam[0], pos[3 * i + 1] - cam[1], pos[3 * i + 2] - cam[2]};
    for (int k = 0; k < 3; ++k) {
      double gp = C.B[k] * a[0] + C.B[3 + k] * a[1] + C.B[6 + k] * a[2];
      g_pos[3 * i + k] = geo_scale * gp;
      g_cam[k] -= gp;
    }
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) gB[3 * r + k] += a[r] * d[k];
  }
  /* rotation rows -> 6D vector by complex-step differentiation of Gram-Schmidt */
  for (int k = 0; k < 6; ++k) {
    double complex a6[6], Bc[9];
    const double h = 1e-30;
    for (int j = 0; j < 6; ++j) a6[j] = cam[3 + j];
    a6[k] += I * h;
    rows_c(a6, Bc);
    double acc = 0.0;
    for (int j = 0; j < 9; ++j) acc += gB[j] * cimag(Bc[j]) / h;
    g_cam[3 + k] = acc;
  }
  /* kappa = s / (W f), orthographic s / W */
  if (P->ortho) {
    g_cam[9] = 0.0;
    g_cam[10] = g_kappa / (double)W;
  } else {
    g_cam[9] = -g_kappa * C.kappa / cam[9];
    g_cam[10] = g_kappa / ((double)W * cam[9]);
  }
  if (P->paper_grad)
    for (int k = 0; k < 11; ++k) g_cam[k] *= 1e-3;
  free(gc);
  free(n_px);
  ctx_free(&C);
}

void orc_render_bwd(const orc_params* P, const double* pos, const double* rad,
                    const double* opa, const double* feat, const double* cam, const double* bg,
                    const double* grad, double* g_pos, double* g_rad, double* g_opa,
                    double* g_feat, double* g_cam, double* g_bg) {
  render_bwd_window(P, pos, rad, opa, feat, cam, bg, grad, 0, 0, P->width, P->height, g_pos, g_rad,
                    g_opa, g_feat, g_cam, g_bg);
}

/* The backward pass with dL/dF given on a window only (zero elsewhere; not
 * with the paper's normalisations, which count every pixel's tracked hits). */
void orc_render_bwd_window(const orc_params* P, const double* pos, const double* rad,
                           const double* opa, const double* feat, const double* cam, const double* bg,
                           const double* grad, int u0, int v0, int ww, int wh, double* g_pos,
                           double* g_rad, double* g_opa, double* g_feat, double* g_cam, double* g_bg) {
  if (P->paper_grad) return;
  render_bwd_window(P, pos, rad, opa, feat, cam, bg, grad, u0, v0, ww, wh, g_pos, g_rad, g_opa,
                    g_feat, g_cam, g_bg);
}

/* Rotation rows in double (for tests of the camera model). */
void orc_rows(const double* rot6, double* B) { rows_f64(rot6, B); }

/* float32 hit predicate of one sphere at one pixel, exported for tests.
 * With ignore_cull set the predicate is evaluated for culled spheres too. */
int orc_hit_f32(const orc_params* P, const double* pos3, double rad, const double* cam, int u, int v,
                int ignore_cull, float* t_out) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  orc_params Q = *P;
  Q.n_spheres = 1;
  ctx_init(&Q, pos3, &rad, cam, NULL, NULL, NULL, &C);
  int hit = 0;
  if (C.pj[0].visible || ignore_cull) {
    float rx = ray_coord_f32(u, P->width, C.kappaf);
    float ry = ray_coord_f32(v, P->height, C.kappaf);
    hit = hit_px(P, &C.pj[0], rx, ry, (float)P->zfar, t_out);
  }
  ctx_free(&C);
  return hit;
}

/* float32 hit predicate of one sphere over the whole image (1 = hit).  With
 * ignore_cull set it is evaluated even when the sphere was culled, so tests
 * can check that culling never drops a sphere that meets a pixel ray. */
void orc_hit_map(const orc_params* P, const double* pos3, double rad, const double* cam,
                 int ignore_cull, uint8_t* map) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  orc_params Q = *P;
  Q.n_spheres = 1;
  ctx_init(&Q, pos3, &rad, cam, NULL, NULL, NULL, &C);
  for (int v = 0; v < P->height; ++v)
    for (int u = 0; u < P->width; ++u) {
      float t;
      int hit = 0;
      if (C.pj[0].visible || ignore_cull) {
        float rx = ray_coord_f32(u, P->width, C.kappaf);
        float ry = ray_coord_f32(v, P->height, C.kappaf);
        hit = hit_px(P, &C.pj[0], rx, ry, (float)P->zfar, &t);
      }
      map[(size_t)v * P->width + u] = (uint8_t)hit;
    }
  ctx_free(&C);
}

/* Forward pass at a list of pixels only (for sampled checks of large
 * workloads): pix holds n_pix (u, v) pairs; outputs are per listed pixel. */
void orc_render_pixels(const orc_params* P, const double* pos, const double* rad,
                       const double* opa, const double* feat, const double* cam, const double* bg,
                       int n_pix, const int32_t* pix, double* image, double* log_d,
                       int32_t* n_hits, int32_t* tracked, float* tracked_t) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  C.pos = pos; C.rad = rad; C.opa = opa; C.feat = feat; C.cam = cam; C.bg = bg;
  ctx_init(P, pos, rad, cam, NULL, NULL, NULL, &C);
  int K = P->n_track, Cn = P->n_channels;
#pragma omp parallel
  {
    hit_rec* hits = (hit_rec*)malloc(sizeof(hit_rec) * (size_t)(P->n_spheres + 1));
#pragma omp for schedule(dynamic, 4)
    for (int q = 0; q < n_pix; ++q) {
      int u = pix[2 * q], v = pix[2 * q + 1];
      int n = pixel_hits(P, &C, u, v, hits);
      log_d[q] = blend_pixel(P, &C, u, v, hits, n, image + (size_t)q * Cn, NULL);
      n_hits[q] = n;
      for (int k = 0; k < K; ++k) {
        tracked[(size_t)q * K + k] = k < n ? hits[k].id : -1;
        tracked_t[(size_t)q * K + k] = k < n ? hits[k].t32 : INFINITY;
      }
    }
    free(hits);
  }
  ctx_free(&C);
}
