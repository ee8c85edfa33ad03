/*
 * ctrex_oracle.c -- plain, slow, FP64 CPU oracle for the CTrex projection /
 * correction / backprojection path (arxiv 2609.30166).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Every routine follows one passage of the paper (cited by section / equation)
 * and, where the paper is silent, one stated reading:
 *
 *   geometry      Sec. 2.2.1 (single-projection geometry, 3x4 projection matrix)
 *   forward A     Sec. 4.1 "Projection operator": ray from source to pixel
 *                 centre, clipped to the volume, sampled with trilinear
 *                 interpolation, samples weighted by path length
 *   sub-angles    Sec. 3.4 / Sec. 4.2.2: pixel value = mean over angular
 *                 sub-projections (extra loop in the projector)
 *   motion        Sec. 2.2.2 "Affine volume pose" (rigid then affine) and
 *                 Sec. 3.1.1 / 4.2.1 (sample coordinates mapped through the
 *                 displacement field before the volume lookup)
 *   correction R  Sec. 4.1 "Correction kernel", Eq. (1) term 2
 *   backproj. CA^T Sec. 4.1 "Backprojection operator", Eq. (1) term 3, with the
 *                 voxel weights w_j of Sec. 3.2 / Sec. 4.3.2
 *   SIRT loop     Eq. (1), Sec. 2.3.1-2.3.2 (all views in one subset)
 *   adjoint, motion gradient: exact transpose / chain rule of the forward
 *                 above (the paper motivates geometry refinement in Sec. 5 but
 *                 prints no formula).
 *
 * Readings where the paper is silent:
 *   R1 the ray is the half line t >= 0 from the source; P is sign-normalised
 *      so that the depth of the volume centre is positive;
 *   R2 fixed step, truncated-midpoint quadrature starting at the entry face;
 *   R3 trilinear interpolation with zero padding outside the voxel grid;
 *   R4 BP samples the correction image bilinearly at the projected voxel
 *      centre (zero outside the detector) and normalises by the column sum of
 *      that same backprojector (C_j = 1 / sum of in-range bilinear weights);
 *   R5 R_i = 1 / (row sum of A) and w_j multiplies after normalisation;
 *   R6 motion: x' = A (R(omega) x + t), y = x' + s_v u(x'), u a uniform cubic
 *      B-spline on an 8^3 control grid spanning the nominal box, clip box
 *      dilated by a fixed margin;
 *   R11 extended field of view (Sec. 3.6, Sec. 4.3.2): the backprojector of
 *      view v sees only detector columns u_lo..u_hi and rows v_lo..v_hi (its
 *      effective edge); taps outside count as off the detector for both the
 *      sum and its normalisation; the forward keeps the whole detector;
 *   R12 sub-voxel backprojection (Sec. 4.3.2, motion blur): with s > 1 the
 *      backprojected value and column sum of a voxel are the means over the
 *      s^3 points at offsets ((a + 1/2)/s - 1/2) voxel on each axis;
 *   R13 aligned cylindrical domain (Sec. 3.5; projector and backprojector
 *      adaptations in Sec. 4.2 / 4.3): a rigid pose maps world x to the
 *      frame q = Rc x + tc, whose z axis is the cylinder axis.  Voxel (i, j,
 *      k) sits at r = (i + 1/2) dr, phi = (j + 1/2) 2 pi / N_phi, z = (k -
 *      (N_z - 1)/2) dz.  A sample at q has index coordinates g_r = r/dr -
 *      1/2 (clamped to >= 0: inside the first ring centre the value of ring
 *      0 is used), g_phi = phi / (2 pi / N_phi) - 1/2 taken modulo N_phi
 *      (periodic), g_z = q_z/dz + (N_z - 1)/2; trilinear interpolation in
 *      these, zero outside in r (beyond ring N_r - 1) and z.  Rays are
 *      clipped to the bounding cylinder r <= N_r dr, |q_z| <= N_z dz / 2;
 *      the step is step_vox * min(dr, dz); the rest of the projector and the
 *      backprojector (at the voxel centres mapped back to world) is as above;
 *   R16 event-based 4D model (Sec. 3.3): three fields per voxel, the initial
 *      value mu0_j, the final value mu1_j and the transition time tau_j; view
 *      v, acquired at time t_v, sees mu0_j where t_v < tau_j and mu1_j
 *      otherwise (one irreversible change per voxel).  The projector
 *      samples that per-view volume (the selection is made per trilinear
 *      tap).  The backprojector splits Eq. (1) term 3 by the same rule: the
 *      views before tau_j update mu0_j, normalised by their own column sum,
 *      the views from tau_j on update mu1_j.  tau is an input (its update
 *      rule is not part of this paper).  Cartesian trilinear projector
 *      without motion, ROI, Joseph or sub-voxel backprojection.
 *
 * Conventions: volume vol[iz][iy][ix] (x fastest), voxel (0,0,0) centred at
 * origin (mm), index coordinate g = (x - origin) / vox.  Projection images
 * proj[view][iv][iu] (u fastest), pixel (iu,iv) centre at detector
 * coordinate (iu,iv).  P[view][sub][3][4] row-major, maps homogeneous world mm
 * to homogeneous pixel coordinates.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Mirror of the ctypes structure in oracle/__init__.py. */
typedef struct {
    int nx, ny, nz;
    double vox[3];
    double origin[3];
    int nu, nv;
    int n_views, n_sub;
    double step_vox;
    const double *P;      /* [n_views][n_sub][12], as given by the caller */
    const double *theta;  /* [n_views][15] (omega, t, A row-major) or NULL */
    const double *coef;   /* [8][8][8][3] (z,y,x,component) or NULL       */
    const double *s_view; /* [n_views] or NULL (then s_v = 0)              */
    double margin;        /* mm, clip-box dilation when motion is on       */
    const int *bp_window; /* [n_views][4] (u_lo, u_hi, v_lo, v_hi) or NULL */
    int bp_subvoxel;      /* > 1: backproject onto s^3 sub-voxel points     */
    /* aligned cylindrical domain (Sec. 3.5, reading R13): when cyl != 0 the
     * grid is (nx, ny, nz) = (N_r, N_phi, N_z) with ring pitch cyl_dr, slice
     * pitch cyl_dz (mm) and sector 2 pi / N_phi; vox and origin are unused */
    int cyl;
    double cyl_dr, cyl_dz;
    const double *cyl_pose; /* [12] row-major 3x4: q = Rc x + tc (world mm -> frame mm) */
    int joseph;             /* 1: classical Joseph projector (reading R14) instead of R2 */
    /* multi-resolution ROI (Sec. 3.7 method B, reading R15): a finer grid
     * inside the context grid's box; volumes are then the context grid's
     * voxels followed by the ROI grid's */
    int roi;
    int roi_n[3];
    double roi_vox[3], roi_origin[3];
    /* event-based 4D model (Sec. 3.3, reading R16): when dyr_tau is set,
     * volumes hold the initial values mu0 followed by the final values mu1
     * (2 nx ny nz each) */
    const double *dyr_tau; /* [nz][ny][nx] transition times, or NULL */
    const double *dyr_t;   /* [n_views] acquisition time of each view */
} or_problem;

/* Per (view, sub-angle) quantities derived from P (Sec. 2.2.1). */
typedef struct {
    double P[12];   /* sign-normalised projection matrix */
    double src[3];  /* source position, mm               */
    double Minv[9]; /* inverse of the left 3x3 block     */
} or_view;

#define OR_E_GEOMETRY (-4)
#define OR_E_ARG (-1)

static double det3(const double *m)
{
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

static void inv3(const double *m, double det, double *r)
{
    r[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    r[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    r[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    r[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    r[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    r[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    r[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    r[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    r[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

/* Cylinder frame -> world: x = Rc^T (q - tc). */
static void cyl_to_world(const or_problem *pb, const double q[3], double x[3])
{
    const double *T = pb->cyl_pose;
    double d[3] = {q[0] - T[3], q[1] - T[7], q[2] - T[11]};
    for (int a = 0; a < 3; ++a) x[a] = T[a] * d[0] + T[4 + a] * d[1] + T[8 + a] * d[2];
}

/* World -> cylinder frame: q = Rc x + tc. */
static void world_to_cyl(const or_problem *pb, const double x[3], double q[3])
{
    const double *T = pb->cyl_pose;
    for (int r = 0; r < 3; ++r) q[r] = T[4 * r] * x[0] + T[4 * r + 1] * x[1] + T[4 * r + 2] * x[2] + T[4 * r + 3];
}

static void volume_centre(const or_problem *pb, double c[3])
{
    if (pb->cyl) {
        const double q0[3] = {0.0, 0.0, 0.0};
        cyl_to_world(pb, q0, c);
        return;
    }
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    for (int a = 0; a < 3; ++a) c[a] = pb->origin[a] + 0.5 * (n[a] - 1) * pb->vox[a];
}

/* Reading R15: the ROI grid as a problem of its own (same views). */
static or_problem roi_part(const or_problem *pb)
{
    or_problem f = *pb;
    f.nx = pb->roi_n[0];
    f.ny = pb->roi_n[1];
    f.nz = pb->roi_n[2];
    for (int a = 0; a < 3; ++a) {
        f.vox[a] = pb->roi_vox[a];
        f.origin[a] = pb->roi_origin[a];
    }
    f.roi = 0;
    return f;
}

static long grid_voxels(const or_problem *pb)
{
    return (long)pb->nx * pb->ny * pb->nz;
}

/*
 * Sec. 2.2.1: one projection is fully described by P = [M | p4].  The source
 * is the point P maps to zero, s = -M^{-1} p4.  Reading R1: P and -P describe
 * the same projection; we pick the sign that gives the volume centre a
 * positive depth (third homogeneous coordinate), so that points in front of
 * the source have positive depth.  A (near-)singular M or a volume centre on
 * the source plane is rejected.
 */
static int setup_view(const double *Pin, const double centre[3], or_view *ov)
{
    double M[9], fro = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            M[3 * r + c] = Pin[4 * r + c];
            fro += M[3 * r + c] * M[3 * r + c];
        }
    fro = sqrt(fro);
    double det = det3(M);
    if (!(fabs(det) > 1e-12 * fro * fro * fro)) return OR_E_GEOMETRY;
    double depth = Pin[8] * centre[0] + Pin[9] * centre[1] + Pin[10] * centre[2] + Pin[11];
    if (!(depth != 0.0)) return OR_E_GEOMETRY;
    double sign = depth > 0.0 ? 1.0 : -1.0;
    for (int k = 0; k < 12; ++k) ov->P[k] = sign * Pin[k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = ov->P[4 * r + c];
    inv3(M, det3(M), ov->Minv);
    const double p4[3] = {ov->P[3], ov->P[7], ov->P[11]};
    for (int r = 0; r < 3; ++r)
        ov->src[r] = -(ov->Minv[3 * r + 0] * p4[0] + ov->Minv[3 * r + 1] * p4[1] +
                       ov->Minv[3 * r + 2] * p4[2]);
    return 0;
}

static or_view *setup_all_views(const or_problem *pb, int *err)
{
    double c[3];
    volume_centre(pb, c);
    int nvs = pb->n_views * pb->n_sub;
    or_view *ov = (or_view *)malloc(sizeof(or_view) * (size_t)(nvs > 0 ? nvs : 1));
    *err = 0;
    for (int k = 0; k < nvs; ++k) {
        int e = setup_view(pb->P + 12 * (size_t)k, c, &ov[k]);
        if (e) {
            *err = e;
            free(ov);
            return NULL;
        }
    }
    return ov;
}

/* Exported: the derived per-(view, sub) quantities, for tests of R1. */
int or_setup_views(const or_problem *pb, double *Pn, double *src, double *Minv)
{
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    int nvs = pb->n_views * pb->n_sub;
    for (int k = 0; k < nvs; ++k) {
        memcpy(Pn + 12 * (size_t)k, ov[k].P, sizeof(double) * 12);
        memcpy(src + 3 * (size_t)k, ov[k].src, sizeof(double) * 3);
        memcpy(Minv + 9 * (size_t)k, ov[k].Minv, sizeof(double) * 9);
    }
    free(ov);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Trilinear interpolation with zero padding (reading R3).                 */
/* ---------------------------------------------------------------------- */

/*
 * Value of the zero-padded trilinear interpolant at index coordinate g, plus
 * the sum of the weights of the taps that fall inside the grid (this is the
 * interpolant of an all-ones volume, used for the row sums) and, if grad is
 * not NULL, the gradient with respect to g inside the cell floor(g).
 */
static double trilinear(const or_problem *pb, const double *vol, const double g[3],
                        double *wsum, double grad[3])
{
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    if (wsum) *wsum = 0.0;
    if (grad) grad[0] = grad[1] = grad[2] = 0.0;
    for (int a = 0; a < 3; ++a)
        if (!(g[a] >= -1.0 && g[a] < (double)n[a])) return 0.0; /* every tap outside */
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]);
        i0[a] = (int)fl;
        f[a] = g[a] - fl;
    }
    double val = 0.0, ws = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                if (ix < 0 || ix >= n[0] || iy < 0 || iy >= n[1] || iz < 0 || iz >= n[2]) continue;
                double wx = dx ? f[0] : 1.0 - f[0];
                double wy = dy ? f[1] : 1.0 - f[1];
                double wz = dz ? f[2] : 1.0 - f[2];
                double vv = vol ? vol[((size_t)iz * n[1] + iy) * n[0] + ix] : 1.0;
                val += wx * wy * wz * vv;
                ws += wx * wy * wz;
                gx += (dx ? 1.0 : -1.0) * wy * wz * vv;
                gy += wx * (dy ? 1.0 : -1.0) * wz * vv;
                gz += wx * wy * (dz ? 1.0 : -1.0) * vv;
            }
    if (wsum) *wsum = ws;
    if (grad) {
        grad[0] = gx;
        grad[1] = gy;
        grad[2] = gz;
    }
    return val;
}

/*
 * Reading R16: the zero-padded trilinear interpolant of the volume that a view
 * acquired at time t sees: each tap takes mu0 (the first half of vol) where
 * t < tau at that voxel, else mu1 (the second half).  wsum as for trilinear().
 */
static double dyr_trilinear(const or_problem *pb, const double *vol, const double g[3], double t, double *wsum)
{
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    const size_t nvox = (size_t)n[0] * n[1] * n[2];
    *wsum = 0.0;
    for (int a = 0; a < 3; ++a)
        if (!(g[a] >= -1.0 && g[a] < (double)n[a])) return 0.0;
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]);
        i0[a] = (int)fl;
        f[a] = g[a] - fl;
    }
    double val = 0.0, ws = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                if (ix < 0 || ix >= n[0] || iy < 0 || iy >= n[1] || iz < 0 || iz >= n[2]) continue;
                double wgt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                size_t j = ((size_t)iz * n[1] + iy) * n[0] + ix;
                if (vol) val += wgt * (t < pb->dyr_tau[j] ? vol[j] : vol[nvox + j]);
                else val += wgt;
                ws += wgt;
            }
    *wsum = ws;
    return val;
}

/*
 * Reading R13: interpolation on the cylindrical grid at index coordinate g =
 * (g_r, g_phi, g_z): g_r clamped to >= 0, phi periodic, zero outside in r and
 * z.  wsum as for trilinear().
 */
static double cyl_interp(const or_problem *pb, const double *vol, const double g[3], double *wsum)
{
    const int nr = pb->nx, np = pb->ny, nz = pb->nz;
    double gr = g[0] < 0.0 ? 0.0 : g[0];
    *wsum = 0.0;
    if (!(gr < (double)nr && g[2] >= -1.0 && g[2] < (double)nz)) return 0.0;
    double fr = floor(gr), fp = floor(g[1]), fz = floor(g[2]);
    int i0 = (int)fr, j0 = (int)fp, k0 = (int)fz;
    double ar = gr - fr, ap = g[1] - fp, az = g[2] - fz;
    double val = 0.0, ws = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dp = 0; dp < 2; ++dp)
            for (int dr = 0; dr < 2; ++dr) {
                int i = i0 + dr, k = k0 + dz;
                int j = ((j0 + dp) % np + np) % np;
                if (i >= nr || k < 0 || k >= nz) continue;
                double wgt = (dr ? ar : 1.0 - ar) * (dp ? ap : 1.0 - ap) * (dz ? az : 1.0 - az);
                val += wgt * (vol ? vol[((size_t)k * np + j) * nr + i] : 1.0);
                ws += wgt;
            }
    *wsum = ws;
    return val;
}

/* Reading R13: frame point q -> cylindrical index coordinates. */
static void cyl_index(const or_problem *pb, const double q[3], double g[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    const double dphi = two_pi / pb->ny;
    double r = sqrt(q[0] * q[0] + q[1] * q[1]);
    double phi = atan2(q[1], q[0]);
    if (phi < 0.0) phi += two_pi;
    g[0] = r / pb->cyl_dr - 0.5;
    g[1] = phi / dphi - 0.5;
    if (g[1] < 0.0) g[1] += pb->ny;
    if (g[1] >= pb->ny) g[1] -= pb->ny;
    g[2] = q[2] / pb->cyl_dz + 0.5 * (pb->nz - 1);
}

/* ---------------------------------------------------------------------- */
/* Motion model (reading R6; Sec. 2.2.2 affine pose, Sec. 3.1 warp).       */
/* ---------------------------------------------------------------------- */

/* Uniform cubic B-spline, support [-2, 2], and its derivative. */
static double bspline3(double t)
{
    double a = fabs(t);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

static double bspline3_d(double t)
{
    double a = fabs(t), s = t < 0.0 ? -1.0 : 1.0;
    if (a < 1.0) return s * (-2.0 * a + 1.5 * a * a);
    if (a < 2.0) return s * (-0.5 * (2.0 - a) * (2.0 - a));
    return 0.0;
}

/* Rodrigues rotation R = I + a K + b K^2, K = [omega]_x, theta = |omega|. */
static void rodrigues_coeffs(double th, double *a, double *b, double *da_over_th,
                             double *db_over_th)
{
    /* a = sin(th)/th, b = (1-cos th)/th^2, and a'(th)/th, b'(th)/th. */
    if (th < 1e-4) {
        double t2 = th * th;
        *a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        *b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *da_over_th = -1.0 / 3.0 + t2 / 30.0;
        *db_over_th = -1.0 / 12.0 + t2 / 180.0;
    } else {
        double s = sin(th), c = cos(th);
        *a = s / th;
        *b = (1.0 - c) / (th * th);
        *da_over_th = (th * c - s) / (th * th * th);
        *db_over_th = (th * s - 2.0 * (1.0 - c)) / (th * th * th * th);
    }
}

static void skew(const double w[3], double K[9])
{
    K[0] = 0.0;   K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2];  K[4] = 0.0;   K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0];  K[8] = 0.0;
}

static void matmul3(const double *A, const double *B, double *C)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

static void matvec3(const double *A, const double *x, double *y)
{
    for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

/* R(omega) and, if dR is not NULL, dR/domega_i for i = 0..2. */
static void rotation(const double w[3], double R[9], double dR[27])
{
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double a, b, dat, dbt;
    rodrigues_coeffs(th, &a, &b, &dat, &dbt);
    double K[9], K2[9];
    skew(w, K);
    matmul3(K, K, K2);
    for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0 ? 1.0 : 0.0) + a * K[k] + b * K2[k];
    if (!dR) return;
    for (int i = 0; i < 3; ++i) {
        double e[3] = {0.0, 0.0, 0.0};
        e[i] = 1.0;
        double E[9], EK[9], KE[9];
        skew(e, E);
        matmul3(E, K, EK);
        matmul3(K, E, KE);
        for (int k = 0; k < 9; ++k)
            dR[9 * i + k] = dat * w[i] * K[k] + a * E[k] + dbt * w[i] * K2[k] + b * (EK[k] + KE[k]);
    }
}

/*
 * B-spline coordinate of x' along axis a: control point i sits at
 * x_min + (i-1) h with h = (box length) / 5, so the box maps to xi in [1, 6];
 * xi is clamped to that range.  Returns whether the clamp was active.
 */
static double spline_coord(const or_problem *pb, int a, double xp, int *clamped)
{
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    double lo = pb->origin[a] - 0.5 * pb->vox[a];
    double h = n[a] * pb->vox[a] / 5.0;
    double xi = (xp - lo) / h + 1.0;
    *clamped = 0;
    if (xi < 1.0) { xi = 1.0; *clamped = 1; }
    if (xi > 6.0) { xi = 6.0; *clamped = 1; }
    return xi;
}

/* Control-point index range [lo, hi] (within 0..7) where beta3(xi - i) != 0. */
static void spline_support(const double xi[3], int lo[3], int hi[3])
{
    for (int a = 0; a < 3; ++a) {
        int f = (int)floor(xi[a]);
        lo[a] = f - 1 < 0 ? 0 : f - 1;
        hi[a] = f + 2 > 7 ? 7 : f + 2;
    }
}

/*
 * Displacement u(x') and, if J is not NULL, its Jacobian du/dx' (row = output
 * component, column = input axis).
 */
static void displacement(const or_problem *pb, const double xp[3], double u[3], double J[9])
{
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    double xi[3];
    int cl[3];
    for (int a = 0; a < 3; ++a) xi[a] = spline_coord(pb, a, xp[a], &cl[a]);
    u[0] = u[1] = u[2] = 0.0;
    if (J) memset(J, 0, sizeof(double) * 9);
    /* beta3(xi - i) vanishes unless |xi - i| < 2: sum over that support only */
    int lo[3], hi[3];
    spline_support(xi, lo, hi);
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                double bx = bspline3(xi[0] - i), by = bspline3(xi[1] - j), bz = bspline3(xi[2] - k);
                const double *c = pb->coef + 3 * (size_t)((k * 8 + j) * 8 + i);
                double wgt = bx * by * bz;
                for (int comp = 0; comp < 3; ++comp) u[comp] += wgt * c[comp];
                if (J) {
                    double hx = n[0] * pb->vox[0] / 5.0, hy = n[1] * pb->vox[1] / 5.0,
                           hz = n[2] * pb->vox[2] / 5.0;
                    double dx = cl[0] ? 0.0 : bspline3_d(xi[0] - i) * by * bz / hx;
                    double dy = cl[1] ? 0.0 : bx * bspline3_d(xi[1] - j) * bz / hy;
                    double dz = cl[2] ? 0.0 : bx * by * bspline3_d(xi[2] - k) / hz;
                    for (int comp = 0; comp < 3; ++comp) {
                        J[3 * comp + 0] += c[comp] * dx;
                        J[3 * comp + 1] += c[comp] * dy;
                        J[3 * comp + 2] += c[comp] * dz;
                    }
                }
            }
}

/*
 * Displacement field u(x') and its Jacobian at n points (Sec. 3.1 deformation,
 * reading R6), exported so that its control-grid placement can be checked on
 * its own: xp [n][3] mm, u [n][3], J [n][9] (row = component, column = axis).
 */
int or_displacement(const or_problem *pb, long n, const double *xp, double *u, double *J)
{
    if (!pb->coef) return -1;
    for (long q = 0; q < n; ++q) displacement(pb, xp + 3 * q, u + 3 * q, J ? J + 9 * q : NULL);
    return 0;
}

/* Motion of view v applied to a nominal sample point x (mm): returns y. */
static void warp_point(const or_problem *pb, int view, const double x[3], double y[3])
{
    if (!pb->theta && !pb->coef) {
        y[0] = x[0]; y[1] = x[1]; y[2] = x[2];
        return;
    }
    double xp[3] = {x[0], x[1], x[2]};
    if (pb->theta) {
        const double *th = pb->theta + 15 * (size_t)view;
        double R[9], q[3];
        rotation(th, R, NULL);
        matvec3(R, x, q);
        for (int a = 0; a < 3; ++a) q[a] += th[3 + a];
        matvec3(th + 6, q, xp);
    }
    double u[3] = {0.0, 0.0, 0.0};
    double s = pb->s_view ? pb->s_view[view] : 0.0;
    if (pb->coef) displacement(pb, xp, u, NULL);
    for (int a = 0; a < 3; ++a) y[a] = xp[a] + s * u[a];
}

/* ---------------------------------------------------------------------- */
/* Forward projector (Sec. 4.1 "Projection operator", readings R1-R3).     */
/* ---------------------------------------------------------------------- */

/* Reading R13: clip the half line to the bounding cylinder of the domain. */
static int clip_ray_cyl(const or_problem *pb, const double s[3], const double d[3], double *t_in,
                        double *t_out)
{
    double qs[3], qe[3], e[3], qd[3];
    world_to_cyl(pb, s, qs);
    for (int a = 0; a < 3; ++a) e[a] = s[a] + d[a];
    world_to_cyl(pb, e, qe);
    for (int a = 0; a < 3; ++a) qd[a] = qe[a] - qs[a];
    double R = pb->nx * pb->cyl_dr, Z = 0.5 * pb->nz * pb->cyl_dz;
    double t0 = 0.0, t1 = INFINITY;
    /* mantle: |qs_xy + t qd_xy|^2 <= R^2 */
    double a = qd[0] * qd[0] + qd[1] * qd[1];
    double b = 2.0 * (qs[0] * qd[0] + qs[1] * qd[1]);
    double c = qs[0] * qs[0] + qs[1] * qs[1] - R * R;
    if (a == 0.0) {
        if (c > 0.0) return 0;
    } else {
        double disc = b * b - 4.0 * a * c;
        if (!(disc > 0.0)) return 0;
        double sq = sqrt(disc);
        double ta = (-b - sq) / (2.0 * a), tb = (-b + sq) / (2.0 * a);
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    /* end caps */
    if (qd[2] == 0.0) {
        if (qs[2] < -Z || qs[2] > Z) return 0;
    } else {
        double ta = (-Z - qs[2]) / qd[2], tb = (Z - qs[2]) / qd[2];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    *t_in = t0;
    *t_out = t1;
    return t1 > t0;
}

/* Clip the half line s + t d, t >= 0, to the (possibly dilated) box. */
static int clip_ray(const or_problem *pb, const double s[3], const double d[3], double *t_in,
                    double *t_out)
{
    if (pb->cyl) return clip_ray_cyl(pb, s, d, t_in, t_out);
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    double m = (pb->theta || pb->coef) ? pb->margin : 0.0;
    double t0 = 0.0, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = pb->origin[a] - 0.5 * pb->vox[a] - m;
        double hi = pb->origin[a] + (n[a] - 0.5) * pb->vox[a] + m;
        if (d[a] == 0.0) {
            if (s[a] < lo || s[a] > hi) return 0;
            continue;
        }
        double ta = (lo - s[a]) / d[a], tb = (hi - s[a]) / d[a];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    *t_in = t0;
    *t_out = t1;
    return t1 > t0;
}

static double step_mm(const or_problem *pb)
{
    if (pb->cyl) return pb->step_vox * (pb->cyl_dr < pb->cyl_dz ? pb->cyl_dr : pb->cyl_dz);
    double v = pb->vox[0];
    if (pb->vox[1] < v) v = pb->vox[1];
    if (pb->vox[2] < v) v = pb->vox[2];
    return pb->step_vox * v;
}

/* Unit direction of the ray through detector point (u, v) of view ov. */
static void ray_direction(const or_view *ov, double u, double v, double d[3])
{
    double m[3];
    for (int r = 0; r < 3; ++r) m[r] = ov->Minv[3 * r] * u + ov->Minv[3 * r + 1] * v + ov->Minv[3 * r + 2];
    double nrm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    for (int r = 0; r < 3; ++r) d[r] = m[r] / nrm;
}

/*
 * Reading R2: segments [a_k, b_k], a_k = t_in + k*Delta, b_k = min(a_k + Delta,
 * t_out), k = 0..ceil(L/Delta)-1; sample at the midpoint, weight b_k - a_k.
 * The callback receives (sample point, weight) for every segment.
 */
typedef void (*sample_fn)(void *ctx, const double x[3], double w);

static void march(const or_problem *pb, const or_view *ov, double u, double v, sample_fn fn,
                  void *ctx)
{
    double d[3], t_in, t_out;
    ray_direction(ov, u, v, d);
    if (!clip_ray(pb, ov->src, d, &t_in, &t_out)) return;
    double L = t_out - t_in, D = step_mm(pb);
    long K = (long)ceil(L / D);
    for (long k = 0; k < K; ++k) {
        double a = t_in + k * D;
        double b = a + D < t_out ? a + D : t_out;
        double w = b - a;
        if (!(w > 0.0)) continue;
        double t = 0.5 * (a + b), x[3];
        for (int r = 0; r < 3; ++r) x[r] = ov->src[r] + t * d[r];
        fn(ctx, x, w);
    }
}

typedef struct {
    const or_problem *pb;
    const double *vol;
    int view;
    double val, rs;
} fwd_acc;

static void to_index(const or_problem *pb, const double x[3], double g[3])
{
    for (int a = 0; a < 3; ++a) g[a] = (x[a] - pb->origin[a]) / pb->vox[a];
}

static void fwd_sample(void *vctx, const double x[3], double w)
{
    fwd_acc *c = (fwd_acc *)vctx;
    double y[3], g[3], ws;
    warp_point(c->pb, c->view, x, y);
    if (c->pb->cyl) {
        double q[3];
        world_to_cyl(c->pb, y, q);
        cyl_index(c->pb, q, g);
        c->val += w * cyl_interp(c->pb, c->vol, g, &ws);
    } else if (c->pb->dyr_tau) {
        to_index(c->pb, y, g);
        c->val += w * dyr_trilinear(c->pb, c->vol, g, c->pb->dyr_t[c->view], &ws);
    } else {
        to_index(c->pb, y, g);
        c->val += w * trilinear(c->pb, c->vol, g, &ws, NULL);
    }
    c->rs += w * ws;
}

/*
 * Reading R14: the Joseph line integral of one ray and its row sum.  Slice
 * k of principal axis m is the plane g_m = k; the crossing point's other two
 * index coordinates are interpolated bilinearly (taps outside the grid
 * contribute nothing); every crossing in front of the source counts with
 * the path length vox_m / |d_m| between neighbouring planes.
 */
static void joseph_ray(const or_problem *pb, const or_view *ov, const double *vol, double u, double v,
                       double *val, double *rs, long *ncross)
{
    long cnt = 0;
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    double d[3], g0[3], dgt[3];
    ray_direction(ov, u, v, d);
    for (int a = 0; a < 3; ++a) {
        g0[a] = (ov->src[a] - pb->origin[a]) / pb->vox[a]; /* source, index coordinates */
        dgt[a] = d[a] / pb->vox[a];                         /* index units per mm */
    }
    int m = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(dgt[a]) > fabs(dgt[m])) m = a;
    const int a1 = m == 0 ? 1 : 0, a2 = m == 2 ? 1 : 2; /* the two in-slice axes, in order */
    const double dl = 1.0 / fabs(dgt[m]);               /* mm between neighbouring planes */
    double sum = 0.0, wsum = 0.0;
    for (int k = 0; k < n[m]; ++k) {
        double t = (k - g0[m]) / dgt[m];
        if (!(t >= 0.0)) continue; /* behind the source */
        double p = g0[a1] + t * dgt[a1], q = g0[a2] + t * dgt[a2];
        double fp = floor(p), fq = floor(q);
        int ip = (int)fp, iq = (int)fq;
        double ap = p - fp, aq = q - fq;
        if (!(p > -1.0 && p < n[a1] && q > -1.0 && q < n[a2])) continue;
        ++cnt;
        for (int dq = 0; dq < 2; ++dq)
            for (int dp = 0; dp < 2; ++dp) {
                int i1 = ip + dp, i2 = iq + dq;
                if (i1 < 0 || i1 >= n[a1] || i2 < 0 || i2 >= n[a2]) continue;
                int idx[3];
                idx[m] = k;
                idx[a1] = i1;
                idx[a2] = i2;
                double wgt = (dp ? ap : 1.0 - ap) * (dq ? aq : 1.0 - aq);
                sum += wgt * (vol ? vol[((size_t)idx[2] * n[1] + idx[1]) * n[0] + idx[0]] : 1.0);
                wsum += wgt;
            }
    }
    *val = dl * sum;
    *rs = dl * wsum;
    if (ncross) *ncross = cnt;
}

/* Reading R2 on one piece [a, b] of a ray: samples of grid g (volume vg). */
static void piece(const or_problem *g, const double *vg, const double s0[3], const double d[3], double a,
                  double b, double *val, double *rs)
{
    double D = step_mm(g);
    long K = (long)ceil((b - a) / D);
    for (long k = 0; k < K; ++k) {
        double ak = a + k * D;
        double bk = ak + D < b ? ak + D : b;
        double w = bk - ak;
        if (!(w > 0.0)) continue;
        double t = 0.5 * (ak + bk), x[3], gi[3], ws;
        for (int r = 0; r < 3; ++r) x[r] = s0[r] + t * d[r];
        to_index(g, x, gi);
        *val += w * trilinear(g, vg, gi, &ws, NULL);
        *rs += w * ws;
    }
}

/* Reading R15: context pieces before and after the ROI box, the ROI piece
 * between, each on its own grid. */
static void roi_ray(const or_problem *pb, const or_view *ov, const double *vol, double u, double v,
                    double *val, double *rs)
{
    double d[3], t0, t1, r0, r1;
    *val = *rs = 0.0;
    ray_direction(ov, u, v, d);
    if (!clip_ray(pb, ov->src, d, &t0, &t1)) return;
    or_problem f = roi_part(pb);
    const double *vf = vol ? vol + grid_voxels(pb) : NULL;
    if (clip_ray(&f, ov->src, d, &r0, &r1) && r1 > t0 && r0 < t1) {
        if (r0 < t0) r0 = t0;
        if (r1 > t1) r1 = t1;
        piece(pb, vol, ov->src, d, t0, r0, val, rs);
        piece(&f, vf, ov->src, d, r0, r1, val, rs);
        piece(pb, vol, ov->src, d, r1, t1, val, rs);
    } else {
        piece(pb, vol, ov->src, d, t0, t1, val, rs);
    }
}

/* Reading R15: samples of the three pieces. */
static long roi_count(const or_problem *pb, const or_view *ov, double u, double v)
{
    double d[3], t0, t1, r0, r1;
    ray_direction(ov, u, v, d);
    if (!clip_ray(pb, ov->src, d, &t0, &t1)) return 0;
    or_problem f = roi_part(pb);
    double Dc = step_mm(pb), Df = step_mm(&f);
    if (clip_ray(&f, ov->src, d, &r0, &r1) && r1 > t0 && r0 < t1) {
        if (r0 < t0) r0 = t0;
        if (r1 > t1) r1 = t1;
        return (long)ceil((r0 - t0) / Dc) + (long)ceil((r1 - r0) / Df) + (long)ceil((t1 - r1) / Dc);
    }
    return (long)ceil((t1 - t0) / Dc);
}

/* Sec. 3.4: a pixel is the mean over its S angular sub-projections. */
static void pixel_value(const or_problem *pb, const or_view *ov, const double *vol, int view,
                        double u, double v, double *val, double *rs)
{
    double sv = 0.0, sr = 0.0;
    for (int s = 0; s < pb->n_sub; ++s) {
        if (pb->roi) {
            double a, b;
            roi_ray(pb, &ov[(size_t)view * pb->n_sub + s], vol, u, v, &a, &b);
            sv += a;
            sr += b;
            continue;
        }
        if (pb->joseph) {
            double a, b;
            joseph_ray(pb, &ov[(size_t)view * pb->n_sub + s], vol, u, v, &a, &b, NULL);
            sv += a;
            sr += b;
            continue;
        }
        fwd_acc c = {pb, vol, view, 0.0, 0.0};
        march(pb, &ov[(size_t)view * pb->n_sub + s], u, v, fwd_sample, &c);
        sv += c.val;
        sr += c.rs;
    }
    *val = sv / pb->n_sub;
    *rs = sr / pb->n_sub;
}

/*
 * A x and the row sums A 1 for the views listed in views[0..n_sel) (all views
 * if views == NULL, n_sel == n_views).  proj, rowsum: [n_sel][nv][nu].
 */
/* The Joseph projector is defined on the Cartesian grid without motion. */
static int joseph_unsupported(const or_problem *pb)
{
    if (pb->roi && (pb->joseph || pb->cyl || pb->theta || pb->coef)) return 1; /* R15: trilinear, no motion */
    if (pb->dyr_tau && (pb->roi || pb->joseph || pb->cyl || pb->theta || pb->coef || pb->bp_subvoxel > 1))
        return 1; /* R16: Cartesian trilinear projector, no motion */
    return pb->joseph && (pb->cyl || pb->theta || pb->coef);
}

int or_forward(const or_problem *pb, const double *vol, const int *views, int n_sel, double *proj,
               double *rowsum)
{
    if (joseph_unsupported(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    long npix = (long)pb->nu * pb->nv;
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < (long)n_sel * npix; ++idx) {
        int k = (int)(idx / npix);
        long p = idx % npix;
        int view = views ? views[k] : k;
        double val, rs;
        pixel_value(pb, ov, vol, view, (double)(p % pb->nu), (double)(p / pb->nu), &val, &rs);
        proj[idx] = val;
        if (rowsum) rowsum[idx] = rs;
    }
    free(ov);
    return 0;
}

/* Same integral for n arbitrary rays (view[i], continuous detector u[i], v[i]). */
int or_forward_rays(const or_problem *pb, const double *vol, const int *view, const double *u,
                    const double *v, long n, double *val, double *rowsum)
{
    if (joseph_unsupported(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) {
        double a, b;
        pixel_value(pb, ov, vol, view[i], u[i], v[i], &a, &b);
        val[i] = a;
        if (rowsum) rowsum[i] = b;
    }
    free(ov);
    return 0;
}

/* Number of samples (segments; for Joseph, slice crossings with at least
 * one tap inside the grid) of every ray of the listed views, summed. */
long or_count_samples(const or_problem *pb, const int *views, int n_sel)
{
    if (joseph_unsupported(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    long total = 0;
    double D = step_mm(pb);
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 16)
    for (long idx = 0; idx < (long)n_sel * pb->nv; ++idx) {
        int k = (int)(idx / pb->nv), iv = (int)(idx % pb->nv);
        int view = views ? views[k] : k;
        for (int s = 0; s < pb->n_sub; ++s)
            for (int iu = 0; iu < pb->nu; ++iu) {
                double d[3], t0, t1;
                const or_view *o = &ov[(size_t)view * pb->n_sub + s];
                if (pb->joseph) {
                    double a, b;
                    long c;
                    joseph_ray(pb, o, NULL, iu, iv, &a, &b, &c);
                    total += c;
                    continue;
                }
                if (pb->roi) {
                    total += roi_count(pb, o, iu, iv);
                    continue;
                }
                ray_direction(o, iu, iv, d);
                if (clip_ray(pb, o->src, d, &t0, &t1)) total += (long)ceil((t1 - t0) / D);
            }
    }
    free(ov);
    return total;
}

/* ---------------------------------------------------------------------- */
/* Correction (Sec. 4.1 "Correction kernel", Eq. (1) term 2, reading R5).  */
/* ---------------------------------------------------------------------- */

/*
 * r_i = R_i (p_i - q_i), R_i = 1/rowsum_i if rowsum_i > eps_R else 0.
 * sums[0] = sum (p - q)^2, sums[1] = sum p^2.
 */
int or_correct(long n, const double *p, const double *q, const double *rowsum, double eps_R,
               double *r, double *sums)
{
    double s0 = 0.0, s1 = 0.0;
    for (long i = 0; i < n; ++i) {
        double e = p[i] - q[i];
        double Ri = rowsum[i] > eps_R ? 1.0 / rowsum[i] : 0.0;
        if (r) r[i] = Ri * e;
        s0 += e * e;
        s1 += p[i] * p[i];
    }
    sums[0] = s0;
    sums[1] = s1;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Voxel-driven backprojection (Sec. 4.1 "Backprojection operator",       */
/* Sec. 4.3.2 weighted BP, reading R4).                                     */
/* ---------------------------------------------------------------------- */

/*
 * For voxel (ix,iy,iz): b = sum_views (1/S) sum_sub bilinear(r_view) at the
 * projected voxel centre, c = the same with r replaced by ones.  r is
 * [n_sel][nv][nu] in the order of views[].
 */
static void bp_point(const or_problem *pb, const or_view *ov, const double *r, const int *views, int n_sel,
                     const double X[3], double tau, double b_out[2], double c_out[2])
{
    double bb[2] = {0.0, 0.0}, cc[2] = {0.0, 0.0};
    size_t npix = (size_t)pb->nu * pb->nv;
    for (int k = 0; k < n_sel; ++k) {
        int view = views ? views[k] : k;
        const double *img = r + k * npix;
        /* reading R16: views from the transition on update the final value */
        const int part = (pb->dyr_tau && !(pb->dyr_t[view] < tau)) ? 1 : 0;
        double b = 0.0, c = 0.0;
        for (int s = 0; s < pb->n_sub; ++s) {
            const double *P = ov[(size_t)view * pb->n_sub + s].P;
            double h[3];
            for (int row = 0; row < 3; ++row)
                h[row] = P[4 * row] * X[0] + P[4 * row + 1] * X[1] + P[4 * row + 2] * X[2] + P[4 * row + 3];
            if (!(h[2] > 0.0)) continue;
            double u = h[0] / h[2], v = h[1] / h[2];
            if (!(u >= -1.0 && u < pb->nu && v >= -1.0 && v < pb->nv)) continue;
            double fu0 = floor(u), fv0 = floor(v);
            int iu0 = (int)fu0, iv0 = (int)fv0;
            double fu = u - fu0, fv = v - fv0;
            int ulo = 0, uhi = pb->nu - 1, vlo = 0, vhi = pb->nv - 1;
            if (pb->bp_window) {
                const int *wd = pb->bp_window + 4 * (size_t)view;
                ulo = wd[0] > ulo ? wd[0] : ulo;
                uhi = wd[1] < uhi ? wd[1] : uhi;
                vlo = wd[2] > vlo ? wd[2] : vlo;
                vhi = wd[3] < vhi ? wd[3] : vhi;
            }
            for (int dv = 0; dv < 2; ++dv)
                for (int du = 0; du < 2; ++du) {
                    int iu = iu0 + du, iv = iv0 + dv;
                    if (iu < ulo || iu > uhi || iv < vlo || iv > vhi) continue;
                    double wgt = (du ? fu : 1.0 - fu) * (dv ? fv : 1.0 - fv);
                    b += wgt * img[(size_t)iv * pb->nu + iu] / pb->n_sub;
                    c += wgt / pb->n_sub;
                }
        }
        bb[part] += b;
        cc[part] += c;
    }
    b_out[0] = bb[0];
    b_out[1] = bb[1];
    c_out[0] = cc[0];
    c_out[1] = cc[1];
}

static void bp_voxel(const or_problem *pb, const or_view *ov, const double *r, const int *views,
                     int n_sel, int ix, int iy, int iz, double b_out[2], double c_out[2])
{
    const int sv = pb->bp_subvoxel > 1 ? pb->bp_subvoxel : 1;
    const int i[3] = {ix, iy, iz};
    const double tau = pb->dyr_tau ? pb->dyr_tau[((size_t)iz * pb->ny + iy) * pb->nx + ix] : 0.0;
    double b[2] = {0.0, 0.0}, c[2] = {0.0, 0.0};
    for (int az = 0; az < sv; ++az)
        for (int ay = 0; ay < sv; ++ay)
            for (int ax = 0; ax < sv; ++ax) {
                const int a[3] = {ax, ay, az};
                double X[3];
                if (pb->cyl) {
                    /* reading R13: sub-point of the cylindrical voxel, mapped to world */
                    double gi[3], q[3];
                    for (int d = 0; d < 3; ++d) gi[d] = i[d] + (a[d] + 0.5) / sv - 0.5;
                    double r = (gi[0] + 0.5) * pb->cyl_dr;
                    double phi = (gi[1] + 0.5) * (6.283185307179586476925286766559 / pb->ny);
                    q[0] = r * cos(phi);
                    q[1] = r * sin(phi);
                    q[2] = (gi[2] - 0.5 * (pb->nz - 1)) * pb->cyl_dz;
                    cyl_to_world(pb, q, X);
                } else {
                    for (int d = 0; d < 3; ++d)
                        X[d] = pb->origin[d] + (i[d] + (a[d] + 0.5) / sv - 0.5) * pb->vox[d];
                }
                double bb[2], cc[2];
                bp_point(pb, ov, r, views, n_sel, X, tau, bb, cc);
                for (int q = 0; q < 2; ++q) {
                    b[q] += bb[q];
                    c[q] += cc[q];
                }
            }
    for (int q = 0; q < 2; ++q) {
        b_out[q] = b[q] / ((double)sv * sv * sv);
        c_out[q] = c[q] / ((double)sv * sv * sv);
    }
}

/*
 * Eq. (1) term 3 with weights: x_j += alpha * w_j * C_j * b_j, C_j = 1/c_j if
 * c_j > eps_C else 0.  x may be NULL (then only b, c are produced); w may be
 * NULL (w = 1); b, c may be NULL.
 */
static int dyrect_unsupported_bp(const or_problem *pb)
{
    return pb->dyr_tau && (pb->cyl || pb->roi || pb->bp_subvoxel > 1);
}

int or_backproject(const or_problem *pb, const double *r, const int *views, int n_sel,
                   const double *w, double alpha, double eps_C, double *x, double *b_out,
                   double *c_out)
{
    if (dyrect_unsupported_bp(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    long nc = grid_voxels(pb);
    or_problem f = pb->roi ? roi_part(pb) : *pb;
    long nvox = nc + (pb->roi ? grid_voxels(&f) : 0);
    const int parts = pb->dyr_tau ? 2 : 1; /* reading R16: mu0 then mu1 */
#pragma omp parallel for schedule(dynamic, 64)
    for (long j = 0; j < nvox; ++j) {
        const or_problem *g = j < nc ? pb : &f; /* reading R15: the ROI voxels follow */
        long jj = j < nc ? j : j - nc;
        int ix = (int)(jj % g->nx), iy = (int)((jj / g->nx) % g->ny), iz = (int)(jj / ((long)g->nx * g->ny));
        double b[2], c[2];
        bp_voxel(g, ov, r, views, n_sel, ix, iy, iz, b, c);
        for (int q = 0; q < parts; ++q) {
            long jo = j + q * nvox;
            if (b_out) b_out[jo] = b[q];
            if (c_out) c_out[jo] = c[q];
            if (x) {
                double C = c[q] > eps_C ? 1.0 / c[q] : 0.0;
                x[jo] += alpha * (w ? w[jo] : 1.0) * C * b[q];
            }
        }
    }
    free(ov);
    return 0;
}

/* b_j, c_j for an explicit list of voxels (flat indices). */
int or_backproject_voxels(const or_problem *pb, const double *r, const int *views, int n_sel,
                          const long *vox, long n_vox, double *b_out, double *c_out)
{
    if (dyrect_unsupported_bp(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    long nc = grid_voxels(pb);
    or_problem f = pb->roi ? roi_part(pb) : *pb;
#pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < n_vox; ++q) {
        long j = vox[q];
        const or_problem *g = (pb->roi && j >= nc) ? &f : pb;
        if (g == &f) j -= nc;
        int ix = (int)(j % g->nx), iy = (int)((j / g->nx) % g->ny), iz = (int)(j / ((long)g->nx * g->ny));
        double b[2], c[2];
        bp_voxel(g, ov, r, views, n_sel, ix, iy, iz, b, c);
        b_out[q] = b[0];
        c_out[q] = c[0];
        if (pb->dyr_tau) { /* reading R16: the mu1 parts follow the mu0 parts */
            b_out[n_vox + q] = b[1];
            c_out[n_vox + q] = c[1];
        }
    }
    free(ov);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Matched adjoint: exact transpose of the forward above.                  */
/* ---------------------------------------------------------------------- */

typedef struct {
    const or_problem *pb;
    int view;
    double y;     /* value scattered along this ray (already / S) */
    double *acc;  /* volume accumulator of this thread           */
} adj_acc;

static void adj_sample(void *vctx, const double x[3], double w)
{
    adj_acc *c = (adj_acc *)vctx;
    const or_problem *pb = c->pb;
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    double yy[3], g[3];
    warp_point(pb, c->view, x, yy);
    to_index(pb, yy, g);
    for (int a = 0; a < 3; ++a)
        if (!(g[a] >= -1.0 && g[a] < (double)n[a])) return;
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]);
        i0[a] = (int)fl;
        f[a] = g[a] - fl;
    }
    const size_t nvox = (size_t)n[0] * n[1] * n[2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                if (ix < 0 || ix >= n[0] || iy < 0 || iy >= n[1] || iz < 0 || iz >= n[2]) continue;
                double wt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                size_t j = ((size_t)iz * n[1] + iy) * n[0] + ix;
                /* reading R16: the tap's value came from mu1 from the transition on */
                if (pb->dyr_tau && !(pb->dyr_t[c->view] < pb->dyr_tau[j])) j += nvox;
                c->acc[j] += c->y * w * wt;
            }
}

/* vol_out (overwritten) = A^T y for y [n_sel][nv][nu]. */
int or_adjoint(const or_problem *pb, const double *y, const int *views, int n_sel, double *vol_out)
{
    /* the transpose of the trilinear projector on the Cartesian grid only */
    if (pb->cyl || pb->joseph || pb->roi || joseph_unsupported(pb)) return OR_E_ARG;
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    size_t nvox = (size_t)pb->nx * pb->ny * pb->nz * (pb->dyr_tau ? 2 : 1);
    long npix = (long)pb->nu * pb->nv;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *buf = (double *)calloc((size_t)nth * nvox, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *acc = buf + (size_t)tid * nvox;
#pragma omp for schedule(dynamic, 64)
        for (long idx = 0; idx < (long)n_sel * npix; ++idx) {
            int k = (int)(idx / npix);
            long p = idx % npix;
            int view = views ? views[k] : k;
            if (y[idx] == 0.0) continue;
            for (int s = 0; s < pb->n_sub; ++s) {
                adj_acc c = {pb, view, y[idx] / pb->n_sub, acc};
                march(pb, &ov[(size_t)view * pb->n_sub + s], (double)(p % pb->nu), (double)(p / pb->nu),
                      adj_sample, &c);
            }
        }
    }
    for (size_t j = 0; j < nvox; ++j) {
        double s = 0.0;
        for (int t = 0; t < nth; ++t) s += buf[(size_t)t * nvox + j];
        vol_out[j] = s;
    }
    free(buf);
    free(ov);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Motion-parameter gradient: chain rule through the warp (reading R6).    */
/* ---------------------------------------------------------------------- */

typedef struct {
    const or_problem *pb;
    const double *vol;
    int view;
    double g;       /* upstream gradient of this ray, already / S */
    double *gth;    /* [15] of this view, this thread             */
    double *gcoef;  /* [8*8*8*3], this thread                      */
} grad_acc;

static void grad_sample(void *vctx, const double x[3], double w)
{
    grad_acc *c = (grad_acc *)vctx;
    const or_problem *pb = c->pb;
    const double *th = pb->theta ? pb->theta + 15 * (size_t)c->view : NULL;
    double s = pb->s_view ? pb->s_view[c->view] : 0.0;
    /* x' = A (R x + t) */
    double R[9], dR[27], q[3], xp[3];
    double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const double *A = th ? th + 6 : I3;
    if (th) {
        rotation(th, R, dR);
        matvec3(R, x, q);
        for (int a = 0; a < 3; ++a) q[a] += th[3 + a];
        matvec3(A, q, xp);
    } else {
        memcpy(q, x, sizeof q);
        memcpy(xp, x, sizeof xp);
    }
    double u[3] = {0, 0, 0}, J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (pb->coef) displacement(pb, xp, u, J);
    double yv[3], gidx[3], gl[3];
    for (int a = 0; a < 3; ++a) yv[a] = xp[a] + s * u[a];
    to_index(pb, yv, gidx);
    trilinear(pb, c->vol, gidx, NULL, gl);
    /* dmu/dy in mm^-1 */
    double gy[3] = {gl[0] / pb->vox[0], gl[1] / pb->vox[1], gl[2] / pb->vox[2]};
    double scale = c->g * w;
    if (scale == 0.0) return;
    /* dmu/dx' = gy^T (I + s J) */
    double gxp[3];
    for (int col = 0; col < 3; ++col)
        gxp[col] = gy[col] + s * (gy[0] * J[col] + gy[1] * J[3 + col] + gy[2] * J[6 + col]);
    if (th) {
        /* d x'/d t = A; d x'/d A_ab = e_a q_b; d x'/d omega_i = A dR_i x */
        for (int col = 0; col < 3; ++col) {
            double v = gxp[0] * A[col] + gxp[1] * A[3 + col] + gxp[2] * A[6 + col];
            c->gth[3 + col] += scale * v;
        }
        for (int a = 0; a < 3; ++a)
            for (int b2 = 0; b2 < 3; ++b2) c->gth[6 + 3 * a + b2] += scale * gxp[a] * q[b2];
        for (int i = 0; i < 3; ++i) {
            double dq[3], dxp[3];
            matvec3(dR + 9 * i, x, dq);
            matvec3(A, dq, dxp);
            c->gth[i] += scale * (gxp[0] * dxp[0] + gxp[1] * dxp[1] + gxp[2] * dxp[2]);
        }
    }
    if (pb->coef && s != 0.0) {
        /* d y / d c_{ijk,comp} = s * beta-product * e_comp */
        double xi[3];
        int cl[3];
        for (int a = 0; a < 3; ++a) xi[a] = spline_coord(pb, a, xp[a], &cl[a]);
        int lo[3], hi[3];
        spline_support(xi, lo, hi);
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    double wgt = bspline3(xi[0] - i) * bspline3(xi[1] - j) * bspline3(xi[2] - k);
                    if (wgt == 0.0) continue;
                    double *gc = c->gcoef + 3 * (size_t)((k * 8 + j) * 8 + i);
                    for (int comp = 0; comp < 3; ++comp) gc[comp] += scale * s * wgt * gy[comp];
                }
    }
}

/*
 * grad_theta [n_views][15] (overwritten for all views, zero for views not
 * listed) and grad_coef [8][8][8][3] (overwritten) of L = sum_i g_i (A x)_i,
 * g [n_sel][nv][nu].  Either output may be NULL.
 */
int or_motion_grad(const or_problem *pb, const double *vol, const double *g, const int *views,
                   int n_sel, double *grad_theta, double *grad_coef)
{
    if (pb->cyl || pb->joseph || pb->roi || pb->dyr_tau) return OR_E_ARG; /* trilinear projector, one Cartesian grid */
    int err;
    or_view *ov = setup_all_views(pb, &err);
    if (!ov) return err;
    long npix = (long)pb->nu * pb->nv;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    size_t nth_len = 15 * (size_t)pb->n_views, ncoef = 8 * 8 * 8 * 3;
    double *bth = (double *)calloc((size_t)nth * nth_len, sizeof(double));
    double *bco = (double *)calloc((size_t)nth * ncoef, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 64)
        for (long idx = 0; idx < (long)n_sel * npix; ++idx) {
            int k = (int)(idx / npix);
            long p = idx % npix;
            int view = views ? views[k] : k;
            if (g[idx] == 0.0) continue;
            for (int s = 0; s < pb->n_sub; ++s) {
                grad_acc c = {pb, vol, view, g[idx] / pb->n_sub,
                              bth + (size_t)tid * nth_len + 15 * (size_t)view,
                              bco + (size_t)tid * ncoef};
                march(pb, &ov[(size_t)view * pb->n_sub + s], (double)(p % pb->nu), (double)(p / pb->nu),
                      grad_sample, &c);
            }
        }
    }
    if (grad_theta)
        for (size_t q = 0; q < nth_len; ++q) {
            double s = 0.0;
            for (int t = 0; t < nth; ++t) s += bth[(size_t)t * nth_len + q];
            grad_theta[q] = s;
        }
    if (grad_coef)
        for (size_t q = 0; q < ncoef; ++q) {
            double s = 0.0;
            for (int t = 0; t < nth; ++t) s += bco[(size_t)t * ncoef + q];
            grad_coef[q] = s;
        }
    free(bth);
    free(bco);
    free(ov);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* SIRT loop: Eq. (1) with one subset holding every view (Sec. 2.3.2).     */
/* ---------------------------------------------------------------------- */

/*
 * Iteration k: q = A x_k, rho_k = ||p - q|| / ||p||, hist[k] = rho_k; stop if
 * rho_k <= tol; otherwise x_{k+1} = x_k + alpha w C B R (p - q).  iters_done =
 * number of updates applied.  Returns 1 if a residual was not finite.
 */
int or_sirt(const or_problem *pb, double *x, const double *p, int max_iter, double alpha,
            const double *w, double tol, double eps_R, double eps_C, double *hist, int *iters_done)
{
    long n = (long)pb->n_views * pb->nu * pb->nv;
    double *q = (double *)malloc(sizeof(double) * n);
    double *rs = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * n);
    int ret = 0, k;
    *iters_done = 0;
    for (k = 0; k < max_iter; ++k) {
        int e = or_forward(pb, x, NULL, pb->n_views, q, rs);
        if (e) { ret = e; break; }
        double sums[2];
        or_correct(n, p, q, rs, eps_R, r, sums);
        double rho = sums[1] > 0.0 ? sqrt(sums[0] / sums[1]) : sqrt(sums[0]);
        if (hist) hist[k] = rho;
        if (!isfinite(rho)) { ret = 1; break; }
        if (rho <= tol) break;
        or_backproject(pb, r, NULL, pb->n_views, w, alpha, eps_C, x, NULL, NULL);
        *iters_done = k + 1;
    }
    free(q);
    free(rs);
    free(r);
    return ret;
}

/* ---------------------------------------------------------------------- */
/* Ordered-subset SIRT: Eq. (1) evaluated on the views of one subset at a   */
/* time (Sec. 2.3.2, index sets P_k).                                       */
/* ---------------------------------------------------------------------- */

/*
 * One cycle visits the subsets in order; subset S updates
 *   x += alpha w C_S B_S R_S (p_S - A_S x),
 * C_S the column sums of the backprojector over the views of S only.
 * Reading (the paper leaves the stopping rule to Rex): the residual of a cycle
 * is the running residual sqrt(sum_S ||p_S - A_S x_(S)||^2 / sum_S ||p_S||^2),
 * each term taken at the iterate x_(S) that subset S starts from (for subsets
 * that partition the views the denominator is ||p||^2); after cycle c it is
 * hist[c], and the loop stops once it is <= tol.  With a single subset holding
 * every view this is SIRT with the test after the update.
 * views: concatenated subset view lists; offsets[0..n_sub_sets].
 */
int or_os_sirt(const or_problem *pb, double *x, const double *p, const int *views, const int *offsets,
               int n_sets, int max_cycles, double alpha, const double *w, double tol, double eps_R,
               double eps_C, double *hist, int *cycles_done)
{
    long npix = (long)pb->nu * pb->nv;
    int maxlen = 0;
    for (int s = 0; s < n_sets; ++s)
        if (offsets[s + 1] - offsets[s] > maxlen) maxlen = offsets[s + 1] - offsets[s];
    double *q = (double *)malloc(sizeof(double) * (size_t)(maxlen > 0 ? maxlen : 1) * npix);
    double *rs = (double *)malloc(sizeof(double) * (size_t)(maxlen > 0 ? maxlen : 1) * npix);
    double *r = (double *)malloc(sizeof(double) * (size_t)(maxlen > 0 ? maxlen : 1) * npix);
    double *ps = (double *)malloc(sizeof(double) * (size_t)(maxlen > 0 ? maxlen : 1) * npix);
    int ret = 0;
    *cycles_done = 0;
    for (int c = 0; c < max_cycles && !ret; ++c) {
        double acc = 0.0, p2 = 0.0;
        for (int s = 0; s < n_sets; ++s) {
            const int *vs = views + offsets[s];
            int n = offsets[s + 1] - offsets[s];
            if (n <= 0) continue;
            int e = or_forward(pb, x, vs, n, q, rs);
            if (e) { ret = e; break; }
            for (int k = 0; k < n; ++k) memcpy(ps + (size_t)k * npix, p + (size_t)vs[k] * npix, sizeof(double) * npix);
            double sums[2];
            or_correct((long)n * npix, ps, q, rs, eps_R, r, sums);
            acc += sums[0];
            p2 += sums[1];
            or_backproject(pb, r, vs, n, w, alpha, eps_C, x, NULL, NULL);
        }
        if (ret) break;
        double rho = p2 > 0.0 ? sqrt(acc / p2) : sqrt(acc);
        if (hist) hist[c] = rho;
        *cycles_done = c + 1;
        if (!isfinite(rho)) { ret = 1; break; }
        if (rho <= tol) break;
    }
    free(q);
    free(rs);
    free(r);
    free(ps);
    return ret;
}
