/*
 * ctrex.h -- C ABI of the GB300 (sm_103a) CTrex projection library.
 *
 * The library implements the projection-correction-backprojection loop of
 * ordered-subset SIRT, Eq. (1) of the CTrex paper (arxiv 2609.30166):
 *
 *     mu_{k+1} = mu_k + alpha C A^T R (p - A mu_k)
 *
 * with A the ray-driven cone-beam projector (Sec. 4.1 "Projection operator"),
 * R the detector-space correction (Sec. 4.1 "Correction kernel") and C A^T the
 * voxel-driven, voxel-weighted backprojector (Sec. 4.1 "Backprojection
 * operator", Sec. 4.3.2).  Geometry is one 3x4 projection matrix per view and
 * angular sub-sample (Sec. 2.2.1, Sec. 3.4); motion is a per-view rigid+affine
 * pose plus a smooth deformation applied during ray traversal (Sec. 2.2.2,
 * Sec. 3.1.1, Sec. 4.2.1).
 *
 * Conventions
 *   volume   vol[nz][ny][nx], x fastest; voxel (ix,iy,iz) centred at
 *            origin + (ix,iy,iz) * vox (mm).
 *   images   proj[k][nv][nu], u fastest; k indexes the views of the call's
 *            view list (all views in order when the list is NULL).  Pixel
 *            (iu,iv) is centred at detector coordinate (iu,iv).
 *   P        double P[n_views][n_sub][3][4], row-major; maps homogeneous
 *            world mm to homogeneous detector coordinates.  P and kappa*P
 *            (kappa != 0) describe the same projection.
 *   dtypes   CTREX_F32 or CTREX_BF16 storage; every sum is accumulated in FP32.
 *
 * Ownership and execution
 *   Every data pointer (volumes, images, weights, gradients, view lists) is a
 *   DEVICE pointer owned by the caller, unless a comment says host.  The
 *   context owns copies of the geometry and motion parameters and its own
 *   scratch buffers.  Calls enqueue work on the context's stream and return
 *   without synchronising, except where stated (sirt_iterate reads one
 *   residual per iteration; the *_host entry points copy their results back).
 *   A context must not be used from two host threads at once.
 *
 * Errors
 *   Every call returns CTREX_OK (0) or a negative CTREX_E_* code; the message
 *   of the last failure is in ctrex_last_error(ctx).  No C++ exception crosses
 *   this interface.  A call that fails argument validation enqueues no work.
 */
#ifndef CTREX_H
#define CTREX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctrex_ctx ctrex_ctx;

typedef enum { CTREX_F32 = 0, CTREX_BF16 = 1 } ctrex_dtype;

enum {
    CTREX_OK = 0,
    CTREX_E_ARG = -1,          /* NULL pointer, bad enum, bad scalar         */
    CTREX_E_SHAPE = -2,        /* size out of range, view index out of range */
    CTREX_E_DTYPE = -3,        /* dtype not supported for this operation     */
    CTREX_E_GEOMETRY = -4,     /* singular P, or depth <= 0 at volume centre */
    CTREX_E_CUDA = -5,         /* CUDA runtime error (message in last_error) */
    CTREX_E_DIVERGED = -6,     /* non-finite residual in sirt_iterate        */
    CTREX_E_DEVICE_CHECK = -7, /* a kernel's own bounds check fired          */
    CTREX_E_NOMEM = -8,        /* device allocation failed                   */
    CTREX_E_STATE = -9         /* call needs set_geometry / set_motion first */
};

/* Volume grid: sizes, voxel pitch (mm) and centre of voxel (0,0,0) (mm). */
typedef struct {
    int nx, ny, nz;
    double vox[3];
    double origin[3];
} ctrex_vol_grid;

/* Detector grid: nu columns (u fastest), nv rows. */
typedef struct {
    int nu, nv;
} ctrex_det_grid;

/*
 * Aligned cylindrical volume domain (Sec. 3.5; projector / backprojector
 * adaptations in Sec. 4.2 / 4.3): n_r rings of pitch dr (mm), n_phi
 * sectors of 2 pi / n_phi, n_z slices of pitch dz (mm).  pose is a rigid
 * 3x4 row-major map q = Rc x + tc from world mm to the cylinder frame, whose
 * z axis is the cylinder axis.  Voxel (i, j, k) sits at frame point r =
 * (i + 1/2) dr, phi = (j + 1/2) 2 pi / n_phi, z = (k - (n_z - 1)/2) dz.
 */
typedef struct {
    int n_r, n_phi, n_z;
    double dr, dz;
    double pose[12];
} ctrex_cyl_grid;

/* Library version string (static storage). */
const char *ctrex_version(void);

/*
 * Create a context on CUDA device `device` that enqueues work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the context; destroy it with ctrex_destroy.
 */
int ctrex_create(ctrex_ctx **out, int device, void *cuda_stream);

/* Free the context and every buffer it owns (synchronises its stream). */
int ctrex_destroy(ctrex_ctx *ctx);

/* Change the stream later calls enqueue on. */
int ctrex_set_stream(ctrex_ctx *ctx, void *cuda_stream);

/* Message of the last failed call on ctx (static text if ctx is NULL). */
const char *ctrex_last_error(const ctrex_ctx *ctx);

/*
 * Synchronise the context's stream and report whether a kernel's own bounds
 * check fired since the last call (a view index outside [0, n_views) in a
 * view list): CTREX_E_DEVICE_CHECK, and the flag is cleared; else CTREX_OK.
 * Kernels never trap: an out-of-range view is skipped (its output is zero).
 */
int ctrex_device_status(ctrex_ctx *ctx);

/*
 * Sec. 2.2.1 single-projection geometry, Sec. 2.2.2 trajectory as a sequence
 * of matrices, Sec. 3.4 angular sub-projections.
 *   P         HOST double [n_views][n_sub][3][4]; copied, may be freed after.
 *   n_views   >= 1; n_sub >= 1 sub-angle matrices per view (motion blur:
 *             a pixel is the mean of its n_sub sub-projections).
 *   vol, det  grids (HOST structs); sizes >= 1, pitches > 0.
 *   step_vox  ray step as a fraction of the smallest voxel pitch, in [0.01, 100].
 * Each P is sign-normalised so that the volume centre has positive depth.
 * Fails with CTREX_E_GEOMETRY if a left 3x3 block is singular
 * (|det| <= 1e-12 |M|_F^3) or the volume centre lies on a source plane.
 * Clears any motion set earlier.
 */
int ctrex_set_geometry(ctrex_ctx *ctx, const double *P, int n_views, int n_sub,
                       const ctrex_vol_grid *vol, const ctrex_det_grid *det, double step_vox);

/*
 * The same projection set-up on the aligned cylindrical domain (Sec. 3.5).
 * Every operator then works on volumes of [n_z][n_phi][n_r] (r fastest):
 *   - the projector clips each ray to the bounding cylinder r <= n_r dr,
 *     |z| <= n_z dz / 2 (instead of the box) and maps each sample to
 *     (r, phi, z) before the lookup: trilinear interpolation in the index
 *     coordinates r/dr - 1/2 (clamped to >= 0: inside the first ring centre
 *     the ring-0 value is used), phi / (2 pi / n_phi) - 1/2 (periodic) and
 *     z/dz + (n_z - 1)/2, zero outside in r and z; fixed step step_vox *
 *     min(dr, dz) as for the box;
 *   - the backprojector maps each voxel point to the frame, then to the
 *     detector; its accumulation, C, w, alpha, windows and sub-voxel points
 *     are unchanged;
 *   - R uses the threshold 1e-6 * min(dr, dz).
 *   P        HOST double [n_views][n_sub][3][4] (world mm -> pixels); the
 *            pose is folded into them, so they are copied.
 *   cyl      HOST grid and pose (pose rotation orthonormal within 1e-9,
 *            det +1, else CTREX_E_ARG); n_phi >= 3.
 * Volumes are sampled through a texture atlas; one that exceeds the
 * device's 2D texture limits fails at the first projection with
 * CTREX_E_SHAPE.  set_motion (with parameters), adjoint_project and
 * motion_grad return CTREX_E_STATE on this domain.  Clears any motion, BP
 * window and earlier geometry; ctrex_set_geometry switches back.
 */
int ctrex_set_geometry_cylinder(ctrex_ctx *ctx, const double *P, int n_views, int n_sub,
                                const ctrex_cyl_grid *cyl, const ctrex_det_grid *det, double step_vox);

/*
 * Sec. 2.2.2 affine volume pose (rigid then affine) and Sec. 3.1.1 / 4.2.1
 * sample-point warping.  Sample point x (mm, volume frame) of view v is
 * mapped to y = x' + s_v u(x'), x' = A_v (R(omega_v) x + t_v), before the
 * volume lookup; u is a uniform cubic B-spline on an 8^3 control grid whose
 * points i = 0..7 sit at box_min + (i - 1) * box_len / 5 per axis (spline
 * coordinate clamped to [1, 6]).
 *   theta   DEVICE float [n_views][15] = (omega(3) Rodrigues, t(3) mm,
 *           A(9) row-major), or NULL for no pose change.
 *   coef    DEVICE float [8][8][8][3] (z, y, x, component; mm), or NULL.
 *   s_view  DEVICE float [n_views] time scale of the deformation, or NULL
 *           (then s_v = 0).
 *   margin  mm in [0, largest box edge]; the ray clip box is the volume box
 *           dilated by this much (fixed, so sample positions do not depend
 *           on theta).
 * The arrays are copied (device to device, on the stream).  Passing all
 * three as NULL switches motion off.
 */
int ctrex_set_motion(ctrex_ctx *ctx, const float *theta, const float *coef, const float *s_view,
                     double margin_mm);

/*
 * Extended field of view (Sec. 3.6, Sec. 4.3.2): per-view detector window of
 * the BACKPROJECTOR.  View v's backprojection sees only detector columns
 * u_lo..u_hi and rows v_lo..v_hi; taps outside count as off the detector for
 * both the sum b and its normalisation c.  The forward projector keeps the
 * whole detector.  Moving the inner edge of an offset-centre-of-rotation scan
 * per view (and per iteration) to a random column between the physical edge
 * and the projected centre of rotation is the paper's remedy for the central
 * field-of-view ring.
 *   window  HOST int32 [n_views][4] = (u_lo, u_hi, v_lo, v_hi), clipped to the
 *           detector; copied (the call synchronises the stream).  NULL resets
 *           to the whole detector.  set_geometry also resets it.
 */
int ctrex_set_bp_window(ctrex_ctx *ctx, const int *window);

/*
 * Sub-voxel backprojection (Sec. 4.3.2, motion-blur compensation: the
 * backprojector accumulates onto a finer voxel grid).  With s > 1 every
 * backprojection (ctrex_back_project and the SIRT / OS-SIRT loops) takes,
 * for voxel j, the means over the s^3 points at index offsets
 * ((a + 1/2)/s - 1/2), a = 0..s-1, on each axis, of the bilinear correction
 * sample and of its in-range weight; C_j is 1 / (that mean weight summed
 * over the views).  The finer grid is not stored.  Equivalent to a
 * backprojection of b and c onto the s-times finer grid followed by the
 * s x s x s block mean.  The forward projector is unchanged.
 *   s        1 (off, the default) .. CTREX_MAX_SUBVOXEL, else CTREX_E_ARG.
 * The setting belongs to the context and survives set_geometry.
 */
#define CTREX_MAX_SUBVOXEL 8
int ctrex_set_bp_subvoxel(ctrex_ctx *ctx, int s);

/*
 * Forward projector of every forward call (fwd_project, fwd_correct, the
 * SIRT loops and count_samples; the backprojector is unchanged):
 *   CTREX_PROJ_TRILINEAR  (default) fixed-step trilinear quadrature, Sec. 4.1.
 *   CTREX_PROJ_JOSEPH     classical Joseph (Sec. 4.1 cites Joseph's method):
 *       the principal axis m of a ray is the one whose index coordinate
 *       changes fastest along it (the lowest on ties); every slice k = 0..N_m-1
 *       crossed in front of the source is interpolated bilinearly at the
 *       crossing (zero outside the grid) and weighted with vox_m / |d_m| (d
 *       the unit direction), the path length between neighbouring planes.
 *       Row sums are the same sum of in-range weights.  count_samples then
 *       counts slice crossings with a tap inside the grid.  The context keeps
 *       the volume as x-, y- and z-slice stacks in one texture atlas (three
 *       copies; CTREX_E_SHAPE at the first projection if it exceeds the
 *       device's 2D texture limits).
 * Joseph is defined on the Cartesian grid without motion: CTREX_E_STATE if
 * the cylindrical domain or motion is set, and set_motion, adjoint_project
 * and motion_grad return CTREX_E_STATE while it is selected.
 * set_geometry_cylinder resets the projector to trilinear.  Unknown kind:
 * CTREX_E_ARG.
 */
/*
 * Multi-resolution ROI (Sec. 3.7; its simultaneous form, where the
 * projector's sampling switches between a high-resolution ROI volume and the
 * low-resolution context volume by ray position).  roi is a second, finer
 * Cartesian grid (same conventions as ctrex_vol_grid) whose box lies inside
 * the grid of set_geometry (the context grid); else CTREX_E_ARG.  Once set,
 * every volume buffer (vol, w) of the projection, backprojection and SIRT
 * calls holds the context grid's voxels followed by the ROI grid's
 * (nx ny nz + roi nx ny nz elements):
 *   - the forward clips each ray to the context box and splits it at the ROI
 *     box; the context pieces and the ROI piece each follow the fixed-step
 *     truncated-midpoint rule with their own grid's step (step_vox times its
 *     smallest pitch) and sample their own grid (zero-padded trilinear);
 *     row sums add over the pieces;
 *   - the backprojector updates both grids, each with its own column sums C
 *     (the context grid everywhere, also under the ROI);
 *   - count_samples counts the samples of all pieces.
 * The ROI path is the trilinear projector on a Cartesian grid without
 * motion: CTREX_E_STATE on the cylindrical domain, with motion or with the
 * Joseph projector (and set_motion, set_projector(JOSEPH) and
 * adjoint_project return CTREX_E_STATE while an ROI is set).  Both grids are
 * sampled through texture atlases (CTREX_E_SHAPE at the first projection if
 * one exceeds the device's 2D texture limits).  NULL removes the ROI;
 * set_geometry and set_geometry_cylinder remove it too.
 */
int ctrex_set_roi(ctrex_ctx *ctx, const ctrex_vol_grid *roi);

/*
 * Event-based 4D reconstruction (Sec. 3.3): temporal behaviour is
 * parameterised per voxel by three fields, an initial value mu0, a final
 * value mu1 and a transition time tau, and the projector and backprojector
 * act on them directly.  Reading: view v, acquired at time t_view[v], sees
 * mu0_j where t_view[v] < tau_j and mu1_j elsewhere (one irreversible change
 * per voxel); the forward projector samples that per-view volume (the choice
 * is made per trilinear tap; weights and row sums are those of the static
 * projector); the backprojector splits Eq. (1) term 3 by the same rule: the
 * views before tau_j update mu0_j, normalised by their own column sum, the
 * others update mu1_j.  tau is an input: its update rule is not part of the
 * paper.  Once set, every volume buffer (vol, w) of fwd_project,
 * fwd_correct, back_project, adjoint_project (the exact transpose with
 * respect to (mu0, mu1)), sirt_iterate, os_sirt_iterate and sirt_host holds
 * mu0 followed by mu1 (2 nx ny nz elements).
 *   tau     DEVICE float [nz][ny][nx] transition times, or NULL to switch
 *           the model off.
 *   t_view  DEVICE float [n_views] acquisition time of each view (same
 *           unit as tau).
 * Both are copied on the stream (the caller may free them once the stream
 * has passed this call).  The context also keeps tau as a texture atlas and
 * the smallest and largest tau of each 8^3 brick (over the brick and the
 * voxel past each upper face; 8 bytes per brick), with which the projector
 * takes one field for a whole footprint when the view's time lies on one
 * side of both (same result as the per-tap choice; a NaN tau keeps its
 * brick on the per-tap path).  Defined for the trilinear projector on the
 * Cartesian grid without motion, ROI or sub-voxel backprojection:
 * CTREX_E_STATE otherwise (and set_motion, set_roi, set_projector(Joseph),
 * set_bp_subvoxel(s > 1) and motion_grad return CTREX_E_STATE while it is
 * on).  CTREX_E_SHAPE if the volume exceeds the device's 2D texture limits.
 * set_geometry and set_geometry_cylinder switch it off.
 */
int ctrex_set_dyrect(ctrex_ctx *ctx, const float *tau, const float *t_view);

#define CTREX_PROJ_TRILINEAR 0
#define CTREX_PROJ_JOSEPH 1
int ctrex_set_projector(ctrex_ctx *ctx, int kind);

/*
 * A x (Sec. 4.1 projection operator; Sec. 3.4 mean over sub-angles; motion
 * if set).  Ray from the source through the pixel centre, clipped to the
 * box, fixed-step truncated-midpoint quadrature with trilinear interpolation
 * (zero outside the grid), weights = segment lengths in mm.
 *   vol      DEVICE [nz][ny][nx] of vol_dtype.
 *   proj     DEVICE [n_idx][nv][nu] of proj_dtype (overwritten).
 *   view_idx DEVICE int32 [n_idx] (each in [0, n_views)), or NULL = all
 *            views (then n_idx must be n_views, or 0 for an empty call).
 *   rowsum   DEVICE float [n_idx][nv][nu] receiving A 1, or NULL.
 */
int ctrex_fwd_project(ctrex_ctx *ctx, const void *vol, int vol_dtype, void *proj, int proj_dtype,
                      float *rowsum, const int *view_idx, int n_idx);

/*
 * Fused A x and correction (Eq. (1) terms 1 and 2, Sec. 4.1 correction
 * kernel): r_i = R_i (p_i - (A x)_i) with R_i = 1 / (A 1)_i if that row sum
 * exceeds 1e-6 * (smallest voxel pitch), else 0.  A x is never stored.
 *   p        DEVICE measured images [n_idx][nv][nu] of p_dtype.
 *   r        DEVICE output [n_idx][nv][nu] of r_dtype (may alias nothing).
 *   sums     DEVICE double [2] receiving (sum (p - Ax)^2, sum p^2) over all
 *            pixels of the listed views (fixed-order reduction: bitwise
 *            reproducible), or NULL.
 */
int ctrex_fwd_correct(ctrex_ctx *ctx, const void *vol, int vol_dtype, const void *p, int p_dtype,
                      void *r, int r_dtype, double *sums, const int *view_idx, int n_idx);

/*
 * Voxel-driven backprojection with normalisation and update (Eq. (1) term
 * 3, Sec. 4.1 backprojection operator, Sec. 4.3.2 weighted BP).  For voxel j,
 * b_j = sum over listed views of (1/n_sub) sum over sub-angles of the
 * bilinear sample of r at the projected voxel centre (zero outside the
 * detector, skipped where the depth is <= 0), c_j = the same sum with r = 1.
 *   out_j = (accumulate ? vol_j : 0) + alpha * w_j * (normalize ? C_j : 1) * b_j
 * with C_j = 1 / c_j if c_j > 1e-6 else 0.
 *   r        DEVICE [n_idx][nv][nu] of r_dtype.
 *   vol      DEVICE [nz][ny][nx] of vol_dtype, read (if accumulate) and written.
 *   w        DEVICE float [nz][ny][nx] voxel weights, or NULL (= 1).
 */
int ctrex_back_project(ctrex_ctx *ctx, const void *r, int r_dtype, void *vol, int vol_dtype,
                       const float *w, float alpha, int normalize, int accumulate,
                       const int *view_idx, int n_idx);

/*
 * Matched adjoint of ctrex_fwd_project (exact transpose, motion included):
 * vol += A^T proj, scattered with FP32 atomics (summation order is not
 * reproducible bit for bit).  The paper has no such operator; it is the
 * transpose of its Sec. 4.1 projector, used for gradients.
 *   proj     DEVICE float [n_idx][nv][nu];  vol  DEVICE float [nz][ny][nx].
 */
int ctrex_adjoint_project(ctrex_ctx *ctx, const float *proj, float *vol, const int *view_idx,
                          int n_idx);

/*
 * Gradient of L = sum_i g_i (A x)_i with respect to the motion parameters
 * set by ctrex_set_motion (chain rule through the warp; the deformation is
 * recomputed, never stored).  Requires motion to be set.
 *   grad_proj   DEVICE float [n_idx][nv][nu] (= g).
 *   grad_theta  DEVICE float [n_views][15], accumulated (+=), or NULL.
 *   grad_coef   DEVICE float [8][8][8][3], accumulated (+=), or NULL.
 */
int ctrex_motion_grad(ctrex_ctx *ctx, const void *vol, int vol_dtype, const float *grad_proj,
                      float *grad_theta, float *grad_coef, const int *view_idx, int n_idx);

/*
 * SIRT (Eq. (1) with one subset holding every view, Sec. 2.3.2).  Iteration
 * k: fused A x_k / correction, rho_k = ||p - A x_k|| / ||p|| (one 16-byte
 * device-to-host read); stop if rho_k <= tol; else backproject with
 * normalisation and update x.  At most max_iter updates.
 *   vol                 DEVICE x_0 in, result out.
 *   p                   DEVICE [n_views][nv][nu] measured images.
 *   w                   DEVICE float voxel weights or NULL.
 *   residual_history    HOST float [max_iter] (entries past the stop are
 *                       left untouched), or NULL.
 *   iters_done          HOST, number of updates applied (may be NULL).
 * Returns CTREX_E_DIVERGED if a residual is not finite.
 */
int ctrex_sirt_iterate(ctrex_ctx *ctx, void *vol, int vol_dtype, const void *p, int p_dtype,
                       int max_iter, float alpha, const float *w, float tol,
                       float *residual_history, int *iters_done);

/*
 * Ordered-subset SIRT (Eq. (1) with index sets P_k, Sec. 2.3.2): one cycle
 * visits the subsets in order; subset S updates
 *   x += alpha w C_S B_S R_S (p_S - A_S x)
 * with the fused forward/correction and the backprojector restricted to the
 * views of S (C_S = column sums over those views).  A single subset of all
 * views is SIRT; one view per subset is SART-like.
 *   vol            DEVICE x_0 in, result out.
 *   p              DEVICE [n_views][nv][nu] measured images (indexed by view).
 *   subset_views   HOST int32, the subsets' view lists concatenated.
 *   subset_offsets HOST int32 [n_sets + 1], subset s = views[off[s] .. off[s+1]),
 *                  off[0] = 0, each subset at most 65535 views.
 *   w              DEVICE float voxel weights or NULL.
 *   residual_history HOST float [max_cycles] or NULL: after cycle k, the
 *                  running residual sqrt(sum_S ||p_S - A_S x_(S)||^2 /
 *                  sum_S ||p_S||^2), each term at the iterate subset S starts
 *                  from (one 16-byte-per-subset read per cycle).
 *   cycles_done    HOST: cycles applied; the loop stops after the first cycle
 *                  whose residual is <= tol.
 * Returns CTREX_E_SHAPE for an out-of-range view, CTREX_E_DIVERGED for a
 * non-finite residual.
 */
int ctrex_os_sirt_iterate(ctrex_ctx *ctx, void *vol, int vol_dtype, const void *p, int p_dtype,
                          const int *subset_views, const int *subset_offsets, int n_sets, int max_cycles,
                          float alpha, const float *w, float tol, float *residual_history, int *cycles_done);

/*
 * Same as ctrex_sirt_iterate with HOST buffers: copies vol (x_0) and p to
 * device buffers owned by the context, iterates, and copies the volume back
 * into vol.  vol_dtype / p_dtype describe the host arrays.  Synchronous.
 * With FP32 projections the first iteration overlaps the upload of p with
 * the forward projection (a copy stream owned by the context; the
 * correction waits for the upload), so the iterates equal those of
 * ctrex_sirt_iterate bitwise and only the first residual norm is summed in
 * another order.  Pinned host memory lets the copies run asynchronously;
 * pageable memory works but the driver stages it.  The context then also
 * holds two FP32 projection-sized scratch buffers and the correction's
 * partial norms (its own, not ctrex_correct_static's shared array).
 */
int ctrex_sirt_host(ctrex_ctx *ctx, void *vol_host, int vol_dtype, const void *p_host, int p_dtype,
                    int max_iter, float alpha, const float *w_host, float tol,
                    float *residual_history, int *iters_done);

/*
 * Exact number of ray samples (segments) of the listed views, summed over
 * all pixels and sub-angles, as the projector kernels count them; result in
 * HOST *out.  Synchronous.
 */
int ctrex_count_samples(ctrex_ctx *ctx, const int *view_idx, int n_idx, long long *out);

/*
 * 3x3x3 convolution, stride 1, zero padding 1 ("same"), as an implicit GEMM
 * on the tcgen05 tensor cores: BF16 operands, FP32 accumulation.  Used by the
 * learned warm start (a 3D U-Net); the paper motivates learned components
 * next to the physics operators (Sec. 5) but specifies none.
 *   x       DEVICE bf16 [nb][d][h][w][cin] (channels last).
 *   wt      DEVICE bf16 [cout][27][cin], tap = kz*9 + ky*3 + kx (k = 0..2
 *           for offsets -1..+1).
 *   bias    DEVICE float [cout] or NULL.
 *   y       DEVICE [nb][d][h][w][cout] of y_dtype (CTREX_F32 or CTREX_BF16),
 *           overwritten with max(conv + bias, 0) if relu else conv + bias.
 *   status  DEVICE int, set to 1 if a tensor-core completion wait expired
 *           (the result is then invalid); never cleared by the library.
 *   stream  cudaStream_t (NULL = legacy default stream).
 * x, wt and y must be 16-byte aligned (CTREX_E_ARG otherwise).
 * The input gradient is this same call on dy with the flipped, transposed
 * weights wt'[ci][26 - tap][co].  Errors: CTREX_E_ARG, CTREX_E_DTYPE,
 * CTREX_E_SHAPE, CTREX_E_CUDA.
 */
int ctrex_conv3d_fwd(const void *x, const void *wt, const float *bias, void *y, int y_dtype, int nb, int d,
                     int h, int w, int cin, int cout, int relu, int *status, void *cuda_stream);

/*
 * Weight gradient of ctrex_conv3d_fwd: dw[co][tap][ci] += sum over voxels of
 * dy[voxel][co] * x[voxel + offset(tap)][ci] (zero outside).  The voxel sum
 * is split across CTAs whose partial sums are added with FP32 atomics (not
 * bitwise reproducible).  x bf16 [nb][d][h][w][cin], dy bf16 [nb][d][h][w][cout],
 * dw DEVICE float [cout][27][cin] (accumulated: zero it first).  cin and
 * cout must be multiples of 8 (CTREX_E_SHAPE otherwise); x and dy must be
 * 16-byte aligned (CTREX_E_ARG otherwise).
 */
int ctrex_conv3d_wgrad(const void *x, const void *dy, float *dw, int nb, int d, int h, int w, int cin,
                       int cout, int *status, void *cuda_stream);

/*
 * Measured ceiling of the texture path: tex2Dgather calls per second on the
 * current device, on a 64 KiB texture that stays in L1 (each call returns a
 * 2x2 footprint, four 32-bit values, per thread).  Allocates and frees a
 * small array; synchronises the stream.  The projectors issue 2 gathers per
 * FP32 sample, 1 per BF16 sample and 1 per backprojected voxel-view.
 */
int ctrex_probe_gather_rate(void *cuda_stream, double *gathers_per_s);

/*
 * Measured L2 read bandwidth of the current device (GB/s, bytes read): a
 * buffer of half the L2 size is read repeatedly with 16-byte L2-only loads
 * (no L1 allocation) by a grid of 8 CTAs per SM, 512 passes timed with CUDA
 * events after one warm pass.  This is the denominator of the graded gather
 * roofline: the projectors' algorithmic gather bytes (8 taps per sample, 4
 * per backprojected voxel-view) over what L2 can deliver.  Allocates and
 * frees the buffer; synchronises the stream.  Errors: CTREX_E_ARG (NULL
 * output), CTREX_E_CUDA.
 */
int ctrex_probe_l2_read_bandwidth(void *cuda_stream, double *gb_per_s);

/*
 * Detector-space correction without any allocation.  The paper has no
 * counterpart: this is an extra entry point for callers that cannot let the
 * library call cudaMalloc (a host whose caching allocator already reserved
 * the device memory, an acquisition loop that must not stall in the driver's
 * allocator, a plugin host that forbids allocation in its callback).
 * It needs no context.  On the current CUDA device it computes, for
 * i < n,  r_i = R_i (p_i - q_i)  with R_i = 1 / rowsum_i if rowsum_i > eps_R
 * else 0, and sums = (sum (p - q)^2, sum p^2) in a fixed-order two-pass
 * reduction -- the same correction ctrex_fwd_correct fuses into the
 * projector, here fed with q = A x and rowsum = A 1 from ctrex_fwd_project.
 *   p, q     DEVICE [n] of dtype (CTREX_F32 or CTREX_BF16); r DEVICE [n]
 *            output of dtype; rowsum DEVICE float [n]; sums DEVICE double
 *            [2] or NULL (then only r is written).
 *   n        0 <= n <= 2^29 (536870912); larger n returns CTREX_E_SHAPE
 *            before any work is enqueued.
 *   stream   cudaStream_t to enqueue on (NULL = legacy default stream).
 * The reduction's scratch is a 1 MiB static device array that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it.  Under CUDA's lazy module loading
 * (the default) that lookup is what loads this file's module, which places
 * the array and the kernels in device memory and may synchronise.  So make
 * one call on each device before any region where allocation or
 * synchronisation is not allowed, and before any stream capture; from the
 * second call on, nothing is allocated.  The cached address belongs to the
 * device's current primary context: after cudaDeviceReset on that device,
 * do not call this function again in the same process (the cache would be
 * stale).  Every call shares the array: calls whose kernels overlap on the
 * GPU race on it and must be serialised by the caller.  Errors:
 * CTREX_E_SHAPE, CTREX_E_DTYPE, CTREX_E_ARG (NULL buffer, eps_R < 0 or NaN),
 * CTREX_E_CUDA (address lookup or launch failed).
 */
int ctrex_correct_static(const void *p, const void *q, const float *rowsum, void *r, int dtype,
                         long long n, float eps_R, double *sums, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CTREX_H */
