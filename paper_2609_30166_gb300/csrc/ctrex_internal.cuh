// ctrex_internal.cuh -- device-side data layout shared by the CUDA kernels of
// libctrex (sm_103a).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctrex.h"

namespace ctrex {

// Per (view, sub-angle) ray parameters, FP32, in voxel-index coordinates
// (g = (x - origin) / vox).  Derived on the host in FP64 from the
// sign-normalised projection matrix (Sec. 2.2.1):
//   ray through detector point (u, v) meets the plane of constant depth
//   through the volume centre at  X(u,v) = ref + (u-uc) qu + (v-vc) qv,
//   and X(u,v) - source = dref + (u-uc) qu + (v-vc) qv   (no cancellation),
// so every sample position is formed relative to a point near the volume,
// never relative to the distant source.
//   P: the projection matrix composed with index -> mm, h = P [ix iy iz 1].
struct ViewGPU {
    float ref[3];
    float dref[3];
    float qu[3];
    float qv[3];
    float P[12];
};
static_assert(sizeof(ViewGPU) == 96, "ViewGPU layout");

// Per-view motion, voxel-index coordinates: g' = M g + b (pose), then
// y = g' + s * u(g') with u in voxels (coefficients pre-divided by vox).
struct MotionGPU {
    float M[9];
    float b[3];
    float s;
    // centred form y - c = (g - c) + D (g - c) + bc about the integer grid
    // centre c = floor((n - 1) / 2) per axis: D = M - I and bc = M c + b - c,
    // both formed in FP64 and rounded once (small for a near-identity pose)
    float bc[3];
    float D[9];
    float pad[3];
};
static_assert(sizeof(MotionGPU) == 112, "MotionGPU layout");

struct Grid {
    int nx, ny, nz;
    int nu, nv;
    int n_views, n_sub;
    float step_mm;       // ray step (mm)
    float vox[3];        // mm
    float uc, vc;        // detector centre coordinates
    float lo[3], hi[3];  // clip box, index coordinates (dilated when motion is on)
    float eps_R;         // row-sum threshold of the correction (mm)
    float inv_sub;       // 1 / n_sub
    float spl_scale[3];  // B-spline coordinate: xi = (g + 1/2) * spl_scale + 1
};

// Aligned cylindrical domain (Sec. 3.5): N_r rings x N_phi sectors x N_z
// slices.  Ray and voxel positions are in the cylinder frame (mm; its z axis
// is the cylinder axis); index coordinates g_r = r / dr - 1/2 (clamped to
// >= 0), g_phi = phi / dphi - 1/2 (periodic), g_z = z / dz + zc.
struct CylGPU {
    int n_r, n_phi, n_z;
    float dr, dphi, dz;              // mm, rad, mm
    float inv_dr, inv_dphi, inv_dz;  // reciprocals
    float zc;                        // (N_z - 1) / 2
    float R, Z;                      // bounding cylinder: radius, half height (mm)
};

// Multi-resolution ROI (Sec. 3.7): a finer grid inside the context grid's
// box.  ROI index coordinates from context ones: g_roi = g_ctx * sc + oc;
// the ROI box in context index coordinates is [lo, hi].
struct RoiGPU {
    float sc[3], oc[3];
    float lo[3], hi[3];
    float step_mm;  // the ROI grid's step
    int n[3];       // the ROI grid's voxels per axis
};

template <typename T> struct Storage;
template <> struct Storage<float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
};
template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p)
    {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// Status word written by kernels whose own bounds checks fire (never trap).
enum : unsigned { DEVCHECK_OOB = 1u };

// ---- host-side launchers (defined in project.cu / backproject.cu / ...) ----

struct Atlas;

// Event-based 4D model (Sec. 3.3): with these set, volume buffers hold mu0
// followed by mu1 (2 nx ny nz elements) and view v sees mu0 at the voxels
// whose transition time tau exceeds t_view[v], mu1 elsewhere.
struct DyrArgs {
    const Atlas *mu1 = nullptr;     // atlas of the final values (the forward's atlas holds mu0)
    const Atlas *tau_atlas = nullptr;
    const float *tau = nullptr;     // device [nz][ny][nx]
    const float *t_view = nullptr;  // device [n_views]
    const float2 *tau_brick = nullptr;  // device: (min, max) of tau per 8^3 brick and its upper neighbours
    int bnx = 0, bny = 0;               // bricks along x and y
};

// The detector-space correction r = R (p - q) with the residual norms
// (sum (p - q)^2, sum p^2) into sums (DEVICE double [2]; NULL: r only), as
// ctrex_correct_static computes it but with caller-owned scratch of
// correct_scratch_pairs(n) double pairs, for any n >= 0 (correct_static.cu).
long long correct_scratch_pairs(long long n);
cudaError_t launch_correct(const void *p, const void *q, const float *rowsum, void *r, int dtype, long long n,
                           float eps_R, double *sums, double *scratch, cudaStream_t stream);

// (min, max) transition time of each 8^3 brick of tau [nz][ny][nx], taken
// over the brick and the voxel past each of its upper faces (within the
// grid).
cudaError_t launch_tau_bricks(const float *tau, int nx, int ny, int nz, float2 *out, cudaStream_t stream);

struct FwdArgs {
    const Grid *grid;           // host copy
    const Atlas *atlas = nullptr;  // volume uploaded into a texture atlas, or nullptr
    const ViewGPU *views;       // device [n_views * n_sub]
    const MotionGPU *motion;    // device [n_views] or nullptr
    const float *coef_idx;      // device [8][8][8][3] voxels, or nullptr
    const void *vol;
    int vol_dtype;
    const int *view_idx;        // device or nullptr
    int n_idx;
    cudaStream_t stream;
    unsigned *devcheck;         // device status word
    int p_by_view = 0;          // correction: measured images indexed by view, not by list position
    const CylGPU *cyl = nullptr;  // cylindrical domain, or nullptr (Cartesian grid)
    int joseph = 0;               // classical Joseph projector; atlas = the three-stack atlas
    const RoiGPU *roi = nullptr;  // multi-resolution ROI: atlas = context grid, roi_atlas = ROI grid
    const Atlas *roi_atlas = nullptr;
    const DyrArgs *dyr = nullptr;  // event-based 4D model, or nullptr
};

cudaError_t launch_forward(const FwdArgs &a, void *proj, int proj_dtype, float *rowsum);
cudaError_t launch_forward_correct(const FwdArgs &a, const void *p, int p_dtype, void *r,
                                   int r_dtype, float *partials, int n_partials_cap,
                                   double *sums);
int forward_partials_needed(const Grid &g, int n_idx);
cudaError_t launch_count_samples(const FwdArgs &a, unsigned long long *out);

struct BpArgs {
    const Grid *grid;
    const Atlas *atlas = nullptr;  // correction images uploaded into a texture atlas, or nullptr
    const int4 *window = nullptr;  // per-view detector window of the backprojector, or nullptr
    const ViewGPU *views;
    const int *view_idx;
    int n_idx;
    const void *r;
    int r_dtype;
    void *vol;
    int vol_dtype;
    const float *w;
    float alpha;
    int normalize;
    int accumulate;
    int subvox = 1;  // sub-voxel points per axis (1 = voxel centre only)
    const CylGPU *cyl = nullptr;  // cylindrical domain, or nullptr (Cartesian grid)
    const DyrArgs *dyr = nullptr;  // event-based 4D model: vol and w hold mu0 then mu1
    cudaStream_t stream;
};
cudaError_t launch_backproject(const BpArgs &a);

cudaError_t launch_adjoint(const FwdArgs &a, const float *proj, float *vol);
cudaError_t launch_motion_grad(const FwdArgs &a, const float *gproj, double *grad_M, double *grad_b,
                               double *grad_coef_idx);
cudaError_t launch_motion_setup(const float *theta, const float *coef, const float *s_view,
                                int n_views, const Grid &g, const double vox[3],
                                const double origin[3], MotionGPU *motion, float *coef_idx,
                                float *dRdw, cudaStream_t stream);
cudaError_t launch_motion_grad_finish(const float *theta, const float *dRdw, const double *grad_M,
                                      const double *grad_b, const double *grad_coef_idx, int n_views,
                                      const Grid &g, const double vox[3], const double origin[3],
                                      float *grad_theta, float *grad_coef, cudaStream_t stream);

}  // namespace ctrex
