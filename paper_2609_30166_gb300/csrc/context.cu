// context.cu -- the C ABI of libctrex: context, geometry and motion set-up,
// operator entry points and the SIRT driver (the paper's Rex / Trajectory
// split, Sec. 2.1-2.3, as a native library).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "atlas.cuh"
#include "ctrex_internal.cuh"

using namespace ctrex;

struct ctrex_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // geometry
    bool has_geom = false;
    Grid grid{};
    double vox[3] = {1, 1, 1}, origin[3] = {0, 0, 0};
    double step_vox = 0.5;
    ViewGPU *d_views = nullptr;
    // motion
    bool has_motion = false;
    double margin = 0.0;
    MotionGPU *d_motion = nullptr;
    float *d_theta = nullptr;     // [n_views][15] copy (or null)
    float *d_coef = nullptr;      // [8][8][8][3] mm
    float *d_coef_idx = nullptr;  // [8][8][8][3] voxels
    float *d_dRdw = nullptr;      // [n_views][27]
    double *d_gM = nullptr, *d_gb = nullptr, *d_gcoef = nullptr;  // gradient scratch (FP64 sums)
    bool coef_valid = false, theta_valid = false;
    // scratch
    float *d_partials = nullptr;
    int partials_cap = 0;
    double *d_sums = nullptr;
    unsigned *d_devcheck = nullptr;
    unsigned long long *d_count = nullptr;
    void *d_r = nullptr;  // SIRT correction images
    size_t r_bytes = 0;
    // texture atlas of the volume read by the forward projector
    AtlasStore vol_atlas;
    Atlas vol_atlas_view;
    // texture atlas of the correction images read by the backprojector
    AtlasStore img_atlas;
    Atlas img_atlas_view;
    bool img_atlas_unfit = false;
    bool atlas_unfit = false;  // geometry exceeds the 2D texture limits: row-major sampling
    // backprojector detector windows (extended field of view), int4 per view
    int4 *d_window = nullptr;
    bool has_window = false;
    // sub-voxel backprojection points per axis (motion blur), 1 = off
    int bp_subvoxel = 1;
    // aligned cylindrical domain (set by ctrex_set_geometry_cylinder)
    bool cyl = false;
    CylGPU cylg{};
    // forward projector: CTREX_PROJ_TRILINEAR or CTREX_PROJ_JOSEPH (three-stack atlas)
    int projector = CTREX_PROJ_TRILINEAR;
    AtlasStore jos_atlas;
    Atlas jos_atlas_view;
    // multi-resolution ROI (set by ctrex_set_roi): a finer grid whose voxels
    // follow the context grid's in every volume buffer
    std::vector<double> hostP;  // world matrices of the current geometry
    double ctr[3] = {0, 0, 0};  // the centre P was sign-normalised with
    bool roi = false;
    Grid roi_grid{};
    ViewGPU *d_views_roi = nullptr;
    RoiGPU roig{};
    AtlasStore roi_atlas;
    Atlas roi_atlas_view;
    // event-based 4D model (set by ctrex_set_dyrect): volume buffers hold
    // the initial values followed by the final values
    bool dyr = false;
    float *d_tau = nullptr;     // [nz][ny][nx] transition times
    float *d_tview = nullptr;   // [n_views] acquisition times
    float2 *d_tau_brick = nullptr;  // (min, max) transition time per 8^3 brick
    AtlasStore dyr_atlas1;      // the final values (the volume atlas holds the initial ones)
    AtlasStore tau_atlas;
    Atlas dyr_atlas1_view, tau_atlas_view;
    DyrArgs dyra{};
    // ordered-subset SIRT: concatenated subset view lists, per-subset norms
    int *d_subset_views = nullptr;
    size_t subset_views_bytes = 0;
    double *d_subset_sums = nullptr;
    size_t subset_sums_bytes = 0;
    // host-buffer entry point scratch
    void *d_hvol = nullptr, *d_hp = nullptr;
    float *d_hw = nullptr;
    size_t hvol_bytes = 0, hp_bytes = 0, hw_bytes = 0;
    // its first iteration overlaps the projections' upload with the forward
    // projection: A x and the row sums (FP32), a copy stream, two events
    void *d_hq = nullptr;
    float *d_hrs = nullptr;
    double *d_hcs = nullptr;  // the correction's partial norms
    size_t hq_bytes = 0, hrs_bytes = 0, hcs_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_vol = nullptr, ev_p = nullptr;
};

namespace {

const char *g_static_err = "ctrex: invalid context";

int fail(ctrex_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(ctrex_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? CTREX_E_NOMEM : CTREX_E_CUDA, "%s: %s (%s)", where,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CT_CUDA(c, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T> void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

int ensure(ctrex_ctx *c, void **p, size_t *have, size_t need, const char *what)
{
    if (*have >= need && *p) return CTREX_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, CTREX_E_NOMEM, "cannot allocate %zu bytes for %s: %s", need, what, cudaGetErrorString(e));
    }
    *have = need;
    return CTREX_OK;
}

size_t dtype_size(int dt) { return dt == CTREX_BF16 ? 2 : 4; }
bool dtype_ok(int dt) { return dt == CTREX_F32 || dt == CTREX_BF16; }

int check_ctx(ctrex_ctx *c)
{
    if (!c) return CTREX_E_ARG;
    return CTREX_OK;
}

int check_views(ctrex_ctx *c, const int *view_idx, int n_idx)
{
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_geometry has not been called");
    if (n_idx < 0 || n_idx > 65535) return fail(c, CTREX_E_SHAPE, "n_idx %d outside [0, 65535]", n_idx);
    if (!view_idx && n_idx != 0 && n_idx != c->grid.n_views)
        return fail(c, CTREX_E_SHAPE, "view_idx is NULL but n_idx (%d) != n_views (%d)", n_idx, c->grid.n_views);
    return CTREX_OK;
}

FwdArgs fwd_args(ctrex_ctx *c, const void *vol, int vdt, const int *view_idx, int n_idx)
{
    FwdArgs a;
    a.grid = &c->grid;
    a.views = c->d_views;
    a.motion = c->has_motion ? c->d_motion : nullptr;
    a.coef_idx = (c->has_motion && c->coef_valid) ? c->d_coef_idx : nullptr;
    a.vol = vol;
    a.vol_dtype = vdt;
    a.view_idx = view_idx;
    a.n_idx = n_idx;
    a.stream = c->stream;
    a.devcheck = c->d_devcheck;
    a.cyl = c->cyl ? &c->cylg : nullptr;
    a.joseph = c->projector == CTREX_PROJ_JOSEPH ? 1 : 0;
    a.roi = c->roi ? &c->roig : nullptr;
    a.dyr = c->dyr ? &c->dyra : nullptr;
    return a;
}

size_t grid_voxels(const Grid &G) { return (size_t)G.nx * G.ny * G.nz; }

// Elements of a volume buffer: the grid, then the ROI grid if one is set;
// with the event-based model the grid's initial then final values.
size_t volume_elems(const ctrex_ctx *c)
{
    return grid_voxels(c->grid) * (c->dyr ? 2 : 1) + (c->roi ? grid_voxels(c->roi_grid) : 0);
}

void dyr_release(ctrex_ctx *c)
{
    c->dyr = false;
    if (c->d_tau) cudaFree(c->d_tau);
    if (c->d_tview) cudaFree(c->d_tview);
    if (c->d_tau_brick) cudaFree(c->d_tau_brick);
    c->d_tau = c->d_tview = nullptr;
    c->d_tau_brick = nullptr;
    atlas_release(c->dyr_atlas1);
    atlas_release(c->tau_atlas);
}

// Uploads vol into the context's texture atlas and points a.atlas at it; if
// the volume does not fit the 2D texture limits the row-major path is used.
int prepare_atlas(ctrex_ctx *c, FwdArgs &a, const void *vol, int vdt)
{
    if (c->projector == CTREX_PROJ_JOSEPH) {
        // x-, y- and z-slice stacks in one atlas; no row-major fallback
        const int nx = c->grid.nx, ny = c->grid.ny, nz = c->grid.nz;
        cudaError_t e = atlas_ensure(c->jos_atlas, nx > ny ? nx : ny, ny > nz ? ny : nz, nx + ny + nz,
                                     vdt == CTREX_BF16, c->device, false);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            return fail(c, CTREX_E_SHAPE, "Joseph projector: volume exceeds the 2D texture limits of the device");
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "Joseph atlas allocation");
        e = atlas_upload_joseph(c->jos_atlas, vol, nx, ny, nz, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "Joseph atlas upload");
        c->jos_atlas_view = atlas_view(c->jos_atlas);
        a.atlas = &c->jos_atlas_view;
        return CTREX_OK;
    }
    if (c->dyr) {
        // initial values into the volume atlas, final values into their own;
        // the transition times were uploaded by set_dyrect; no row-major fallback
        const size_t off = grid_voxels(c->grid) * dtype_size(vdt);
        AtlasStore *st[2] = {&c->vol_atlas, &c->dyr_atlas1};
        Atlas *vw[2] = {&c->vol_atlas_view, &c->dyr_atlas1_view};
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = atlas_ensure(*st[i], c->grid.nx, c->grid.ny, c->grid.nz, vdt == CTREX_BF16, c->device,
                                         false);
            if (e == cudaErrorInvalidValue) {
                cudaGetLastError();
                return fail(c, CTREX_E_SHAPE, "event model: the volume exceeds the 2D texture limits of the device");
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "event-model atlas allocation");
            e = atlas_upload(*st[i], static_cast<const char *>(vol) + (i ? off : 0), c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "event-model atlas upload");
            *vw[i] = atlas_view(*st[i]);
        }
        c->dyra.mu1 = &c->dyr_atlas1_view;
        c->dyra.tau_atlas = &c->tau_atlas_view;
        a.atlas = &c->vol_atlas_view;
        return CTREX_OK;
    }
    if (c->roi) {
        // context and ROI grids in atlases of their own; no row-major fallback
        const size_t off = grid_voxels(c->grid) * dtype_size(vdt);
        const Grid *gs[2] = {&c->grid, &c->roi_grid};
        AtlasStore *st[2] = {&c->vol_atlas, &c->roi_atlas};
        Atlas *vw[2] = {&c->vol_atlas_view, &c->roi_atlas_view};
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = atlas_ensure(*st[i], gs[i]->nx, gs[i]->ny, gs[i]->nz, vdt == CTREX_BF16, c->device, false);
            if (e == cudaErrorInvalidValue) {
                cudaGetLastError();
                return fail(c, CTREX_E_SHAPE, "ROI projection: a grid exceeds the 2D texture limits of the device");
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "ROI atlas allocation");
            e = atlas_upload(*st[i], static_cast<const char *>(vol) + (i ? off : 0), c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "ROI atlas upload");
            *vw[i] = atlas_view(*st[i]);
        }
        a.atlas = &c->vol_atlas_view;
        a.roi_atlas = &c->roi_atlas_view;
        return CTREX_OK;
    }
    if (c->cyl) {
        // cylindrical domain: z-slice tiles of N_r x (N_phi + 1), the last row
        // repeating sector 0; no row-major fallback
        cudaError_t e = atlas_ensure(c->vol_atlas, c->grid.nx, c->grid.ny, c->grid.nz, vdt == CTREX_BF16, c->device,
                                     false, true);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            return fail(c, CTREX_E_SHAPE, "cylindrical volume exceeds the 2D texture limits of the device");
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "volume atlas allocation");
        e = atlas_upload(c->vol_atlas, vol, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "volume atlas upload");
        c->vol_atlas_view = atlas_view(c->vol_atlas);
        a.atlas = &c->vol_atlas_view;
        return CTREX_OK;
    }
    if (c->atlas_unfit) return CTREX_OK;
    // BF16 volumes: slice pairs packed in 32-bit texels, one gather per sample
    cudaError_t e = atlas_ensure(c->vol_atlas, c->grid.nx, c->grid.ny, c->grid.nz, vdt == CTREX_BF16, c->device,
                                 vdt == CTREX_BF16);
    if (e == cudaErrorInvalidValue) {
        cudaGetLastError();
        c->atlas_unfit = true;
        return CTREX_OK;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "volume atlas allocation");
    e = atlas_upload(c->vol_atlas, vol, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "volume atlas upload");
    c->vol_atlas_view = atlas_view(c->vol_atlas);
    a.atlas = &c->vol_atlas_view;
    return CTREX_OK;
}

// 3x3 helpers (FP64, host)
double det3(const double *m)
{
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) + m[2] * (m[3] * m[7] - m[4] * m[6]);
}

void inv3(const double *m, double *r)
{
    const double d = det3(m);
    r[0] = (m[4] * m[8] - m[5] * m[7]) / d;
    r[1] = (m[2] * m[7] - m[1] * m[8]) / d;
    r[2] = (m[1] * m[5] - m[2] * m[4]) / d;
    r[3] = (m[5] * m[6] - m[3] * m[8]) / d;
    r[4] = (m[0] * m[8] - m[2] * m[6]) / d;
    r[5] = (m[2] * m[3] - m[0] * m[5]) / d;
    r[6] = (m[3] * m[7] - m[4] * m[6]) / d;
    r[7] = (m[1] * m[6] - m[0] * m[7]) / d;
    r[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

void set_clip_box(ctrex_ctx *c)
{
    const int n[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    const double m = c->has_motion ? c->margin : 0.0;
    for (int a = 0; a < 3; ++a) {
        c->grid.lo[a] = (float)(-0.5 - m / c->vox[a]);
        c->grid.hi[a] = (float)(n[a] - 0.5 + m / c->vox[a]);
    }
}

}  // namespace

extern "C" {

const char *ctrex_version(void) { return "ctrex-gb300 0.1 (sm_103a)"; }

const char *ctrex_last_error(const ctrex_ctx *c) { return c ? c->err.c_str() : g_static_err; }

int ctrex_create(ctrex_ctx **out, int device, void *stream)
{
    if (!out) return CTREX_E_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CTREX_E_CUDA;
    }
    ctrex_ctx *c = new (std::nothrow) ctrex_ctx();
    if (!c) return CTREX_E_NOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    DeviceGuard g(device);
    if (cudaMalloc((void **)&c->d_sums, 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_devcheck, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_count, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        ctrex_destroy(c);
        return CTREX_E_NOMEM;
    }
    cudaMemset(c->d_devcheck, 0, sizeof(unsigned));
    *out = c;
    return CTREX_OK;
}

int ctrex_destroy(ctrex_ctx *c)
{
    if (!c) return CTREX_E_ARG;
    {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        dfree(c->d_views);
        dfree(c->d_motion);
        dfree(c->d_theta);
        dfree(c->d_coef);
        dfree(c->d_coef_idx);
        dfree(c->d_dRdw);
        dfree(c->d_gM);
        dfree(c->d_gb);
        dfree(c->d_gcoef);
        dfree(c->d_partials);
        dfree(c->d_sums);
        dfree(c->d_devcheck);
        dfree(c->d_count);
        dfree(c->d_r);
        dfree(c->d_hvol);
        dfree(c->d_hp);
        dfree(c->d_hw);
        dfree(c->d_hq);
        dfree(c->d_hrs);
        dfree(c->d_hcs);
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
        if (c->ev_vol) cudaEventDestroy(c->ev_vol);
        if (c->ev_p) cudaEventDestroy(c->ev_p);
        dfree(c->d_subset_views);
        dfree(c->d_window);
        dfree(c->d_subset_sums);
        atlas_release(c->vol_atlas);
        atlas_release(c->img_atlas);
        atlas_release(c->jos_atlas);
        atlas_release(c->roi_atlas);
        dfree(c->d_views_roi);
        dyr_release(c);
    }
    delete c;
    return CTREX_OK;
}

int ctrex_set_stream(ctrex_ctx *c, void *stream)
{
    if (!c) return CTREX_E_ARG;
    c->stream = (cudaStream_t)stream;
    return CTREX_OK;
}

int ctrex_device_status(ctrex_ctx *c)
{
    if (!c) return CTREX_E_ARG;
    DeviceGuard g(c->device);
    unsigned h = 0;
    CT_CUDA(c, cudaMemcpyAsync(&h, c->d_devcheck, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h) {
        CT_CUDA(c, cudaMemsetAsync(c->d_devcheck, 0, sizeof(unsigned), c->stream));
        return fail(c, CTREX_E_DEVICE_CHECK, "a kernel bounds check fired (flags 0x%x): view index out of range", h);
    }
    return CTREX_OK;
}

// Shared by the Cartesian and the cylindrical set-up.  P maps the frame the
// grid is indexed in (mm) to pixels; voxel i of axis a sits at origin[a] +
// i vox[a] in that frame; ctr is the volume centre (sign normalisation of P);
// min_pitch the smallest physical pitch (step and row-sum threshold).
// Per-(view, sub) FP32 parameters of P on a grid (vox, origin); ctr fixes
// the sign normalisation.
static int compute_views(ctrex_ctx *c, const double *P, int nvs, int n_sub, const double vox[3],
                         const double origin[3], const double ctr[3], double uc, double vc, std::vector<ViewGPU> &hv)
{
    hv.assign((size_t)nvs, ViewGPU{});
    for (int q = 0; q < nvs; ++q) {
        const double *Pi = P + 12 * (size_t)q;
        double M[9], fro = 0.0;
        for (int k = 0; k < 12; ++k)
            if (!isfinite(Pi[k])) return fail(c, CTREX_E_GEOMETRY, "view %d sub %d: non-finite matrix", q / n_sub, q % n_sub);
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                M[3 * r + cc] = Pi[4 * r + cc];
                fro += M[3 * r + cc] * M[3 * r + cc];
            }
        fro = sqrt(fro);
        if (!(fabs(det3(M)) > 1e-12 * fro * fro * fro))
            return fail(c, CTREX_E_GEOMETRY, "view %d sub %d: singular projection matrix", q / n_sub, q % n_sub);
        const double depth = Pi[8] * ctr[0] + Pi[9] * ctr[1] + Pi[10] * ctr[2] + Pi[11];
        if (!(depth != 0.0))
            return fail(c, CTREX_E_GEOMETRY, "view %d sub %d: volume centre on the source plane", q / n_sub, q % n_sub);
        const double sgn = depth > 0 ? 1.0 : -1.0;
        double Pn[12];
        for (int k = 0; k < 12; ++k) Pn[k] = sgn * Pi[k];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) M[3 * r + cc] = Pn[4 * r + cc];
        double Mi[9];
        inv3(M, Mi);
        double src[3];
        for (int r = 0; r < 3; ++r) src[r] = -(Mi[3 * r] * Pn[3] + Mi[3 * r + 1] * Pn[7] + Mi[3 * r + 2] * Pn[11]);
        const double lam = sgn * depth;  // depth of the volume centre, > 0
        ViewGPU &V = hv[(size_t)q];
        for (int a = 0; a < 3; ++a) {
            const double mc = Mi[3 * a] * uc + Mi[3 * a + 1] * vc + Mi[3 * a + 2];
            const double dref = lam * mc;  // X(uc,vc) - source, mm
            V.dref[a] = (float)(dref / vox[a]);
            V.ref[a] = (float)((src[a] + dref - origin[a]) / vox[a]);
            V.qu[a] = (float)(lam * Mi[3 * a] / vox[a]);
            V.qv[a] = (float)(lam * Mi[3 * a + 1] / vox[a]);
        }
        // h = Pn [origin + vox * i; 1]
        for (int r = 0; r < 3; ++r) {
            double acc = Pn[4 * r + 3];
            for (int a = 0; a < 3; ++a) {
                V.P[4 * r + a] = (float)(Pn[4 * r + a] * vox[a]);
                acc += Pn[4 * r + a] * origin[a];
            }
            V.P[4 * r + 3] = (float)acc;
        }
    }
    return CTREX_OK;
}

static int build_geometry(ctrex_ctx *c, const double *P, int n_views, int n_sub, const int n[3], const double vox[3],
                          const double origin[3], const double ctr[3], double min_pitch, const ctrex_det_grid *det,
                          double step_vox)
{
    DeviceGuard g(c->device);
    const int nvs = n_views * n_sub;
    std::vector<ViewGPU> hv;
    const double uc = 0.5 * (det->nu - 1), vc = 0.5 * (det->nv - 1);
    int e = compute_views(c, P, nvs, n_sub, vox, origin, ctr, uc, vc, hv);
    if (e) return e;
    // the world matrices and the centre, for a later ROI grid
    c->hostP.assign(P, P + 12 * (size_t)nvs);
    for (int a = 0; a < 3; ++a) c->ctr[a] = ctr[a];
    dfree(c->d_views);
    dfree(c->d_views_roi);
    c->roi = false;
    atlas_release(c->roi_atlas);
    dyr_release(c);
    dfree(c->d_window);
    c->has_window = false;
    // motion buffers are sized by n_views: drop them with the old geometry
    dfree(c->d_motion);
    dfree(c->d_dRdw);
    dfree(c->d_theta);
    dfree(c->d_coef);
    dfree(c->d_coef_idx);
    dfree(c->d_gM);
    dfree(c->d_gb);
    dfree(c->d_gcoef);
    c->coef_valid = c->theta_valid = false;
    CT_CUDA(c, cudaMalloc((void **)&c->d_views, sizeof(ViewGPU) * (size_t)nvs));
    CT_CUDA(c, cudaMemcpy(c->d_views, hv.data(), sizeof(ViewGPU) * (size_t)nvs, cudaMemcpyHostToDevice));
    Grid &G = c->grid;
    G.nx = n[0];
    G.ny = n[1];
    G.nz = n[2];
    G.nu = det->nu;
    G.nv = det->nv;
    G.n_views = n_views;
    G.n_sub = n_sub;
    const double minv = min_pitch;
    for (int a = 0; a < 3; ++a) {
        c->vox[a] = vox[a];
        c->origin[a] = origin[a];
        G.vox[a] = (float)vox[a];
        G.spl_scale[a] = (float)(5.0 / n[a]);
    }
    c->step_vox = step_vox;
    G.step_mm = (float)(step_vox * minv);
    G.uc = (float)uc;
    G.vc = (float)vc;
    G.eps_R = (float)(1e-6 * minv);
    G.inv_sub = (float)(1.0 / n_sub);
    c->has_motion = false;
    c->cyl = false;
    c->has_geom = true;
    c->atlas_unfit = false;
    c->img_atlas_unfit = false;
    set_clip_box(c);
    return CTREX_OK;
}


int ctrex_set_geometry(ctrex_ctx *c, const double *P, int n_views, int n_sub, const ctrex_vol_grid *vol,
                       const ctrex_det_grid *det, double step_vox)
{
    if (!c) return CTREX_E_ARG;
    if (!P || !vol || !det) return fail(c, CTREX_E_ARG, "set_geometry: NULL argument");
    if (n_views < 1 || n_sub < 1 || (long long)n_views * n_sub > (1 << 24))
        return fail(c, CTREX_E_SHAPE, "set_geometry: bad n_views %d / n_sub %d", n_views, n_sub);
    if (vol->nx < 1 || vol->ny < 1 || vol->nz < 1 || (long long)vol->nx * vol->ny * vol->nz >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_geometry: volume %d x %d x %d unsupported", vol->nx, vol->ny, vol->nz);
    if (det->nu < 1 || det->nv < 1 || det->nv > 4 * 65535 || (long long)det->nu * det->nv >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_geometry: detector %d x %d unsupported", det->nu, det->nv);
    for (int a = 0; a < 3; ++a)
        if (!(vol->vox[a] > 0.0) || !isfinite(vol->origin[a]))
            return fail(c, CTREX_E_ARG, "set_geometry: voxel pitch must be > 0 and origin finite");
    // bounded step keeps every ray's sample count (and kernel run time) bounded
    if (!(step_vox >= 1e-2 && step_vox <= 100.0))
        return fail(c, CTREX_E_ARG, "set_geometry: step_vox must lie in [0.01, 100]");
    const int n[3] = {vol->nx, vol->ny, vol->nz};
    double ctr[3], minv = vol->vox[0];
    for (int a = 0; a < 3; ++a) {
        ctr[a] = vol->origin[a] + 0.5 * (n[a] - 1) * vol->vox[a];
        minv = fmin(minv, vol->vox[a]);
    }
    return build_geometry(c, P, n_views, n_sub, n, vol->vox, vol->origin, ctr, minv, det, step_vox);
}

int ctrex_set_geometry_cylinder(ctrex_ctx *c, const double *P, int n_views, int n_sub, const ctrex_cyl_grid *cyl,
                                const ctrex_det_grid *det, double step_vox)
{
    if (!c) return CTREX_E_ARG;
    if (!P || !cyl || !det) return fail(c, CTREX_E_ARG, "set_geometry_cylinder: NULL argument");
    if (n_views < 1 || n_sub < 1 || (long long)n_views * n_sub > (1 << 24))
        return fail(c, CTREX_E_SHAPE, "set_geometry_cylinder: bad n_views %d / n_sub %d", n_views, n_sub);
    if (cyl->n_r < 1 || cyl->n_phi < 3 || cyl->n_z < 1 ||
        (long long)cyl->n_r * (cyl->n_phi + 1) * cyl->n_z >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_geometry_cylinder: grid %d x %d x %d unsupported", cyl->n_r, cyl->n_phi,
                    cyl->n_z);
    if (det->nu < 1 || det->nv < 1 || det->nv > 4 * 65535 || (long long)det->nu * det->nv >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_geometry_cylinder: detector %d x %d unsupported", det->nu, det->nv);
    if (!(cyl->dr > 0.0 && isfinite(cyl->dr) && cyl->dz > 0.0 && isfinite(cyl->dz)))
        return fail(c, CTREX_E_ARG, "set_geometry_cylinder: dr and dz must be finite and > 0");
    if (!(step_vox >= 1e-2 && step_vox <= 100.0))
        return fail(c, CTREX_E_ARG, "set_geometry_cylinder: step_vox must lie in [0.01, 100]");
    // the pose must be a rigid motion: Rc orthonormal with det +1
    const double *T = cyl->pose;
    for (int k = 0; k < 12; ++k)
        if (!isfinite(T[k])) return fail(c, CTREX_E_ARG, "set_geometry_cylinder: non-finite pose");
    double Rc[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Rc[3 * r + k] = T[4 * r + k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double d = Rc[i] * Rc[j] + Rc[3 + i] * Rc[3 + j] + Rc[6 + i] * Rc[6 + j];
            if (fabs(d - (i == j ? 1.0 : 0.0)) > 1e-9)
                return fail(c, CTREX_E_ARG, "set_geometry_cylinder: pose rotation is not orthonormal");
        }
    if (!(det3(Rc) > 0.0)) return fail(c, CTREX_E_ARG, "set_geometry_cylinder: pose rotation is a reflection");
    // P_q = P [Rc^T | -Rc^T tc]: the matrices act on cylinder-frame mm
    const size_t nvs = (size_t)n_views * n_sub;
    std::vector<double> Pq(12 * nvs);
    const double tc[3] = {T[3], T[7], T[11]};
    double inv[12];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) inv[4 * r + k] = Rc[3 * k + r];
        inv[4 * r + 3] = -(Rc[r] * tc[0] + Rc[3 + r] * tc[1] + Rc[6 + r] * tc[2]);
    }
    for (size_t q = 0; q < nvs; ++q) {
        const double *Pi = P + 12 * q;
        double *Po = Pq.data() + 12 * q;
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 4; ++k) {
                double acc = k == 3 ? Pi[4 * r + 3] : 0.0;
                for (int m = 0; m < 3; ++m) acc += Pi[4 * r + m] * inv[4 * m + k];
                Po[4 * r + k] = acc;
            }
    }
    const int n[3] = {cyl->n_r, cyl->n_phi, cyl->n_z};
    const double one[3] = {1.0, 1.0, 1.0}, zero[3] = {0.0, 0.0, 0.0};
    const int e = build_geometry(c, Pq.data(), n_views, n_sub, n, one, zero, zero, fmin(cyl->dr, cyl->dz), det,
                                 step_vox);
    if (e) return e;
    CylGPU &C = c->cylg;
    const double two_pi = 6.283185307179586476925286766559;
    C.n_r = cyl->n_r;
    C.n_phi = cyl->n_phi;
    C.n_z = cyl->n_z;
    C.dr = (float)cyl->dr;
    C.dphi = (float)(two_pi / cyl->n_phi);
    C.dz = (float)cyl->dz;
    C.inv_dr = (float)(1.0 / cyl->dr);
    C.inv_dphi = (float)(cyl->n_phi / two_pi);
    C.inv_dz = (float)(1.0 / cyl->dz);
    C.zc = (float)(0.5 * (cyl->n_z - 1));
    C.R = (float)(cyl->n_r * cyl->dr);
    C.Z = (float)(0.5 * cyl->n_z * cyl->dz);
    // bounding box of the cylinder (frame mm), for anything that reads the clip box
    for (int a = 0; a < 2; ++a) {
        c->grid.lo[a] = -C.R;
        c->grid.hi[a] = C.R;
    }
    c->grid.lo[2] = -C.Z;
    c->grid.hi[2] = C.Z;
    c->cyl = true;
    c->projector = CTREX_PROJ_TRILINEAR;
    return CTREX_OK;
}

int ctrex_set_motion(ctrex_ctx *c, const float *theta, const float *coef, const float *s_view, double margin_mm)
{
    if (!c) return CTREX_E_ARG;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_motion before set_geometry");
    if ((c->cyl || c->roi || c->dyr || c->projector == CTREX_PROJ_JOSEPH) && (theta || coef || s_view))
        return fail(c, CTREX_E_STATE, "set_motion: the motion model is defined for the trilinear projector on the "
                                      "Cartesian grid only, without the event model");
    double box = 0.0;
    const int nn[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    for (int a = 0; a < 3; ++a) box = fmax(box, nn[a] * c->vox[a]);
    if (!(margin_mm >= 0.0 && margin_mm <= box))
        return fail(c, CTREX_E_ARG, "set_motion: margin must lie in [0, largest box edge]");
    DeviceGuard g(c->device);
    if (!theta && !coef && !s_view) {
        c->has_motion = false;
        set_clip_box(c);
        return CTREX_OK;
    }
    const int V = c->grid.n_views;
    if (!c->d_motion) {
        CT_CUDA(c, cudaMalloc((void **)&c->d_motion, sizeof(MotionGPU) * (size_t)V));
        CT_CUDA(c, cudaMalloc((void **)&c->d_dRdw, sizeof(float) * 27 * (size_t)V));
        CT_CUDA(c, cudaMalloc((void **)&c->d_theta, sizeof(float) * 15 * (size_t)V));
        CT_CUDA(c, cudaMalloc((void **)&c->d_coef, sizeof(float) * 1536));
        CT_CUDA(c, cudaMalloc((void **)&c->d_coef_idx, sizeof(float) * 1536));
        CT_CUDA(c, cudaMalloc((void **)&c->d_gM, sizeof(double) * 9 * (size_t)V));
        CT_CUDA(c, cudaMalloc((void **)&c->d_gb, sizeof(double) * 3 * (size_t)V));
        CT_CUDA(c, cudaMalloc((void **)&c->d_gcoef, sizeof(double) * 1536));
    }
    const float *th = nullptr;
    if (theta) {
        CT_CUDA(c, cudaMemcpyAsync(c->d_theta, theta, sizeof(float) * 15 * (size_t)V, cudaMemcpyDeviceToDevice, c->stream));
        th = c->d_theta;
    }
    const float *co = nullptr;
    if (coef) {
        CT_CUDA(c, cudaMemcpyAsync(c->d_coef, coef, sizeof(float) * 1536, cudaMemcpyDeviceToDevice, c->stream));
        co = c->d_coef;
    }
    const float *sv = nullptr;
    // s_view is consumed by the set-up kernel straight from the caller's buffer
    if (s_view) sv = s_view;
    c->margin = margin_mm;
    c->has_motion = true;
    cudaError_t e = launch_motion_setup(th, co, sv, V, c->grid, c->vox, c->origin, c->d_motion, c->d_coef_idx,
                                        c->d_dRdw, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "motion set-up");
    c->coef_valid = co != nullptr;
    c->theta_valid = th != nullptr;
    set_clip_box(c);
    return CTREX_OK;
}

int ctrex_set_bp_window(ctrex_ctx *c, const int *window)
{
    if (!c) return CTREX_E_ARG;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_bp_window before set_geometry");
    if (!window) {
        c->has_window = false;
        return CTREX_OK;
    }
    const int V = c->grid.n_views;
    std::vector<int4> hw((size_t)V);
    for (int v = 0; v < V; ++v) {
        const int *q = window + 4 * (size_t)v;
        hw[(size_t)v] = make_int4(q[0] > 0 ? q[0] : 0, q[1] < c->grid.nu - 1 ? q[1] : c->grid.nu - 1,
                                  q[2] > 0 ? q[2] : 0, q[3] < c->grid.nv - 1 ? q[3] : c->grid.nv - 1);
    }
    DeviceGuard g(c->device);
    if (!c->d_window) CT_CUDA(c, cudaMalloc((void **)&c->d_window, sizeof(int4) * (size_t)V));
    CT_CUDA(c, cudaMemcpyAsync(c->d_window, hw.data(), sizeof(int4) * (size_t)V, cudaMemcpyHostToDevice, c->stream));
    CT_CUDA(c, cudaStreamSynchronize(c->stream));  // hw is a local buffer
    c->has_window = true;
    return CTREX_OK;
}

int ctrex_set_roi(ctrex_ctx *c, const ctrex_vol_grid *roi)
{
    if (!c) return CTREX_E_ARG;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_roi before set_geometry");
    DeviceGuard g(c->device);
    if (!roi) {
        c->roi = false;
        dfree(c->d_views_roi);
        atlas_release(c->roi_atlas);
        return CTREX_OK;
    }
    if (c->cyl || c->has_motion || c->dyr || c->projector != CTREX_PROJ_TRILINEAR)
        return fail(c, CTREX_E_STATE, "set_roi: the ROI projector is the trilinear one on a Cartesian grid without "
                                      "motion or the event model");
    if (roi->nx < 1 || roi->ny < 1 || roi->nz < 1 ||
        (long long)roi->nx * roi->ny * roi->nz + (long long)grid_voxels(c->grid) >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_roi: grid %d x %d x %d unsupported", roi->nx, roi->ny, roi->nz);
    const int n[3] = {roi->nx, roi->ny, roi->nz}, nc[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (!(roi->vox[a] > 0.0) || !isfinite(roi->vox[a]) || !isfinite(roi->origin[a]))
            return fail(c, CTREX_E_ARG, "set_roi: voxel pitch must be > 0 and origin finite");
        // the ROI box must lie inside the context grid's box
        lo[a] = roi->origin[a] - 0.5 * roi->vox[a];
        hi[a] = roi->origin[a] + (n[a] - 0.5) * roi->vox[a];
        const double clo = c->origin[a] - 0.5 * c->vox[a], chi = c->origin[a] + (nc[a] - 0.5) * c->vox[a];
        const double tol = 1e-9 * (chi - clo);
        if (lo[a] < clo - tol || hi[a] > chi + tol)
            return fail(c, CTREX_E_ARG, "set_roi: the ROI box leaves the context grid's box on axis %d", a);
    }
    const int nvs = c->grid.n_views * c->grid.n_sub;
    std::vector<ViewGPU> hv;
    int e = compute_views(c, c->hostP.data(), nvs, c->grid.n_sub, roi->vox, roi->origin, c->ctr, c->grid.uc,
                          c->grid.vc, hv);
    if (e) return e;
    dfree(c->d_views_roi);
    CT_CUDA(c, cudaMalloc((void **)&c->d_views_roi, sizeof(ViewGPU) * (size_t)nvs));
    CT_CUDA(c, cudaMemcpy(c->d_views_roi, hv.data(), sizeof(ViewGPU) * (size_t)nvs, cudaMemcpyHostToDevice));
    Grid &F = c->roi_grid;
    F = c->grid;
    F.nx = n[0];
    F.ny = n[1];
    F.nz = n[2];
    double minf = roi->vox[0];
    for (int a = 0; a < 3; ++a) {
        F.vox[a] = (float)roi->vox[a];
        minf = fmin(minf, roi->vox[a]);
        F.lo[a] = -0.5f;
        F.hi[a] = (float)(n[a] - 0.5);
    }
    F.step_mm = (float)(c->step_vox * minf);
    RoiGPU &R = c->roig;
    for (int a = 0; a < 3; ++a) {
        R.sc[a] = (float)(c->vox[a] / roi->vox[a]);
        R.oc[a] = (float)((c->origin[a] - roi->origin[a]) / roi->vox[a]);
        R.lo[a] = (float)((lo[a] - c->origin[a]) / c->vox[a]);
        R.hi[a] = (float)((hi[a] - c->origin[a]) / c->vox[a]);
    }
    R.step_mm = F.step_mm;
    for (int a = 0; a < 3; ++a) R.n[a] = n[a];
    c->roi = true;
    return CTREX_OK;
}

int ctrex_set_projector(ctrex_ctx *c, int kind)
{
    if (!c) return CTREX_E_ARG;
    if (kind != CTREX_PROJ_TRILINEAR && kind != CTREX_PROJ_JOSEPH)
        return fail(c, CTREX_E_ARG, "set_projector: unknown projector %d", kind);
    if (kind == CTREX_PROJ_JOSEPH && (c->cyl || c->has_motion || c->roi || c->dyr))
        return fail(c, CTREX_E_STATE, "set_projector: the Joseph projector is defined on the Cartesian grid "
                                      "without motion or the event model");
    c->projector = kind;
    if (kind != CTREX_PROJ_JOSEPH) atlas_release(c->jos_atlas);
    return CTREX_OK;
}

int ctrex_set_bp_subvoxel(ctrex_ctx *c, int s)
{
    if (!c) return CTREX_E_ARG;
    if (s < 1 || s > CTREX_MAX_SUBVOXEL) return fail(c, CTREX_E_ARG, "set_bp_subvoxel: s must be in [1, 8]");
    if (s > 1 && c->dyr) return fail(c, CTREX_E_STATE, "set_bp_subvoxel: not defined with the event model");
    c->bp_subvoxel = s;
    return CTREX_OK;
}

int ctrex_set_dyrect(ctrex_ctx *c, const float *tau, const float *t_view)
{
    if (!c) return CTREX_E_ARG;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_dyrect before set_geometry");
    DeviceGuard g(c->device);
    if (!tau) {
        dyr_release(c);
        return CTREX_OK;
    }
    if (!t_view) return fail(c, CTREX_E_ARG, "set_dyrect: t_view is NULL");
    if (c->cyl || c->roi || c->has_motion || c->projector != CTREX_PROJ_TRILINEAR || c->bp_subvoxel > 1)
        return fail(c, CTREX_E_STATE, "set_dyrect: the event model is defined for the trilinear projector on one "
                                      "Cartesian grid, without motion, ROI or sub-voxel backprojection");
    if (2 * (long long)grid_voxels(c->grid) >= (1LL << 31))
        return fail(c, CTREX_E_SHAPE, "set_dyrect: the two value fields exceed 2^31 elements");
    const size_t nvox = grid_voxels(c->grid), V = (size_t)c->grid.n_views;
    if (!c->d_tau) CT_CUDA(c, cudaMalloc((void **)&c->d_tau, sizeof(float) * nvox));
    if (!c->d_tview) CT_CUDA(c, cudaMalloc((void **)&c->d_tview, sizeof(float) * V));
    CT_CUDA(c, cudaMemcpyAsync(c->d_tau, tau, sizeof(float) * nvox, cudaMemcpyDeviceToDevice, c->stream));
    CT_CUDA(c, cudaMemcpyAsync(c->d_tview, t_view, sizeof(float) * V, cudaMemcpyDeviceToDevice, c->stream));
    cudaError_t e = atlas_ensure(c->tau_atlas, c->grid.nx, c->grid.ny, c->grid.nz, false, c->device, false);
    if (e == cudaErrorInvalidValue) {
        cudaGetLastError();
        dyr_release(c);
        return fail(c, CTREX_E_SHAPE, "set_dyrect: the volume exceeds the 2D texture limits of the device");
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "transition-time atlas allocation");
    e = atlas_upload(c->tau_atlas, c->d_tau, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "transition-time atlas upload");
    c->tau_atlas_view = atlas_view(c->tau_atlas);
    const int bnx = (c->grid.nx + 7) / 8, bny = (c->grid.ny + 7) / 8, bnz = (c->grid.nz + 7) / 8;
    if (!c->d_tau_brick)
        CT_CUDA(c, cudaMalloc((void **)&c->d_tau_brick, sizeof(float2) * (size_t)bnx * bny * bnz));
    e = launch_tau_bricks(c->d_tau, c->grid.nx, c->grid.ny, c->grid.nz, c->d_tau_brick, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "transition-time bricks");
    c->dyra.tau_brick = c->d_tau_brick;
    c->dyra.bnx = bnx;
    c->dyra.bny = bny;
    c->dyra.tau = c->d_tau;
    c->dyra.t_view = c->d_tview;
    c->dyra.tau_atlas = &c->tau_atlas_view;
    c->dyra.mu1 = &c->dyr_atlas1_view;
    c->dyr = true;
    return CTREX_OK;
}

int ctrex_fwd_project(ctrex_ctx *c, const void *vol, int vdt, void *proj, int pdt, float *rowsum,
                      const int *view_idx, int n_idx)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (n_idx == 0) return CTREX_OK;  // nothing to project
    if (!vol || !proj) return fail(c, CTREX_E_ARG, "fwd_project: NULL buffer");
    if (!dtype_ok(vdt) || !dtype_ok(pdt)) return fail(c, CTREX_E_DTYPE, "fwd_project: bad dtype");
    DeviceGuard g(c->device);
    FwdArgs a = fwd_args(c, vol, vdt, view_idx, n_idx);
    e = prepare_atlas(c, a, vol, vdt);
    if (e) return e;
    cudaError_t ce = launch_forward(a, proj, pdt, rowsum);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "fwd_project launch");
    return CTREX_OK;
}

static int ensure_partials(ctrex_ctx *c, int n_idx)
{
    const int need = forward_partials_needed(c->grid, n_idx);
    if (need <= c->partials_cap) return CTREX_OK;
    size_t have = (size_t)c->partials_cap * 2 * sizeof(float);
    int e = ensure(c, (void **)&c->d_partials, &have, (size_t)need * 2 * sizeof(float), "residual partials");
    if (e) return e;
    c->partials_cap = need;
    return CTREX_OK;
}

int ctrex_fwd_correct(ctrex_ctx *c, const void *vol, int vdt, const void *p, int pdt, void *r, int rdt,
                      double *sums, const int *view_idx, int n_idx)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (n_idx == 0) {  // empty view list: zero norms, no images
        if (sums) CT_CUDA(c, cudaMemsetAsync(sums, 0, 2 * sizeof(double), c->stream));
        return CTREX_OK;
    }
    if (!vol || !p || !r) return fail(c, CTREX_E_ARG, "fwd_correct: NULL buffer");
    if (!dtype_ok(vdt) || !dtype_ok(pdt) || !dtype_ok(rdt)) return fail(c, CTREX_E_DTYPE, "fwd_correct: bad dtype");
    if (pdt != rdt) return fail(c, CTREX_E_DTYPE, "fwd_correct: p and r must share one dtype");
    DeviceGuard g(c->device);
    e = ensure_partials(c, n_idx);
    if (e) return e;
    FwdArgs a = fwd_args(c, vol, vdt, view_idx, n_idx);
    e = prepare_atlas(c, a, vol, vdt);
    if (e) return e;
    cudaError_t ce = launch_forward_correct(a, p, pdt, r, rdt, c->d_partials, c->partials_cap, sums);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "fwd_correct launch");
    return CTREX_OK;
}

int ctrex_back_project(ctrex_ctx *c, const void *r, int rdt, void *vol, int vdt, const float *w, float alpha,
                       int normalize, int accumulate, const int *view_idx, int n_idx)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (!vol || (!r && n_idx > 0)) return fail(c, CTREX_E_ARG, "back_project: NULL buffer");
    if (!dtype_ok(vdt) || !dtype_ok(rdt)) return fail(c, CTREX_E_DTYPE, "back_project: bad dtype");
    if (!isfinite(alpha)) return fail(c, CTREX_E_ARG, "back_project: alpha not finite");
    DeviceGuard g(c->device);
    BpArgs a;
    a.grid = &c->grid;
    a.views = c->d_views;
    a.view_idx = view_idx;
    a.n_idx = n_idx;
    a.r = r;
    a.r_dtype = rdt;
    a.vol = vol;
    a.vol_dtype = vdt;
    a.w = w;
    a.alpha = alpha;
    a.normalize = normalize ? 1 : 0;
    a.accumulate = accumulate ? 1 : 0;
    a.stream = c->stream;
    a.window = c->has_window ? c->d_window : nullptr;
    a.subvox = c->bp_subvoxel;
    a.cyl = c->cyl ? &c->cylg : nullptr;
    a.dyr = c->dyr ? &c->dyra : nullptr;
    if (n_idx > 0 && !c->img_atlas_unfit) {
        cudaError_t ae = atlas_ensure(c->img_atlas, c->grid.nu, c->grid.nv, n_idx, rdt == CTREX_BF16, c->device);
        if (ae == cudaErrorInvalidValue) {
            cudaGetLastError();
            c->img_atlas_unfit = true;
        } else if (ae != cudaSuccess) {
            return cuda_fail(c, ae, "image atlas allocation");
        } else {
            ae = atlas_upload(c->img_atlas, r, c->stream);
            if (ae != cudaSuccess) return cuda_fail(c, ae, "image atlas upload");
            c->img_atlas_view = atlas_view(c->img_atlas);
            a.atlas = &c->img_atlas_view;
        }
    }
    cudaError_t ce = launch_backproject(a);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "back_project launch");
    if (c->roi) {  // the ROI grid's voxels follow the context grid's
        const size_t nc = grid_voxels(c->grid);
        a.grid = &c->roi_grid;
        a.views = c->d_views_roi;
        a.vol = static_cast<char *>(vol) + nc * dtype_size(vdt);
        a.w = w ? w + nc : nullptr;
        ce = launch_backproject(a);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "back_project launch (ROI grid)");
    }
    return CTREX_OK;
}

int ctrex_adjoint_project(ctrex_ctx *c, const float *proj, float *vol, const int *view_idx, int n_idx)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (c->cyl || c->roi || c->projector == CTREX_PROJ_JOSEPH)
        return fail(c, CTREX_E_STATE, "adjoint_project: the transpose of the trilinear projector on one Cartesian "
                                      "grid only");
    if (n_idx == 0) return CTREX_OK;
    if (!proj || !vol) return fail(c, CTREX_E_ARG, "adjoint_project: NULL buffer");
    DeviceGuard g(c->device);
    cudaError_t ce = launch_adjoint(fwd_args(c, nullptr, CTREX_F32, view_idx, n_idx), proj, vol);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "adjoint_project launch");
    return CTREX_OK;
}

int ctrex_motion_grad(ctrex_ctx *c, const void *vol, int vdt, const float *gproj, float *grad_theta,
                      float *grad_coef, const int *view_idx, int n_idx)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (!c->has_motion || c->dyr) return fail(c, CTREX_E_STATE, "motion_grad: set_motion has not been called");
    if (n_idx == 0) return CTREX_OK;
    if (!vol || !gproj) return fail(c, CTREX_E_ARG, "motion_grad: NULL buffer");
    if (!dtype_ok(vdt)) return fail(c, CTREX_E_DTYPE, "motion_grad: bad dtype");
    if (grad_theta && !c->theta_valid)
        return fail(c, CTREX_E_STATE, "motion_grad: grad_theta requested but no theta was set");
    if (grad_coef && !c->coef_valid)
        return fail(c, CTREX_E_STATE, "motion_grad: grad_coef requested but no coefficients were set");
    DeviceGuard g(c->device);
    const int V = c->grid.n_views;
    CT_CUDA(c, cudaMemsetAsync(c->d_gM, 0, sizeof(double) * 9 * (size_t)V, c->stream));
    CT_CUDA(c, cudaMemsetAsync(c->d_gb, 0, sizeof(double) * 3 * (size_t)V, c->stream));
    CT_CUDA(c, cudaMemsetAsync(c->d_gcoef, 0, sizeof(double) * 1536, c->stream));
    cudaError_t ce = launch_motion_grad(fwd_args(c, vol, vdt, view_idx, n_idx), gproj, c->d_gM, c->d_gb,
                                        grad_coef ? c->d_gcoef : nullptr);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "motion_grad launch");
    ce = launch_motion_grad_finish(c->theta_valid ? c->d_theta : nullptr, c->d_dRdw, c->d_gM, c->d_gb, c->d_gcoef, V,
                                   c->grid, c->vox, c->origin, grad_theta, grad_coef, c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "motion_grad finish");
    return CTREX_OK;
}

int ctrex_sirt_iterate(ctrex_ctx *c, void *vol, int vdt, const void *p, int pdt, int max_iter, float alpha,
                       const float *w, float tol, float *hist, int *iters_done)
{
    if (!c) return CTREX_E_ARG;
    if (iters_done) *iters_done = 0;
    int e = check_views(c, nullptr, c->has_geom ? c->grid.n_views : 0);
    if (e) return e;
    if (!vol || !p) return fail(c, CTREX_E_ARG, "sirt_iterate: NULL buffer");
    if (!dtype_ok(vdt) || !dtype_ok(pdt)) return fail(c, CTREX_E_DTYPE, "sirt_iterate: bad dtype");
    if (max_iter < 0) return fail(c, CTREX_E_ARG, "sirt_iterate: max_iter < 0");
    DeviceGuard g(c->device);
    const int V = c->grid.n_views;
    const size_t rb = (size_t)V * c->grid.nu * c->grid.nv * dtype_size(pdt);
    e = ensure(c, &c->d_r, &c->r_bytes, rb, "SIRT correction images");
    if (e) return e;
    e = ensure_partials(c, V);
    if (e) return e;
    for (int k = 0; k < max_iter; ++k) {
        FwdArgs a = fwd_args(c, vol, vdt, nullptr, V);
        e = prepare_atlas(c, a, vol, vdt);
        if (e) return e;
        cudaError_t ce = launch_forward_correct(a, p, pdt, c->d_r, pdt, c->d_partials, c->partials_cap, c->d_sums);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "sirt: fwd_correct");
        double s[2];
        CT_CUDA(c, cudaMemcpyAsync(s, c->d_sums, sizeof s, cudaMemcpyDeviceToHost, c->stream));
        CT_CUDA(c, cudaStreamSynchronize(c->stream));
        const double rho = s[1] > 0.0 ? sqrt(s[0] / s[1]) : sqrt(s[0]);
        if (hist) hist[k] = (float)rho;
        if (!isfinite(rho)) return fail(c, CTREX_E_DIVERGED, "sirt: residual not finite at iteration %d", k);
        if (rho <= (double)tol) break;
        int be = ctrex_back_project(c, c->d_r, pdt, vol, vdt, w, alpha, 1, 1, nullptr, V);
        if (be) return be;
        if (iters_done) *iters_done = k + 1;
    }
    return ctrex_device_status(c);
}

int ctrex_os_sirt_iterate(ctrex_ctx *c, void *vol, int vdt, const void *p, int pdt, const int *subset_views,
                          const int *subset_offsets, int n_sets, int max_cycles, float alpha, const float *w,
                          float tol, float *hist, int *cycles_done)
{
    if (!c) return CTREX_E_ARG;
    if (cycles_done) *cycles_done = 0;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_geometry has not been called");
    if (!vol || !p || !subset_views || !subset_offsets) return fail(c, CTREX_E_ARG, "os_sirt: NULL argument");
    if (!dtype_ok(vdt) || !dtype_ok(pdt)) return fail(c, CTREX_E_DTYPE, "os_sirt: bad dtype");
    if (n_sets < 1 || max_cycles < 0) return fail(c, CTREX_E_ARG, "os_sirt: need n_sets >= 1, max_cycles >= 0");
    const int V = c->grid.n_views;
    if (subset_offsets[0] != 0) return fail(c, CTREX_E_ARG, "os_sirt: subset_offsets[0] must be 0");
    int maxlen = 0;
    for (int s = 0; s < n_sets; ++s) {
        const int n = subset_offsets[s + 1] - subset_offsets[s];
        if (n < 0 || n > 65535) return fail(c, CTREX_E_SHAPE, "os_sirt: subset %d has size %d", s, n);
        if (n > maxlen) maxlen = n;
    }
    const int total = subset_offsets[n_sets];
    for (int i = 0; i < total; ++i)
        if (subset_views[i] < 0 || subset_views[i] >= V)
            return fail(c, CTREX_E_SHAPE, "os_sirt: view %d out of range", subset_views[i]);
    DeviceGuard g(c->device);
    int e = ensure(c, (void **)&c->d_subset_views, &c->subset_views_bytes, sizeof(int) * (size_t)(total > 0 ? total : 1),
                   "subset view lists");
    if (e) return e;
    e = ensure(c, (void **)&c->d_subset_sums, &c->subset_sums_bytes, sizeof(double) * 2 * (size_t)n_sets,
               "subset residual norms");
    if (e) return e;
    const size_t rb = (size_t)(maxlen > 0 ? maxlen : 1) * c->grid.nu * c->grid.nv * dtype_size(pdt);
    e = ensure(c, &c->d_r, &c->r_bytes, rb, "correction images");
    if (e) return e;
    e = ensure_partials(c, maxlen > 0 ? maxlen : 1);
    if (e) return e;
    if (total > 0)
        CT_CUDA(c, cudaMemcpyAsync(c->d_subset_views, subset_views, sizeof(int) * (size_t)total, cudaMemcpyHostToDevice,
                                   c->stream));
    CT_CUDA(c, cudaMemsetAsync(c->d_subset_sums, 0, sizeof(double) * 2 * (size_t)n_sets, c->stream));
    std::vector<double> sums(2 * (size_t)n_sets);
    for (int k = 0; k < max_cycles; ++k) {
        for (int s = 0; s < n_sets; ++s) {
            const int n = subset_offsets[s + 1] - subset_offsets[s];
            if (n == 0) continue;
            const int *vs = c->d_subset_views + subset_offsets[s];
            FwdArgs a = fwd_args(c, vol, vdt, vs, n);
            a.p_by_view = 1;
            e = prepare_atlas(c, a, vol, vdt);
            if (e) return e;
            cudaError_t ce = launch_forward_correct(a, p, pdt, c->d_r, pdt, c->d_partials, c->partials_cap,
                                                    c->d_subset_sums + 2 * (size_t)s);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "os_sirt: fwd_correct");
            int be = ctrex_back_project(c, c->d_r, pdt, vol, vdt, w, alpha, 1, 1, vs, n);
            if (be) return be;
        }
        CT_CUDA(c, cudaMemcpyAsync(sums.data(), c->d_subset_sums, sizeof(double) * 2 * (size_t)n_sets,
                                   cudaMemcpyDeviceToHost, c->stream));
        CT_CUDA(c, cudaStreamSynchronize(c->stream));
        double acc = 0.0, p2 = 0.0;
        for (int s = 0; s < n_sets; ++s) {
            if (subset_offsets[s + 1] == subset_offsets[s]) continue;
            acc += sums[2 * (size_t)s];
            p2 += sums[2 * (size_t)s + 1];
        }
        const double rho = p2 > 0.0 ? sqrt(acc / p2) : sqrt(acc);
        if (hist) hist[k] = (float)rho;
        if (cycles_done) *cycles_done = k + 1;
        if (!isfinite(rho)) return fail(c, CTREX_E_DIVERGED, "os_sirt: residual not finite in cycle %d", k);
        if (rho <= (double)tol) break;
    }
    return ctrex_device_status(c);
}

int ctrex_sirt_host(ctrex_ctx *c, void *vol_h, int vdt, const void *p_h, int pdt, int max_iter, float alpha,
                    const float *w_h, float tol, float *hist, int *iters_done)
{
    if (!c) return CTREX_E_ARG;
    if (!c->has_geom) return fail(c, CTREX_E_STATE, "set_geometry has not been called");
    if (!vol_h || !p_h) return fail(c, CTREX_E_ARG, "sirt_host: NULL buffer");
    if (!dtype_ok(vdt) || !dtype_ok(pdt)) return fail(c, CTREX_E_DTYPE, "sirt_host: bad dtype");
    DeviceGuard g(c->device);
    const Grid &G = c->grid;
    const size_t nvox = volume_elems(c);
    const size_t vb = nvox * dtype_size(vdt);
    const size_t pb = (size_t)G.n_views * G.nu * G.nv * dtype_size(pdt);
    int e = ensure(c, &c->d_hvol, &c->hvol_bytes, vb, "host-SIRT volume");
    if (e) return e;
    e = ensure(c, &c->d_hp, &c->hp_bytes, pb, "host-SIRT projections");
    if (e) return e;
    const float *dw = nullptr;
    if (w_h) {
        e = ensure(c, (void **)&c->d_hw, &c->hw_bytes, nvox * sizeof(float), "host-SIRT weights");
        if (e) return e;
        CT_CUDA(c, cudaMemcpyAsync(c->d_hw, w_h, nvox * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        dw = c->d_hw;
    }
    CT_CUDA(c, cudaMemcpyAsync(c->d_hvol, vol_h, vb, cudaMemcpyHostToDevice, c->stream));
    if (iters_done) *iters_done = 0;
    int first = 0;  // iterations done here, before ctrex_sirt_iterate takes over
    if (pdt == CTREX_F32 && max_iter >= 1) {
        // First iteration: the projections (the larger upload) travel on a
        // copy stream while the forward projection runs; the correction
        // r = R (p - A x) waits for them (the kernels of
        // ctrex_correct_static with this context's own scratch).  Same
        // arithmetic as the fused correction (A x and the row sums are FP32
        // either way); only the residual norms are summed in another order.
        const size_t npix = (size_t)G.n_views * G.nu * G.nv;
        e = ensure(c, &c->d_hq, &c->hq_bytes, npix * sizeof(float), "host-SIRT forward projection");
        if (e) return e;
        e = ensure(c, (void **)&c->d_hrs, &c->hrs_bytes, npix * sizeof(float), "host-SIRT row sums");
        if (e) return e;
        e = ensure(c, &c->d_r, &c->r_bytes, npix * sizeof(float), "SIRT correction images");
        if (e) return e;
        const size_t pairs = (size_t)correct_scratch_pairs((long long)npix);
        e = ensure(c, (void **)&c->d_hcs, &c->hcs_bytes, 2 * sizeof(double) * pairs, "host-SIRT correction partials");
        if (e) return e;
        if (!c->copy_stream) CT_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->ev_vol) CT_CUDA(c, cudaEventCreateWithFlags(&c->ev_vol, cudaEventDisableTiming));
        if (!c->ev_p) CT_CUDA(c, cudaEventCreateWithFlags(&c->ev_p, cudaEventDisableTiming));
        CT_CUDA(c, cudaEventRecord(c->ev_vol, c->stream));  // the volume's upload (and earlier work) first
        CT_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_vol, 0));
        CT_CUDA(c, cudaMemcpyAsync(c->d_hp, p_h, pb, cudaMemcpyHostToDevice, c->copy_stream));
        CT_CUDA(c, cudaEventRecord(c->ev_p, c->copy_stream));
        FwdArgs a = fwd_args(c, c->d_hvol, vdt, nullptr, G.n_views);
        e = prepare_atlas(c, a, c->d_hvol, vdt);
        if (e) return e;
        cudaError_t ce = launch_forward(a, c->d_hq, CTREX_F32, c->d_hrs);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "sirt_host: forward projection");
        CT_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_p, 0));
        ce = launch_correct(c->d_hp, c->d_hq, c->d_hrs, c->d_r, CTREX_F32, (long long)npix, G.eps_R, c->d_sums,
                            c->d_hcs, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "sirt_host: correction of the first iteration");
        double s[2];
        CT_CUDA(c, cudaMemcpyAsync(s, c->d_sums, sizeof s, cudaMemcpyDeviceToHost, c->stream));
        CT_CUDA(c, cudaStreamSynchronize(c->stream));
        const double rho = s[1] > 0.0 ? sqrt(s[0] / s[1]) : sqrt(s[0]);
        if (hist) hist[0] = (float)rho;
        if (!isfinite(rho)) return fail(c, CTREX_E_DIVERGED, "sirt: residual not finite at iteration 0");
        first = 1;
        if (rho <= (double)tol) {
            max_iter = first;  // converged before the first update
        } else {
            e = ctrex_back_project(c, c->d_r, CTREX_F32, c->d_hvol, vdt, dw, alpha, 1, 1, nullptr, G.n_views);
            if (e) return e;
            if (iters_done) *iters_done = 1;
        }
    } else {
        CT_CUDA(c, cudaMemcpyAsync(c->d_hp, p_h, pb, cudaMemcpyHostToDevice, c->stream));
    }
    int rest = 0;
    e = ctrex_sirt_iterate(c, c->d_hvol, vdt, c->d_hp, pdt, max_iter - first, alpha, dw, tol,
                           hist ? hist + first : nullptr, &rest);
    if (iters_done && max_iter - first > 0) *iters_done = first + rest;
    if (e) return e;
    CT_CUDA(c, cudaMemcpyAsync(vol_h, c->d_hvol, vb, cudaMemcpyDeviceToHost, c->stream));
    CT_CUDA(c, cudaStreamSynchronize(c->stream));
    return CTREX_OK;
}

int ctrex_count_samples(ctrex_ctx *c, const int *view_idx, int n_idx, long long *out)
{
    if (!c) return CTREX_E_ARG;
    int e = check_views(c, view_idx, n_idx);
    if (e) return e;
    if (!out) return fail(c, CTREX_E_ARG, "count_samples: NULL output");
    DeviceGuard g(c->device);
    cudaError_t ce = launch_count_samples(fwd_args(c, nullptr, CTREX_F32, view_idx, n_idx), c->d_count);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "count_samples launch");
    unsigned long long h = 0;
    CT_CUDA(c, cudaMemcpyAsync(&h, c->d_count, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CT_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = (long long)h;
    return CTREX_OK;
}

}  // extern "C"
