"""Python binding of libctrex (ctypes): argument marshalling only.

Every operation runs in the CUDA kernels of ``libctrex.so``; this module only
checks tensor shapes, dtypes and devices, and passes raw device pointers and
the current torch stream through the C ABI declared in ``include/ctrex.h``.
There is no CPU fallback: if the library is missing, loading fails loudly.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# CTREX_LIB may point at another build of the same sources (e.g. a variant
# compiled with different tuning flags); the default is the in-tree build.
LIB_PATH = os.environ.get("CTREX_LIB") or os.path.join(_HERE, "libctrex.so")

F32, BF16 = 0, 1
OK = 0
ERRORS = {
    -1: "CTREX_E_ARG", -2: "CTREX_E_SHAPE", -3: "CTREX_E_DTYPE", -4: "CTREX_E_GEOMETRY",
    -5: "CTREX_E_CUDA", -6: "CTREX_E_DIVERGED", -7: "CTREX_E_DEVICE_CHECK", -8: "CTREX_E_NOMEM",
    -9: "CTREX_E_STATE",
}

# Every symbol include/ctrex.h declares.
EXPORTS = (
    "ctrex_version", "ctrex_create", "ctrex_destroy", "ctrex_set_stream", "ctrex_last_error",
    "ctrex_device_status", "ctrex_set_geometry", "ctrex_set_motion", "ctrex_fwd_project",
    "ctrex_fwd_correct", "ctrex_back_project", "ctrex_adjoint_project", "ctrex_motion_grad",
    "ctrex_sirt_iterate", "ctrex_sirt_host", "ctrex_count_samples", "ctrex_correct_static",
    "ctrex_conv3d_fwd", "ctrex_conv3d_wgrad", "ctrex_os_sirt_iterate", "ctrex_set_bp_window",
    "ctrex_probe_gather_rate", "ctrex_probe_l2_read_bandwidth", "ctrex_set_dyrect", "ctrex_set_bp_subvoxel", "ctrex_set_geometry_cylinder", "ctrex_set_projector",
    "ctrex_set_roi",
)

PROJ_TRILINEAR, PROJ_JOSEPH = 0, 1

# Largest n ctrex_correct_static accepts (its static scratch holds 65536 CTA partials of 8192 elements).
CORRECT_STATIC_MAX_N = 1 << 29


class CtrexError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class VolGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vox", ctypes.c_double * 3), ("origin", ctypes.c_double * 3)]


class DetGrid(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_int), ("nv", ctypes.c_int)]


class CylGrid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("n_phi", ctypes.c_int), ("n_z", ctypes.c_int),
                ("dr", ctypes.c_double), ("dz", ctypes.c_double), ("pose", ctypes.c_double * 12)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libctrex.so (built by ``__graft_entry__.build()``); no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libctrex.so not found at {path}: run __graft_entry__.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i, d, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float
    ip, fp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    sig = {
        "ctrex_version": ([], ctypes.c_char_p),
        "ctrex_create": ([ctypes.POINTER(vp), i, vp], i),
        "ctrex_destroy": ([vp], i),
        "ctrex_set_stream": ([vp, vp], i),
        "ctrex_last_error": ([vp], ctypes.c_char_p),
        "ctrex_device_status": ([vp], i),
        "ctrex_set_geometry": ([vp, ctypes.POINTER(d), i, i, ctypes.POINTER(VolGrid),
                                ctypes.POINTER(DetGrid), d], i),
        "ctrex_set_motion": ([vp, vp, vp, vp, d], i),
        "ctrex_fwd_project": ([vp, vp, i, vp, i, vp, vp, i], i),
        "ctrex_fwd_correct": ([vp, vp, i, vp, i, vp, i, vp, vp, i], i),
        "ctrex_back_project": ([vp, vp, i, vp, i, vp, f, i, i, vp, i], i),
        "ctrex_adjoint_project": ([vp, vp, vp, vp, i], i),
        "ctrex_motion_grad": ([vp, vp, i, vp, vp, vp, vp, i], i),
        "ctrex_sirt_iterate": ([vp, vp, i, vp, i, i, f, vp, f, fp, ip], i),
        "ctrex_sirt_host": ([vp, vp, i, vp, i, i, f, vp, f, fp, ip], i),
        "ctrex_count_samples": ([vp, vp, i, ctypes.POINTER(ctypes.c_longlong)], i),
        "ctrex_correct_static": ([vp, vp, vp, vp, i, ctypes.c_longlong, f, vp, vp], i),
        "ctrex_conv3d_fwd": ([vp, vp, vp, vp, i, i, i, i, i, i, i, i, vp, vp], i),
        "ctrex_conv3d_wgrad": ([vp, vp, vp, i, i, i, i, i, i, vp, vp], i),
        "ctrex_os_sirt_iterate": ([vp, vp, i, vp, i, ip, ip, i, i, f, vp, f, fp, ip], i),
        "ctrex_set_bp_window": ([vp, ip], i),
        "ctrex_set_bp_subvoxel": ([vp, i], i),
        "ctrex_set_projector": ([vp, i], i),
        "ctrex_set_roi": ([vp, ctypes.POINTER(VolGrid)], i),
        "ctrex_set_geometry_cylinder": ([vp, ctypes.POINTER(d), i, i, ctypes.POINTER(CylGrid),
                                         ctypes.POINTER(DetGrid), d], i),
        "ctrex_probe_gather_rate": ([vp, ctypes.POINTER(d)], i),
        "ctrex_probe_l2_read_bandwidth": ([vp, ctypes.POINTER(d)], i),
        "ctrex_set_dyrect": ([vp, vp, vp], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported dtype {t.dtype} (float32 or bfloat16)")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """One libctrex context bound to a CUDA device (work goes on the current
    torch stream of that device at each call)."""

    def __init__(self, device=None):
        self.lib = load_library()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", int(device) if not isinstance(device, torch.device) else device.index or 0)
        h = ctypes.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self.lib.ctrex_create(ctypes.byref(h), self.device.index, ctypes.c_void_p(stream))
        if rc != OK:
            raise CtrexError(rc, "ctrex_create failed")
        self._h = h
        self.vol_shape = None
        self.det_shape = None
        self.n_views = 0
        self.n_sub = 0

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.ctrex_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ----------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            msg = self.lib.ctrex_last_error(self._h)
            raise CtrexError(rc, msg.decode() if msg else "")

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self._check(self.lib.ctrex_set_stream(self._h, ctypes.c_void_p(s)))

    def _dev(self, t, name, shape=None, dtypes=(torch.float32, torch.bfloat16)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}, got {t.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.dtype not in dtypes:
            raise TypeError(f"{name}: dtype {t.dtype} not in {dtypes}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
        return t

    def _views(self, view_idx):
        if view_idx is None:
            return None, self.n_views
        if not isinstance(view_idx, torch.Tensor):
            view_idx = torch.as_tensor(np.asarray(view_idx, dtype=np.int32), device=self.device)
        view_idx = self._dev(view_idx.to(torch.int32).contiguous(), "view_idx", dtypes=(torch.int32,))
        return view_idx, int(view_idx.numel())

    # -- C ABI mirrors ------------------------------------------------------
    def set_geometry(self, P, vol_shape, vox, origin, det, step_vox=0.5):
        """P: float64 array [V, S, 3, 4] (or [V, 3, 4]); vol_shape (nz, ny, nx);
        vox, origin in (x, y, z) mm; det (nu, nv)."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        if P.ndim == 3:
            P = P[:, None]
        V, S = P.shape[:2]
        nz, ny, nx = (int(s) for s in vol_shape)
        vg = VolGrid(nx, ny, nz, (ctypes.c_double * 3)(*vox), (ctypes.c_double * 3)(*origin))
        dg = DetGrid(int(det[0]), int(det[1]))
        self._check(self.lib.ctrex_set_geometry(self._h, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                V, S, ctypes.byref(vg), ctypes.byref(dg), float(step_vox)))
        self.vol_shape = (nz, ny, nx)
        self.grid_shape = self.vol_shape
        self.roi_shape = None
        self.det_shape = (int(det[1]), int(det[0]))
        self.n_views, self.n_sub = V, S

    def set_roi(self, roi_shape=None, vox=None, origin=None):
        """A finer ROI grid (roi_shape (nz, ny, nx), vox and origin (x, y, z)
        mm) inside the grid: volumes then become flat [context voxels, ROI
        voxels].  None removes it."""
        if roi_shape is None:
            self._check(self.lib.ctrex_set_roi(self._h, None))
            self.vol_shape, self.roi_shape = self.grid_shape, None
            return
        nz, ny, nx = (int(s) for s in roi_shape)
        vg = VolGrid(nx, ny, nz, (ctypes.c_double * 3)(*vox), (ctypes.c_double * 3)(*origin))
        self._check(self.lib.ctrex_set_roi(self._h, ctypes.byref(vg)))
        self.roi_shape = (nz, ny, nx)
        gz, gy, gx = self.grid_shape
        self.vol_shape = (gz * gy * gx + nz * ny * nx,)

    def split_volume(self, vol):
        """(context grid view, ROI grid view) of a flat multi-resolution volume."""
        gz, gy, gx = self.grid_shape
        n = gz * gy * gx
        return vol[:n].view(self.grid_shape), vol[n:].view(self.roi_shape)

    def set_geometry_cylinder(self, P, n_r, n_phi, n_z, dr, dz, det, pose=None, step_vox=0.5):
        """The aligned cylindrical domain: n_r rings of dr mm, n_phi sectors,
        n_z slices of dz mm; pose [3, 4] maps world mm to the cylinder frame
        (identity if None).  Volumes are then [n_z, n_phi, n_r]."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        if P.ndim == 3:
            P = P[:, None]
        V, S = P.shape[:2]
        if pose is None:
            pose = np.hstack([np.eye(3), np.zeros((3, 1))])
        pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(12)
        cg = CylGrid(int(n_r), int(n_phi), int(n_z), float(dr), float(dz), (ctypes.c_double * 12)(*pose))
        dg = DetGrid(int(det[0]), int(det[1]))
        self._check(self.lib.ctrex_set_geometry_cylinder(
            self._h, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), V, S, ctypes.byref(cg), ctypes.byref(dg),
            float(step_vox)))
        self.vol_shape = (int(n_z), int(n_phi), int(n_r))
        self.grid_shape = self.vol_shape
        self.roi_shape = None
        self.det_shape = (int(det[1]), int(det[0]))
        self.n_views, self.n_sub = V, S

    def set_motion(self, theta=None, coef=None, s_view=None, margin=0.0):
        self._sync_stream()
        args = []
        for t, name, shape in ((theta, "theta", (self.n_views, 15)), (coef, "coef", (8, 8, 8, 3)),
                               (s_view, "s_view", (self.n_views,))):
            if t is not None:
                t = self._dev(t, name, shape, dtypes=(torch.float32,))
            args.append(t)
        self._motion_keep = args  # the set-up kernel reads them on the stream
        self._check(self.lib.ctrex_set_motion(self._h, *[_ptr(a) for a in args], float(margin)))

    def set_bp_window(self, window=None):
        """Per-view backprojection detector windows [n_views, 4] = (u_lo, u_hi,
        v_lo, v_hi) (extended field of view), or None for the whole detector."""
        if window is None:
            self._check(self.lib.ctrex_set_bp_window(self._h, None))
            return
        win = np.ascontiguousarray(window, dtype=np.int32)
        if win.shape != (self.n_views, 4):
            raise ValueError(f"window must be [{self.n_views}, 4]")
        self._sync_stream()
        self._check(self.lib.ctrex_set_bp_window(self._h, win.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))

    def set_projector(self, kind="trilinear"):
        """Forward projector: "trilinear" (default) or "joseph"."""
        k = {"trilinear": PROJ_TRILINEAR, "joseph": PROJ_JOSEPH}[kind]
        self._check(self.lib.ctrex_set_projector(self._h, k))

    def set_dyrect(self, tau=None, t_view=None):
        """Event-based 4D model (Sec. 3.3): tau [nz, ny, nx] transition times
        and t_view [n_views] acquisition times (float32 device tensors);
        volumes then become [2, nz, ny, nx] = (initial values, final values).
        None switches it off."""
        self._sync_stream()
        if tau is None:
            self._check(self.lib.ctrex_set_dyrect(self._h, None, None))
            self.vol_shape = self.grid_shape
            return
        tau = self._dev(tau, "tau", self.grid_shape, dtypes=(torch.float32,))
        t_view = self._dev(t_view, "t_view", (self.n_views,), dtypes=(torch.float32,))
        self._dyr_keep = (tau, t_view)  # copied on the stream
        self._check(self.lib.ctrex_set_dyrect(self._h, _ptr(tau), _ptr(t_view)))
        self.vol_shape = (2,) + tuple(self.grid_shape)

    def set_bp_subvoxel(self, s=1):
        """Sub-voxel backprojection: s^3 points per voxel (1 = off)."""
        self._check(self.lib.ctrex_set_bp_subvoxel(self._h, int(s)))

    def fwd_project(self, vol, proj=None, rowsum=None, view_idx=None, out_dtype=None):
        self._sync_stream()
        vol = self._dev(vol, "vol", self.vol_shape)
        vi, n = self._views(view_idx)
        shape = (n,) + self.det_shape
        if proj is None:
            proj = torch.empty(shape, dtype=out_dtype or vol.dtype, device=self.device)
        proj = self._dev(proj, "proj", shape)
        if rowsum is not None:
            rowsum = self._dev(rowsum, "rowsum", shape, dtypes=(torch.float32,))
        self._check(self.lib.ctrex_fwd_project(self._h, _ptr(vol), _dt(vol), _ptr(proj), _dt(proj),
                                               _ptr(rowsum), _ptr(vi), n))
        return proj

    def fwd_correct(self, vol, p, r=None, sums=None, view_idx=None):
        self._sync_stream()
        vol = self._dev(vol, "vol", self.vol_shape)
        vi, n = self._views(view_idx)
        shape = (n,) + self.det_shape
        p = self._dev(p, "p", shape)
        if r is None:
            r = torch.empty(shape, dtype=p.dtype, device=self.device)
        r = self._dev(r, "r", shape)
        if sums is None:
            sums = torch.empty(2, dtype=torch.float64, device=self.device)
        sums = self._dev(sums, "sums", (2,), dtypes=(torch.float64,))
        self._check(self.lib.ctrex_fwd_correct(self._h, _ptr(vol), _dt(vol), _ptr(p), _dt(p), _ptr(r), _dt(r),
                                               _ptr(sums), _ptr(vi), n))
        return r, sums

    def back_project(self, r, vol=None, w=None, alpha=1.0, normalize=True, accumulate=True, view_idx=None,
                     vol_dtype=torch.float32):
        self._sync_stream()
        vi, n = self._views(view_idx)
        r = self._dev(r, "r", (n,) + self.det_shape)
        if vol is None:
            vol = torch.zeros(self.vol_shape, dtype=vol_dtype, device=self.device)
        vol = self._dev(vol, "vol", self.vol_shape)
        if w is not None:
            w = self._dev(w, "w", self.vol_shape, dtypes=(torch.float32,))
        self._check(self.lib.ctrex_back_project(self._h, _ptr(r), _dt(r), _ptr(vol), _dt(vol), _ptr(w),
                                                float(alpha), int(bool(normalize)), int(bool(accumulate)),
                                                _ptr(vi), n))
        return vol

    def adjoint_project(self, proj, vol=None, view_idx=None):
        self._sync_stream()
        vi, n = self._views(view_idx)
        proj = self._dev(proj, "proj", (n,) + self.det_shape, dtypes=(torch.float32,))
        if vol is None:
            vol = torch.zeros(self.vol_shape, dtype=torch.float32, device=self.device)
        vol = self._dev(vol, "vol", self.vol_shape, dtypes=(torch.float32,))
        self._check(self.lib.ctrex_adjoint_project(self._h, _ptr(proj), _ptr(vol), _ptr(vi), n))
        return vol

    def motion_grad(self, vol, grad_proj, grad_theta=None, grad_coef=None, view_idx=None, want_theta=True,
                    want_coef=True):
        self._sync_stream()
        vol = self._dev(vol, "vol", self.vol_shape)
        vi, n = self._views(view_idx)
        grad_proj = self._dev(grad_proj, "grad_proj", (n,) + self.det_shape, dtypes=(torch.float32,))
        if want_theta and grad_theta is None:
            grad_theta = torch.zeros((self.n_views, 15), dtype=torch.float32, device=self.device)
        if want_coef and grad_coef is None:
            grad_coef = torch.zeros((8, 8, 8, 3), dtype=torch.float32, device=self.device)
        if grad_theta is not None:
            grad_theta = self._dev(grad_theta, "grad_theta", (self.n_views, 15), dtypes=(torch.float32,))
        if grad_coef is not None:
            grad_coef = self._dev(grad_coef, "grad_coef", (8, 8, 8, 3), dtypes=(torch.float32,))
        self._check(self.lib.ctrex_motion_grad(self._h, _ptr(vol), _dt(vol), _ptr(grad_proj), _ptr(grad_theta),
                                               _ptr(grad_coef), _ptr(vi), n))
        return grad_theta, grad_coef

    def sirt_iterate(self, vol, p, max_iter, alpha=1.0, w=None, tol=0.0):
        self._sync_stream()
        vol = self._dev(vol, "vol", self.vol_shape)
        p = self._dev(p, "p", (self.n_views,) + self.det_shape)
        if w is not None:
            w = self._dev(w, "w", self.vol_shape, dtypes=(torch.float32,))
        hist = np.full(max(max_iter, 1), np.nan, dtype=np.float32)
        done = ctypes.c_int(0)
        self._check(self.lib.ctrex_sirt_iterate(self._h, _ptr(vol), _dt(vol), _ptr(p), _dt(p), int(max_iter),
                                                float(alpha), _ptr(w), float(tol),
                                                hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                ctypes.byref(done)))
        return vol, hist[:max_iter], done.value

    def os_sirt_iterate(self, vol, p, subsets, max_cycles, alpha=1.0, w=None, tol=0.0):
        """Ordered-subset SIRT over ``subsets`` (a list of view lists)."""
        self._sync_stream()
        vol = self._dev(vol, "vol", self.vol_shape)
        p = self._dev(p, "p", (self.n_views,) + self.det_shape)
        if w is not None:
            w = self._dev(w, "w", self.vol_shape, dtypes=(torch.float32,))
        views = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in subsets]),
                                     dtype=np.int32)
        offsets = np.ascontiguousarray(np.cumsum([0] + [len(s) for s in subsets]), dtype=np.int32)
        hist = np.full(max(max_cycles, 1), np.nan, dtype=np.float32)
        done = ctypes.c_int(0)
        ip = ctypes.POINTER(ctypes.c_int)
        self._check(self.lib.ctrex_os_sirt_iterate(
            self._h, _ptr(vol), _dt(vol), _ptr(p), _dt(p), views.ctypes.data_as(ip), offsets.ctypes.data_as(ip),
            len(subsets), int(max_cycles), float(alpha), _ptr(w), float(tol),
            hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(done)))
        return vol, hist[:max_cycles], done.value

    def sirt_host(self, vol_host, p_host, max_iter, alpha=1.0, w_host=None, tol=0.0):
        """SIRT on HOST tensors (CPU, ideally pinned): the library copies in,
        iterates and copies the volume back into vol_host."""
        self._sync_stream()
        for t, name in ((vol_host, "vol"), (p_host, "p")):
            if t.device.type != "cpu" or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor")
        if w_host is not None and (w_host.device.type != "cpu" or w_host.dtype != torch.float32):
            raise ValueError("w must be a float32 CPU tensor")
        hist = np.full(max(max_iter, 1), np.nan, dtype=np.float32)
        done = ctypes.c_int(0)
        self._check(self.lib.ctrex_sirt_host(self._h, _ptr(vol_host), _dt(vol_host), _ptr(p_host), _dt(p_host),
                                             int(max_iter), float(alpha), _ptr(w_host), float(tol),
                                             hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                             ctypes.byref(done)))
        return vol_host, hist[:max_iter], done.value

    def count_samples(self, view_idx=None):
        self._sync_stream()
        vi, n = self._views(view_idx)
        out = ctypes.c_longlong(0)
        self._check(self.lib.ctrex_count_samples(self._h, _ptr(vi), n, ctypes.byref(out)))
        return int(out.value)

    def device_status(self):
        self._sync_stream()
        self._check(self.lib.ctrex_device_status(self._h))


def correct_static(p, q, rowsum, r=None, sums=None, eps_R=0.0):
    """r = R (p - q) and (sum (p-q)^2, sum p^2) without any allocation in the
    library (for callers that cannot let it call cudaMalloc); see
    ``ctrex_correct_static`` in include/ctrex.h.  Runs on the device of p, on
    the current torch stream.  Calls that overlap on the GPU share one static
    scratch array and race: serialise them.  Every tensor is checked before
    the call, so a wrong output buffer is refused instead of being written
    past its end."""
    lib = load_library()
    dev = p.device if isinstance(p, torch.Tensor) else None
    for t, name in ((p, "p"), (q, "q"), (rowsum, "rowsum")):
        if not isinstance(t, torch.Tensor) or t.device != dev or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous tensor on {dev}")
    if p.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("p must be float32 or bfloat16")
    if q.dtype != p.dtype or q.shape != p.shape or rowsum.shape != p.shape or rowsum.dtype != torch.float32:
        raise ValueError("q must match p; rowsum must be float32 of p's shape")
    if r is not None and (not isinstance(r, torch.Tensor) or r.dtype != p.dtype or r.shape != p.shape
                          or r.device != dev or not r.is_contiguous()):
        raise ValueError("r must be a contiguous tensor of p's dtype, shape and device")
    if sums is not None and (not isinstance(sums, torch.Tensor) or sums.dtype != torch.float64
                             or sums.numel() < 2 or sums.device != dev or not sums.is_contiguous()):
        raise ValueError("sums must be a contiguous float64 tensor of at least 2 elements on p's device")
    n = p.numel()
    if n > CORRECT_STATIC_MAX_N:
        raise ValueError(f"correct_static: n = {n} exceeds the static scratch limit {CORRECT_STATIC_MAX_N}")
    if dev.type != "cuda":
        raise ValueError("correct_static runs on a CUDA device only (there is no CPU fallback)")
    if r is None:
        r = torch.empty_like(p)
    if sums is None:
        sums = torch.empty(2, dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        rc = lib.ctrex_correct_static(_ptr(p), _ptr(q), _ptr(rowsum), _ptr(r), _dt(p), n, float(eps_R),
                                      _ptr(sums), ctypes.c_void_p(stream))
    if rc != OK:
        raise CtrexError(rc, f"ctrex_correct_static failed (n = {n})")
    return r, sums


_conv_status = {}


def _status(dev):
    st = _conv_status.get(dev)
    if st is None:
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        _conv_status[dev] = st
    return st


def conv_status_check(dev=None):
    """Raise if a tensor-core completion wait expired in an earlier conv call."""
    dev = torch.device("cuda", torch.cuda.current_device()) if dev is None else dev
    st = _status(dev)
    if int(st.item()) != 0:
        st.zero_()
        raise CtrexError(-5, "a tcgen05 completion wait expired in a conv kernel")


def conv3d(x, wt, bias=None, relu=False, out_dtype=torch.bfloat16):
    """3x3x3 'same' convolution on the tensor cores.  x bf16 [N, D, H, W, Cin]
    (channels last), wt bf16 [Cout, 27, Cin]; returns [N, D, H, W, Cout]."""
    lib = load_library()
    if x.dtype != torch.bfloat16 or wt.dtype != torch.bfloat16:
        raise TypeError("conv3d takes bfloat16 x and weights")
    if x.dim() != 5 or wt.dim() != 3 or wt.shape[1] != 27 or wt.shape[2] != x.shape[4]:
        raise ValueError(f"conv3d: x {tuple(x.shape)}, wt {tuple(wt.shape)}")
    x, wt = x.contiguous(), wt.contiguous()
    nb, d, h, w, cin = x.shape
    cout = wt.shape[0]
    y = torch.empty((nb, d, h, w, cout), dtype=out_dtype, device=x.device)
    if bias is not None:
        bias = bias.float().contiguous()
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):  # the library launches on the current device
        rc = lib.ctrex_conv3d_fwd(_ptr(x), _ptr(wt), _ptr(bias), _ptr(y), _dt(y), nb, d, h, w, cin, cout, int(relu),
                                  _ptr(_status(x.device)), ctypes.c_void_p(stream))
    if rc != OK:
        raise CtrexError(rc, f"ctrex_conv3d_fwd failed for x {tuple(x.shape)}, wt {tuple(wt.shape)}")
    return y


def conv3d_wgrad(x, dy, dw=None):
    """dw [Cout, 27, Cin] (float32, accumulated) of conv3d for input x and
    output gradient dy (both bf16, channels last)."""
    lib = load_library()
    x, dy = x.contiguous(), dy.contiguous()
    nb, d, h, w, cin = x.shape
    cout = dy.shape[4]
    if dw is None:
        dw = torch.zeros((cout, 27, cin), dtype=torch.float32, device=x.device)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):
        rc = lib.ctrex_conv3d_wgrad(_ptr(x), _ptr(dy), _ptr(dw), nb, d, h, w, cin, cout, _ptr(_status(x.device)),
                                    ctypes.c_void_p(stream))
    if rc != OK:
        raise CtrexError(rc, "ctrex_conv3d_wgrad failed")
    return dw


def flip_weights(wt):
    """wt [Cout, 27, Cin] -> the weights of the input-gradient convolution,
    [Cin, 27, Cout] with the taps reversed (a copy, no arithmetic)."""
    return wt.flip(1).transpose(0, 2).contiguous()


def probe_gather_rate(device=None):
    """Measured tex2Dgather calls per second (L1-resident texture)."""
    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = ctypes.c_double(0.0)
    with torch.cuda.device(dev):
        rc = lib.ctrex_probe_gather_rate(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream),
                                         ctypes.byref(out))
    if rc != OK:
        raise CtrexError(rc, "gather-rate probe failed")
    return out.value


def probe_l2_read_bandwidth(device=None):
    """Measured L2 read bandwidth in GB/s (16-byte L2-only loads over half
    of L2)."""
    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = ctypes.c_double(0.0)
    with torch.cuda.device(dev):
        rc = lib.ctrex_probe_l2_read_bandwidth(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream),
                                               ctypes.byref(out))
    if rc != OK:
        raise CtrexError(rc, "L2 read-bandwidth probe failed")
    return out.value


def context_for_cylinder(ccfg, P=None, device=None):
    """A Context on the cylindrical domain of an ``inputs.CylConfig``."""
    from . import inputs

    if P is None:
        P = inputs.projection_matrices(ccfg.base)
    ctx = Context(device)
    b = ccfg.base
    ctx.set_geometry_cylinder(P, ccfg.n_r, ccfg.n_phi, ccfg.n_z, ccfg.dr, ccfg.dz, (b.nu, b.nv),
                              pose=inputs.cylinder_pose(ccfg), step_vox=ccfg.step_vox)
    return ctx


def context_for(cfg, P=None, device=None):
    """A Context with the geometry of an ``inputs.Config`` already set."""
    from . import inputs

    if P is None:
        P = inputs.projection_matrices(cfg)
    ctx = Context(device)
    ctx.set_geometry(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)
    return ctx
