"""FP64 CPU oracle for the CTrex projection / correction / backprojection path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
never does.  The arithmetic lives in ``ctrex_oracle.c`` (plain C, FP64,
OpenMP), which shares no code with the CUDA path; this module only marshals
numpy arrays through ctypes and builds the shared object on first use.

Each wrapper names the paper passage its C routine follows:

* ``forward``/``forward_rays``  -- Sec. 4.1 projection operator (A), Sec. 3.4
  angular sub-projections, Sec. 3.1 / 4.2.1 warped sampling.
* ``correct``                   -- Sec. 4.1 correction kernel, Eq. (1) term 2.
* ``backproject``               -- Sec. 4.1 backprojection operator with C and
  alpha, Eq. (1) term 3; Sec. 3.2 / 4.3.2 voxel weights.
* ``adjoint``, ``motion_grad``  -- transpose and chain rule of ``forward``
  (Sec. 5 motivates geometry refinement; no formula is printed).
* ``displacement``              -- the Sec. 3.1 deformation field on its own.
* ``Problem(dyrect=...)``       -- Sec. 3.3 event-based 4D model (initial and
  final values, transition times) in the projector, backprojector, adjoint
  and SIRT.
* ``sirt``                      -- Eq. (1) iterated, all views in one subset.
* ``os_sirt``                   -- Eq. (1) on ordered subsets of views (Sec. 2.3.2).

Parity status: every routine is pinned by ``tests/test_oracle_pins.py``
(closed forms, analytic phantoms, adjointness, invariances, brute force and
finite differences); none is "parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import platform
import struct
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctrex_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EPS_C = 1e-6


def _native(path):
    machine = {"x86_64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine())
    try:
        with open(path, "rb") as f:
            head = f.read(20)
        return head[:4] == b"\x7fELF" and struct.unpack("<H", head[18:20])[0] == machine
    except OSError:
        return False


def build(force: bool = False) -> str:
    """Compile ctrex_oracle.c into liboracle.so (gcc, OpenMP, IEEE FP64)."""
    if (force or not os.path.exists(_LIB) or not _native(_LIB)
            or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


class _CProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("vox", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("n_views", ctypes.c_int), ("n_sub", ctypes.c_int),
        ("step_vox", ctypes.c_double),
        ("P", _dp), ("theta", _dp), ("coef", _dp), ("s_view", _dp),
        ("margin", ctypes.c_double), ("bp_window", _ip), ("bp_subvoxel", ctypes.c_int),
        ("cyl", ctypes.c_int), ("cyl_dr", ctypes.c_double), ("cyl_dz", ctypes.c_double),
        ("cyl_pose", _dp), ("joseph", ctypes.c_int),
        ("roi", ctypes.c_int), ("roi_n", ctypes.c_int * 3), ("roi_vox", ctypes.c_double * 3),
        ("roi_origin", ctypes.c_double * 3), ("dyr_tau", _dp), ("dyr_t", _dp),
    ]


def _declare(lib):
    pp = ctypes.POINTER(_CProblem)
    lib.or_setup_views.argtypes = [pp, _dp, _dp, _dp]
    lib.or_forward.argtypes = [pp, _dp, _ip, ctypes.c_int, _dp, _dp]
    lib.or_forward_rays.argtypes = [pp, _dp, _ip, _dp, _dp, ctypes.c_long, _dp, _dp]
    lib.or_count_samples.argtypes = [pp, _ip, ctypes.c_int]
    lib.or_count_samples.restype = ctypes.c_long
    lib.or_correct.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, _dp, _dp]
    lib.or_backproject.argtypes = [pp, _dp, _ip, ctypes.c_int, _dp, ctypes.c_double,
                                   ctypes.c_double, _dp, _dp, _dp]
    lib.or_backproject_voxels.argtypes = [pp, _dp, _ip, ctypes.c_int, _lp, ctypes.c_long, _dp, _dp]
    lib.or_adjoint.argtypes = [pp, _dp, _ip, ctypes.c_int, _dp]
    lib.or_motion_grad.argtypes = [pp, _dp, _dp, _ip, ctypes.c_int, _dp, _dp]
    lib.or_displacement.argtypes = [pp, ctypes.c_long, _dp, _dp, _dp]
    lib.or_sirt.argtypes = [pp, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, _dp, _ip]
    lib.or_os_sirt.argtypes = [pp, _dp, _dp, _ip, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _ip]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, typ=_dp):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


class Problem:
    """Geometry (and optional motion) of one projection problem, FP64.

    P: [n_views, n_sub, 3, 4]; vol_shape (nz, ny, nx); vox, origin in (x, y, z)
    order, mm; det (nu, nv); theta [n_views, 15]; coef [8, 8, 8, 3]; s_view
    [n_views].  cyl = (dr, dz, pose[3, 4]) switches to the aligned cylindrical
    domain (reading R13): vol_shape is then (N_z, N_phi, N_r) and vox, origin
    are unused.  dyrect = (tau [nz, ny, nx], t_view [n_views]) switches on the
    event-based 4D model (Sec. 3.3, reading R16): volumes are then
    [2, nz, ny, nx], the initial values followed by the final values.
    """

    def __init__(self, P, vol_shape, vox, origin, det, step_vox=0.5, theta=None, coef=None,
                 s_view=None, margin=0.0, bp_window=None, bp_subvoxel=1, cyl=None, joseph=False, roi=None,
                 dyrect=None):
        P = _f64(P)
        if P.ndim == 3:
            P = P[:, None]
        self.P = P
        self.n_views, self.n_sub = P.shape[0], P.shape[1]
        self.nz, self.ny, self.nx = (int(s) for s in vol_shape)
        self.vox = tuple(float(v) for v in vox)
        self.origin = tuple(float(v) for v in origin)
        self.nu, self.nv = (int(d) for d in det)
        self.step_vox = float(step_vox)
        self.theta = None if theta is None else _f64(theta)
        self.coef = None if coef is None else _f64(coef)
        self.s_view = None if s_view is None else _f64(s_view)
        self.margin = float(margin)
        self.bp_window = None if bp_window is None else np.ascontiguousarray(bp_window, dtype=np.int32)
        self.bp_subvoxel = int(bp_subvoxel)
        self.joseph = bool(joseph)
        self.roi = None
        if roi is not None:  # (roi_shape (nz, ny, nx), vox (x, y, z), origin (x, y, z))
            rshape, rvox, rorg = roi
            self.roi = (tuple(int(v) for v in rshape), tuple(float(v) for v in rvox),
                        tuple(float(v) for v in rorg))
        self.dyrect = None
        if dyrect is not None:
            tau, tv = dyrect
            tau, tv = _f64(tau), _f64(tv)
            assert tau.shape == (self.nz, self.ny, self.nx) and tv.shape == (self.n_views,)
            self.dyrect = (tau, tv)
        self.cyl = None
        if cyl is not None:
            dr, dz, pose = cyl
            self.cyl = (float(dr), float(dz), _f64(pose).reshape(3, 4).copy())
        cdr, cdz, cpose = self.cyl if self.cyl else (0.0, 0.0, None)
        self._c = _CProblem(self.nx, self.ny, self.nz, (ctypes.c_double * 3)(*self.vox),
                            (ctypes.c_double * 3)(*self.origin), self.nu, self.nv, self.n_views,
                            self.n_sub, self.step_vox, _ptr(self.P), _ptr(self.theta),
                            _ptr(self.coef), _ptr(self.s_view), self.margin, _ptr(self.bp_window, _ip),
                            self.bp_subvoxel, 1 if self.cyl else 0, cdr, cdz, _ptr(cpose),
                            1 if self.joseph else 0, 1 if self.roi else 0,
                            (ctypes.c_int * 3)(*(self.roi[0][::-1] if self.roi else (0, 0, 0))),
                            (ctypes.c_double * 3)(*(self.roi[1] if self.roi else (0.0, 0.0, 0.0))),
                            (ctypes.c_double * 3)(*(self.roi[2] if self.roi else (0.0, 0.0, 0.0))),
                            _ptr(self.dyrect[0] if self.dyrect else None),
                            _ptr(self.dyrect[1] if self.dyrect else None))

    @property
    def grid_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def vol_shape(self):
        """Shape of a volume argument: the grid, or with an ROI the flat
        concatenation of the context grid's and the ROI grid's voxels."""
        if self.roi:
            rz, ry, rx = self.roi[0]
            return (self.nz * self.ny * self.nx + rz * ry * rx,)
        if self.dyrect:
            return (2, self.nz, self.ny, self.nx)
        return (self.nz, self.ny, self.nx)

    @property
    def min_vox(self):
        if self.cyl:
            return min(self.cyl[0], self.cyl[1])
        return min(self.vox)

    @property
    def eps_R(self):
        return 1e-6 * self.min_vox

    def _replace(self, **kw):
        args = dict(P=self.P, vol_shape=self.grid_shape, vox=self.vox, origin=self.origin,
                    det=(self.nu, self.nv), step_vox=self.step_vox, theta=self.theta, coef=self.coef,
                    s_view=self.s_view, margin=self.margin, bp_window=self.bp_window,
                    bp_subvoxel=self.bp_subvoxel, cyl=self.cyl, joseph=self.joseph, roi=self.roi,
                    dyrect=self.dyrect)
        args.update(kw)
        return Problem(**args)

    def with_motion(self, theta=None, coef=None, s_view=None, margin=0.0):
        return self._replace(theta=theta, coef=coef, s_view=s_view, margin=margin)

    def with_P(self, P):
        return self._replace(P=P)

    def with_subvoxel(self, s):
        """The same problem whose backprojector averages s^3 sub-voxel points."""
        return self._replace(bp_subvoxel=s)

    def with_roi(self, roi_shape, roi_vox, roi_origin):
        """The same problem with a finer ROI grid (reading R15): roi_shape
        (nz, ny, nx), roi_vox and roi_origin (x, y, z) mm."""
        return self._replace(roi=(roi_shape, roi_vox, roi_origin))

    def with_joseph(self, on=True):
        """The same problem with the classical Joseph projector (reading R14)."""
        return self._replace(joseph=on)

    def with_dyrect(self, tau, t_view):
        """The same problem with the event-based 4D model (reading R16)."""
        return self._replace(dyrect=(tau, t_view))

    def with_window(self, bp_window):
        """The same problem whose backprojector sees per-view detector windows
        [n_views, 4] = (u_lo, u_hi, v_lo, v_hi) (extended field of view)."""
        return self._replace(bp_window=bp_window)


def cylinder_problem(P, n_r, n_phi, n_z, dr, dz, det, pose=None, step_vox=0.5):
    """A problem on the aligned cylindrical domain: N_r rings of pitch dr,
    N_phi sectors, N_z slices of pitch dz (mm); pose [3, 4] maps world mm to
    the cylinder frame (identity if None)."""
    if pose is None:
        pose = np.hstack([np.eye(3), np.zeros((3, 1))])
    return Problem(P, (n_z, n_phi, n_r), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), det, step_vox,
                   cyl=(dr, dz, pose))


def _views(pb, views):
    if views is None:
        return None, pb.n_views
    v = np.ascontiguousarray(views, dtype=np.int32)
    return v, len(v)


def _check(ret):
    if ret != 0:
        raise ValueError(f"oracle error {ret}")


def setup_views(pb):
    lib = _load()
    n = pb.n_views * pb.n_sub
    Pn, src, Minv = np.zeros((n, 12)), np.zeros((n, 3)), np.zeros((n, 9))
    _check(lib.or_setup_views(ctypes.byref(pb._c), _ptr(Pn), _ptr(src), _ptr(Minv)))
    return Pn.reshape(pb.n_views, pb.n_sub, 3, 4), src.reshape(pb.n_views, pb.n_sub, 3), \
        Minv.reshape(pb.n_views, pb.n_sub, 3, 3)


def forward(pb, vol, views=None):
    """(A x, A 1) for the listed views: two arrays [n_sel, nv, nu]."""
    lib = _load()
    vol = _f64(vol)
    assert vol.shape == pb.vol_shape
    v, n = _views(pb, views)
    proj = np.zeros((n, pb.nv, pb.nu))
    rs = np.zeros((n, pb.nv, pb.nu))
    _check(lib.or_forward(ctypes.byref(pb._c), _ptr(vol), _ptr(v, _ip), n, _ptr(proj), _ptr(rs)))
    return proj, rs


def forward_rays(pb, vol, view, u, v):
    """Ray integrals at arbitrary detector points (view[i], u[i], v[i])."""
    lib = _load()
    vol = _f64(vol)
    view = np.ascontiguousarray(view, dtype=np.int32)
    u, v = _f64(u), _f64(v)
    n = len(view)
    val, rs = np.zeros(n), np.zeros(n)
    _check(lib.or_forward_rays(ctypes.byref(pb._c), _ptr(vol), _ptr(view, _ip), _ptr(u), _ptr(v), n,
                               _ptr(val), _ptr(rs)))
    return val, rs


def count_samples(pb, views=None):
    lib = _load()
    v, n = _views(pb, views)
    c = int(lib.or_count_samples(ctypes.byref(pb._c), _ptr(v, _ip), n))
    if c < 0:
        raise ValueError(f"oracle error {c}")
    return c


def correct(p, q, rowsum, eps_R):
    """(r, sum (p-q)^2, sum p^2) of Eq. (1) term 2."""
    lib = _load()
    p, q, rowsum = _f64(p), _f64(q), _f64(rowsum)
    r = np.zeros_like(p)
    sums = np.zeros(2)
    _check(lib.or_correct(p.size, _ptr(p), _ptr(q), _ptr(rowsum), eps_R, _ptr(r), _ptr(sums)))
    return r, sums[0], sums[1]


def backproject(pb, r, views=None, w=None, alpha=1.0, x=None, eps_C=EPS_C):
    """(x_new, b, c): Eq. (1) term 3 on x (zeros if None) from r [n_sel, nv, nu]."""
    lib = _load()
    r = _f64(r)
    v, n = _views(pb, views)
    assert r.shape == (n, pb.nv, pb.nu)
    x = np.zeros(pb.vol_shape) if x is None else _f64(x).copy()
    w = None if w is None else _f64(w)
    b = np.zeros(pb.vol_shape)
    c = np.zeros(pb.vol_shape)
    _check(lib.or_backproject(ctypes.byref(pb._c), _ptr(r), _ptr(v, _ip), n, _ptr(w), alpha, eps_C,
                              _ptr(x), _ptr(b), _ptr(c)))
    return x, b, c


def backproject_voxels(pb, r, vox_flat, views=None):
    """(b, c) at the listed flat voxel indices (with the event-based model:
    arrays [2, n], the initial-value parts then the final-value parts)."""
    lib = _load()
    r = _f64(r)
    v, n = _views(pb, views)
    vox_flat = np.ascontiguousarray(vox_flat, dtype=np.int64)
    shape = (2, len(vox_flat)) if pb.dyrect else (len(vox_flat),)
    b = np.zeros(shape)
    c = np.zeros(shape)
    _check(lib.or_backproject_voxels(ctypes.byref(pb._c), _ptr(r), _ptr(v, _ip), n,
                                     _ptr(vox_flat, _lp), len(vox_flat), _ptr(b), _ptr(c)))
    return b, c


def adjoint(pb, y, views=None):
    """A^T y for y [n_sel, nv, nu] (matched transpose of ``forward``)."""
    lib = _load()
    y = _f64(y)
    v, n = _views(pb, views)
    out = np.zeros(pb.vol_shape)
    _check(lib.or_adjoint(ctypes.byref(pb._c), _ptr(y), _ptr(v, _ip), n, _ptr(out)))
    return out


def motion_grad(pb, vol, g, views=None):
    """(dL/dtheta [n_views, 15], dL/dcoef [8, 8, 8, 3]) for L = <g, A x>."""
    lib = _load()
    vol, g = _f64(vol), _f64(g)
    v, n = _views(pb, views)
    gt = np.zeros((pb.n_views, 15))
    gc = np.zeros((8, 8, 8, 3))
    _check(lib.or_motion_grad(ctypes.byref(pb._c), _ptr(vol), _ptr(g), _ptr(v, _ip), n, _ptr(gt),
                              _ptr(gc)))
    return gt, gc


def displacement(pb, pts):
    """(u [n, 3], du/dx' [n, 3, 3]) of the B-spline deformation (Sec. 3.1,
    reading R6) at world points pts [n, 3] (mm), from ``pb.coef``."""
    lib = _load()
    pts = _f64(pts).reshape(-1, 3)
    u = np.zeros_like(pts)
    J = np.zeros((len(pts), 3, 3))
    _check(lib.or_displacement(ctypes.byref(pb._c), len(pts), _ptr(pts), _ptr(u), _ptr(J)))
    return u, J


def sirt(pb, p, max_iter, alpha=1.0, w=None, tol=0.0, x0=None, eps_C=EPS_C):
    """(x, residual history, iterations done) of Eq. (1) with all views."""
    lib = _load()
    p = _f64(p)
    x = np.zeros(pb.vol_shape) if x0 is None else _f64(x0).copy()
    w = None if w is None else _f64(w)
    hist = np.full(max_iter, np.nan)
    done = ctypes.c_int(0)
    ret = lib.or_sirt(ctypes.byref(pb._c), _ptr(x), _ptr(p), max_iter, alpha, _ptr(w), tol, pb.eps_R,
                      eps_C, _ptr(hist), ctypes.byref(done))
    if ret < 0:
        raise ValueError(f"oracle error {ret}")
    return x, hist, done.value, ret


def os_sirt(pb, p, subsets, max_cycles, alpha=1.0, w=None, tol=0.0, x0=None, eps_C=EPS_C):
    """(x, residual history per cycle, cycles done, status) of ordered-subset
    SIRT over the list of view lists ``subsets``."""
    lib = _load()
    p = _f64(p)
    x = np.zeros(pb.vol_shape) if x0 is None else _f64(x0).copy()
    w = None if w is None else _f64(w)
    views = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in subsets]), dtype=np.int32)
    offsets = np.ascontiguousarray(np.cumsum([0] + [len(s) for s in subsets]), dtype=np.int32)
    hist = np.full(max_cycles, np.nan)
    done = ctypes.c_int(0)
    ret = lib.or_os_sirt(ctypes.byref(pb._c), _ptr(x), _ptr(p), _ptr(views, _ip), _ptr(offsets, _ip), len(subsets),
                         max_cycles, alpha, _ptr(w), tol, pb.eps_R, eps_C, _ptr(hist), ctypes.byref(done))
    if ret < 0:
        raise ValueError(f"oracle error {ret}")
    return x, hist, done.value, ret
