"""Seeded synthetic inputs: configurations, trajectories, phantoms, motion.

This module holds none of the reconstruction arithmetic.  It builds the
*inputs* that the CUDA path and the FP64 oracle both consume: per-view 3x4
projection matrices (the "Trajectory" of Sec. 2.1 / 2.2.2), volumes of
analytic objects, and motion parameters.  Random numbers come from
``numpy.random.Generator(PCG64(seed))``, drawn in the order documented in each
builder, so every input is reproducible from its seed.

Shared physical set-up (all configurations): source-object distance 200 mm,
source-detector distance 400 mm, a 32 mm cubic field of view centred at the
world origin (voxel = 32/N mm), a 96 mm wide detector (pitch = 96/nu mm, rows
with the same pitch), circular view v at angle 2*pi*v/V about z.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SOD = 200.0
SDD = 400.0
BOX = 32.0
DET_WIDTH = 96.0


@dataclasses.dataclass(frozen=True)
class Config:
    """One workload: volume edge n, detector nu x nv, views, sub-angles."""

    name: str
    n: int
    nu: int
    nv: int
    n_views: int
    n_sub: int = 1
    trajectory: str = "circular"      # circular | perturbed | helical | offset
    det_offset: float = 0.0           # offset: lateral detector shift (pixels), centre of rotation off-centre
    seed: int = 1
    helical_turns: float = 0.0
    z_span: float = 0.0               # helical: source z runs -z_span .. +z_span (mm)
    step_vox: float = 0.5
    n_ellipsoids: int = 10
    n_blobs: int = 0
    textured: bool = False
    motion: bool = False
    margin: float = 0.0               # mm, clip-box dilation with motion
    sirt_iters: int = 10
    box: float = BOX
    det_width: float = DET_WIDTH

    @property
    def vox(self) -> float:
        return self.box / self.n

    @property
    def pitch(self) -> float:
        return self.det_width / self.nu

    @property
    def origin(self) -> tuple:
        o = -0.5 * self.box + 0.5 * self.vox
        return (o, o, o)

    @property
    def vol_shape(self) -> tuple:
        return (self.n, self.n, self.n)

    def scaled(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


# Workloads (names describe them; sizes as stated).
CIRCULAR_64 = Config("circular-64^3-96^2-90v", n=64, nu=96, nv=96, n_views=90, seed=1,
                     sirt_iters=10)
PERTURBED_512 = Config("perturbed-512^3-768^2-720v", n=512, nu=768, nv=768, n_views=720,
                       trajectory="perturbed", seed=2, n_blobs=40, sirt_iters=50)
HELICAL_256 = Config("helical-256^3-512x384-1440v-S4", n=256, nu=512, nv=384, n_views=1440,
                     n_sub=4, trajectory="helical", seed=3, helical_turns=2.0, z_span=36.0)
MOTION_256 = Config("motion-256^3-384^2-360v", n=256, nu=384, nv=384, n_views=360, seed=4,
                    motion=True, margin=0.5)
MOTION_FD_32 = Config("motion-fd-32^3-48^2-24v", n=32, nu=48, nv=48, n_views=24, seed=4,
                      motion=True, margin=0.5)
SPARSE_128 = Config("sparse-128^3-192^2-60v", n=128, nu=192, nv=192, n_views=60, seed=0,
                    textured=True)

CONFIGS = {c.name: c for c in (CIRCULAR_64, PERTURBED_512, HELICAL_256, MOTION_256, MOTION_FD_32,
                               SPARSE_128)}


# ---------------------------------------------------------------------------
# Trajectories: per-view projection matrices (inputs to both sides)
# ---------------------------------------------------------------------------

def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def cone_matrix(src, det_centre, u_axis, v_axis, nu, nv) -> np.ndarray:
    """3x4 matrix mapping world mm to homogeneous pixel indices.

    Pixel (iu, iv) centre sits at d0 + iu*u_axis + iv*v_axis with
    d0 = det_centre - (nu-1)/2 u_axis - (nv-1)/2 v_axis; the matrix is
    Mc^{-1} [I | -src] with Mc = [u_axis | v_axis | d0 - src].
    """
    src = np.asarray(src, float)
    u_axis = np.asarray(u_axis, float)
    v_axis = np.asarray(v_axis, float)
    d0 = np.asarray(det_centre, float) - 0.5 * (nu - 1) * u_axis - 0.5 * (nv - 1) * v_axis
    Mc = np.stack([u_axis, v_axis, d0 - src], axis=1)
    Mi = np.linalg.inv(Mc)
    return np.concatenate([Mi, -(Mi @ src)[:, None]], axis=1)


def _circular_pose(angle: float, z: float, cfg: Config):
    R = rot_z(angle)
    src = R @ np.array([-SOD, 0.0, 0.0]) + np.array([0.0, 0.0, z])
    ctr = R @ np.array([SDD - SOD, 0.0, 0.0]) + np.array([0.0, 0.0, z])
    u = R @ np.array([0.0, cfg.pitch, 0.0])
    v = np.array([0.0, 0.0, cfg.pitch])
    return src, ctr, u, v


def detector_frames(cfg: Config):
    """Per (view, sub) source, detector centre, u axis, v axis: arrays [V, S, 3].

    circular:  angle 2*pi*v/V, z = 0.
    offset:    circular with the detector shifted by ``det_offset`` pixels along
               u (offset centre of rotation, extended field of view).
    perturbed: circular, then per view (draw order: du, dv in pixels U[-2, 2];
               tilt U[-0.5, 0.5] deg about the detector normal; source jitter
               3 x U[-0.2, 0.2] mm) the detector is offset by du*u + dv*v,
               its u/v axes are rotated in-plane by the tilt and the source is
               displaced.
    helical:   V views over ``helical_turns`` turns, angle a_v = 2*pi*turns*v/V,
               z = -z_span + p*a_v with p = 2*z_span / (2*pi*turns) (mm/rad);
               sub-angle s of view v at a_v + (s + 1/2 - S/2) * da / S with da
               the view increment, z interpolated the same way.
    The sub-angle rule is also used by circular trajectories with n_sub > 1.
    """
    V, S = cfg.n_views, cfg.n_sub
    srcs = np.zeros((V, S, 3))
    ctrs = np.zeros((V, S, 3))
    us = np.zeros((V, S, 3))
    vs = np.zeros((V, S, 3))
    if cfg.trajectory == "helical":
        total = 2.0 * math.pi * cfg.helical_turns
        da = total / V
        p = 2.0 * cfg.z_span / total
    else:
        da = 2.0 * math.pi / V
        p = 0.0
    rng = np.random.Generator(np.random.PCG64(cfg.seed)) if cfg.trajectory == "perturbed" else None
    for v in range(V):
        if rng is not None:
            du, dv = rng.uniform(-2.0, 2.0, size=2)
            tilt = math.radians(rng.uniform(-0.5, 0.5))
            jitter = rng.uniform(-0.2, 0.2, size=3)
        for s in range(S):
            a = v * da + (s + 0.5 - 0.5 * S) * da / S
            z = (-cfg.z_span + p * a) if cfg.trajectory == "helical" else 0.0
            src, ctr, u, w = _circular_pose(a, z, cfg)
            if cfg.trajectory == "offset":
                ctr = ctr + cfg.det_offset * u
            if rng is not None:
                n = np.cross(u, w)
                n /= np.linalg.norm(n)
                ctr = ctr + du * u + dv * w
                c, sn = math.cos(tilt), math.sin(tilt)
                u, w = c * u + sn * np.cross(n, u), c * w + sn * np.cross(n, w)
                src = src + jitter
            srcs[v, s], ctrs[v, s], us[v, s], vs[v, s] = src, ctr, u, w
    return srcs, ctrs, us, vs


def projection_matrices(cfg: Config) -> np.ndarray:
    """P [V, S, 3, 4] (float64) for the configuration's trajectory."""
    srcs, ctrs, us, vs = detector_frames(cfg)
    V, S = cfg.n_views, cfg.n_sub
    P = np.zeros((V, S, 3, 4))
    for v in range(V):
        for s in range(S):
            P[v, s] = cone_matrix(srcs[v, s], ctrs[v, s], us[v, s], vs[v, s], cfg.nu, cfg.nv)
    return P


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

def random_rotation(rng) -> np.ndarray:
    """Uniform rotation from a random unit quaternion (4 normal draws)."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclasses.dataclass
class Ellipsoid:
    centre: np.ndarray     # mm
    semi_axes: np.ndarray  # mm
    rot: np.ndarray        # columns = principal axes
    density: float
    texture: Optional[np.ndarray] = None  # [8, 4]: kx, ky, kz (1/mm), phase


@dataclasses.dataclass
class Blob:
    centre: np.ndarray
    sigma: float
    amplitude: float


def draw_objects(cfg: Config, seed: Optional[int] = None):
    """Ellipsoids then blobs, drawn from PCG64(seed or cfg.seed) in this order.

    Ellipsoid: full axes U[3, 20] mm (3 draws), rotation (4 normals), centre
    uniform in the box shrunk by the largest semi-axis (3 draws), density
    U[0.1, 1]; textured phantoms add 8 sinusoids (direction 3 normals,
    |k| U[0.2, 1] 1/mm, phase U[0, 2 pi]).  Blob: sigma U[0.3, 2] mm,
    amplitude U[0.05, 0.5], centre uniform in the box shrunk by 3 sigma.
    """
    rng = np.random.Generator(np.random.PCG64(cfg.seed if seed is None else seed))
    half = 0.5 * cfg.box
    ells = []
    for _ in range(cfg.n_ellipsoids):
        semi = 0.5 * rng.uniform(3.0, 20.0, size=3)
        rot = random_rotation(rng)
        r = float(semi.max())
        centre = rng.uniform(-half + r, half - r, size=3)
        dens = float(rng.uniform(0.1, 1.0))
        tex = None
        if cfg.textured:
            tex = np.zeros((8, 4))
            for k in range(8):
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
                tex[k, :3] = d * rng.uniform(0.2, 1.0)
                tex[k, 3] = rng.uniform(0.0, 2.0 * math.pi)
        ells.append(Ellipsoid(centre, semi, rot, dens, tex))
    blobs = []
    for _ in range(cfg.n_blobs):
        sigma = float(rng.uniform(0.3, 2.0))
        amp = float(rng.uniform(0.05, 0.5))
        centre = rng.uniform(-half + 3 * sigma, half - 3 * sigma, size=3)
        blobs.append(Blob(centre, sigma, amp))
    return ells, blobs


def _axis_coords(cfg: Config, sub: int, torch_mod, device):
    """Sub-sample coordinates along one axis: [n, sub] (mm)."""
    off = (torch_mod.arange(sub, dtype=torch_mod.float64, device=device) + 0.5) / sub - 0.5
    i = torch_mod.arange(cfg.n, dtype=torch_mod.float64, device=device)
    return cfg.origin[0] + (i[:, None] + off[None, :]) * cfg.vox


def voxelize(cfg: Config, ells, blobs, sub: int = 4, device: str = "cpu", dtype=None):
    """Volume [n, n, n] (z, y, x): mean of the object sum over sub^3 sub-samples.

    Overlapping objects add.  Ellipsoid indicator (times its density, times
    1 + 0.3 * mean of its sinusoids if textured) is evaluated on the sub-sample
    grid inside its bounding box; an isotropic Gaussian blob is separable, so
    its sub-sample mean is the product of three per-axis means.
    """
    import torch

    vol = torch.zeros(cfg.vol_shape, dtype=torch.float64, device=device)
    ax = _axis_coords(cfg, sub, torch, device)          # [n, sub]
    n = cfg.n
    for e in ells:
        r = float(e.semi_axes.max())
        lo = [max(0, int(math.floor((e.centre[a] - r - cfg.origin[0]) / cfg.vox)) - 1) for a in range(3)]
        hi = [min(n, int(math.ceil((e.centre[a] + r - cfg.origin[0]) / cfg.vox)) + 2) for a in range(3)]
        Q = torch.tensor((e.rot / e.semi_axes[None, :]).T, dtype=torch.float64, device=device)
        c = torch.tensor(e.centre, dtype=torch.float64, device=device)
        xs = ax[lo[0]:hi[0]] - c[0]
        ys = ax[lo[1]:hi[1]] - c[1]
        for z0 in range(lo[2], hi[2], 16):
            z1 = min(hi[2], z0 + 16)
            zs = ax[z0:z1] - c[2]
            # local coordinates: q = Q (x - c); broadcast [z, sz, y, sy, x, sx]
            Z = zs[:, :, None, None, None, None]
            Y = ys[None, None, :, :, None, None]
            X = xs[None, None, None, None, :, :]
            q2 = 0.0
            for row in range(3):
                qr = Q[row, 0] * X + Q[row, 1] * Y + Q[row, 2] * Z
                q2 = q2 + qr * qr
            inside = (q2 <= 1.0).to(torch.float64)
            if e.texture is not None:
                tex = 0.0
                for k in range(8):
                    kx, ky, kz, ph = (float(t) for t in e.texture[k])
                    tex = tex + torch.sin(kx * (X + c[0]) + ky * (Y + c[1]) + kz * (Z + c[2]) + ph)
                inside = inside * (1.0 + 0.3 * tex / 8.0)
            val = inside.mean(dim=(1, 3, 5)) * e.density
            vol[z0:z1, lo[1]:hi[1], lo[0]:hi[0]] += val
    for b in blobs:
        g = []
        for a in range(3):
            d = ax - float(b.centre[a])
            g.append(torch.exp(-0.5 * d * d / (b.sigma * b.sigma)).mean(dim=1))
        vol += b.amplitude * g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
    if dtype is not None:
        vol = vol.to(dtype)
    return vol


def phantom(cfg: Config, seed: Optional[int] = None, device: str = "cpu", sub: int = 4):
    """Voxelised phantom of the configuration (float64 torch tensor)."""
    ells, blobs = draw_objects(cfg, seed)
    return voxelize(cfg, ells, blobs, sub=sub, device=device)


# ---------------------------------------------------------------------------
# Event-based 4D scenes (Sec. 3.3): initial values, final values, transition
# times per voxel, for a scan during which regions change irreversibly
# ---------------------------------------------------------------------------

def view_times(cfg: Config) -> np.ndarray:
    """Acquisition time of each view: t_v = v / (V - 1), the scan running
    from 0 to 1."""
    return np.arange(cfg.n_views, dtype=np.float64) / max(cfg.n_views - 1, 1)


def dyrect_fields(cfg: Config, seed: Optional[int] = None, n_events: int = 8, device: str = "cpu", sub: int = 4):
    """(mu0, mu1, tau) of a scene in which n_events ellipsoidal regions change
    attenuation once during the scan (fluid invading a pore network, a phase
    transition): mu0 = the configuration's phantom; region k adds delta_k to
    it (voxelised like the phantom), and a planar front sweeps through the
    region, so a voxel changes when the front reaches its centre:
        tau = t0_k + dur_k ((x - c_k) . n_k + r_k) / (2 r_k),
    r_k the region's largest semi-axis.  Voxels outside every region get
    tau = 2 (after the scan); overlapping regions keep the earliest time.
    Draws from PCG64(seed or cfg.seed, offset 1000), per region in this
    order: full axes U[4, 16] mm (3), rotation (4 normals), centre in the
    box shrunk by r_k (3), delta_k U[-0.4, 0.6], front direction (3
    normals), start t0_k U[0.05, 0.6], duration dur_k U[0.2, 0.5].
    Returns float64 torch tensors [n, n, n] on device."""
    import torch

    mu0 = phantom(cfg, seed, device, sub)
    rng = np.random.Generator(np.random.PCG64((cfg.seed if seed is None else seed) + 1000))
    half = 0.5 * cfg.box
    mu1 = mu0.clone()
    tau = torch.full(cfg.vol_shape, 2.0, dtype=torch.float64, device=device)
    idx = torch.arange(cfg.n, dtype=torch.float64, device=device)
    xc = cfg.origin[0] + idx * cfg.vox
    for _ in range(n_events):
        semi = 0.5 * rng.uniform(4.0, 16.0, size=3)
        rot = random_rotation(rng)
        r = float(semi.max())
        centre = rng.uniform(-half + r, half - r, size=3)
        delta = float(rng.uniform(-0.4, 0.6))
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        t0 = float(rng.uniform(0.05, 0.6))
        dur = float(rng.uniform(0.2, 0.5))
        region = voxelize(cfg, [Ellipsoid(centre, semi, rot, delta)], [], sub=sub, device=device)
        mu1 += region
        front = t0 + dur * ((xc[None, None, :] - centre[0]) * nrm[0] + (xc[None, :, None] - centre[1]) * nrm[1]
                            + (xc[:, None, None] - centre[2]) * nrm[2] + r) / (2.0 * r)
        tau = torch.where(region != 0, torch.minimum(tau, front), tau)
    return mu0, mu1, tau


# ---------------------------------------------------------------------------
# Aligned cylindrical domain (Sec. 3.5): a vial on the scanner's trajectory
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class CylConfig:
    """A cylindrical reconstruction domain of N_r rings x N_phi sectors x N_z
    slices inside a bounding cylinder of the given radius and height, scanned
    on the trajectory (views, detector) of ``base``.  The cylinder axis is
    tilted by ``tilt_deg`` (about x, then y) against the rotation axis and
    its centre sits at ``shift`` (mm): the misalignment the domain's rigid
    pose absorbs."""

    name: str
    base: Config
    n_r: int
    n_phi: int
    n_z: int
    radius: float = 15.0
    height: float = 30.0
    tilt_deg: tuple = (0.8, -0.6)
    shift: tuple = (0.4, -0.3, 0.2)
    seed: int = 7
    n_inclusions: int = 12

    @property
    def dr(self) -> float:
        return self.radius / self.n_r

    @property
    def dz(self) -> float:
        return self.height / self.n_z

    @property
    def vol_shape(self) -> tuple:
        return (self.n_z, self.n_phi, self.n_r)

    @property
    def step_vox(self) -> float:
        return self.base.step_vox

    def scaled(self, **kw) -> "CylConfig":
        return dataclasses.replace(self, **kw)


CYL_SMALL = CylConfig("cylinder-24x64x32-64^2-60v",
                      CIRCULAR_64.scaled(name="perturbed-64^2-60v", nu=64, nv=64, n_views=60,
                                         trajectory="perturbed", seed=8),
                      n_r=24, n_phi=64, n_z=32)
CYL_VIAL = CylConfig("cylinder-256x1024x512-768^2-720v", PERTURBED_512, n_r=256, n_phi=1024, n_z=512)


def cylinder_pose(ccfg: CylConfig) -> np.ndarray:
    """3x4 rigid map q = Rc x + tc from world mm to the cylinder frame (axis =
    frame z): Rc = (Ry(b) Rx(a))^T for the tilt (a, b), and the frame origin
    at ``shift``."""
    a, b = (math.radians(t) for t in ccfg.tilt_deg)
    ca, sa, cb, sb = math.cos(a), math.sin(a), math.cos(b), math.sin(b)
    rx = np.array([[1.0, 0.0, 0.0], [0.0, ca, -sa], [0.0, sa, ca]])
    ry = np.array([[cb, 0.0, sb], [0.0, 1.0, 0.0], [-sb, 0.0, cb]])
    Rc = (ry @ rx).T
    tc = -Rc @ np.asarray(ccfg.shift, float)
    return np.hstack([Rc, tc[:, None]])


def cyl_phantom(ccfg: CylConfig, seed: Optional[int] = None, device: str = "cpu", sub: int = 2):
    """A vial phantom on the cylindrical grid [N_z, N_phi, N_r] (float64
    torch tensor), defined in the cylinder frame (radius R, height H):

    - glass wall 0.86 R <= r <= 0.94 R, -0.46 H <= z <= 0.40 H, and bottom
      r <= 0.94 R, -0.46 H <= z < -0.42 H: density 1;
    - frozen solution r < 0.86 R, -0.42 H <= z <= 0.15 H: density
      0.35 (1 + 0.15 sin(2 pi r / (R/6) + psi)) (concentric layers);
    - n_inclusions ellipsoids inside the solution (pores and crystals).

    Draw order from PCG64(seed or ccfg.seed): psi U[0, 2 pi]; per inclusion
    radius 0.75 R sqrt(U), angle U[0, 2 pi], z U[-0.38 H, 0.10 H], full axes
    3 x U[0.6, 3] mm, rotation (4 normals), density U[-0.25, 0.25].  Each
    voxel is the mean over sub^3 points spread evenly over its (r, phi, z)
    cell."""
    import torch

    rng = np.random.Generator(np.random.PCG64(ccfg.seed if seed is None else seed))
    R, H = ccfg.radius, ccfg.height
    psi = float(rng.uniform(0.0, 2.0 * math.pi))
    incl = []
    for _ in range(ccfg.n_inclusions):
        rc = 0.75 * R * math.sqrt(rng.uniform())
        ph = rng.uniform(0.0, 2.0 * math.pi)
        zc = rng.uniform(-0.38 * H, 0.10 * H)
        semi = 0.5 * rng.uniform(0.6, 3.0, size=3)
        rot = random_rotation(rng)
        dens = float(rng.uniform(-0.25, 0.25))
        incl.append((np.array([rc * math.cos(ph), rc * math.sin(ph), zc]), semi, rot, dens))
    f64 = dict(dtype=torch.float64, device=device)
    off = (torch.arange(sub, **f64) + 0.5) / sub - 0.5
    r = ((torch.arange(ccfg.n_r, **f64)[:, None] + 0.5 + off[None, :]) * ccfg.dr).reshape(-1)
    phi = ((torch.arange(ccfg.n_phi, **f64)[:, None] + 0.5 + off[None, :]) * (2 * math.pi / ccfg.n_phi)).reshape(-1)
    zall = ((torch.arange(ccfg.n_z, **f64)[:, None] - 0.5 * (ccfg.n_z - 1) + off[None, :]) * ccfg.dz)
    cphi, sphi = torch.cos(phi), torch.sin(phi)
    vol = torch.zeros(ccfg.vol_shape, **f64)
    chunk = 8
    for k0 in range(0, ccfg.n_z, chunk):
        k1 = min(ccfg.n_z, k0 + chunk)
        z = zall[k0:k1].reshape(-1)[:, None, None]        # [kz*sub, 1, 1]
        rr = r[None, None, :]                               # [1, 1, nr*sub]
        val = torch.zeros((z.shape[0], 1, rr.shape[2]), **f64)
        wall = (rr >= 0.86 * R) & (rr <= 0.94 * R) & (z >= -0.46 * H) & (z <= 0.40 * H)
        bottom = (rr <= 0.94 * R) & (z >= -0.46 * H) & (z < -0.42 * H)
        sol = (rr < 0.86 * R) & (z >= -0.42 * H) & (z <= 0.15 * H)
        layers = 0.35 * (1.0 + 0.15 * torch.sin(2 * math.pi * rr / (R / 6.0) + psi))
        val = val + (wall | bottom).to(torch.float64) + sol.to(torch.float64) * layers
        val = val.expand(-1, phi.shape[0], -1).clone()     # [kz*sub, nphi*sub, nr*sub]
        zlo, zhi = float(z.min()), float(z.max())
        for c, semi, rot, dens in incl:
            rmax = float(semi.max())
            if c[2] + rmax < zlo or c[2] - rmax > zhi:
                continue
            Q = torch.tensor((rot / semi[None, :]).T, **f64)
            X = rr * cphi[None, :, None] - float(c[0])
            Y = rr * sphi[None, :, None] - float(c[1])
            Z = z - float(c[2])
            q2 = 0.0
            for row in range(3):
                qr = Q[row, 0] * X + Q[row, 1] * Y + Q[row, 2] * Z
                q2 = q2 + qr * qr
            val += dens * (q2 <= 1.0).to(torch.float64)
        nz = k1 - k0
        vol[k0:k1] = val.view(nz, sub, ccfg.n_phi, sub, ccfg.n_r, sub).mean(dim=(1, 3, 5))
    return vol


# ---------------------------------------------------------------------------
# Multi-resolution ROI (Sec. 3.7): a coarse context grid and a fine ROI cube
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class RoiConfig:
    """A context grid (``base``: its n, box and trajectory) and a cubic ROI
    grid of roi_n voxels over a roi_box mm cube centred at roi_centre."""

    name: str
    base: Config
    roi_n: int
    roi_box: float
    roi_centre: tuple = (0.0, 0.0, 0.0)

    @property
    def roi_vox(self) -> float:
        return self.roi_box / self.roi_n

    @property
    def roi_origin(self) -> tuple:
        return tuple(c - 0.5 * self.roi_box + 0.5 * self.roi_vox for c in self.roi_centre)

    @property
    def roi_shape(self) -> tuple:
        return (self.roi_n,) * 3


# context 256^3 over the 32 mm field of view (0.125 mm) and an ROI of 256^3
# over the central 8 mm (0.03125 mm, 4 times finer), on the 720-view
# trajectory of the 512^3 workload
ROI_FOCUS = RoiConfig("roi-256^3+256^3x4-768^2-720v", PERTURBED_512.scaled(n=256), roi_n=256, roi_box=8.0,
                      roi_centre=(0.6, -0.4, 0.3))


def roi_phantom(rcfg: RoiConfig, seed: Optional[int] = None, device: str = "cpu", sub: int = 2):
    """(context volume, ROI volume): the objects of ``draw_objects(base)``
    voxelised on both grids (sub^3 sub-samples per voxel), so the two
    resolutions describe the same object."""
    ells, blobs = draw_objects(rcfg.base, seed)
    ctx = voxelize(rcfg.base, ells, blobs, sub=sub, device=device)
    # the ROI grid as a cubic Config centred at the origin, objects shifted by -roi_centre
    sh = np.asarray(rcfg.roi_centre, float)
    ells_r = [Ellipsoid(e.centre - sh, e.semi_axes, e.rot, e.density, e.texture) for e in ells]
    blobs_r = [Blob(b.centre - sh, b.sigma, b.amplitude) for b in blobs]
    roi_grid = rcfg.base.scaled(n=rcfg.roi_n, box=rcfg.roi_box)
    roi = voxelize(roi_grid, ells_r, blobs_r, sub=sub, device=device)
    return ctx, roi


# ---------------------------------------------------------------------------
# Motion parameters
# ---------------------------------------------------------------------------

def motion_params(cfg: Config, seed: Optional[int] = None):
    """theta [V, 15] = (omega, t, A row-major), coef [8, 8, 8, 3], s_view [V].

    Draw order from PCG64(seed or cfg.seed + 1000): per view omega 3 x U[-1, 1]
    deg, t 3 x U[-0.5, 0.5] mm, A = I + 9 x U[-0.01, 0.01]; then coefficients
    8*8*8*3 x U[-1, 1], rescaled so that the largest control-point vector has
    length 3 voxels (a B-spline is a convex combination of its coefficients, so
    the displacement never exceeds that).  s_v = v / (V - 1).
    """
    rng = np.random.Generator(np.random.PCG64((cfg.seed if seed is None else seed) + 1000))
    V = cfg.n_views
    theta = np.zeros((V, 15))
    for v in range(V):
        theta[v, 0:3] = np.radians(rng.uniform(-1.0, 1.0, size=3))
        theta[v, 3:6] = rng.uniform(-0.5, 0.5, size=3)
        theta[v, 6:15] = (np.eye(3) + rng.uniform(-0.01, 0.01, size=(3, 3))).reshape(9)
    coef = rng.uniform(-1.0, 1.0, size=(8, 8, 8, 3))
    coef *= 3.0 * cfg.vox / np.linalg.norm(coef, axis=-1).max()
    s_view = np.arange(V, dtype=np.float64) / max(V - 1, 1)
    return theta, coef, s_view


def identity_theta(n_views: int) -> np.ndarray:
    th = np.zeros((n_views, 15))
    th[:, 6:15] = np.eye(3).reshape(9)
    return th


# ---------------------------------------------------------------------------
# Ordered-subset schedules (the index sets P_k of Sec. 2.3.2)
# ---------------------------------------------------------------------------

def _bit_reversal_order(n):
    bits = max(1, (n - 1).bit_length())
    order = sorted(range(n), key=lambda i: int(format(i, f"0{bits}b")[::-1], 2))
    return order


def subsets_cyclic(n_views, n_subsets, spread=True):
    """Interleaved subsets {s, s + n, s + 2n, ...}; with ``spread`` they are
    visited in bit-reversed order so consecutive subsets are far apart in
    angle (a geometry-dependent ordering).  Every view appears exactly once."""
    sets = [list(range(s, n_views, n_subsets)) for s in range(n_subsets)]
    if spread:
        sets = [sets[i] for i in _bit_reversal_order(n_subsets)]
    return [s for s in sets if s]


def subsets_random(n_views, n_subsets, seed):
    """A seeded random permutation of the views cut into n_subsets
    near-equal contiguous pieces."""
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n_views)
    return [list(map(int, c)) for c in np.array_split(perm, n_subsets) if len(c)]


def efov_windows(cfg, u_cor, seed):
    """Per-view backprojection windows [V, 4] = (u_lo, u_hi, v_lo, v_hi) for an
    offset-centre-of-rotation scan whose rotation axis projects at column
    ``u_cor``: the inner detector edge is moved, per view, to a column drawn
    uniformly from [0, u_cor] (between the physical edge and the projected
    centre of rotation); PCG64(seed), one draw per view."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = rng.integers(0, int(u_cor) + 1, size=cfg.n_views)
    win = np.zeros((cfg.n_views, 4), dtype=np.int32)
    win[:, 0] = lo
    win[:, 1] = cfg.nu - 1
    win[:, 2] = 0
    win[:, 3] = cfg.nv - 1
    return win
