"""Seeded synthetic scenes: density grids, source sets and optical layouts.

This module only *generates inputs*.  It holds none of the image generator's
arithmetic (no ray generation, integration, refraction or deposit), so both the
CUDA library and the CPU oracle can consume its output without sharing code.

The paper's own experiment uses DNS density data (Sec. 4) that is not
available; the fields below stand in for it:

* ``c0``  BOS linear-gradient slab: 32^3 grid over 50x50x10 mm, rho rising
  linearly 1.20 -> 1.26 kg/m^3 along y, K = 0.225e-3 m^3/kg; 64x64 dot grid
  0.5 m before the volume mid-plane, 100 rays per dot, Euler step 0.1 mm; ideal
  thin lens f = 105 mm, f/8, M = 0.1; 256x256 sensor, 17 um pitch.
* ``c1``  PIV uniform medium (n = 1.000277): 1e4 particles uniform in a
  50x50x1 mm sheet, 1e4 rays each; thick biconvex lens (R = +-0.1 m, 10 mm,
  n = 1.5), f/4, M = 0.2; the sheet centred 2 mm before and 2 mm behind the
  plane of focus (two frames); 1024x1024 sensor, 17 um pitch.
* ``c2``  BOS turbulence-like field: 256^3 grid over a 0.1 m cube, Gaussian
  random field with a k^-5/3 energy spectrum, mean 1.2 kg/m^3, 5 % rms; 1e5
  random dots, 1e3 rays each; RK4 step 0.2 mm; the thick lens at f/8, M = 0.1
  focused on the dot plane; 1024x1024 sensor.
* ``c3``  64 frames of uneven size mixing shock slabs, linear gradients and
  turbulence fields (grids 64^3-256^3, 1e3-1e5 sources, 1e3-1e4 rays/source).
* ``c4``  Tomo-PIV scale: 1e5 particles inside a 100x100x30 mm turbulence
  field (256^3), 1e4 rays each, thick lens f/4 M = 0.2 focused on the volume
  centre, 2048x2048 sensor.
* ``table1``  the simulated BOS experiment of Sec. 4 with the geometry of
  Table 1: a 2-D Gaussian random density slice with a k^-5/3 inertial range
  and a dissipation cutoff at 8 cycles per box (the paper's DNS slice is
  resolved into its dissipation range), 256^2 nodes over 32x32 mm, mean
  1.225 kg/m^3, 5 % rms, stacked along z over 10 mm (the paper stacks its
  slice the same way), K = 0.226e-3 m^3/kg; dots 0.25 m (Z_D) before the
  volume mid-plane, the lens 0.75 m (Z_A) after it, f = 105 mm, f/11 (M =
  f / (Z_A + Z_D - f) = 0.117, printed as 0.12); 512x512 sensor of 10 um
  pixels with 20 random dots per 32x32 pixels (5,120 dots), 1e4 rays each;
  RK4 step 0.1 mm.

Every generator takes a ``scale`` that shrinks ray and source counts (and the
grid, where stated) for tests, keeping geometry, spacing and distributions.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SPHERE, PLANE, IDEAL_THIN, STOP, MIRROR, LENS_ARRAY = 0, 1, 2, 3, 4, 5
EULER, RK4 = 0, 1

K_AIR = 0.225e-3          # m^3/kg, the Gladstone-Dale constant the workloads use
RHO_AIR = 1.2             # kg/m^3
LAMBDA_GREEN = 532e-9     # m, effective wavelength for white light (Sec. 3.4)


@dataclasses.dataclass
class Surface:
    type: int
    z: float
    R: float = 0.0          # signed radius (spheres, mirrors); lenslet pitch (lens arrays)
    f: float = 0.0
    n_after: float = 1.0
    clear_r: float = 1.0

    def as_row(self):
        return [float(self.type), self.z, self.R, self.f, self.n_after, self.clear_r]


@dataclasses.dataclass
class Mie:
    """Mie radiance of the rays of PIV particles (Sec. 3.1): sphere diameter,
    laser wavelength (vacuum), index of the medium, the particle's index
    relative to it, laser direction and polarisation (None = unpolarised),
    and the angle table size."""
    diameter: float = 1e-6
    wavelength: float = 532e-9
    n_medium: float = 1.000277
    m_re: float = 1.45 / 1.000277
    m_im: float = 0.0
    laser_dir: tuple = (1.0, 0.0, 0.0)
    polarisation: Optional[tuple] = (0.0, 1.0, 0.0)
    n_angles: int = 1801


@dataclasses.dataclass
class Optics:
    surfaces: List[Surface]
    n_object: float
    aim_z: float
    aim_r: float
    sensor_z: float
    pitch: float
    width: int
    height: int
    f_number: float
    magnification: float
    wavelength: float = LAMBDA_GREEN
    dtau_rule: int = 0     # 0: Eq. 8 as printed (2.44 pi ...), 1: textbook 2.44
    sensor_tilt_x: float = 0.0   # radians about x, then
    sensor_tilt_y: float = 0.0   # radians about y (the sensor turns about its centre)
    mie: Optional["Mie"] = None  # Mie radiance of the rays (None: every ray weighs 1)

    def surface_array(self) -> np.ndarray:
        return np.array([s.as_row() for s in self.surfaces], dtype=np.float64).reshape(-1, 6)


@dataclasses.dataclass
class Medium:
    rho: np.ndarray          # float32 [nz, ny, nx], kg/m^3
    origin: tuple            # metres, node (0,0,0)
    spacing: tuple           # metres between nodes
    K: float = K_AIR

    @property
    def dims(self):
        nz, ny, nx = self.rho.shape
        return nx, ny, nz

    def extent(self):
        nx, ny, nz = self.dims
        return tuple(o + (n - 1) * h for o, n, h in zip(self.origin, (nx, ny, nz), self.spacing))


@dataclasses.dataclass
class Frame:
    """One image: a medium (or None for a uniform ambient), sources, rays."""
    medium: Optional[Medium]
    optics: Optics
    sources: np.ndarray      # float64 [S, 3]
    rays_per_source: int
    seed: int
    integrator: int
    step: float
    frame_index: int = 0

    @property
    def n_rays(self) -> int:
        return int(self.sources.shape[0]) * int(self.rays_per_source)


# --------------------------------------------------------------------------
# density fields
# --------------------------------------------------------------------------
def linear_gradient_rho(nx, ny, nz, rho0=1.20, rho1=1.26, axis=1) -> np.ndarray:
    """rho rising linearly from rho0 at the first node to rho1 at the last
    node along ``axis`` (0 = x, 1 = y, 2 = z)."""
    n = (nx, ny, nz)[axis]
    ramp = rho0 + (rho1 - rho0) * np.arange(n, dtype=np.float64) / (n - 1)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    rho = np.broadcast_to(ramp.reshape(shape), (nz, ny, nx))
    return np.ascontiguousarray(rho, dtype=np.float32)


def uniform_rho(nx, ny, nz, rho=1.2311) -> np.ndarray:
    return np.full((nz, ny, nx), rho, dtype=np.float32)


def turbulence_rho(n, seed, mean=1.2, rms_frac=0.05, shape=None) -> np.ndarray:
    """Periodic Gaussian random field with energy spectrum E(k) ~ k^-5/3, so
    |rho_hat(k)| ~ |k|^-11/6 in 3-D; k = 0 removed; scaled to ``rms_frac`` of
    ``mean``.  ``shape`` = (nz, ny, nx) overrides the cube n^3."""
    import scipy.fft as sfft
    if shape is None:
        shape = (n, n, n)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape, dtype=np.float32)
    spec = sfft.rfftn(white, workers=-1)
    kz = np.fft.fftfreq(shape[0]) * shape[0]
    ky = np.fft.fftfreq(shape[1]) * shape[1]
    kx = np.fft.rfftfreq(shape[2]) * shape[2]
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2).astype(np.float32)
    k2[0, 0, 0] = 1.0
    amp = k2 ** np.float32(-11.0 / 12.0)
    amp[0, 0, 0] = 0.0
    spec *= amp
    field = sfft.irfftn(spec, s=shape, workers=-1).astype(np.float64)
    field -= field.mean()
    field /= field.std()
    return (mean * (1.0 + rms_frac * field)).astype(np.float32)


def turbulence_slice_rho(n, seed, mean=1.225, rms_frac=0.05, k_cut=None) -> np.ndarray:
    """Periodic 2-D Gaussian random field [n, n] with energy spectrum
    E(k) ~ k^-5/3, so |rho_hat(k)| ~ |k|^-4/3 in 2-D, times a dissipation
    cutoff exp(-(k / k_cut)^2) on the energy when k_cut (cycles per box) is
    given; k = 0 removed; scaled to ``rms_frac`` of ``mean``."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n))
    spec = np.fft.rfft2(white)
    ky = np.fft.fftfreq(n) * n
    kx = np.fft.rfftfreq(n) * n
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    k2[0, 0] = 1.0
    amp = k2 ** (-2.0 / 3.0)
    if k_cut is not None:
        amp = amp * np.exp(-0.5 * k2 / (k_cut * k_cut))
    amp[0, 0] = 0.0
    field = np.fft.irfft2(spec * amp, s=(n, n))
    field -= field.mean()
    field /= field.std()
    return mean * (1.0 + rms_frac * field)


def shock_rho(nx, ny, nz, spacing_y, rho1=1.2, ratio=2.5, width=0.5e-3, y_shock=None) -> np.ndarray:
    """Normal-shock slab: rho1 -> ratio*rho1 across a tanh profile of width
    ``width`` centred at ``y_shock`` (default: the middle of the grid)."""
    y = np.arange(ny, dtype=np.float64) * spacing_y
    if y_shock is None:
        y_shock = 0.5 * (ny - 1) * spacing_y
    prof = rho1 + (ratio * rho1 - rho1) * 0.5 * (1.0 + np.tanh((y - y_shock) / width))
    rho = np.broadcast_to(prof.reshape(1, ny, 1), (nz, ny, nx))
    return np.ascontiguousarray(rho, dtype=np.float32)


# --------------------------------------------------------------------------
# optical layouts
# --------------------------------------------------------------------------
def _thick_lens_matrix(R1, R2, d, n_glass, n0):
    """Paraxial (y, n*u) system matrix of a thick lens between its vertices;
    used only to place the lens and sensor of a scene."""
    P1 = (n_glass - n0) / R1
    P2 = (n0 - n_glass) / R2
    ref1 = np.array([[1.0, 0.0], [-P1, 1.0]])
    tr = np.array([[1.0, d / n_glass], [0.0, 1.0]])
    ref2 = np.array([[1.0, 0.0], [-P2, 1.0]])
    return ref2 @ tr @ ref1


def thick_lens_layout(z_object, M, f_number, n0, R1=0.1, R2=-0.1, d=0.01, n_glass=1.5,
                      pitch=17e-6, width=1024, height=1024, clear_r=0.03):
    """Biconvex lens focused on the plane z = z_object with |magnification| M,
    stop (entrance aperture) at the front vertex.  Returns an ``Optics``."""
    S = _thick_lens_matrix(R1, R2, d, n_glass, n0)
    A, B, C, D = S[0, 0], S[0, 1], S[1, 0], S[1, 1]
    P = -C
    efl = n0 / P
    # object distance u = s_o / n0 so that the imaged magnification is -M
    u = (1.0 / M + D) / P
    v = (A * u + B) * M
    s_o, s_i = u * n0, v * n0
    zv1 = z_object + s_o
    zv2 = zv1 + d
    a = efl / (2.0 * f_number)
    surfaces = [
        Surface(STOP, zv1, clear_r=a),
        Surface(SPHERE, zv1, R=R1, n_after=n_glass, clear_r=clear_r),
        Surface(SPHERE, zv2, R=R2, n_after=n0, clear_r=clear_r),
    ]
    return Optics(surfaces=surfaces, n_object=n0, aim_z=zv1, aim_r=a, sensor_z=zv2 + s_i,
                  pitch=pitch, width=width, height=height, f_number=f_number, magnification=M)


def ideal_lens_layout(z_object, M, f, f_number, n0, pitch=17e-6, width=256, height=256):
    """Ideal thin lens at distance s_o = f (1 + 1/M) after the object plane."""
    s_o = f * (1.0 + 1.0 / M)
    s_i = f * (1.0 + M)
    zl = z_object + s_o
    a = f / (2.0 * f_number)
    surfaces = [
        Surface(STOP, zl, clear_r=a),
        Surface(IDEAL_THIN, zl, f=f, n_after=n0, clear_r=a * 1.5),
    ]
    return Optics(surfaces=surfaces, n_object=n0, aim_z=zl, aim_r=a, sensor_z=zl + s_i,
                  pitch=pitch, width=width, height=height, f_number=f_number, magnification=M)


# --------------------------------------------------------------------------
# source sets
# --------------------------------------------------------------------------
def dot_grid(nx, ny, pitch, z=0.0) -> np.ndarray:
    xs = (np.arange(nx) - 0.5 * (nx - 1)) * pitch
    ys = (np.arange(ny) - 0.5 * (ny - 1)) * pitch
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1).astype(np.float64)


def uniform_points(n, lo, hi, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.random((n, 3))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def _n_ambient(rho=RHO_AIR, K=K_AIR):
    return 1.0 + K * rho


def c0(scale: float = 1.0, rays_per_source: int = 100) -> List[Frame]:
    """BOS linear-gradient slab (409,600 rays at scale 1)."""
    n0 = _n_ambient()
    Lx, Ly, Lz = 0.05, 0.05, 0.01
    zc = 0.5
    N = 32
    rho = linear_gradient_rho(N, N, N, 1.20, 1.26, axis=1)
    med = Medium(rho, (-Lx / 2, -Ly / 2, zc - Lz / 2), (Lx / (N - 1), Ly / (N - 1), Lz / (N - 1)))
    opt = ideal_lens_layout(0.0, 0.1, 0.105, 8.0, n0, width=256, height=256)
    nd = max(1, int(round(64 * math.sqrt(scale))))
    src = dot_grid(nd, nd, 0.68e-3 * 64 / nd, z=0.0)
    rps = max(1, int(round(rays_per_source)))
    return [Frame(med, opt, src, rps, seed=0, integrator=EULER, step=0.1e-3)]


def c1(scale: float = 1.0) -> List[Frame]:
    """PIV uniform medium, thick lens, sheet 2 mm before / after focus."""
    n0 = 1.000277
    rho_u = (n0 - 1.0) / K_AIR
    opt = thick_lens_layout(0.0, 0.2, 4.0, n0, width=1024, height=1024)
    n_src = max(1, int(round(10000 * scale)))
    rps = max(1, int(round(10000 * min(1.0, scale * 100))))
    frames = []
    for fi, dz in enumerate((-2e-3, 2e-3)):
        lo = (-0.025, -0.025, dz - 0.5e-3)
        hi = (0.025, 0.025, dz + 0.5e-3)
        rho = uniform_rho(16, 16, 4, rho_u)
        med = Medium(rho, lo, (0.05 / 15, 0.05 / 15, 1e-3 / 3))
        src = uniform_points(n_src, lo, hi, seed=1 + 100 * fi)
        frames.append(Frame(med, opt, src, rps, seed=1, integrator=RK4, step=0.2e-3, frame_index=fi))
    return frames


def c2(scale: float = 1.0, grid: Optional[int] = None) -> List[Frame]:
    """BOS turbulence field (1e8 rays at scale 1)."""
    n0 = _n_ambient()
    N = grid if grid is not None else 256
    L = 0.1
    zc = 0.5
    rho = turbulence_rho(N, seed=2)
    med = Medium(rho, (-L / 2, -L / 2, zc - L / 2), (L / (N - 1),) * 3)
    opt = thick_lens_layout(0.0, 0.1, 8.0, n0, width=1024, height=1024)
    fov = 1024 * 17e-6 / 0.1
    n_src = max(1, int(round(100000 * scale)))
    rps = max(1, int(round(1000 * min(1.0, scale * 100))))
    src = uniform_points(n_src, (-fov / 2, -fov / 2, 0.0), (fov / 2, fov / 2, 0.0), seed=2)
    return [Frame(med, opt, src, rps, seed=2, integrator=RK4, step=0.2e-3)]


def c4(scale: float = 1.0, grid: Optional[int] = None) -> List[Frame]:
    """Tomo-PIV scale: particles inside a turbulence volume (1e9 rays at scale 1)."""
    n0 = _n_ambient()
    N = grid if grid is not None else 256
    Lx, Ly, Lz = 0.1, 0.1, 0.03
    rho = turbulence_rho(N, seed=4)
    med = Medium(rho, (-Lx / 2, -Ly / 2, -Lz / 2), (Lx / (N - 1), Ly / (N - 1), Lz / (N - 1)))
    opt = thick_lens_layout(0.0, 0.2, 4.0, n0, width=2048, height=2048)
    n_src = max(1, int(round(100000 * scale)))
    rps = max(1, int(round(10000 * min(1.0, scale * 100))))
    src = uniform_points(n_src, (-Lx / 2, -Ly / 2, -Lz / 2), (Lx / 2, Ly / 2, Lz / 2), seed=4)
    return [Frame(med, opt, src, rps, seed=4, integrator=RK4, step=0.2e-3)]


def c3(scale: float = 1.0, n_frames: int = 64, max_grid: int = 256) -> List[Frame]:
    """64 frames of uneven size: N_src = 10^U(3,5), grid from {64..256},
    field kind in rotation (shock, gradient, turbulence), rays/source =
    10^U(3,4); the C2 optics."""
    n0 = _n_ambient()
    rng = np.random.default_rng(3)
    opt = thick_lens_layout(0.0, 0.1, 8.0, n0, width=1024, height=1024)
    fov = 1024 * 17e-6 / 0.1
    L = 0.1
    zc = 0.5
    grids = [g for g in (64, 96, 128, 192, 256) if g <= max_grid]
    frames = []
    turb_cache = {}
    for f in range(n_frames):
        n_src = int(round(10 ** rng.uniform(3, 5) * scale)) or 1
        N = int(grids[rng.integers(len(grids))])
        rps = int(round(10 ** rng.uniform(3, 4) * min(1.0, scale * 100))) or 1
        kind = f % 3
        h = L / (N - 1)
        if kind == 0:
            rho = shock_rho(N, N, N, h)
        elif kind == 1:
            rho = linear_gradient_rho(N, N, N, 1.20, 1.26, axis=1)
        else:
            if N not in turb_cache:
                turb_cache[N] = turbulence_rho(N, seed=300 + N)
            rho = turb_cache[N]
        med = Medium(rho, (-L / 2, -L / 2, zc - L / 2), (h, h, h))
        src = uniform_points(n_src, (-fov / 2, -fov / 2, 0.0), (fov / 2, fov / 2, 0.0), seed=3000 + f)
        frames.append(Frame(med, opt, src, rps, seed=3, integrator=RK4, step=0.2e-3, frame_index=f))
    return frames


TABLE1 = {"Z_A": 0.75, "Z_D": 0.25, "Lx": 0.032, "Ly": 0.032, "Lz": 0.010, "f": 0.105, "f_number": 11.0,
          "M_printed": 0.12, "pitch": 10e-6, "dots_per_32x32_px": 20, "K": 0.226e-3, "rho_scale": 1.225}


def table1(scale: float = 1.0, grid: Optional[int] = None, rays_per_source: int = 10000,
           sensor: int = 512) -> List[Frame]:
    """The BOS experiment of Sec. 4 with the Table 1 geometry (5.12e7 rays at
    scale 1): a z-stacked 2-D turbulence slice, dots Z_D before the volume
    mid-plane, an ideal thin lens Z_A after it."""
    t = TABLE1
    K = t["K"]
    n0 = 1.0 + K * t["rho_scale"]
    N = grid if grid is not None else 256
    nz = 11
    rho2 = turbulence_slice_rho(N, seed=5, mean=t["rho_scale"], rms_frac=0.05, k_cut=8.0)
    rho = np.ascontiguousarray(np.broadcast_to(rho2[None, :, :], (nz, N, N)), dtype=np.float32)
    z_mid = t["Z_D"]
    med = Medium(rho, (-t["Lx"] / 2, -t["Ly"] / 2, z_mid - t["Lz"] / 2),
                 (t["Lx"] / (N - 1), t["Ly"] / (N - 1), t["Lz"] / (nz - 1)), K)
    # the lens at Z_A + Z_D from the dots, focused on them
    M = t["f"] / (t["Z_A"] + t["Z_D"] - t["f"])
    opt = ideal_lens_layout(0.0, M, t["f"], t["f_number"], n0, pitch=t["pitch"], width=sensor, height=sensor)
    n_dots = max(1, int(round(t["dots_per_32x32_px"] * sensor * sensor / 1024.0 * scale)))
    half = 0.5 * sensor * t["pitch"] / M
    src = uniform_points(n_dots, (-half, -half, 0.0), (half, half, 0.0), seed=5)
    rps = max(1, int(round(rays_per_source * min(1.0, scale * 100))))
    return [Frame(med, opt, src, rps, seed=5, integrator=RK4, step=0.1e-3)]


WORKLOADS = {"c0": c0, "c1": c1, "c2": c2, "c3": c3, "c4": c4, "table1": table1}
