"""CPU FP64 oracle for the PIV/BOS ray-tracing image generator.

TEST INFRASTRUCTURE.  This package is a plain, slow, independently written
restatement of the method of arXiv 1812.05902 (Sec. 3): light-field
generation (Sec. 3.1), tracing through density gradients with Eq. 1 and the
Runge-Kutta scheme of Eqs. 3-6 or the first-order scheme (Sec. 3.2), optical
elements with Eq. 7 (Sec. 3.3), and sensor deposit with Eq. 8 (Sec. 3.4).
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference leg of ``bench.py`` may use it; the product library never does.
It shares no code with the CUDA library.

The arithmetic lives in ``pivbos_oracle.c`` (C11, FP64, compiled with
``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes.  Every function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pivbos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpivbos_oracle.so")
_lock = threading.Lock()
_lib = None

SPHERE, PLANE, IDEAL_THIN, STOP, MIRROR, LENS_ARRAY = 0, 1, 2, 3, 4, 5
EULER, RK4 = 0, 1
REACHED, KILLED_STOP, KILLED_MISS, KILLED_TIR, KILLED_OFF_SENSOR, KILLED_MAXSTEP = range(6)

RAY_STATE = np.dtype([
    ("vol_pos", "<f8", (3,)), ("vol_dir", "<f8", (3,)),
    ("sensor_xy", "<f8", (2,)), ("sensor_dir", "<f8", (3,)),
    ("status", "<i4"), ("steps", "<i4"), ("opl", "<f8"),
])


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            D = ctypes.c_double
            I = ctypes.c_int
            I64 = ctypes.c_int64
            U32 = ctypes.c_uint32
            U64 = ctypes.c_uint64
            L.om_philox4x64.argtypes = [P, P, P]
            L.om_u01.argtypes = [U64]
            L.om_u01.restype = D
            L.om_lens_point.argtypes = [U64, U32, U32, U32, D, D, P]
            L.om_medium_build.argtypes = [P, I, I, I, P, P, D]
            L.om_medium_build.restype = P
            L.om_medium_free.argtypes = [P]
            L.om_medium_nodes.argtypes = [P, P, P, P, P]
            L.om_sample_many.argtypes = [P, P, I64, P, P]
            L.om_sigma_from_eq8.argtypes = [D, D, D, I]
            L.om_sigma_from_eq8.restype = D
            L.om_optics_build.argtypes = [P, I, D, D, D, D, D, I, I, D]
            L.om_optics_build.restype = P
            L.om_optics_free.argtypes = [P]
            L.om_refract.argtypes = [P, P, D, D, P]
            L.om_refract.restype = I
            L.om_sphere_hit.argtypes = [P, P, D, D, P]
            L.om_sphere_hit.restype = I
            L.om_max_steps.argtypes = [P, D]
            L.om_max_steps.restype = I
            L.om_trace.argtypes = [P, P, P, U64, U32, U32, U32, I, D, P]
            L.om_trace.restype = I
            L.om_deposit.argtypes = [P, D, D, P, I]
            L.om_deposit.restype = I
            L.om_render.argtypes = [P, P, P, I64, ctypes.c_int32, I64, I64, U64, U32, I, D, P, P, I]
            L.om_trace_many.argtypes = [P, P, P, ctypes.c_int32, P, I64, U64, U32, I, D, P, I]
            L.om_threads.restype = I
            L.om_line_gradient_integral.argtypes = [P, P, P, P]
            L.om_optics_tilt_sensor.argtypes = [P, D, D]
            L.om_reflect.argtypes = [P, P, P]
            L.om_trace_optics.argtypes = [P, P, P, P]
            L.om_trace_optics.restype = I
            L.om_mie.argtypes = [D, D, D, I, P, P]
            L.om_mie.restype = I
            L.om_optics_radiance.argtypes = [P, P, I, P, P]
            L.om_ray_weight.argtypes = [P, P, U64, U32, U32, U32]
            L.om_ray_weight.restype = D
            L.om_advect.argtypes = [P, I64, P, I, I, I, P, P, D, P]
            L.om_image_u16.argtypes = [P, I64, D, P]
            L.om_line_gradient_integral.restype = I
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x64(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().om_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(w: int) -> float:
    return lib().om_u01(int(w))


def lens_point(seed, source_id, ray_id, frame, aim_r, aim_z) -> np.ndarray:
    p = np.zeros(3)
    lib().om_lens_point(seed, source_id, ray_id, frame, aim_r, aim_z, _ptr(p))
    return p


def sigma_eq8(f_number, M, wavelength, rule=0) -> float:
    return lib().om_sigma_from_eq8(f_number, M, wavelength, rule)


def refract(d, N, n_i, n_f):
    d = np.ascontiguousarray(d, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.float64)
    out = np.zeros(3)
    ok = lib().om_refract(_ptr(d), _ptr(N), n_i, n_f, _ptr(out))
    return (out if ok else None)


def sphere_hit(P, d, zv, R):
    P = np.array(P, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    N = np.zeros(3)
    ok = lib().om_sphere_hit(_ptr(P), _ptr(d), zv, R, _ptr(N))
    return (P, N) if ok else None


class Medium:
    """Node values n-1 and grad n built from rho (Eq. 1, central differences)."""

    def __init__(self, rho, origin, spacing, K):
        self.rho = np.ascontiguousarray(rho, dtype=np.float32)
        nz, ny, nx = self.rho.shape
        self.dims = (nx, ny, nz)
        o = np.ascontiguousarray(origin, dtype=np.float64)
        h = np.ascontiguousarray(spacing, dtype=np.float64)
        self.origin, self.spacing = tuple(float(v) for v in o), tuple(float(v) for v in h)
        self.h = lib().om_medium_build(_ptr(self.rho), nx, ny, nz, _ptr(o), _ptr(h), float(K))
        if not self.h:
            raise ValueError("oracle medium needs at least 2 nodes per axis")

    @classmethod
    def from_scene(cls, m):
        return cls(m.rho, m.origin, m.spacing, m.K)

    def nodes(self):
        nx, ny, nz = self.dims
        out = [np.zeros((nz, ny, nx)) for _ in range(4)]
        lib().om_medium_nodes(self.h, *[_ptr(a) for a in out])
        return out

    def sample(self, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        dn = np.zeros(len(pts))
        g = np.zeros((len(pts), 3))
        lib().om_sample_many(self.h, _ptr(pts), len(pts), _ptr(dn), _ptr(g))
        return dn, g

    def z_mid(self):
        """z of the mid-plane of the box"""
        return self.origin[2] + 0.5 * (self.dims[2] - 1) * self.spacing[2]

    def max_steps(self, step):
        return lib().om_max_steps(self.h, step)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.om_medium_free(h)
            self.h = None


class Optics:
    def __init__(self, surfaces, n_object, aim_z, aim_r, sensor_z, pitch, W, H, sigma):
        self.surf = np.ascontiguousarray(surfaces, dtype=np.float64).reshape(-1, 6)
        self.W, self.H, self.pitch, self.sigma = int(W), int(H), float(pitch), float(sigma)
        self.h = lib().om_optics_build(_ptr(self.surf), len(self.surf), n_object, aim_z, aim_r,
                                       sensor_z, pitch, int(W), int(H), float(sigma))
        if not self.h:
            raise ValueError("bad optics")

    @classmethod
    def from_scene(cls, o):
        sigma = sigma_eq8(o.f_number, o.magnification, o.wavelength, o.dtau_rule)
        opt = cls(o.surface_array(), o.n_object, o.aim_z, o.aim_r, o.sensor_z, o.pitch,
                  o.width, o.height, sigma)
        tx, ty = getattr(o, "sensor_tilt_x", 0.0), getattr(o, "sensor_tilt_y", 0.0)
        if tx != 0.0 or ty != 0.0:
            opt.tilt_sensor(tx, ty)
        mie_cfg = getattr(o, "mie", None)
        if mie_cfg is not None:
            s12, _ = mie(mie_size_parameter(mie_cfg.diameter, mie_cfg.wavelength, mie_cfg.n_medium),
                         mie_cfg.m_re, mie_cfg.m_im, mie_cfg.n_angles)
            opt.radiance(s12, mie_cfg.laser_dir, mie_cfg.polarisation)
        return opt

    def radiance(self, s12, laser_dir, polarisation=None):
        """Mie radiance per ray (Sec. 3.1): table s12 [n, 2] of |S1|^2, |S2|^2 at
        angles 0..pi, laser direction, polarisation (None = unpolarised)"""
        self._rad = np.ascontiguousarray(s12, dtype=np.float64).reshape(-1, 2)
        L = np.ascontiguousarray(laser_dir, dtype=np.float64)
        pol = None if polarisation is None else np.ascontiguousarray(polarisation, dtype=np.float64)
        lib().om_optics_radiance(self.h, _ptr(self._rad), len(self._rad), _ptr(L),
                                 None if pol is None else _ptr(pol))
        return self

    def tilt_sensor(self, tilt_x, tilt_y):
        """turn the sensor about its centre: tilt_x about x, then tilt_y about y (radians)"""
        lib().om_optics_tilt_sensor(self.h, float(tilt_x), float(tilt_y))
        return self

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.om_optics_free(h)
            self.h = None


def _mh(medium):
    return medium.h if medium is not None else None


def trace(medium, optics, source, seed, source_id, ray_id, frame, integrator, step):
    st = np.zeros(1, dtype=RAY_STATE)
    s = np.ascontiguousarray(source, dtype=np.float64)
    lib().om_trace(_mh(medium), optics.h, _ptr(s), seed, source_id, ray_id, frame,
                   integrator, step, _ptr(st))
    return st[0]


def trace_many(medium, optics, sources, rays_per_source, ray_ids, seed, frame, integrator, step,
               threads=0):
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
    ids = np.ascontiguousarray(ray_ids, dtype=np.int64)
    out = np.zeros(len(ids), dtype=RAY_STATE)
    lib().om_trace_many(_mh(medium), optics.h, _ptr(src), int(rays_per_source), _ptr(ids), len(ids),
                        seed, frame, integrator, step, _ptr(out), threads)
    return out


def mie_size_parameter(diameter, wavelength, n_medium):
    """x = pi d n_medium / lambda (lambda in vacuum)"""
    return np.pi * diameter * n_medium / wavelength


def mie(x, m_re, m_im=0.0, n_angles=181):
    """Mie scattering by a homogeneous sphere (``om_mie``): returns (s12 [n, 2] =
    |S1|^2, |S2|^2 at theta = 0..pi, {q_ext, q_sca, re_s0, terms})."""
    s12 = np.zeros((n_angles, 2))
    q = np.zeros(4)
    if not lib().om_mie(float(x), float(m_re), float(m_im), int(n_angles), _ptr(s12), _ptr(q)):
        raise ValueError("bad Mie input")
    return s12, {"q_ext": q[0], "q_sca": q[1], "re_s0": q[2], "terms": int(q[3])}


def ray_weight(optics, src, seed, source_id, ray_id, frame):
    s = np.ascontiguousarray(src, dtype=np.float64)
    return lib().om_ray_weight(optics.h, _ptr(s), seed, source_id, ray_id, frame)


def advect(sources, vel, origin, spacing, dt):
    """Second frame of an image pair: particles moved over dt by the velocity
    field vel [nz, ny, nx, 3] (explicit midpoint rule, trilinear samples)."""
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(vel, dtype=np.float32)
    nz, ny, nx, _ = v.shape
    o = np.ascontiguousarray(origin, dtype=np.float64)
    h = np.ascontiguousarray(spacing, dtype=np.float64)
    out = np.zeros_like(src)
    lib().om_advect(_ptr(src), len(src), _ptr(v), nx, ny, nz, _ptr(o), _ptr(h), float(dt), _ptr(out))
    return out


def image_u16(image, full_scale):
    """16-bit image: full_scale rays read 65535 (rounded, clipped)."""
    img = np.ascontiguousarray(image, dtype=np.int64)
    out = np.zeros(img.shape, dtype=np.uint16)
    lib().om_image_u16(_ptr(img), img.size, float(full_scale), _ptr(out))
    return out


def reflect(d, N):
    d = np.ascontiguousarray(d, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.float64)
    out = np.zeros(3)
    lib().om_reflect(_ptr(d), _ptr(N), _ptr(out))
    return out


def trace_optics(optics, P, d):
    """The optics and sensor stages alone from point P, unit direction d."""
    st = np.zeros(1, dtype=RAY_STATE)
    P = np.ascontiguousarray(P, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    lib().om_trace_optics(optics.h, _ptr(P), _ptr(d), _ptr(st))
    return st[0]


def deposit(optics, px, py, image=None):
    if image is None:
        image = np.zeros((optics.H, optics.W), dtype=np.int64)
    lib().om_deposit(optics.h, px, py, _ptr(image), 0)
    return image


def render(medium, optics, sources, rays_per_source, seed, frame, integrator, step,
           image=None, first_ray=0, ray_count=None, threads=0):
    """Render (part of) a frame: rays [first_ray, first_ray + ray_count) of the
    flattened (source, ray) index.  Returns (image int64 [H, W], stats[6])."""
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
    if image is None:
        image = np.zeros((optics.H, optics.W), dtype=np.int64)
    total = len(src) * int(rays_per_source)
    if ray_count is None:
        ray_count = total - first_ray
    stats = np.zeros(6, dtype=np.int64)
    lib().om_render(_mh(medium), optics.h, _ptr(src), len(src), int(rays_per_source),
                    int(first_ray), int(ray_count), seed, frame, integrator, step,
                    _ptr(image), _ptr(stats), threads)
    return image, stats


def render_frame(frame, image=None, first_ray=0, ray_count=None, threads=0):
    """Render a ``scenes.Frame`` with the oracle."""
    med = Medium.from_scene(frame.medium) if frame.medium is not None else None
    opt = Optics.from_scene(frame.optics)
    return render(med, opt, frame.sources, frame.rays_per_source, frame.seed, frame.frame_index,
                  frame.integrator, frame.step, image=image, first_ray=first_ray,
                  ray_count=ray_count, threads=threads)


# --------------------------------------------------------------------------
# Sec. 4: the simulated BOS experiment (per-dot displacements, Eq. 9, and
# the regular-grid map the paper draws them on)
# --------------------------------------------------------------------------
def line_gradient_integral(medium, s, c):
    """Integral over z of the sampled (dn/dx, dn/dy) along the line from s
    toward c, over its part inside the box (``om_line_gradient_integral``).
    Returns (integral [2], pieces)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(2)
    k = lib().om_line_gradient_integral(medium.h, _ptr(s), _ptr(c), _ptr(out))
    return out, k


def eq9_displacements(medium, dots, aim_z, magnification, n_object, pitch):
    """Eq. 9 for every dot, in pixels of the sensor frame.

    Delta X = (M Z_D / n0) * integral of grad n dz, the integral taken along
    the dot's chief ray (toward the centre of the lens at z = aim_z), Z_D
    from the dot to the mid-plane of the box.  A ray bent by epsilon seems to
    come from a dot shifted by -Z_D epsilon; the lens inverts the real image
    (the sensor frame is not flipped), so the dot's image moves by
    +M Z_D epsilon."""
    dots = np.ascontiguousarray(dots, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(dots), 2))
    zm = medium.z_mid()
    for q, d in enumerate(dots):
        I, _ = line_gradient_integral(medium, d, (0.0, 0.0, aim_z))
        out[q] = magnification * (zm - d[2]) * I / n_object / pitch
    return out


def bos_displacements(medium, optics, dots, rays_per_dot, seed, frame, integrator, step, threads=0,
                      dot_ids=None):
    """Sec. 4: every ray of a dot traced through the medium and, with the same
    lens point, through the uniform medium; over the rays that reach the
    sensor both times: the mean sensor position without the medium
    (centroid, px), the mean of (with - without) (displacement, px) and the
    number of such pairs.  Dots without a pair get NaN.  dot_ids (optional)
    restricts the result to those dots of the set (ray k of dot d keeps its
    lens point)."""
    dots = np.ascontiguousarray(dots, dtype=np.float64).reshape(-1, 3)
    sel = np.arange(len(dots), dtype=np.int64) if dot_ids is None else np.asarray(dot_ids, dtype=np.int64)
    n = len(sel)
    ids = (sel[:, None] * int(rays_per_dot) + np.arange(int(rays_per_dot))[None, :]).ravel()
    a = trace_many(medium, optics, dots, rays_per_dot, ids, seed, frame, integrator, step, threads)
    b = trace_many(None, optics, dots, rays_per_dot, ids, seed, frame, integrator, step, threads)
    ok = ((a["status"] == REACHED) & (b["status"] == REACHED)).reshape(n, rays_per_dot)
    pa = a["sensor_xy"].reshape(n, rays_per_dot, 2)
    pb = b["sensor_xy"].reshape(n, rays_per_dot, 2)
    cnt = ok.sum(1)
    centroid = np.full((n, 2), np.nan)
    disp = np.full((n, 2), np.nan)
    for q in range(n):
        if cnt[q]:
            centroid[q] = pb[q][ok[q]].mean(0)
            disp[q] = (pa[q][ok[q]] - pb[q][ok[q]]).mean(0)
    return centroid, disp, cnt.astype(np.int32)


def regrid_bilinear(xy, values, grid_w, grid_h, x0, y0, cell, min_weight=0.0):
    """Sec. 4: scattered per-dot values onto a regular grid by bilinear
    interpolation.  Reading: a point at grid coordinates (u, v) =
    ((x - x0) / cell, (y - y0) / cell) inside [0, W-1] x [0, H-1] gives the
    four nodes of its cell its value with the bilinear weights
    (1-fu)(1-fv), fu(1-fv), (1-fu)fv, fu fv; a node holds the weighted mean
    of what it received, NaN if its summed weight is zero or below
    min_weight.  Returns (values [H, W, 2], weight [H, W])."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    values = np.asarray(values, dtype=np.float64).reshape(-1, 2)
    acc = np.zeros((grid_h, grid_w, 2))
    wsum = np.zeros((grid_h, grid_w))
    for (x, y), v in zip(xy, values):
        if not (np.isfinite(v).all() and np.isfinite(x) and np.isfinite(y)):
            continue
        u, t = (x - x0) / cell, (y - y0) / cell
        if not (0.0 <= u <= grid_w - 1 and 0.0 <= t <= grid_h - 1):
            continue
        i = min(int(np.floor(u)), grid_w - 2)
        j = min(int(np.floor(t)), grid_h - 2)
        fu, fv = u - i, t - j
        for di, dj, w in ((0, 0, (1 - fu) * (1 - fv)), (1, 0, fu * (1 - fv)),
                          (0, 1, (1 - fu) * fv), (1, 1, fu * fv)):
            acc[j + dj, i + di] += w * v
            wsum[j + dj, i + di] += w
    out = np.full((grid_h, grid_w, 2), np.nan)
    keep = (wsum > 0.0) & (wsum >= min_weight)
    out[keep] = acc[keep] / wsum[keep][:, None]
    return out, wsum


def threads() -> int:
    return lib().om_threads()
