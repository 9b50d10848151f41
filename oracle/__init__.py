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

SPHERE, PLANE, IDEAL_THIN, STOP = 0, 1, 2, 3
EULER, RK4 = 0, 1
REACHED, KILLED_STOP, KILLED_MISS, KILLED_TIR, KILLED_OFF_SENSOR, KILLED_MAXSTEP = range(6)

RAY_STATE = np.dtype([
    ("vol_pos", "<f8", (3,)), ("vol_dir", "<f8", (3,)),
    ("sensor_xy", "<f8", (2,)), ("sensor_dir", "<f8", (3,)),
    ("status", "<i4"), ("steps", "<i4"),
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
        return cls(o.surface_array(), o.n_object, o.aim_z, o.aim_r, o.sensor_z, o.pitch,
                   o.width, o.height, sigma)

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


def threads() -> int:
    return lib().om_threads()
