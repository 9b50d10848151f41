"""Thin ctypes binding of libpivbos.so (include/pivbos.h).

Argument marshalling only: every step of the ray-tracing path runs in the
CUDA kernels of the library.  PyTorch is used for device memory and streams:
functions that take device buffers accept CUDA tensors (their ``data_ptr()``
is passed) and run on ``torch.cuda.current_stream()`` unless a stream is
given.  If the library is missing, importing the binding raises; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpivbos.so")
TESTING_LIB_PATH = os.path.join(_HERE, "libpivbos_testing.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_OVERFLOW, ERR_UNSUPPORTED = range(7)
RAY_REACHED, RAY_STOP, RAY_MISS, RAY_TIR, RAY_OFF_SENSOR, RAY_MAXSTEP = range(6)
RAY_NSTATUS = 6
SURF_SPHERE, SURF_PLANE, SURF_IDEAL_THIN, SURF_STOP, SURF_MIRROR, SURF_LENS_ARRAY = range(6)
EULER, RK4 = 0, 1
MAX_SURFACES = 16
MAX_WINDOW = 12

RAY_STATE = np.dtype([
    ("vol_pos", "<f8", (3,)), ("vol_dir", "<f8", (3,)),
    ("sensor_xy", "<f8", (2,)), ("sensor_dir", "<f8", (3,)),
    ("status", "<i4"), ("steps", "<i4"), ("opl", "<f8"),
])
assert RAY_STATE.itemsize == 104


class pivbos_surface(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32), ("z_vertex", ctypes.c_double),
                ("radius", ctypes.c_double), ("focal", ctypes.c_double), ("n_after", ctypes.c_double),
                ("clear_radius", ctypes.c_double)]


class pivbos_frame_desc(ctypes.Structure):
    _fields_ = [("medium", ctypes.c_void_p), ("optics", ctypes.c_void_p), ("sources", ctypes.c_void_p),
                ("n_sources", ctypes.c_int64), ("rays_per_source", ctypes.c_int32), ("frame", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("step", ctypes.c_double), ("image", ctypes.c_void_p),
                ("stats", ctypes.c_void_p)]


class pivbos_tuning(ctypes.Structure):
    _fields_ = [("rays_per_cta", ctypes.c_int32), ("cell_cache", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class pivbos_surrogate_cfg(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_int64), ("n_val", ctypes.c_int64), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("err_budget_px", ctypes.c_float),
                ("budget_margin", ctypes.c_float), ("min_bin_count", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("ref_plane_z", ctypes.c_double), ("born_segments", ctypes.c_int32),
                ("use_network", ctypes.c_int32), ("table_columns_per_cell", ctypes.c_int32),
                ("table_levels_per_cell", ctypes.c_int32)]


_REPORT_SCALARS = ("train_loss", "train_steps", "val_rms_px", "val_rms_px_born", "val_rms_px_straight",
                   "val_rms_px_served", "val_served_frac", "val_served_frac_born", "val_served_frac_straight",
                   "steps_saved_frac", "steps_saved_frac_born", "steps_saved_frac_straight",
                   "val_status_flip_frac", "n_val_reached", "n_val_box", "seconds_table", "seconds_data",
                   "seconds_train", "seconds_validate", "table_bytes", "born_segments",
                   "table_columns_per_cell")
_REPORT_VECTORS = (("pilot_rms_px_born_k", 6), ("target_rms", 4), ("correction_rms", 4),
                   ("sensor_px_per_unit", 4))
_REPORT_TAIL = ("network_trained", "val_served_frac_net")


class pivbos_surrogate_report(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in _REPORT_SCALARS] +
                [(n, ctypes.c_double * k) for n, k in _REPORT_VECTORS] +
                [(n, ctypes.c_double) for n in _REPORT_TAIL])

    def as_dict(self):
        d = {n: getattr(self, n) for n in _REPORT_SCALARS + _REPORT_TAIL}
        for n, _ in _REPORT_VECTORS:
            d[n] = list(getattr(self, n))
        return d


class PivbosError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("pivbos status %d: %s" % (status, msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpivbos.so is not built (run __graft_entry__.build() or "
                          "python paper_1812_05902_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    I32, I64, U32, U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "pivbos_medium_create": ([P, I, I, I, I, P, P, D, P, P], I),
        "pivbos_medium_refill": ([P, P, I, P], I),
        "pivbos_medium_destroy": ([P], None),
        "pivbos_optics_create": ([P, I, D, D, D, D, D, D, I, D, D, I, I, P], I),
        "pivbos_optics_destroy": ([P], None),
        "pivbos_optics_tilt_sensor": ([P, D, D, P], I),
        "pivbos_mie": ([D, D, D, D, D, I, P, P], I),
        "pivbos_optics_radiance": ([P, P, P, P, I, P], I),
        "pivbos_advect_sources": ([P, I64, P, I, I, I, P, P, D, P, P], I),
        "pivbos_image_u16": ([P, I64, D, P, P], I),
        "pivbos_selftest_wait_timeout": ([U32, P], I),
        "pivbos_render": ([P, P, P, I64, I, I32, U64, U32, I, D, P, I, P, P], I),
        "pivbos_trace_exit_states": ([P, P, P, I64, I, I32, U64, U32, I, D, P, I64, P, P], I),
        "pivbos_image_finalize": ([P, I64, P, P], I),
        "pivbos_sync": ([P], I),
        "pivbos_last_error": ([], ctypes.c_char_p),
        "pivbos_timing_enable": ([I], I),
        "pivbos_timing_reset": ([], I),
        "pivbos_timing_read": ([ctypes.c_char_p, ctypes.POINTER(D), ctypes.POINTER(I64)], I),
        "pivbos_version": ([], ctypes.c_char_p),
        "pivbos_kernel_launches": ([], I64),
        "pivbos_render_noalloc": ([P, P, P, I64, I32, U64, U32, I, D, P, P, P], I),
        "pivbos_default_tuning": ([P], I),
        "pivbos_render_range": ([P, P, P, I64, I64, I, I32, U64, U32, I, D, P, I, P, P], I),
        "pivbos_batch_create": ([P, I, I, P, P], I),
        "pivbos_batch_render": ([P, P], I),
        "pivbos_batch_destroy": ([P], None),
        "pivbos_autotune": ([P, I, D, I32, P, P, P], I),
        "pivbos_surrogate_default_cfg": ([P], I),
        "pivbos_surrogate_train": ([P, I, P, P, P, P], I),
        "pivbos_surrogate_render": ([P, P, P, P], I),
        "pivbos_surrogate_render_range": ([P, P, I64, P, P], I),
        "pivbos_surrogate_sensor": ([P, P, P, I64, P, P, P, P], I),
        "pivbos_surrogate_report_get": ([P, P], I),
        "pivbos_surrogate_destroy": ([P], None),
        "pivbos_bos_displacements": ([P, P, P, I64, I32, U64, U32, I, D, P, P, P, P], I),
        "pivbos_bos_displacements_range": ([P, P, P, I64, I64, I32, U64, U32, I, D, P, P, P, P], I),
        "pivbos_bos_theory": ([P, P, P, I64, P, P], I),
        "pivbos_regrid_bilinear": ([P, P, I64, I, I, D, D, D, D, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()
EXPORTED = ("pivbos_medium_create", "pivbos_medium_refill", "pivbos_medium_destroy", "pivbos_optics_create",
            "pivbos_optics_destroy", "pivbos_render", "pivbos_trace_exit_states", "pivbos_image_finalize",
            "pivbos_sync", "pivbos_last_error", "pivbos_timing_enable", "pivbos_timing_reset",
            "pivbos_timing_read", "pivbos_version", "pivbos_kernel_launches", "pivbos_render_noalloc",
            "pivbos_default_tuning", "pivbos_batch_create", "pivbos_batch_render", "pivbos_batch_destroy",
            "pivbos_autotune", "pivbos_render_range",
            "pivbos_surrogate_default_cfg", "pivbos_surrogate_train", "pivbos_surrogate_render",
            "pivbos_surrogate_render_range",
            "pivbos_surrogate_sensor", "pivbos_surrogate_report_get", "pivbos_surrogate_destroy",
            "pivbos_bos_displacements", "pivbos_bos_displacements_range", "pivbos_bos_theory", "pivbos_regrid_bilinear", "pivbos_optics_tilt_sensor",
            "pivbos_mie", "pivbos_optics_radiance", "pivbos_advect_sources", "pivbos_image_u16",
            "pivbos_selftest_wait_timeout")
TESTING_EXPORTED = ("pivbos_mlp_forward", "pivbos_mlp_train_forward", "pivbos_mlp_loss_grad",
                    "pivbos_mlp_adam_steps", "pivbos_surrogate_net_apply", "pivbos_probe_l1_bandwidth",
                    "pivbos_plan_bins")
MLP_PARAMS = 52228
NOALLOC_MAX_SOURCES = 1 << 17


def lib():
    return _lib


_tlib = None


def testing_lib():
    """libpivbos_testing.so (include/pivbos_testing.h): the checking and
    measurement hooks, loaded on first use."""
    global _tlib
    if _tlib is None:
        if not os.path.exists(TESTING_LIB_PATH):
            raise ImportError("libpivbos_testing.so is not built")
        T = ctypes.CDLL(TESTING_LIB_PATH)
        P, I, D, I32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int32
        sig = {
            "pivbos_mlp_forward": ([P, P, I32, P], I),
            "pivbos_mlp_train_forward": ([P, P, I32, P], I),
            "pivbos_mlp_loss_grad": ([P, P, P, I32, P, P], I),
            "pivbos_mlp_adam_steps": ([P, P, P, P, I32, I32, P, P], I),
            "pivbos_surrogate_net_apply": ([P, P, P, P, I32, P], I),
            "pivbos_probe_l1_bandwidth": ([ctypes.POINTER(D)], I),
            "pivbos_plan_bins": ([P, P, P, P, I32, I32, D, I32, I32, P, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(T, name)
            f.argtypes = args
            f.restype = res
        _tlib = T
    return _tlib


def _check(st):
    if st != OK:
        raise PivbosError(st, _lib.pivbos_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _addr(buf):
    """(address, on_device) of a CUDA tensor or a C-contiguous numpy array."""
    if buf is None:
        return None, 0
    if hasattr(buf, "data_ptr"):
        if buf.is_cuda:
            if not buf.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(buf.data_ptr()), 1
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(buf.data_ptr()), 0
    if not buf.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(buf.ctypes.data), 0


# ---------------------------------------------------------------------------
# C-named entry points (same names and argument order as include/pivbos.h)
# ---------------------------------------------------------------------------
def pivbos_medium_create(rho, nx, ny, nz, origin, spacing, K_GD, stream=None):
    p, on_dev = _addr(rho)
    o = (ctypes.c_double * 3)(*origin)
    h = (ctypes.c_double * 3)(*spacing)
    out = ctypes.c_void_p()
    _check(_lib.pivbos_medium_create(p, on_dev, nx, ny, nz, o, h, K_GD, _stream(stream), ctypes.byref(out)))
    return out


def pivbos_medium_refill(m, rho, stream=None):
    p, on_dev = _addr(rho)
    _check(_lib.pivbos_medium_refill(m, p, on_dev, _stream(stream)))


def pivbos_medium_destroy(m):
    _lib.pivbos_medium_destroy(m)


def pivbos_optics_create(surfaces, n_object, aim_z, aim_radius, f_number, magnification, wavelength,
                         dtau_rule, sensor_z, pixel_pitch, width, height):
    n = len(surfaces)
    arr = (pivbos_surface * max(n, 1))()
    for i, s in enumerate(surfaces):
        arr[i] = pivbos_surface(int(s[0]), 0, *[float(v) for v in s[1:6]])
    out = ctypes.c_void_p()
    _check(_lib.pivbos_optics_create(arr if n else None, n, n_object, aim_z, aim_radius, f_number, magnification,
                                     wavelength, dtau_rule, sensor_z, pixel_pitch, width, height,
                                     ctypes.byref(out)))
    return out


def pivbos_optics_tilt_sensor(o, tilt_x, tilt_y):
    """A new optics handle: `o` with its sensor turned about its centre."""
    out = ctypes.c_void_p()
    _check(_lib.pivbos_optics_tilt_sensor(o, tilt_x, tilt_y, ctypes.byref(out)))
    return out


def pivbos_mie(diameter, wavelength, n_medium, m_re, m_im=0.0, n_angles=1801):
    """Mie scattering of a sphere on the GPU: (s12 [n, 2] of |S1|^2, |S2|^2,
    {q_ext, q_sca, re_s0, terms})."""
    s12 = np.zeros((n_angles, 2))
    q = np.zeros(4)
    _check(_lib.pivbos_mie(diameter, wavelength, n_medium, m_re, m_im, n_angles, s12.ctypes.data, q.ctypes.data))
    return s12, {"q_ext": q[0], "q_sca": q[1], "re_s0": q[2], "terms": int(q[3])}


def pivbos_optics_radiance(o, laser_dir, polarisation, s12):
    """A new optics handle: `o` with Mie radiance weights per ray."""
    s12 = np.ascontiguousarray(s12, dtype=np.float64).reshape(-1, 2)
    L = (ctypes.c_double * 3)(*laser_dir)
    pol = (ctypes.c_double * 3)(*polarisation) if polarisation is not None else None
    out = ctypes.c_void_p()
    _check(_lib.pivbos_optics_radiance(o, L, pol, s12.ctypes.data, len(s12), ctypes.byref(out)))
    return out


def pivbos_optics_destroy(o):
    _lib.pivbos_optics_destroy(o)


def pivbos_render(m, o, sources, n_sources, rays_per_source, seed, frame, integrator, step, image,
                  stats=None, stream=None):
    sp, s_dev = _addr(sources)
    ip, i_dev = _addr(image)
    st_p, _ = _addr(stats)
    _check(_lib.pivbos_render(m, o, sp, n_sources, s_dev, rays_per_source, seed, frame, integrator, step,
                              ip, i_dev, st_p, _stream(stream)))


def pivbos_render_range(m, o, sources, n_sources, first_source, rays_per_source, seed, frame, integrator, step,
                        image, stats=None, stream=None):
    sp, s_dev = _addr(sources)
    ip, i_dev = _addr(image)
    st_p, _ = _addr(stats)
    _check(_lib.pivbos_render_range(m, o, sp, n_sources, first_source, s_dev, rays_per_source, seed, frame,
                                    integrator, step, ip, i_dev, st_p, _stream(stream)))


def pivbos_render_noalloc(m, o, sources, n_sources, rays_per_source, seed, frame, integrator, step, image,
                          stats=None, stream=None):
    """pivbos_render without any allocation: sources, image (and stats) must be
    CUDA tensors; scratch comes from a fixed device array in the library."""
    sp, _ = _addr(sources)
    ip, _ = _addr(image)
    st_p, _ = _addr(stats)
    _check(_lib.pivbos_render_noalloc(m, o, sp, n_sources, rays_per_source, seed, frame, integrator, step,
                                      ip, st_p, _stream(stream)))


def frame_desc(medium, optics, sources, n_sources, rays_per_source, frame, seed, step, image, stats=None):
    return pivbos_frame_desc(medium, optics, ctypes.c_void_p(sources.data_ptr()), n_sources, rays_per_source,
                             frame, seed, step, ctypes.c_void_p(image.data_ptr()),
                             ctypes.c_void_p(stats.data_ptr()) if stats is not None else None)


def pivbos_default_tuning():
    t = pivbos_tuning()
    _check(_lib.pivbos_default_tuning(ctypes.byref(t)))
    return t


def pivbos_batch_create(descs, integrator, tuning=None):
    arr = (pivbos_frame_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(_lib.pivbos_batch_create(arr, len(descs), integrator, ctypes.byref(tuning) if tuning else None,
                                    ctypes.byref(out)))
    return out


def pivbos_batch_render(batch, stream=None):
    _check(_lib.pivbos_batch_render(batch, _stream(stream)))


def pivbos_batch_destroy(batch):
    _lib.pivbos_batch_destroy(batch)


def pivbos_autotune(desc, integrator, tol_px, n_sample_rays, stream=None):
    step = ctypes.c_double()
    t = pivbos_tuning()
    _check(_lib.pivbos_autotune(ctypes.byref(desc), integrator, tol_px, n_sample_rays, ctypes.byref(step),
                                ctypes.byref(t), _stream(stream)))
    return step.value, t


def pivbos_mlp_forward(params, x):
    """The inference forward (testing library)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros((x.shape[0], 4), dtype=np.float32)
    _check(testing_lib().pivbos_mlp_forward(params.ctypes.data, x.ctypes.data, x.shape[0], y.ctypes.data))
    return y


def pivbos_mlp_train_forward(params, x):
    """The training forward (testing library)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros((x.shape[0], 4), dtype=np.float32)
    _check(testing_lib().pivbos_mlp_train_forward(params.ctypes.data, x.ctypes.data, x.shape[0], y.ctypes.data))
    return y


def pivbos_mlp_loss_grad(params, x, t):
    """Training forward and backward of the mean squared error (testing library)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(testing_lib().pivbos_mlp_loss_grad(params.ctypes.data, x.ctypes.data, t.ctypes.data, x.shape[0],
                                              g.ctypes.data, ctypes.byref(loss)))
    return loss.value, g


def pivbos_mlp_adam_steps(params, m, v, grads, t0, lr):
    """Adam steps of the training kernel on host state (testing library):
    returns (params, m, v, bf16 weight bits)."""
    params = np.array(params, dtype=np.float32)
    m = np.array(m, dtype=np.float32)
    v = np.array(v, dtype=np.float32)
    grads = np.ascontiguousarray(grads, dtype=np.float32).reshape(-1, MLP_PARAMS)
    lr = np.ascontiguousarray(lr, dtype=np.float32)
    wbf = np.zeros(51712, dtype=np.uint16)
    _check(testing_lib().pivbos_mlp_adam_steps(params.ctypes.data, m.ctypes.data, v.ctypes.data, grads.ctypes.data,
                                               grads.shape[0], t0, lr.ctypes.data, wbf.ctypes.data))
    return params, m, v, wbf


def pivbos_surrogate_net_apply(params, x, b, t_scale):
    """The surrogate render's network kernel: r = b + MLP(x) * t_scale (testing library)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    ts = np.ascontiguousarray(t_scale, dtype=np.float32)
    r = np.zeros((x.shape[0], 4), dtype=np.float32)
    _check(testing_lib().pivbos_surrogate_net_apply(params.ctypes.data, x.ctypes.data, b.ctypes.data, ts.ctypes.data,
                                                    x.shape[0], r.ctypes.data))
    return r


def pivbos_surrogate_default_cfg():
    c = pivbos_surrogate_cfg()
    _check(_lib.pivbos_surrogate_default_cfg(ctypes.byref(c)))
    return c


def pivbos_surrogate_train(desc, integrator, cfg=None, stream=None):
    """Train a surrogate on a frame; returns (handle, report)."""
    out = ctypes.c_void_p()
    rep = pivbos_surrogate_report()
    _check(_lib.pivbos_surrogate_train(ctypes.byref(desc), integrator, ctypes.byref(cfg) if cfg else None,
                                       ctypes.byref(out), ctypes.byref(rep), _stream(stream)))
    return out, rep


def pivbos_surrogate_render(sg, desc, count_fallback=False, stream=None):
    """Render a frame with the surrogate; returns the number of plain-traced
    rays when count_fallback (the call then synchronises), else None."""
    n = ctypes.c_int64()
    _check(_lib.pivbos_surrogate_render(sg, ctypes.byref(desc), ctypes.byref(n) if count_fallback else None,
                                        _stream(stream)))
    return n.value if count_fallback else None


def pivbos_surrogate_render_range(sg, desc, first_source, count_fallback=False, stream=None):
    """The surrogate render of the frame's sources as the range starting at
    global source index first_source (sharding one image)."""
    n = ctypes.c_int64()
    _check(_lib.pivbos_surrogate_render_range(sg, ctypes.byref(desc), first_source,
                                              ctypes.byref(n) if count_fallback else None, _stream(stream)))
    return n.value if count_fallback else None


def pivbos_surrogate_sensor(sg, desc, ray_ids, sensor_xy, flags, status, stream=None):
    rp, _ = _addr(ray_ids)
    _check(_lib.pivbos_surrogate_sensor(sg, ctypes.byref(desc), rp, int(ray_ids.numel()), _addr(sensor_xy)[0],
                                        _addr(flags)[0], _addr(status)[0], _stream(stream)))


def pivbos_surrogate_report_get(sg):
    rep = pivbos_surrogate_report()
    _check(_lib.pivbos_surrogate_report_get(sg, ctypes.byref(rep)))
    return rep


def pivbos_surrogate_destroy(sg):
    _lib.pivbos_surrogate_destroy(sg)


def pivbos_trace_exit_states(m, o, sources, n_sources, rays_per_source, seed, frame, integrator, step,
                             ray_ids, n_rays, out, stream=None):
    sp, s_dev = _addr(sources)
    rp, _ = _addr(ray_ids)
    op, _ = _addr(out)
    _check(_lib.pivbos_trace_exit_states(m, o, sp, n_sources, s_dev, rays_per_source, seed, frame,
                                         integrator, step, rp, n_rays, op, _stream(stream)))


def pivbos_bos_displacements(m, o, dots, n_dots, rays_per_dot, seed, frame, integrator, step, centroid=None,
                             displacement=None, n_pairs=None, stream=None):
    """Sec. 4: per-dot mean sensor position without the medium, mean
    displacement (with - without) and pair count; CUDA tensors."""
    _check(_lib.pivbos_bos_displacements(m, o, _addr(dots)[0], n_dots, rays_per_dot, seed, frame, integrator, step,
                                         _addr(centroid)[0], _addr(displacement)[0], _addr(n_pairs)[0],
                                         _stream(stream)))


def pivbos_bos_displacements_range(m, o, dots, n_dots, first_dot, rays_per_dot, seed, frame, integrator, step,
                                   centroid=None, displacement=None, n_pairs=None, stream=None):
    """pivbos_bos_displacements for dots [first_dot, first_dot + n_dots) of a larger set."""
    _check(_lib.pivbos_bos_displacements_range(m, o, _addr(dots)[0], n_dots, first_dot, rays_per_dot, seed, frame,
                                               integrator, step, _addr(centroid)[0], _addr(displacement)[0],
                                               _addr(n_pairs)[0], _stream(stream)))


def pivbos_bos_theory(m, o, dots, n_dots, displacement, stream=None):
    """Eq. 9 per dot (pixels) along the dot's chief ray; CUDA tensors."""
    _check(_lib.pivbos_bos_theory(m, o, _addr(dots)[0], n_dots, _addr(displacement)[0], _stream(stream)))


def pivbos_regrid_bilinear(xy, values, n, grid_w, grid_h, x0, y0, cell, min_weight, out, weight=None,
                           stream=None):
    """Scattered values onto a regular grid by bilinear weights; CUDA tensors."""
    _check(_lib.pivbos_regrid_bilinear(_addr(xy)[0], _addr(values)[0], n, grid_w, grid_h, x0, y0, cell, min_weight,
                                       _addr(out)[0], _addr(weight)[0], _stream(stream)))


def pivbos_advect_sources(sources, n_sources, velocity, origin, spacing, dt, out, stream=None):
    """Second frame of an image pair: sources moved by the velocity field
    (CUDA tensor [nz, ny, nx, 3]) over dt; CUDA tensors."""
    nz, ny, nx = (int(v) for v in velocity.shape[:3])
    o = (ctypes.c_double * 3)(*origin)
    h = (ctypes.c_double * 3)(*spacing)
    _check(_lib.pivbos_advect_sources(_addr(sources)[0], n_sources, _addr(velocity)[0], nx, ny, nz, o, h, dt,
                                      _addr(out)[0], _stream(stream)))


def pivbos_image_u16(image, n_pixels, full_scale, out, stream=None):
    """16-bit image (full_scale rays read 65535); CUDA tensors (out uint16)."""
    _check(_lib.pivbos_image_u16(_addr(image)[0], n_pixels, full_scale, _addr(out)[0], _stream(stream)))


def pivbos_probe_l1_bandwidth():
    """Measured L1 bandwidth for coalesced 16-byte loads (bytes/s; testing library)."""
    v = ctypes.c_double()
    _check(testing_lib().pivbos_probe_l1_bandwidth(ctypes.byref(v)))
    return v.value


def pivbos_plan_bins(err2n, err2p, steps, counts, min_count, budget2, segments, with_net=True):
    """The surrogate's per-bin plan (testing library, host only): returns
    (served bool [n], network bool [n], {err2, steps, rays, net_rays, cost})."""
    err2n = np.ascontiguousarray(err2n, dtype=np.float64)
    err2p = np.ascontiguousarray(err2p, dtype=np.float64)
    steps = np.ascontiguousarray(steps, dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    n = counts.size
    served = np.zeros(max(n // 32, 1), dtype=np.uint32)
    network = np.zeros_like(served)
    out = np.zeros(5)
    _check(testing_lib().pivbos_plan_bins(err2n.ctypes.data, err2p.ctypes.data, steps.ctypes.data, counts.ctypes.data,
                                          n, min_count, float(budget2), segments, 1 if with_net else 0,
                                          served.ctypes.data, network.ctypes.data, out.ctypes.data))
    bits = lambda w: ((w[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1).astype(bool)
    return bits(served), bits(network), dict(zip(("err2", "steps", "rays", "net_rays", "cost"), out))


def pivbos_selftest_wait_timeout(polls, stream=None):
    """Enqueue the bounded-wait self-test (the next pivbos_sync reports the timeout)."""
    _check(_lib.pivbos_selftest_wait_timeout(polls, _stream(stream)))


def pivbos_image_finalize(image, n_pixels, out, stream=None):
    ip, _ = _addr(image)
    op, _ = _addr(out)
    _check(_lib.pivbos_image_finalize(ip, n_pixels, op, _stream(stream)))


def pivbos_sync(stream=None):
    _check(_lib.pivbos_sync(_stream(stream)))


def pivbos_last_error():
    return _lib.pivbos_last_error().decode()


def pivbos_timing_enable(on=True):
    _check(_lib.pivbos_timing_enable(1 if on else 0))


def pivbos_timing_reset():
    _check(_lib.pivbos_timing_reset())


def pivbos_timing_read(prefix):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.pivbos_timing_read(prefix.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def pivbos_kernel_launches():
    return int(_lib.pivbos_kernel_launches())


def pivbos_version():
    return _lib.pivbos_version().decode()


# ---------------------------------------------------------------------------
# RAII helpers over scenes.Frame descriptions
# ---------------------------------------------------------------------------
class Medium:
    def __init__(self, scene_medium, rho=None, stream=None):
        r = scene_medium.rho if rho is None else rho
        if not hasattr(r, "data_ptr"):
            r = np.ascontiguousarray(r, dtype=np.float32)
        nx, ny, nz = scene_medium.dims
        self.h = pivbos_medium_create(r, nx, ny, nz, scene_medium.origin, scene_medium.spacing,
                                      scene_medium.K, stream)

    def refill(self, rho, stream=None):
        pivbos_medium_refill(self.h, rho, stream)

    def close(self):
        if getattr(self, "h", None):
            pivbos_medium_destroy(self.h)
            self.h = None

    __del__ = close


class Optics:
    def __init__(self, so):
        self.W, self.H = so.width, so.height
        self.h = pivbos_optics_create([s.as_row() for s in so.surfaces], so.n_object, so.aim_z, so.aim_r,
                                      so.f_number, so.magnification, so.wavelength, so.dtau_rule,
                                      so.sensor_z, so.pitch, so.width, so.height)
        tx, ty = getattr(so, "sensor_tilt_x", 0.0), getattr(so, "sensor_tilt_y", 0.0)
        if tx != 0.0 or ty != 0.0:
            flat = self.h
            self.h = pivbos_optics_tilt_sensor(flat, tx, ty)
            pivbos_optics_destroy(flat)
        mie = getattr(so, "mie", None)
        if mie is not None:
            s12, _ = pivbos_mie(mie.diameter, mie.wavelength, mie.n_medium, mie.m_re, mie.m_im, mie.n_angles)
            plain = self.h
            self.h = pivbos_optics_radiance(plain, mie.laser_dir, mie.polarisation, s12)
            pivbos_optics_destroy(plain)

    def close(self):
        if getattr(self, "h", None):
            pivbos_optics_destroy(self.h)
            self.h = None

    __del__ = close
