"""Shared helpers of the GPU parity tests: run a scenes.Frame through the CUDA
library (via the C-ABI binding) and through the oracle, and compare."""
import json
import math
import os

import numpy as np

import oracle
from paper_1812_05902_gb300 import scenes

TOL_PX = 1e-5       # sensor position, pixels
TOL_RAD = 1e-6      # direction, radians
TOL_IMG = 1e-4      # image, relative L2
# optical path inside the box (m): the GPU's last, clipped step is an FP32
# parameter (~1e-11 m of path); the integral is summed in double-float
TOL_OPL = 1e-10


def torch_cuda():
    import torch
    return torch


def gpu_handles(frame):
    from paper_1812_05902_gb300 import pivbos as P
    med = P.Medium(frame.medium) if frame.medium is not None else None
    opt = P.Optics(frame.optics)
    return med, opt


def gpu_states(frame, ids, handles=None):
    torch = torch_cuda()
    from paper_1812_05902_gb300 import pivbos as P
    med, opt = handles if handles is not None else gpu_handles(frame)
    src = torch.tensor(frame.sources, dtype=torch.float64, device="cuda")
    ids_t = torch.tensor(np.asarray(ids, dtype=np.int64), device="cuda")
    out = torch.empty(len(ids) * P.RAY_STATE.itemsize, dtype=torch.uint8, device="cuda")
    P.pivbos_trace_exit_states(med.h if med else None, opt.h, src, len(frame.sources), frame.rays_per_source,
                               frame.seed, frame.frame_index, frame.integrator, frame.step, ids_t, len(ids), out)
    P.pivbos_sync()
    return np.frombuffer(out.cpu().numpy().tobytes(), dtype=P.RAY_STATE)


def oracle_states(frame, ids):
    med = oracle.Medium.from_scene(frame.medium) if frame.medium is not None else None
    opt = oracle.Optics.from_scene(frame.optics)
    return oracle.trace_many(med, opt, frame.sources, frame.rays_per_source, np.asarray(ids, dtype=np.int64),
                             frame.seed, frame.frame_index, frame.integrator, frame.step)


def gpu_render(frame, image=None, handles=None, stats=True):
    torch = torch_cuda()
    from paper_1812_05902_gb300 import pivbos as P
    med, opt = handles if handles is not None else gpu_handles(frame)
    W, H = frame.optics.width, frame.optics.height
    if image is None:
        image = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda") if stats else None
    src = torch.tensor(frame.sources, dtype=torch.float64, device="cuda")
    P.pivbos_render(med.h if med else None, opt.h, src, len(frame.sources), frame.rays_per_source, frame.seed,
                    frame.frame_index, frame.integrator, frame.step, image, st)
    P.pivbos_sync()
    return image.cpu().numpy(), (st.cpu().numpy() if stats else None)


def angles(d):
    return np.stack([np.arctan2(d[:, 0], d[:, 2]), np.arctan2(d[:, 1], d[:, 2])], axis=1)


def _log(kind, res):
    path = os.environ.get("PIVBOS_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"kind": kind, **res}) + "\n")


def compare_states(g, o, pitch, vol_scale, max_status_mismatch_frac=2e-4, label="", exact=False):
    """g, o: RAY_STATE arrays for the same rays.  vol_scale: metres in the
    volume per pixel on the sensor (the tolerance on the exit line is
    TOL_PX * vol_scale).  Computes every error, then asserts; returns them.

    The GPU takes its aperture, clear-radius, hemisphere and TIR decisions on
    the FP32 leading parts of double-float values, the oracle in FP64, so a
    ray within ~1e-7 (relative) of such an edge may be decided differently:
    about 1e-7 of the rays of a render.  Samples may therefore differ in
    max(2, max_status_mismatch_frac * n) statuses and in one step (the
    final, clipped step's decision); with exact=True (the small scenes
    compared ray by ray) every status and every step count must agree."""
    n = len(o)
    same = g["status"] == o["status"]
    res = {"label": label, "n": n, "status_mismatch": int(np.sum(~same))}
    ga, oa = angles(g["vol_dir"]), angles(o["vol_dir"])
    res["vol_angle"] = float(np.max(np.abs(ga - oa))) if n else 0.0
    z = o["vol_pos"][:, 2]
    t = (z - g["vol_pos"][:, 2]) / g["vol_dir"][:, 2]
    xg = g["vol_pos"][:, :2] + t[:, None] * g["vol_dir"][:, :2]
    res["vol_line_m"] = float(np.max(np.abs(xg - o["vol_pos"][:, :2]))) if n else 0.0
    res["vol_line_tol_m"] = TOL_PX * vol_scale
    both = same & (o["status"] == oracle.REACHED)
    res["reached"] = int(np.sum(both))
    if np.any(both):
        res["sensor_px"] = float(np.max(np.abs(g["sensor_xy"][both] - o["sensor_xy"][both])))
        res["sensor_angle"] = float(np.max(np.abs(angles(g["sensor_dir"][both]) - angles(o["sensor_dir"][both]))))
    steps_same = same & (o["steps"] > 0)
    if np.any(steps_same):
        res["steps_diff"] = int(np.max(np.abs(g["steps"][steps_same] - o["steps"][steps_same])))
    if "opl" in (g.dtype.names or ()) and "opl" in (o.dtype.names or ()):
        # rays whose step counts agree (a clipped last step decided the other
        # way changes the path by up to a step)
        ok = same & (g["steps"] == o["steps"])
        res["opl_m"] = float(np.max(np.abs(g["opl"][ok] - o["opl"][ok]))) if np.any(ok) else 0.0
    _log("states", res)
    if exact:
        assert res["status_mismatch"] == 0, res
        assert np.array_equal(g["steps"], o["steps"]), res
    assert res["status_mismatch"] <= max(2, int(max_status_mismatch_frac * n)), res
    assert res["vol_angle"] <= TOL_RAD, res
    assert res["vol_line_m"] <= res["vol_line_tol_m"], res
    if "sensor_px" in res:
        assert res["sensor_px"] <= TOL_PX, res
        assert res["sensor_angle"] <= TOL_RAD, res
    if "steps_diff" in res:
        assert res["steps_diff"] <= 1, res
    if "opl_m" in res:
        assert res["opl_m"] <= TOL_OPL, res
    return res


def compare_images(img_g, img_o, st_g, st_o, frame, label="", exact_status=False, n=None):
    """Images of the same rays: exact 2^32-per-ray totals on both sides, the
    per-status counts (equal with exact_status, else within the edge-decision
    allowance of compare_states) and relative L2 <= TOL_IMG.  n: the rays
    rendered (default: the frame's)."""
    n = frame.n_rays if n is None else n
    a = img_g.astype(np.float64)
    b = img_o.astype(np.float64)
    rel = math.sqrt(np.sum((a - b) ** 2)) / max(math.sqrt(np.sum(b * b)), 1.0)
    _log("image", {"label": label, "n": n, "rel_l2": rel, "reached_gpu": int(st_g[0]), "reached_oracle": int(st_o[0])})
    assert st_g.sum() == n and st_o.sum() == n
    # exact totals on both sides: every ray that reaches adds 2^32
    assert img_g.sum() == int(st_g[0]) << 32
    assert img_o.sum() == int(st_o[0]) << 32
    if exact_status:
        assert np.array_equal(st_g, st_o), (st_g, st_o)
    assert np.all(np.abs(st_g - st_o) <= max(2, 2e-4 * n)), (st_g, st_o)
    assert rel <= TOL_IMG, rel
    return rel


def vol_scale(frame):
    """metres at the volume per sensor pixel for the exit-line tolerance: a
    lateral shift of the exit line by dx moves the image by about M dx."""
    return frame.optics.pitch / frame.optics.magnification
