"""Benchmark: rays/s traced to the sensor on one GB300 (and N by torchrun).

Default workload (config C4, Tomo-PIV scale): 1e5 particles inside a
100x100x30 mm k^-5/3 turbulence field on a 256^3 grid, 1e4 rays each (1e9
rays per image), RK4 with 0.2 mm steps, the thick biconvex lens at f/4 and
M = 0.2 focused on the volume centre, 2048x2048 sensor.  The metric compares
the plain tracer with the surrogate path (learned ray map + plain fallback)
at <= 0.01 px RMS sensor error against the oracle, so the line times three
arms on the same image:
  * plain       -- Morton sort, the fused trace/optics/deposit kernel,
                   finalisation;
  * surrogate   -- the trained ray map (first-order projection plus the
                   tcgen05 network's correction) for rays in served bins,
                   the plain tracer for the rest (the line's value);
  * projection  -- the same without the network (what the learned part is
                   measured against).
A step is one image of an arm.  The medium (Eq. 1 and the node gradients)
is built once per density field and the surrogate trained once per field:
both are outside the timed steps and reported with the images per field at
which the surrogate breaks even.  Inputs are resident on the GPU when the
timed region starts; L2 is flushed between timed steps.  The e2e figures run
the same steps with host buffers (sources in, image out).  The line also
reports the RMS sensor error of both surrogate arms against the plain tracer
(1e6 rays) and against the oracle (2e5 rays), and carries the C1 (PIV
uniform medium), Table 1 (Sec. 4 BOS experiment) and 16-bit conversion
figures as sub-objects.

With N ranks (torchrun) the image's sources are split into N contiguous
ranges; every rank renders its range (global ray indices, so the sum is the
single-GPU image bit for bit) and one NCCL all-reduce sums the int64 images:
strong scaling of one image.

--workload c0/c1/c2 time the plain tracer alone on that config, c3 the
64-frame batch, table1 the Sec. 4 experiment; --surrogate --workload c2 the
surrogate on the C2 BOS field.

--impl reference times the CPU oracle (the paper's method written plainly in
FP64 C) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1812_05902_gb300 import scenes  # noqa: E402

WORKLOAD_NAMES = {
    "c0": "BOS linear-gradient slab, 32^3 grid, 64x64 dots x 100 rays, Euler 0.1 mm, ideal lens f/8 M=0.1, 256^2",
    "c1": "PIV uniform medium n=1.000277, 1e4 particles x 1e4 rays in a 50x50x1 mm sheet, thick biconvex lens "
          "R=+-0.1 m d=10 mm n=1.5 f/4 M=0.2, sheet -2 mm and +2 mm from focus (2 images), 1024^2 17 um",
    "c2": "BOS k^-5/3 turbulence 256^3 over 0.1 m, 1e5 dots x 1e3 rays, RK4 0.2 mm, thick lens f/8 M=0.1, 1024^2",
    "c4": "Tomo-PIV 1e5 particles x 1e4 rays in a 100x100x30 mm 256^3 turbulence field, RK4 0.2 mm, thick lens "
          "f/4 M=0.2, 2048^2",
    "c3": "64 frames in one persistent graph-replayed launch: 10^U(3,5) sources, grids 64^3-256^3, shock / "
          "gradient / turbulence in rotation, 10^U(3,4) rays/source, RK4 0.2 mm, thick lens f/8 M=0.1, 1024^2",
    "table1": "BOS experiment of Sec. 4 with the Table 1 geometry: z-stacked 2-D k^-5/3 density slice 256^2 over "
              "32x32x10 mm, Z_D 0.25 m, Z_A 0.75 m, f 105 mm f/11, 512^2 sensor 10 um, 5,120 dots x 1e4 rays, "
              "RK4 0.1 mm; per-dot mean displacement (every ray traced with and without the medium), Eq. 9 "
              "theory and the bilinear 16 px grid map",
}
METRIC = "rays/s traced to sensor at 1 GB300 (plain vs surrogate at ≤0.01 px RMS error)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


_GRID = [None]   # --grid: a smaller C4 field for profiling captures only


def _frames(workload, scale=1.0):
    """The workload's frames; scale < 1 shrinks source and ray counts (used
    only for profiling captures, never for a reported number)."""
    if workload == "c1":
        return scenes.c1(scale=scale)
    if workload == "c0":
        return scenes.c0(scale=scale)
    if workload == "c2":
        return scenes.c2(scale=scale)
    if workload == "c4":
        return scenes.c4(scale=scale, grid=_GRID[0])
    if workload == "c3":
        return scenes.c3(scale=scale)
    if workload == "table1":
        return scenes.table1(scale=scale)
    raise SystemExit("unknown workload %s" % workload)


# ----------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ----------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# roofline of the dominant kernel
# ----------------------------------------------------------------------------
# The render kernel is bound by instruction issue on the FP32/INT32 pipes
# (no FP64 left on the path, no tensor-core work, DRAM and L2 lightly used),
# so its roofline is the SM issue rate: 152 SMs x 128 lanes x clock.  The
# algorithmic work of one ray is a static count of FP32/INT32 lane operations
# of the double-float and FP32 formulation, per stage:
#   ray generation (Philox4x64-10, lens point, direction)  710
#   volume entry + exit to the optics                       470
#   each integration step: RK4 430, first-order 160
#   per surface: sphere 530, stop/plane/ideal lens 80
#   sensor plane 125, spot deposit 450, bookkeeping 40
OPS_RAY_BASE = 710 + 470 + 125 + 450 + 40
OPS_STEP = {scenes.RK4: 430.0, scenes.EULER: 160.0}
OPS_SURF = {scenes.SPHERE: 530.0, scenes.PLANE: 80.0, scenes.IDEAL_THIN: 80.0, scenes.STOP: 80.0,
            scenes.MIRROR: 530.0, scenes.LENS_ARRAY: 120.0}
# extended optics: a flat mirror is a clear-radius test; a turned sensor's
# general plane intersection costs ~150 more than the square sensor; a Mie
# radiance weight (acos, table lookup, scattering-plane projection) ~70
OPS_FLAT_MIRROR = 80.0
OPS_TILT = 150.0
OPS_MIE = 70.0
ISSUE_LANES_PER_SM = 128
N_SM = 152


# the sources each profiled kernel is compiled from
KERNEL_SOURCES = {
    "render": ("render.cu", "render_chunk.cuh", "trace.cuh", "df64.cuh", "common.cuh"),
    "surrogate": ("surrogate.cu", "surrogate_kernels.cuh", "mlp_tc.cuh", "umma.cuh", "mlp.cuh", "trace.cuh",
                  "df64.cuh", "common.cuh"),
    "bos": ("bos.cu", "trace.cuh", "df64.cuh", "common.cuh"),
}


def kernel_source_hash(kind="render"):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1812_05902_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(record, kind="render", rays_per_cta=None, scale_to_rays=None):
    """DRAM bytes per launch from a committed ncu record (profiles/<record>.json),
    or None when the kernel's sources changed since it was taken, or when the
    record names a launch geometry (rays per CTA) other than the current one.
    A record taken on a smaller launch (its rays_per_launch) is scaled to
    scale_to_rays rays in proportion (the field and image parts of the
    traffic do not grow with the rays, so the scaled figure is an upper
    bound), unless the record says its traffic is the launch's fixed part
    (scales_with_rays false: used as it is)."""
    try:
        with open(os.path.join(ROOT, "profiles", record + ".json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash(kind):
        return None
    if rays_per_cta is not None and rec.get("rays_per_cta", rays_per_cta) != rays_per_cta:
        return None
    b = float(rec["dram_bytes_read"] + rec["dram_bytes_write"])
    if scale_to_rays and rec.get("rays_per_launch") and rec.get("scales_with_rays", True):
        b *= scale_to_rays / float(rec["rays_per_launch"])
    return int(b)


def render_rays_per_cta(frames, step_integrator_dense):
    """Rays per CTA the library's render uses (its rule: PIVBOS_RAYS_PER_CTA if
    set, else 2048 in a dense medium, 256 otherwise)."""
    v = os.environ.get("PIVBOS_RAYS_PER_CTA")
    if v and v.isdigit() and 256 <= int(v) <= (1 << 20):
        return int(v)
    return 2048 if step_integrator_dense else 256


def ops_per_ray(frame, mean_steps):
    o = frame.optics
    surf = sum(OPS_FLAT_MIRROR if (s.type == scenes.MIRROR and s.R == 0.0) else OPS_SURF[s.type]
               for s in o.surfaces)
    extra = (OPS_TILT if (o.sensor_tilt_x or o.sensor_tilt_y) else 0.0) + (OPS_MIE if o.mie is not None else 0.0)
    return OPS_RAY_BASE + surf + extra + OPS_STEP[frame.integrator] * mean_steps


OPTICS_VARIANTS = ("plain", "mie", "plenoptic", "tilted", "mirror")


def apply_optics_variant(frames, variant):
    """The workload's camera with an optical extension of Sec. 3.3-3.4 (a copy
    per frame): Mie radiance of a polarised laser, a lenslet array 0.5 mm
    before the sensor (plenoptic), a sensor turned by 0.05 / -0.03 rad, or a
    flat fold mirror before the stop."""
    import dataclasses
    if variant == "plain":
        return
    for fr in frames:
        o = fr.optics
        if variant == "mie":
            fr.optics = dataclasses.replace(o, mie=scenes.Mie())
        elif variant == "plenoptic":
            fr.optics = dataclasses.replace(o, surfaces=list(o.surfaces) + [
                scenes.Surface(scenes.LENS_ARRAY, o.sensor_z - 5e-4, R=1e-4, f=5e-4, clear_r=0.05)])
        elif variant == "tilted":
            fr.optics = dataclasses.replace(o, sensor_tilt_x=0.05, sensor_tilt_y=-0.03)
        elif variant == "mirror":
            fr.optics = dataclasses.replace(o, surfaces=[scenes.Surface(scenes.MIRROR, o.aim_z - 0.05, R=0.0,
                                                                        clear_r=0.2)] + list(o.surfaces))
        else:
            raise SystemExit("unknown optics variant %s" % variant)


def measure_image_u16(P, dev, n=16384 * 16384, reps=5):
    """HBM roofline of the 16-bit conversion on a 16384^2 image (2 GiB of
    int64 in, 0.5 GiB out): CUDA events over `reps` launches."""
    import torch
    img = torch.randint(0, 1 << 40, (n,), dtype=torch.int64, device=dev)
    out = torch.empty(n, dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        P.pivbos_image_u16(img, n, 100.0, out)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        P.pivbos_image_u16(img, n, 100.0, out)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / reps * 1e-3
    peaks, src_kind = _peaks()
    gbs = n * 10 / t / 1e9
    del img, out
    return {"kernel": "image_u16_kernel", "pixels": n, "ms_per_launch": round(t * 1e3, 3), "bound": "hbm",
            "achieved": round(gbs, 1), "unit": "GB/s", "peak": peaks.get("hbm_gbs", 6800.0),
            "frac": round(gbs / peaks.get("hbm_gbs", 6800.0), 4), "bytes_per_pixel": 10,
            "peak_source": "%s hbm_gbs" % src_kind}


# field gathers: 8 corners x 16 B per evaluation of D; RK4 evaluates 3 times per step
GATHER_BYTES_PER_EVAL = 8 * 16
EVALS_PER_STEP = {scenes.RK4: 3, scenes.EULER: 1}
L1_BYTES_PER_CLK_PER_SM = 128


_L1_PEAK = {}


def measured_l1_gbs(P):
    """The L1 data path's measured bandwidth for 16-byte loads (GB/s), from
    the library's probe; taken once per process, outside any timed region."""
    if "v" not in _L1_PEAK:
        try:
            _L1_PEAK["v"] = P.pivbos_probe_l1_bandwidth() / 1e9
        except Exception:
            _L1_PEAK["v"] = None
    return _L1_PEAK["v"]


def roofline(frames, mean_steps, render_ms, render_launches, sm_max_mhz, traffic=None, l1_gbs=None, ray_frac=1.0):
    """Issue and gather rooflines of a render launch (ray_frac: the share of
    a frame's rays one launch traces, for sharded images)."""
    if render_launches == 0:
        return None
    t = render_ms / render_launches * 1e-3
    rays = ray_frac * sum(f.n_rays for f in frames) / len(frames)
    ops = ray_frac * sum(ops_per_ray(f, ms) * f.n_rays for f, ms in zip(frames, mean_steps)) / len(frames)
    achieved = ops / t / 1e12
    clk = (sm_max_mhz or 2070.0) * 1e6
    peak = N_SM * ISSUE_LANES_PER_SM * clk / 1e12
    out = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
           "frac": round(achieved / peak, 4), "traffic": traffic,
           "kernel": "render_kernel", "op": "FP32/INT32 lane operation (1 per lane instruction)",
           "peak_source": "issue rate derived from 152 SMs x 128 lanes x max SM clock",
           "ops_per_ray": round(ops / rays, 1), "launch_ms": round(t * 1e3, 4), "rays_per_launch": int(rays)}
    if all(f.medium is not None for f in frames):
        # the same launch against the L1 data path, for the field gathers
        gbytes = ray_frac * sum(GATHER_BYTES_PER_EVAL * EVALS_PER_STEP[f.integrator] * ms * f.n_rays
                                for f, ms in zip(frames, mean_steps)) / len(frames)
        gpeak = N_SM * L1_BYTES_PER_CLK_PER_SM * clk / 1e9
        out["gather"] = {"bound": "l1", "achieved": round(gbytes / t / 1e9, 1), "peak": round(gpeak, 1),
                         "unit": "GB/s", "frac": round(gbytes / t / 1e9 / gpeak, 4),
                         "bytes_per_ray": round(gbytes / rays, 1),
                         "peak_source": "152 SMs x 128 B/clk L1 data path x max SM clock"}
        if l1_gbs:
            out["gather"].update({"peak_measured": round(l1_gbs, 1),
                                  "frac_measured": round(gbytes / t / 1e9 / l1_gbs, 4),
                                  "peak_measured_source": "pivbos_probe_l1_bandwidth: coalesced 16-byte loads "
                                                          "from an L1-resident 48 KB buffer on every SM"})
    return out


def mean_steps(P, frame, opt, med, src_d, n=65536):
    """Mean integration steps per ray on a seeded sample of the frame's rays
    (outside the timed region), for the algorithmic operation count."""
    import torch
    rng = np.random.default_rng(12345)
    ids = torch.tensor(np.unique(rng.integers(0, frame.n_rays, n)), dtype=torch.int64, device="cuda")
    out = torch.empty(len(ids) * P.RAY_STATE.itemsize, dtype=torch.uint8, device="cuda")
    P.pivbos_trace_exit_states(med.h if med else None, opt.h, src_d, len(frame.sources), frame.rays_per_source,
                               frame.seed, frame.frame_index, frame.integrator, frame.step, ids, len(ids), out)
    P.pivbos_sync()
    st = np.frombuffer(out.cpu().numpy().tobytes(), dtype=P.RAY_STATE)
    return float(st["steps"].mean())


# ----------------------------------------------------------------------------
# CPU oracle (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------
def oracle_sample(frames, seconds_target=12.0, max_rays=None):
    import oracle
    fr = frames[0]
    med = oracle.Medium.from_scene(fr.medium) if fr.medium is not None else None
    opt = oracle.Optics.from_scene(fr.optics)
    threads = oracle.threads()
    chunk = 200000
    done, t_total = 0, 0.0
    img = np.zeros((fr.optics.height, fr.optics.width), dtype=np.int64)
    while t_total < seconds_target and (max_rays is None or done < max_rays):
        t0 = time.perf_counter()
        oracle.render(med, opt, fr.sources, fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator,
                      fr.step, image=img, first_ray=done, ray_count=chunk)
        t_total += time.perf_counter() - t0
        done += chunk
        if done >= fr.n_rays:
            break
    return done / t_total, threads, done, t_total


def c4_subset(fr, n_sources=10000, rays=100):
    """The fixed subset of an image the oracle baselines use: rays 0..rays-1
    of its first n_sources sources (the same Philox counters as in the full
    image, whatever its rays per source)."""
    import copy
    sub = copy.copy(fr)
    sub.sources = fr.sources[:n_sources]
    sub.rays_per_source = min(rays, fr.rays_per_source)
    return sub


def oracle_subset_rate(fr, seconds_cap=30.0):
    """The oracle's rays/s on the fixed 1e6-ray subset of the image (first
    1e4 sources x 100 rays), all host cores; fewer sources if a first chunk
    says the whole subset would exceed seconds_cap."""
    import oracle
    sub = c4_subset(fr)
    med = oracle.Medium.from_scene(sub.medium) if sub.medium is not None else None
    opt = oracle.Optics.from_scene(sub.optics)
    img = np.zeros((sub.optics.height, sub.optics.width), dtype=np.int64)
    t0 = time.perf_counter()
    first = 50000
    oracle.render(med, opt, sub.sources, sub.rays_per_source, sub.seed, sub.frame_index, sub.integrator, sub.step,
                  image=img, first_ray=0, ray_count=first)
    t_first = time.perf_counter() - t0
    budget = int(max(first, min(sub.n_rays, first * seconds_cap / max(t_first, 1e-9))))
    done = first
    if budget > first:
        oracle.render(med, opt, sub.sources, sub.rays_per_source, sub.seed, sub.frame_index, sub.integrator,
                      sub.step, image=img, first_ray=first, ray_count=budget - first)
        done = budget
    t = time.perf_counter() - t0
    return {"value": done / t, "unit": "rays/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "rays 0-%d of the first %d sources (%d rays, the fixed image subset), %.1f s of CPU work"
                      % (sub.rays_per_source - 1, min(len(sub.sources), (done + sub.rays_per_source - 1)
                                                      // sub.rays_per_source), done, t)}


def config_for(args):
    """The line's config object (both arms print the same one)."""
    wl = args.workload
    if wl == "c4" and not args.surrogate:
        cfg = {"workload": WORKLOAD_NAMES["c4"] + ("" if args.scale == 1.0 else " (scaled by %g)" % args.scale)
               + ("" if not getattr(args, "grid", None) else " (grid %d^3)" % args.grid),
               "name": "c4", "arms": "plain tracer vs surrogate (projection + tcgen05 network, plain fallback) "
                                     "vs projection alone",
               "budget_px_rms": 0.01, "rays_per_step": 0, "l2": "flushed between steps (inputs also > L2)"}
    elif args.surrogate:
        cfg = {"workload": WORKLOAD_NAMES[wl] + " - surrogate path", "name": wl + "-surrogate",
               "rays_per_step": 0, "l2": "flushed between steps"}
    else:
        cfg = {"workload": WORKLOAD_NAMES[wl] + ("" if args.scale == 1.0 else " (scaled by %g)" % args.scale),
               "name": wl, "optics": args.optics, "rays_per_step": 0, "l2": "flushed between steps"}
    frames = _frames(wl, args.scale)
    cfg["rays_per_step"] = sum(f.n_rays for f in frames) if not (wl == "c4" or args.surrogate) else frames[0].n_rays
    cfg["parallelism"] = ("single GPU" if args.gpus <= 1 else
                          ("one image sharded by source ranges + NCCL int64 all-reduce" if wl == "c4"
                           else "replicas (weak)"))
    return cfg


# ----------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The oracle on the host cores, on this workload's config: every step
    traces a bounded sample of the image's rays (the fixed subset: rays 0..99
    of the first 1e4 sources, continued cyclically); ms_per_step is the wall
    time those rays took, value the rays traced per second."""
    if rank != 0:
        return
    import oracle
    frames = _frames(args.workload, args.scale)
    fr = frames[0]
    sub = c4_subset(fr) if fr.rays_per_source > 100 else fr
    med = oracle.Medium.from_scene(sub.medium) if sub.medium is not None else None
    opt = oracle.Optics.from_scene(sub.optics)
    img = np.zeros((sub.optics.height, sub.optics.width), dtype=np.int64)
    # size a step to ~2.5 s of CPU work from a short probe (whole run: a minute or two)
    t0 = time.perf_counter()
    oracle.render(med, opt, sub.sources, sub.rays_per_source, sub.seed, sub.frame_index, sub.integrator, sub.step,
                  image=img, first_ray=0, ray_count=20000)
    rate0 = 20000 / max(time.perf_counter() - t0, 1e-9)
    per_step = int(min(sub.n_rays, max(20000, rate0 * min(2.5, 150.0 / max(args.steps + args.warmup, 1)))))
    pos = 0

    def step():
        nonlocal pos
        done = 0
        while done < per_step:
            n = min(per_step - done, sub.n_rays - pos)
            oracle.render(med, opt, sub.sources, sub.rays_per_source, sub.seed, sub.frame_index, sub.integrator,
                          sub.step, image=img, first_ray=pos, ray_count=n)
            done += n
            pos = (pos + n) % sub.n_rays
        return done

    for _ in range(args.warmup):
        step()
    traced, secs = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        traced += step()
        secs += time.perf_counter() - t0
    value = traced / secs
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "strong" if (args.workload == "c4" and args.gpus > 1) else "weak",
        "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": config_for(args),
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": "%d rays per step from the image's fixed subset (rays 0..%d of the first %d "
                                   "sources), %.2f s per step; the plain method (the oracle has no surrogate)"
                                   % (per_step, sub.rays_per_source - 1, len(sub.sources), secs / args.steps)},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "rays_per_step_traced": per_step,
    }
    print(json.dumps(out), flush=True)


def measure_plain(args, workload, rank, world, steps, warmup, with_e2e=True, with_cpu=True):
    """A plain-tracer workload (C0, C1, C2): per step the medium build, the
    Morton ordering, the render kernel and the finalisation of every image
    (weak scaling across ranks: every rank renders its own images).  Returns
    the measurement as a dict."""
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    from paper_1812_05902_gb300 import pivbos as P

    frames = _frames(workload, args.scale)
    apply_optics_variant(frames, args.optics)
    for fr in frames:
        fr.seed = fr.seed + 1000003 * rank
    opt = P.Optics(frames[0].optics)
    W, H = frames[0].optics.width, frames[0].optics.height
    rho_d = [torch.tensor(fr.medium.rho, device=dev) for fr in frames]
    src_d = [torch.tensor(fr.sources, dtype=torch.float64, device=dev) for fr in frames]
    meds = [P.Medium(fr.medium, rho=rho_d[i]) for i, fr in enumerate(frames)]
    img = torch.zeros((H, W), dtype=torch.int64, device=dev)
    fimg = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in frames]
    stats = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        for i, fr in enumerate(frames):
            P.pivbos_medium_refill(meds[i].h, rho_d[i])
            img.zero_()
            P.pivbos_render(meds[i].h, opt.h, src_d[i], len(fr.sources), fr.rays_per_source, fr.seed,
                            fr.frame_index, fr.integrator, fr.step, img, stats)
            P.pivbos_image_finalize(img, H * W, fimg[i])

    step()
    P.pivbos_sync()
    # exact-total check of an image (outside the timed region)
    stats.zero_()
    step()
    P.pivbos_sync()
    st = stats.cpu().numpy()
    assert int(st.sum()) == sum(fr.n_rays for fr in frames)

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    timer = ArmTimer(P, torch, flush, world)
    ms, launches, kt = timer(step, steps, warmup, ("render", "medium", "sort", "finalize"))
    clk = clocks.stop()
    rays_step = sum(fr.n_rays for fr in frames)
    value = rays_step * steps * world / (ms * 1e-3)

    # e2e: the same step through the C ABI with host buffers: host density,
    # host sources in; the host image out (the render call copies)
    e2e = None
    if with_e2e and not args.no_e2e:
        rho_h = [torch.tensor(fr.medium.rho).pin_memory() for fr in frames]
        src_h = [torch.tensor(fr.sources, dtype=torch.float64).pin_memory() for fr in frames]
        img_h = torch.zeros((H, W), dtype=torch.int64).pin_memory()
        fimg_h = torch.empty((H, W), dtype=torch.float32).pin_memory()

        def step_host():
            for i, fr in enumerate(frames):
                P.pivbos_medium_refill(meds[i].h, rho_h[i])
                img_h.zero_()
                P.pivbos_render(meds[i].h, opt.h, src_h[i], len(fr.sources), fr.rays_per_source, fr.seed,
                                fr.frame_index, fr.integrator, fr.step, img_h, stats)
                # the same finalisation as the device-timed step
                img.copy_(img_h, non_blocking=True)
                P.pivbos_image_finalize(img, H * W, fimg[i])
                fimg_h.copy_(fimg[i], non_blocking=True)

        step_host()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, steps)):
            flush.fill_(1)
            step_host()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        h2d = sum(r.numel() * 4 + s.numel() * 8 + H * W * 8 * 2 for r, s in zip(rho_h, src_h))
        e2e = {"value": rays_step * max(1, steps) * world / dt, "unit": "rays/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int((H * W * 8 + H * W * 4) * len(frames)),
               "note": "wall clock including the L2 flush of every step"}

    msteps = [mean_steps(P, fr, opt, meds[i], src_d[i]) for i, fr in enumerate(frames)]
    dense = all(f.medium is not None and (f.medium.dims[2] - 1) * f.medium.spacing[2] / f.step *
                (3 if f.integrator == scenes.RK4 else 1) >= 64 for f in frames)
    rk = kt["render"]
    rf = roofline(frames, msteps, rk["ms_per_launch"] or 0.0, 1 if rk["ms_per_launch"] else 0,
                  clk.get("sm_max_mhz"),
                  recorded_traffic("render_%s_traffic" % workload, rays_per_cta=render_rays_per_cta(frames, dense),
                                   scale_to_rays=sum(f.n_rays for f in frames) / len(frames))
                  if args.scale == 1.0 and args.optics == "plain" else None,
                  l1_gbs=measured_l1_gbs(P) if all(f.medium is not None for f in frames) else None)
    cpu = None
    if with_cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, done, t = oracle_sample(frames, seconds_target=12.0)
        cpu = {"value": v, "unit": "rays/s", "cores": threads, "kind": "oracle",
               "sample": "first %d rays (source order) of image 1, %.1f s of CPU work" % (done, t)}
    return {"workload": WORKLOAD_NAMES[workload], "name": workload, "value": value, "unit": "rays/s",
            "ms_per_step": ms / steps, "steps": steps, "warmup": warmup, "rays_per_step": rays_step,
            "images_per_step": len(frames), "gpu_launches": launches, "clocks": clk, "kernels": kt,
            "mean_steps_per_ray": msteps, "roofline": rf, "e2e": e2e, "cpu_baseline": cpu}


def run_gpu_sub(args, workload):
    """A plain workload's figures as a sub-object of the default line."""
    return measure_plain(args, workload, 0, 1, steps=3, warmup=2, with_e2e=True, with_cpu=True)


def run_gpu(args, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1812_05902_gb300 import build as libbuild
    libbuild.build()
    res = measure_plain(args, args.workload, rank, world, args.steps, args.warmup)
    if rank == 0:
        out = {
            "metric": METRIC, "value": res["value"], "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (double-float f32 pairs for positions/directions)",
            "data": "synthetic", "config": config_for(args), "gpu_launches": res["gpu_launches"],
            "clocks": res["clocks"], "roofline": res["roofline"], "e2e": res["e2e"],
            "cpu_baseline": res["cpu_baseline"], "impl": "pivbos", "plain": res,
        }
        print(json.dumps(out), flush=True)


MLP_FLOP_PER_RAY = 2 * (16 * 128 + 3 * 128 * 128 + 128 * 4)   # one forward of the surrogate network


def shard_range(n, rank, world):
    """Contiguous source range [lo, hi) of rank `rank` among `world` (the
    library's sharding rule, shard.source_range)."""
    from paper_1812_05902_gb300.shard import source_range
    first, count = source_range(n, world, rank)
    return first, first + count


class ArmTimer:
    """Times K steps of one arm (CUDA events on the launching stream, L2
    flushed before each step outside the events, max over ranks) and reads
    the library's per-kernel timings of those steps."""

    def __init__(self, P, torch, flush, world):
        self.P, self.torch, self.flush, self.world = P, torch, flush, world

    def __call__(self, fn, steps, warmup, kernels=()):
        P, torch = self.P, self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        stream = torch.cuda.current_stream()
        P.pivbos_timing_reset()
        P.pivbos_timing_enable(True)
        l0 = P.pivbos_kernel_launches()
        ev = []
        for _ in range(steps):
            self.flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        launches = P.pivbos_kernel_launches() - l0
        P.pivbos_timing_enable(False)
        ms = sum(a.elapsed_time(b) for a, b in ev)
        if self.world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        kt = {}
        for k in kernels:
            kms, kn = P.pivbos_timing_read(k)
            kt[k] = {"ms_per_step": kms / steps, "launches_per_step": kn / steps,
                     "ms_per_launch": kms / kn if kn else None}
        return ms, int(launches), kt


def surrogate_error(P, torch, oracle, fr, med, opt, src, sg, desc, n_plain=1_000_000, n_oracle=200_000, seed=777):
    """RMS sensor error (px) of a trained surrogate's path on seeded random
    rays of the image: against the plain tracer (n_plain rays) and against
    the oracle (the first n_oracle of them); rays whose status differs
    (a ray grazing a stop) are counted, not averaged in.  Also the plain
    tracer's own worst error against the oracle on the same rays."""
    dev = src.device
    ids = np.random.default_rng(seed).choice(fr.n_rays, n_plain, replace=False).astype(np.int64)
    ids_t = torch.tensor(ids, device=dev)
    xy = torch.empty((len(ids), 2), dtype=torch.float64, device=dev)
    flags = torch.empty(len(ids), dtype=torch.int32, device=dev)
    sst = torch.empty(len(ids), dtype=torch.int32, device=dev)
    P.pivbos_surrogate_sensor(sg, desc, ids_t, xy, flags, sst)
    out = torch.empty(len(ids) * P.RAY_STATE.itemsize, dtype=torch.uint8, device=dev)
    P.pivbos_trace_exit_states(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.seed, fr.frame_index,
                               fr.integrator, fr.step, ids_t, len(ids), out)
    P.pivbos_sync()
    plain = np.frombuffer(out.cpu().numpy().tobytes(), dtype=P.RAY_STATE)
    xy, flags, sst = xy.cpu().numpy(), flags.cpu().numpy(), sst.cpu().numpy()
    ok = (sst == 0) & (plain["status"] == 0)
    d = xy[ok] - plain["sensor_xy"][ok]
    res = {"rms_px_vs_plain": float(np.sqrt((d ** 2).sum(1).mean())), "rays_vs_plain": int(ok.sum()),
           "status_differs_vs_plain": int(((sst == 0) != (plain["status"] == 0)).sum()),
           "served_frac_sample": float((flags[ok] == 0).mean())}
    om = oracle.Medium.from_scene(fr.medium)
    oo = oracle.Optics.from_scene(fr.optics)
    t0 = time.perf_counter()
    ost = oracle.trace_many(om, oo, fr.sources, fr.rays_per_source, ids[:n_oracle], fr.seed, fr.frame_index,
                            fr.integrator, fr.step)
    t_or = time.perf_counter() - t0
    ok_o = (sst[:n_oracle] == 0) & (ost["status"] == 0)
    do = xy[:n_oracle][ok_o] - ost["sensor_xy"][ok_o]
    both = (plain["status"][:n_oracle] == ost["status"]) & (ost["status"] == 0)
    res.update({"rms_px_vs_oracle": float(np.sqrt((do ** 2).sum(1).mean())), "rays_vs_oracle": int(ok_o.sum()),
                "status_differs_vs_oracle": int(((sst[:n_oracle] == 0) != (ost["status"] == 0)).sum()),
                "plain_max_err_px_vs_oracle": float(np.max(np.abs(plain["sensor_xy"][:n_oracle][both] -
                                                                  ost["sensor_xy"][both]))),
                "plain_status_mismatch_vs_oracle": int((plain["status"][:n_oracle] != ost["status"]).sum()),
                "oracle_seconds": round(t_or, 2)})
    return res


# FP32/INT32 lane operations per ray served by the surrogate's finish kernel:
# exit line from the straight line and the residual (40), the lens in FP32
# (two spheres 2 x 130, the stop 20), the sensor plane (125), the spot
# deposit (450), list reads and bookkeeping (20)
OPS_FINISH_RAY = 40 + 2 * 130 + 20 + 125 + 450 + 20
# ... and per ray of the direct pass (a surrogate without the network: the
# prep and finish kernels' work in one kernel), besides the finish work of
# each served ray: ray generation in FP32 from the Philox words (330), the
# box test (40), entry point, features and bin (60), the one-segment
# projection's two table lookups with their first moments (2 x 110), the
# fallback-list ballot (10)
OPS_DIRECT_RAY = 330 + 40 + 60 + 2 * 110 + 10
TIGHT_BUDGET_PX = 0.001


def run_c4(args, rank, world):
    """The default line: C4, plain tracer vs the surrogate path (the value),
    the network forced on every served ray, and a tight-budget comparison."""
    import torch
    import oracle
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1812_05902_gb300 import build as libbuild
    libbuild.build()
    from paper_1812_05902_gb300 import pivbos as P
    if world > 1:
        import torch.distributed as dist
    fr = _frames("c4", args.scale)[0]
    n_src = len(fr.sources)
    lo, hi = shard_range(n_src, rank, world)
    W, H = fr.optics.width, fr.optics.height
    rho_d = torch.tensor(fr.medium.rho, device=dev)
    opt = P.Optics(fr.optics)
    src_all = torch.tensor(fr.sources, dtype=torch.float64, device=dev)
    src = src_all[lo:hi].contiguous()
    img = torch.zeros((H, W), dtype=torch.int64, device=dev)
    fimg = torch.empty((H, W), dtype=torch.float32, device=dev)
    stats = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    timer = ArmTimer(P, torch, flush, world)
    rays = fr.n_rays
    # A1 once per density field: the medium build, timed on its own
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    med = P.Medium(fr.medium, rho=rho_d)
    torch.cuda.synchronize()
    a.record(stream)
    med.refill(rho_d)
    b.record(stream)
    torch.cuda.synchronize()
    medium_ms = a.elapsed_time(b)
    desc_all = P.frame_desc(med.h, opt.h, src_all, n_src, fr.rays_per_source, fr.frame_index, fr.seed, fr.step,
                            img, stats)
    desc = P.frame_desc(med.h, opt.h, src, hi - lo, fr.rays_per_source, fr.frame_index, fr.seed, fr.step, img, stats)

    def reduce():
        if world > 1:
            dist.all_reduce(img, op=dist.ReduceOp.SUM)

    def plain_step():
        img.zero_()
        P.pivbos_render_range(med.h, opt.h, src, hi - lo, lo, fr.rays_per_source, fr.seed, fr.frame_index,
                              fr.integrator, fr.step, img, stats)
        reduce()
        P.pivbos_image_finalize(img, H * W, fimg)

    def sur_step(g):
        def f():
            img.zero_()
            P.pivbos_surrogate_render_range(g, desc, lo)
            reduce()
            P.pivbos_image_finalize(img, H * W, fimg)
        return f

    def wall(fn):
        fn()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        if world > 1:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        return rays * max(1, args.steps) / dt

    sur_kernels = ("surrogate_direct", "surrogate_prep", "surrogate_net", "surrogate_finish", "surrogate_fallback",
                   "sort")

    def surrogate_arm(label, with_e2e=False, **cfg_fields):
        """Train a surrogate (outside the timed region; every rank trains the
        same one), time its render, measure its error; returns the arm."""
        cfg = P.pivbos_surrogate_default_cfg()
        for k, v in cfg_fields.items():
            setattr(cfg, k, v)
        t0 = time.perf_counter()
        g, rep = P.pivbos_surrogate_train(desc_all, fr.integrator, cfg)
        train_s = time.perf_counter() - t0
        try:
            ms, launches, kt = timer(sur_step(g), args.steps, args.warmup, sur_kernels)
            n_fb = P.pivbos_surrogate_render(g, desc_all, count_fallback=True)
            e2e = None
            if with_e2e and not args.no_e2e:
                src_h = torch.tensor(fr.sources[lo:hi], dtype=torch.float64).pin_memory()
                fimg_h = torch.empty((H, W), dtype=torch.float32).pin_memory()

                def e2e_step():
                    src.copy_(src_h, non_blocking=True)
                    sur_step(g)()
                    fimg_h.copy_(fimg, non_blocking=True)

                e2e = {"value": wall(e2e_step), "unit": "rays/s", "h2d_bytes_per_step": int(src_h.numel() * 8),
                       "d2h_bytes_per_step": int(H * W * 4),
                       "path": "pinned host sources -> device, pivbos_surrogate_render_range, "
                               "pivbos_image_finalize, float image -> pinned host"}
            err = (surrogate_error(P, torch, oracle, fr, med, opt, src_all, g, desc_all)
                   if rank == 0 and not args.only else None)
        finally:
            P.pivbos_surrogate_destroy(g)
        r = rep.as_dict()
        t = ms * 1e-3 / args.steps
        return {"label": label, "config": {k: v for k, v in cfg_fields.items()},
                "rays_per_s": rays * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
                "gpu_launches": launches, "served_frac": (rays - n_fb) / rays,
                "served_frac_network": r["val_served_frac_net"], "fallback_rays": int(n_fb),
                "network_trained": bool(r["network_trained"]), "born_segments": r["born_segments"],
                "train_seconds": round(train_s, 3), "kernels": kt, "error": err, "report": r, "e2e": e2e,
                "_t": t}

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if args.only in ("surrogate", "network"):
        # a profiling capture of one surrogate arm (no line is printed)
        surrogate_arm(args.only, use_network=-1 if args.only == "surrogate" else 1)
        clocks.stop()
        return
    ms_plain, l_plain, k_plain = timer(plain_step, args.steps, args.warmup, ("render", "sort"))
    if args.only == "plain":
        clocks.stop()
        return
    img_plain = img.clone() if world > 1 and rank == 0 else None
    sur = surrogate_arm("surrogate (automatic predictor choice, the default)", with_e2e=True)
    net = surrogate_arm("network's correction on every served ray", use_network=1)
    tight = {"budget_px": TIGHT_BUDGET_PX}
    if not args.no_tight:
        tight["projection"] = surrogate_arm("projection alone", use_network=0, err_budget_px=TIGHT_BUDGET_PX)
        tight["surrogate"] = surrogate_arm("automatic predictor choice", err_budget_px=TIGHT_BUDGET_PX)
    clk = clocks.stop()
    if world > 1 and rank == 0:
        # the sharded image is the single-GPU image, bit for bit
        ref = torch.zeros_like(img)
        P.pivbos_render(med.h, opt.h, src_all, n_src, fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator,
                        fr.step, ref)
        P.pivbos_sync()
        assert torch.equal(ref, img_plain), "sharded image differs from the single-GPU image"
    e2e_plain = None
    if not args.no_e2e:
        src_h = torch.tensor(fr.sources[lo:hi], dtype=torch.float64).pin_memory()
        img_h = torch.zeros((H, W), dtype=torch.int64).pin_memory()
        fimg_h = torch.empty((H, W), dtype=torch.float32).pin_memory()

        def e2e_plain_step():
            # the C ABI copies host sources in and the host image out itself
            img_h.zero_()
            P.pivbos_render_range(med.h, opt.h, src_h, hi - lo, lo, fr.rays_per_source, fr.seed, fr.frame_index,
                                  fr.integrator, fr.step, img_h)
            if world > 1:
                img.copy_(img_h, non_blocking=True)
                reduce()
                P.pivbos_image_finalize(img, H * W, fimg)
                fimg_h.copy_(fimg, non_blocking=True)

        e2e_plain = {"value": wall(e2e_plain_step), "unit": "rays/s",
                     "h2d_bytes_per_step": int(src_h.numel() * 8 + H * W * 8),
                     "d2h_bytes_per_step": int(H * W * 8 + (H * W * 4 if world > 1 else 0)),
                     "path": "pivbos_render_range with host sources and a host image (the call copies)"}
    v_plain = rays * args.steps / (ms_plain * 1e-3)
    v_sur = sur["rays_per_s"]
    peaks, src_kind = _peaks()
    peak_tf = peaks.get("bf16_tflops", 1900.0)
    clk_hz = (clk.get("sm_max_mhz") or 2070.0) * 1e6

    def net_roofline(arm):
        k = arm["kernels"]["surrogate_net"]
        if not k["ms_per_launch"]:
            return None
        served_net = arm["served_frac_network"] * rays / world
        per_launch = served_net / k["launches_per_step"]
        achieved = per_launch * MLP_FLOP_PER_RAY / (k["ms_per_launch"] * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak_tf, "unit": "TFLOP/s",
                "frac": round(achieved / peak_tf, 4),
                "traffic": (recorded_traffic("surrogate_net_c4_traffic", "surrogate", scale_to_rays=per_launch)
                            if args.scale == 1.0 and world == 1 else None),
                "kernel": "surr_net_kernel", "op": "BF16 MLP forward on tcgen05, %d FLOP per ray it corrects"
                                                   % MLP_FLOP_PER_RAY,
                "peak_source": "%s bf16_tflops (burst)" % src_kind, "launch_ms": round(k["ms_per_launch"], 3),
                "rays_per_launch": int(per_launch)}

    def finish_roofline(arm):
        k = arm["kernels"]["surrogate_finish"]
        if not k["ms_per_launch"]:
            return None
        per_launch = arm["served_frac"] * rays / world / k["launches_per_step"]
        achieved = per_launch * OPS_FINISH_RAY / (k["ms_per_launch"] * 1e-3) / 1e12
        peak = N_SM * ISSUE_LANES_PER_SM * clk_hz / 1e12
        return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": (recorded_traffic("surrogate_finish_c4_traffic", "surrogate", scale_to_rays=per_launch)
                            if args.scale == 1.0 and world == 1 else None),
                "kernel": "surr_finish_kernel", "op": "FP32/INT32 lane operation, %d per served ray" % OPS_FINISH_RAY,
                "peak_source": "issue rate derived from 152 SMs x 128 lanes x max SM clock",
                "launch_ms": round(k["ms_per_launch"], 3), "rays_per_launch": int(per_launch)}

    def direct_roofline(arm):
        k = arm["kernels"]["surrogate_direct"]
        if not k["ms_per_launch"]:
            return None
        per_launch = rays / world / k["launches_per_step"]
        ops = OPS_DIRECT_RAY + arm["served_frac"] * OPS_FINISH_RAY
        achieved = per_launch * ops / (k["ms_per_launch"] * 1e-3) / 1e12
        peak = N_SM * ISSUE_LANES_PER_SM * clk_hz / 1e12
        return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": (recorded_traffic("surrogate_direct_c4_traffic", "surrogate", scale_to_rays=per_launch)
                            if args.scale == 1.0 and world == 1 else None),
                "kernel": "surr_direct_kernel",
                "op": "FP32/INT32 lane operation, %d per ray and %d more per served ray"
                      % (OPS_DIRECT_RAY, OPS_FINISH_RAY),
                "peak_source": "issue rate derived from 152 SMs x 128 lanes x max SM clock",
                "launch_ms": round(k["ms_per_launch"], 3), "rays_per_launch": int(per_launch)}

    for arm in [sur, net] + [tight[k] for k in ("projection", "surrogate") if k in tight]:
        arm["rooflines"] = {"surr_net_kernel": net_roofline(arm), "surr_finish_kernel": finish_roofline(arm),
                            "surr_direct_kernel": direct_roofline(arm)}
    # the headline's roofline: the surrogate step's dominant kernel
    ks = sur["kernels"]
    dom = max(("surrogate_direct", "surrogate_net", "surrogate_finish", "surrogate_prep"),
              key=lambda k: ks[k]["ms_per_step"])
    rf = sur["rooflines"][{"surrogate_direct": "surr_direct_kernel", "surrogate_net": "surr_net_kernel"}
                          .get(dom, "surr_finish_kernel")]
    if rf is not None:
        rf = dict(rf, dominant_kernel_share=round(ks[dom]["ms_per_step"] / sur["ms_per_step"], 4))
    # the plain arm's render kernel: the gather roofline (128 B per field
    # evaluation through L1) and the issue roofline
    msteps = mean_steps(P, fr, opt, med, src_all)
    rk = k_plain["render"]
    rf_plain = None
    if rk["ms_per_launch"]:
        rf_plain = roofline([fr], [msteps], rk["ms_per_launch"], 1, clk.get("sm_max_mhz"),
                            recorded_traffic("render_c4_traffic", "render", rays_per_cta=2048,
                                             scale_to_rays=rays / world)
                            if args.scale == 1.0 and world == 1 else None,
                            l1_gbs=measured_l1_gbs(P), ray_frac=1.0 / world)
    # once per density field: the medium build, and the surrogate's table,
    # data and (when the network is trained) training
    t_plain = ms_plain * 1e-3 / args.steps
    amort = {"medium_build_ms": round(medium_ms, 2)}
    for name, arm in (("surrogate", sur), ("network", net)):
        amort[name] = {"build_seconds": arm["train_seconds"],
                       "break_even_images": (arm["train_seconds"] / (t_plain - arm["_t"])) if t_plain > arm["_t"]
                       else None,
                       "rays_per_s_one_image_incl_build": rays / (arm["train_seconds"] + arm["_t"]),
                       "rays_per_s_ten_images_incl_build": 10 * rays / (arm["train_seconds"] + 10 * arm["_t"])}
    amort["plain_rays_per_s_one_image_incl_medium"] = rays / (medium_ms * 1e-3 + t_plain)
    amort["note"] = ("every arm needs the medium; a surrogate is built once per density field and serves every "
                     "image rendered through that field")
    for arm in [sur, net] + [tight[k] for k in ("projection", "surrogate") if k in tight]:
        arm.pop("_t", None)
    c1 = t1 = u16 = None
    if world == 1 and not args.no_table1:
        try:
            c1 = run_gpu_sub(args, "c1")
        except Exception as exc:   # reported, never hidden
            c1 = {"error": "%s: %s" % (type(exc).__name__, exc)}
        try:
            t1 = run_table1(args, rank, world, steps=3, warmup=1, embedded=True)
        except Exception as exc:
            t1 = {"error": "%s: %s" % (type(exc).__name__, exc)}
        try:
            u16 = measure_image_u16(P, dev)
        except Exception as exc:
            u16 = {"error": "%s: %s" % (type(exc).__name__, exc)}
    c3 = None
    if world == 1 and not args.no_batch:
        try:
            c3 = measure_batch(args, rank, world, steps=1, warmup=1)
        except Exception as exc:
            c3 = {"error": "%s: %s" % (type(exc).__name__, exc)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_subset_rate(fr)
    if rank == 0:
        out = {
            "metric": METRIC, "value": v_sur, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sur["ms_per_step"], "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f32 projection, optics and deposit weights; bf16 network with f32 accumulation where it "
                     "runs; double-float pairs on the plain path; int64 image",
            "data": "synthetic", "config": config_for(args),
            "gpu_launches": sur["gpu_launches"], "clocks": clk, "roofline": rf, "e2e": sur["e2e"],
            "cpu_baseline": cpu, "impl": "pivbos",
            "plain_rays_per_s": v_plain, "surrogate_rays_per_s": v_sur, "speedup_vs_plain": v_sur / v_plain,
            "rms_px_vs_oracle": (sur["error"] or {}).get("rms_px_vs_oracle"),
            "surrogate": sur, "network": net, "tight_budget": tight,
            "plain": {"rays_per_s": v_plain, "ms_per_step": ms_plain / args.steps, "gpu_launches": l_plain,
                      "kernels": k_plain, "mean_steps_per_ray": msteps, "roofline": rf_plain, "e2e": e2e_plain},
            "per_density_field": amort,
        }
        if c1 is not None:
            out["c1"] = c1
        if t1 is not None:
            out["table1"] = t1
        if u16 is not None:
            out["image_u16"] = u16
        if c3 is not None:
            out["c3"] = c3
        print(json.dumps(out), flush=True)


def run_surrogate(args, rank, world, steps, warmup, embedded, workload="c4"):
    """A workload with the surrogate (C4, or the C2 BOS field): returns the
    measurement as a dict."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    fr = _frames(workload, args.scale)[0]
    fr.seed = fr.seed + 1000003 * rank
    med = P.Medium(fr.medium, rho=torch.tensor(fr.medium.rho, device=dev))
    opt = P.Optics(fr.optics)
    W, H = fr.optics.width, fr.optics.height
    src = torch.tensor(fr.sources, dtype=torch.float64, device=dev)
    img = torch.zeros((H, W), dtype=torch.int64, device=dev)
    fimg = torch.empty((H, W), dtype=torch.float32, device=dev)
    stats = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device=dev)
    desc = P.frame_desc(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.frame_index, fr.seed, fr.step,
                        img, stats)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sg, rep = P.pivbos_surrogate_train(desc, fr.integrator, P.pivbos_surrogate_default_cfg())
    train_wall = time.perf_counter() - t0

    def plain_step():
        img.zero_()
        P.pivbos_render(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.seed, fr.frame_index,
                        fr.integrator, fr.step, img, stats)
        P.pivbos_image_finalize(img, H * W, fimg)

    def surrogate_step():
        img.zero_()
        P.pivbos_surrogate_render(sg, desc)
        P.pivbos_image_finalize(img, H * W, fimg)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        P.pivbos_timing_reset()   # kernel timings of the timed steps only
        timed.launches0 = P.pivbos_kernel_launches()
        ev = []
        for _ in range(steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    try:
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.3)
        ms_plain = timed(plain_step)
        P.pivbos_timing_reset()
        P.pivbos_timing_enable(True)
        ms_sur = timed(surrogate_step)
        launches = P.pivbos_kernel_launches() - timed.launches0
        P.pivbos_timing_enable(False)
        clk = clocks.stop()
        k_ms, k_n = P.pivbos_timing_read("surrogate_net")
        p_ms, p_n = P.pivbos_timing_read("surrogate_prep")
        q_ms, q_n = P.pivbos_timing_read("surrogate_finish")
        d_ms, d_n = P.pivbos_timing_read("surrogate_direct")
        f_ms, f_n = P.pivbos_timing_read("surrogate_fallback")
        n_fb = P.pivbos_surrogate_render(sg, desc, count_fallback=True)
        # error of the surrogate path: against the plain tracer on 10^6 rays,
        # against the oracle on a few thousand of them
        ids = np.random.default_rng(777).choice(fr.n_rays, 1_000_000, replace=False).astype(np.int64)
        ids_t = torch.tensor(ids, device=dev)
        xy = torch.empty((len(ids), 2), dtype=torch.float64, device=dev)
        flags = torch.empty(len(ids), dtype=torch.int32, device=dev)
        sst = torch.empty(len(ids), dtype=torch.int32, device=dev)
        P.pivbos_surrogate_sensor(sg, desc, ids_t, xy, flags, sst)
        out = torch.empty(len(ids) * P.RAY_STATE.itemsize, dtype=torch.uint8, device=dev)
        P.pivbos_trace_exit_states(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.seed,
                                   fr.frame_index, fr.integrator, fr.step, ids_t, len(ids), out)
        P.pivbos_sync()
        plain = np.frombuffer(out.cpu().numpy().tobytes(), dtype=P.RAY_STATE)
        xy, flags, sst = xy.cpu().numpy(), flags.cpu().numpy(), sst.cpu().numpy()
        ok = (sst == 0) & (plain["status"] == 0)
        d = xy[ok] - plain["sensor_xy"][ok]
        rms_plain = float(np.sqrt((d ** 2).sum(1).mean()))
        n_or = 3000
        om = oracle.Medium.from_scene(fr.medium)
        oo = oracle.Optics.from_scene(fr.optics)
        ost = oracle.trace_many(om, oo, fr.sources, fr.rays_per_source, ids[:n_or], fr.seed, fr.frame_index,
                                fr.integrator, fr.step)
        ok_o = (sst[:n_or] == 0) & (ost["status"] == 0)
        do = xy[:n_or][ok_o] - ost["sensor_xy"][ok_o]
        rms_oracle = float(np.sqrt((do ** 2).sum(1).mean()))
        e2e = None
        if not embedded and not args.no_e2e:
            # sources from pinned host memory in, the float image out, every step
            src_h = torch.tensor(fr.sources, dtype=torch.float64).pin_memory()
            img_h = torch.empty((H, W), dtype=torch.float32).pin_memory()

            def e2e_step():
                src.copy_(src_h, non_blocking=True)
                surrogate_step()
                img_h.copy_(fimg, non_blocking=True)

            e2e_step()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for _ in range(max(1, steps)):
                e2e_step()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t1
            e2e = {"value": fr.n_rays * max(1, steps) * world / dt, "unit": "rays/s",
                   "h2d_bytes_per_step": int(src_h.numel() * 8), "d2h_bytes_per_step": int(H * W * 4)}
    finally:
        P.pivbos_surrogate_destroy(sg)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_plain, ms_sur], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_plain, ms_sur = float(t[0]), float(t[1])
    rays = fr.n_rays
    v_plain = rays * steps * world / (ms_plain * 1e-3)
    v_sur = rays * steps * world / (ms_sur * 1e-3)
    served = rays - n_fb
    k_launch_s = k_ms / steps * 1e-3   # the network kernels of one render
    peaks, src_kind = _peaks()
    peak_tf = peaks.get("bf16_tflops", 1900.0)
    achieved = served * MLP_FLOP_PER_RAY / k_launch_s / 1e12 if k_n else None
    res = {
        "workload": WORKLOAD_NAMES[workload], "name": workload, "rays_per_step": rays,
        "plain_rays_per_s": v_plain, "surrogate_rays_per_s": v_sur, "speedup": v_sur / v_plain,
        "ms_per_step_plain": ms_plain / steps, "ms_per_step_surrogate": ms_sur / steps,
        "rms_err_px_vs_plain": rms_plain, "rms_err_px_vs_oracle": rms_oracle, "oracle_rays": int(ok_o.sum()),
        "sampled_rays": int(ok.sum()), "budget_px": 0.01,
        "served_frac": served / rays, "fallback_rays": int(n_fb),
        "kernel_ms_per_render": {"prep": p_ms / steps, "net": k_ms / steps, "finish": q_ms / steps,
                                 "direct": d_ms / steps,
                                 "fallback": f_ms / max(f_n, 1)},
        "train_seconds": train_wall, "report": rep.as_dict(),
        "roofline": ({"bound": "tensor", "achieved": round(achieved, 2), "peak": peak_tf, "unit": "TFLOP/s",
                      "frac": round(achieved / peak_tf, 4),
                      "traffic": (recorded_traffic("surrogate_%s_traffic" % workload, "surrogate")
                                  if args.scale == 1.0 else None), "kernel": "surr_net_kernel",
                      "op": "BF16 MLP forward (tcgen05), %d FLOP per served ray" % MLP_FLOP_PER_RAY,
                      "peak_source": "%s bf16_tflops" % src_kind} if achieved else None),
        "clocks": clk, "gpu_launches": int(launches), "steps": steps, "warmup": warmup, "e2e": e2e,
    }
    return res


def run_surrogate_line(args, rank, world):
    """--surrogate: the C4 line with the surrogate path as the value."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1812_05902_gb300 import build as libbuild
    libbuild.build()
    wl = args.workload if args.workload in ("c2", "c4") else "c4"
    res = run_surrogate(args, rank, world, steps=args.steps, warmup=args.warmup, embedded=False, workload=wl)
    fr = _frames(wl, args.scale)[0]
    e2e = res.pop("e2e")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, done, t = oracle_sample([fr], seconds_target=12.0)
        cpu = {"value": v, "unit": "rays/s", "cores": threads, "kind": "oracle",
               "sample": "first %d rays (source order) of the image, %.1f s of CPU work (plain method)" % (done, t)}
    if rank == 0:
        out = {
            "metric": METRIC, "value": res["surrogate_rays_per_s"], "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step_surrogate"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 network / f32 projection and optics (double-float pairs)", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[wl] + " - surrogate path", "name": wl + "-surrogate",
                       "rays_per_step": res["rays_per_step"], "l2": "flushed between steps",
                       "parallelism": "replicas (weak)" if world > 1 else "single GPU"},
            "gpu_launches": res["gpu_launches"], "clocks": res["clocks"], "roofline": res["roofline"],
            "e2e": e2e, "cpu_baseline": cpu, "impl": "pivbos", "surrogate": res,
        }
        print(json.dumps(out), flush=True)


# A ray pair of the BOS experiment: the traced ray without its deposit, the
# same ray through the uniform medium (generation, optics, sensor), and the
# fixed-point conversion of its four coordinates plus the warp's segmented
# reduction (~100 lane operations).
OPS_PAIR_EXTRA = 710 + 125 + 40 + 100 - 450


def run_table1(args, rank, world, steps, warmup, embedded):
    """The BOS experiment of Sec. 4 (Table 1 geometry): per step, the per-dot
    displacements of every ray pair, the Eq. 9 theory per dot and the
    bilinear grid map of the displacements.  Returns the measurement."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    fr = _frames("table1", args.scale)[0]
    fr.seed = fr.seed + 1000003 * rank
    med = P.Medium(fr.medium, rho=torch.tensor(fr.medium.rho, device=dev))
    opt = P.Optics(fr.optics)
    n = len(fr.sources)
    W = fr.optics.width
    cell = 16.0
    G = int(W // cell) + 1
    dots = torch.tensor(fr.sources, dtype=torch.float64, device=dev)
    cen = torch.empty((n, 2), dtype=torch.float64, device=dev)
    disp = torch.empty((n, 2), dtype=torch.float64, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    th = torch.empty((n, 2), dtype=torch.float64, device=dev)
    grid = torch.empty((G, G, 2), dtype=torch.float64, device=dev)
    gw = torch.empty((G, G), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        P.pivbos_bos_displacements(med.h, opt.h, dots, n, fr.rays_per_source, fr.seed, fr.frame_index,
                                   fr.integrator, fr.step, cen, disp, cnt)
        P.pivbos_bos_theory(med.h, opt.h, dots, n, th)
        P.pivbos_regrid_bilinear(cen, disp, n, G, G, 0.0, 0.0, cell, 0.05, grid, gw)

    for _ in range(warmup):
        step()
    P.pivbos_sync()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    P.pivbos_timing_reset()
    P.pivbos_timing_enable(True)
    launches0 = P.pivbos_kernel_launches()
    ev = []
    for _ in range(steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    launches = P.pivbos_kernel_launches() - launches0
    P.pivbos_timing_enable(False)
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    k_ms, k_n = P.pivbos_timing_read("bos_pairs")
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    rays = fr.n_rays
    value = rays * steps * world / (ms * 1e-3)
    c = cnt.cpu().numpy()
    d = disp.cpu().numpy()
    tt = th.cpu().numpy()
    ok = c > 0.9 * fr.rays_per_source
    agree = {}
    for q, name in enumerate(("x", "y")):
        agree[name] = {"corr": round(float(np.corrcoef(d[ok, q], tt[ok, q])[0, 1]), 4),
                       "slope": round(float(np.sum(d[ok, q] * tt[ok, q]) / np.sum(tt[ok, q] ** 2)), 4),
                       "rms_traced_px": round(float(np.sqrt(np.mean(d[ok, q] ** 2))), 4),
                       "rms_eq9_px": round(float(np.sqrt(np.mean(tt[ok, q] ** 2))), 4)}
    # roofline of the pair kernel: FP32/INT32 issue, and the L1 gather path
    ms_steps = mean_steps(P, fr, opt, med, dots)
    rf = roofline([fr], [ms_steps], k_ms, k_n, clk.get("sm_max_mhz"),
                  recorded_traffic("bos_table1_traffic", "bos") if args.scale == 1.0 else None,
                  l1_gbs=measured_l1_gbs(P))
    if rf is not None:
        clk_hz = (clk.get("sm_max_mhz") or 2070.0) * 1e6
        t_launch = k_ms / k_n * 1e-3
        ops = (ops_per_ray(fr, ms_steps) + OPS_PAIR_EXTRA + sum(OPS_SURF[sf.type] for sf in fr.optics.surfaces))
        peak = N_SM * ISSUE_LANES_PER_SM * clk_hz / 1e12
        rf.update({"achieved": round(ops * rays / t_launch / 1e12, 3), "frac": round(ops * rays / t_launch / 1e12 / peak, 4),
                   "kernel": "bos_pairs_kernel", "ops_per_ray": round(ops, 1)})
    e2e = None
    if not embedded and not args.no_e2e:
        # dots from pinned host memory in; per-dot results and the grid map out
        dots_h = torch.tensor(fr.sources, dtype=torch.float64).pin_memory()
        out_h = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in (cen, disp, cnt, th, grid)]

        def e2e_step():
            dots.copy_(dots_h, non_blocking=True)
            step()
            for h, x in zip(out_h, (cen, disp, cnt, th, grid)):
                h.copy_(x, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(max(1, steps)):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        e2e = {"value": rays * max(1, steps) * world / dt, "unit": "rays/s",
               "h2d_bytes_per_step": int(dots_h.numel() * 8),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in out_h))}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        om = oracle.Medium.from_scene(fr.medium)
        oo = oracle.Optics.from_scene(fr.optics)
        ids = np.arange(0, n, max(1, n // 1024))[:1024]
        t0 = time.perf_counter()
        done = 0
        for q in ids:
            oracle.bos_displacements(om, oo, fr.sources, fr.rays_per_source, fr.seed, fr.frame_index,
                                     fr.integrator, fr.step, dot_ids=[q])
            done += fr.rays_per_source
            if time.perf_counter() - t0 > (5.0 if embedded else 12.0):
                break
        t_cpu = time.perf_counter() - t0
        cpu = {"value": done / t_cpu, "unit": "rays/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": "all rays of %d dots (each traced with and without the medium), %.1f s of CPU work"
                         % (done // fr.rays_per_source, t_cpu)}
    return {"workload": WORKLOAD_NAMES["table1"], "name": "table1", "rays_per_step": rays, "value": value,
            "ms_per_step": ms / steps, "kernel_ms_per_step": k_ms / max(k_n, 1), "mean_steps": ms_steps,
            "dots": n, "dots_with_pairs": int((c > 0).sum()), "eq9_agreement": agree, "roofline": rf,
            "clocks": clk, "gpu_launches": int(launches), "steps": steps, "warmup": warmup, "e2e": e2e,
            "cpu_baseline": cpu}


def run_table1_line(args, rank, world):
    """--workload table1: the BOS experiment of Sec. 4 as the line's value."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1812_05902_gb300 import build as libbuild
    libbuild.build()
    res = run_table1(args, rank, world, steps=args.steps, warmup=args.warmup, embedded=False)
    if rank == 0:
        out = {
            "metric": METRIC, "value": res.pop("value"), "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (double-float f32 pairs for positions/directions), int64 fixed-point sums",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES["table1"], "name": "table1", "rays_per_step": res["rays_per_step"],
                       "counting": "a ray is counted once though traced twice (with and without the medium)",
                       "l2": "flushed between steps",
                       "parallelism": "replicas (weak)" if world > 1 else "single GPU"},
            "gpu_launches": res.pop("gpu_launches"), "clocks": res.pop("clocks"), "roofline": res.pop("roofline"),
            "e2e": res.pop("e2e"), "cpu_baseline": res.pop("cpu_baseline"), "impl": "pivbos", "table1": res,
        }
        print(json.dumps(out), flush=True)


def measure_batch(args, rank, world, steps, warmup):
    """C3: all frames in one persistent launch (CUDA graph replay per step);
    returns the measurement."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    from paper_1812_05902_gb300 import pivbos as P
    frames = _frames("c3", args.scale)
    for fr in frames:
        fr.seed = fr.seed + 1000003 * rank
    opt = P.Optics(frames[0].optics)
    meds, srcs, imgs, descs = [], [], [], []
    for fr in frames:
        meds.append(P.Medium(fr.medium, rho=torch.tensor(fr.medium.rho, device=dev)))
        srcs.append(torch.tensor(fr.sources, dtype=torch.float64, device=dev))
        imgs.append(torch.zeros((fr.optics.height, fr.optics.width), dtype=torch.int64, device=dev))
        descs.append(P.frame_desc(meds[-1].h, opt.h, srcs[-1], len(fr.sources), fr.rays_per_source,
                                  fr.frame_index, fr.seed, fr.step, imgs[-1]))
    batch = P.pivbos_batch_create(descs, scenes.RK4, None)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    try:
        clocks = Clocks(local)
        clocks.start()
        time.sleep(0.3)
        timer = ArmTimer(P, torch, flush, world)
        ms, launches, kt = timer(lambda: P.pivbos_batch_render(batch), steps, warmup, ("batch",))
        clk = clocks.stop()
    finally:
        P.pivbos_batch_destroy(batch)
    rays = sum(fr.n_rays for fr in frames)
    return {"workload": WORKLOAD_NAMES["c3"], "name": "c3", "frames": len(frames), "rays_per_step": rays,
            "value": rays * steps * world / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms / steps,
            "steps": steps, "warmup": warmup, "gpu_launches": launches, "clocks": clk}


def run_batch(args, rank, world):
    """C3: all frames in one persistent launch (CUDA graph replay per step)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1812_05902_gb300 import build as libbuild
    libbuild.build()
    res = measure_batch(args, rank, world, args.steps, args.warmup)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": res["value"], "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (double-float f32 pairs for positions/directions)",
            "data": "synthetic", "config": dict(config_for(args), frames=res["frames"]),
            "gpu_launches": res["gpu_launches"], "clocks": res["clocks"], "roofline": None, "e2e": None,
            "cpu_baseline": None, "impl": "pivbos", "batch": res}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pivbos", choices=["pivbos", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOAD_NAMES))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=None,
                    help="C4 field nodes per axis (profiling captures only; default 256)")
    ap.add_argument("--only", choices=("plain", "surrogate", "network"), default=None,
                    help="C4: run one arm's timed steps and print nothing (profiling captures)")
    ap.add_argument("--no-batch", action="store_true", help="skip the C3 batch sub-object of the default line")
    ap.add_argument("--no-tight", action="store_true",
                    help="skip the tight-budget comparison of the default line")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the C1, Sec. 4 BOS and 16-bit conversion sub-objects of the default line")
    ap.add_argument("--optics", default="plain", choices=OPTICS_VARIANTS,
                    help="the workload's camera with an optical extension (plain render workloads only)")
    ap.add_argument("--surrogate", action="store_true",
                    help="the surrogate path alone as the value (workload c2; c4's default line has all arms)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (profiling captures only; the JSON line says so)")
    args = ap.parse_args()
    _GRID[0] = args.grid
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.surrogate:
            run_surrogate_line(args, rank, world)
        elif args.workload == "c4":
            run_c4(args, rank, world)
        elif args.workload == "c3":
            run_batch(args, rank, world)
        elif args.workload == "table1":
            run_table1_line(args, rank, world)
        else:
            run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
