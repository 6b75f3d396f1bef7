#!/usr/bin/env python
"""Hypothesis-scoring throughput of the hand tracker at Kinect scale.

Workload (the Kinect-scale configuration): a 30-frame seeded trajectory of
320x240 uint16 depth frames with a 600 mm background plane, N(0, 3 mm) noise,
5% holes and 2% flipped skin pixels; per frame a 64-particle swarm runs 40
generations of pose_fk -> render_score_batch -> pso_step, tracking from the
previous frame's global best.  One step = one frame (one CUDA graph).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line.  `value` is evals/s with the frames resident in HBM;
`e2e` adds the host->device copy of each frame and the read-back of the
result.  Under torchrun (N > 1) every rank tracks its own sequence (replicas;
the swarm needs no exchange), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H = 320, 240
PARTICLES, GENS, FRAMES = 64, 40, 30
HOST_WALL_FRAMES = 240
METRIC = "hypothesis evals/s (render+cost, 320x240 ROI)"
WORKLOAD = ("Kinect-scale tracking: 320x240 uint16 depth + uint8 skin frames (600 mm plane, N(0,3 mm) noise, "
            "5% holes, 2% skin flips), 64 particles x 40 generations per frame, 30-frame seeded trajectory")
FP32_LANES_PER_SM = 128
XU_PER_SM_CLK = 16  # MUFU (square root, reciprocal) results per SM per clock: 4 per SM sub-partition
# Algorithmic work of one ray-primitive test (a pixel inside a primitive's
# exact screen box), the textbook per-pixel test counted once per primitive
# kind (an FMA counts 2 FLOP; the primitive's local ray origin o = -M C and
# the quadric's constant term are per-primitive, not per-test, work):
#   every test:  local direction h = M (a, b, 1): 3 x 2 FMA = 12;
#     ellipsoid  A = h.h (5), B = o.h (5), disc = B^2 - A C (3), disc >= 0 (1)            = 26
#     cone       w = kappa h_y (1), A = h_x^2 + h_z^2 - w^2 (5),
#                B = o_x h_x + o_z h_z - (1 + kappa o_y) w (5), disc (3), disc >= 0 (1)   = 27
#   a hit adds:  ellipsoid  s = (-B - sqrt(disc)) / A: 2, t > 0: 1, nearest depth: 1  = 4 FLOP, 2 XU
#                cone       q = -(B + sign(B) sqrt(disc)): 1, s1 = q / A, s2 = C / q: 2,
#                           y = o_y + s h_y (x2): 4, |y| <= 1 (x2): 2, t > 0 (x2): 2,
#                           nearest: 1                                                  = 12 FLOP, 3 XU
# and a test hits with probability pi / 4, the fraction of its tight
# axis-aligned box that an ellipse covers (oracle renders of 640x480 poses
# give 0.66 hits per box pixel with the 1-pixel box margin).  So a test is
# 26 + 4 pi/4 = 29.1 FLOP and 1.57 XU (ellipsoid), 27 + 12 pi/4 = 36.4 FLOP
# and 2.36 XU (cone).  The kernels decide coverage and the roots with fewer
# operations (quadratic polynomials in the pixel offsets); the tally stays the
# unit of work, so a faster kernel reads higher.
HIT_FILL = math.pi / 4
TALLY = {0: (26.0, 4.0, 2.0), 1: (27.0, 12.0, 3.0)}  # kind: (FLOP per test, FLOP per hit, XU per hit)
FLOP_PER_TEST = {k: t + HIT_FILL * h for k, (t, h, _) in TALLY.items()}
XU_PER_TEST = {k: HIT_FILL * x for k, (_, _, x) in TALLY.items()}
TALLY_BASIS = ("pixel-exact primitive boxes x per-test tally of the textbook ray-quadric test: ellipsoid "
               f"{FLOP_PER_TEST[0]:.1f} FLOP + {XU_PER_TEST[0]:.2f} XU, cone {FLOP_PER_TEST[1]:.1f} FLOP + "
               f"{XU_PER_TEST[1]:.2f} XU (miss part + pi/4 x hit part; derivation in bench.py and DESIGN)")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample")
    ap.add_argument("--profile", action="store_true", help="short run for an ncu launch list")
    ap.add_argument("--no-roofline", action="store_true", help="skip the render roofline replay")
    ap.add_argument("--no-sub-rooflines", action="store_true",
                    help="skip the render rooflines of the batched (64 sequences) and 640x480 workloads")
    ap.add_argument("--no-frame-path", action="store_true",
                    help="skip the second measurement through track_frame (one launch per frame)")
    ap.add_argument("--render", default="tune", help="render kernel: tune (timed on the workload first), auto, "
                    "units, tiles32x16, tiles32x32, tiles64x32, tiles64x64")
    ap.add_argument("--ctas", type=int, default=0, help="render CTAs per particle (0 = automatic)")
    ap.add_argument("--workload", choices=["kinect", "batch", "fullframe", "render", "equaltime", "polish"],
                    default="kinect",
                    help="kinect: one 320x240 sequence (the headline); batch: 64 sequences with uneven ROIs and P; "
                         "fullframe: 640x480 sequence, s/frame to <= 5 deg at several swarm sizes; polish: the "
                         "gradient polish's kernels for 8 particles; render: "
                         "render_score_batch alone on one frame (--roi, the first of --particles, --render; for "
                         "profiling one kernel); equaltime: hybrid 64 x 20 + polish against plain PSO given the "
                         "same time per frame, on the 320x240 sequence")
    ap.add_argument("--particles", default="256,1024,4096", help="fullframe: swarm sizes")
    ap.add_argument("--frames", type=int, default=None, help="fullframe: frames of the sequence (default 100); "
                    "equaltime: frames of the Kinect-scale sequence (default 30)")
    ap.add_argument("--gens", default="5,10,20,50", help="fullframe: generation budgets per frame")
    ap.add_argument("--roi", default="640,480", help="fullframe: ROI W,H (the Kinect camera scaled to it)")
    ap.add_argument("--methods", default="plain,hybrid",
                    help="fullframe: plain (PSO) and/or hybrid (PSO + gradient polish of the k best particles)")
    ap.add_argument("--polish", default="8,5", help="fullframe: hybrid polish: particles k, descent steps")
    ap.add_argument("--log", default="", help="fullframe: append JSON lines (every generation's best and mean E "
                    "and the best pose's joint error, one line per setting) to this file; the per-generation "
                    "copies add a little time to every frame")
    ap.add_argument("--kc", default="0,0", help="fullframe: kc variant and penetration weight (rad/mm): 0 = the "
                    "paper's, 1 = plus the interpenetration of different fingers, 2 = interpenetration only")
    args = ap.parse_args()
    args.frames_given = args.frames is not None
    if args.frames is None:
        args.frames = 100
    return args


# ---- host-side helpers ---------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


CSRC = os.path.join(ROOT, "paper_2005_07068_b300", "csrc")
# the render kernels' sources, and the committed ncu summary taken on them
KERNEL_SOURCES = {
    "units": ["render_score.cu", "hs_units.cuh", "hs_render.cuh", "hs_args.cuh", "hs_device.cuh"],
    "tiles": ["render_tiles.cu", "hs_render.cuh", "hs_args.cuh", "hs_device.cuh"],
    "frame": ["frame.cu", "hs_units.cuh", "hs_step.cuh", "hs_fk.cuh", "hs_render.cuh", "hs_args.cuh", "hs_device.cuh"],
    "strips": ["render_strips.cu", "hs_units.cuh", "hs_render.cuh", "hs_args.cuh", "hs_device.cuh"],
}
PROFILE_FILES = {("kinect", "units"): "render_units_kinect_320x240.txt",
                 ("batch", "tiles"): "render_tiles64x32_batch_64seq.txt",
                 ("kinect", "frame"): "track_frame_kinect_320x240.txt",
                 ("fullframe640x480P4096", "strips"): "render_strips8x32_fullframe_640x480.txt"}


def source_sha256(kind: str) -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_traffic(workload: str, kernel: str):
    """dram bytes per launch from the committed ncu summary of this workload's
    render kernel, if it was taken on the kernel's current source; else None."""
    kind = kernel if kernel in ("units", "frame") else "strips" if kernel.startswith("strips") else "tiles"
    name = PROFILE_FILES.get((workload, kind))
    if name is None:
        return None
    try:
        kv = {}
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != source_sha256(kind) or kv.get("kernel") != kernel:
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml)."""
    CLOCK_SM = 1

    def __init__(self, index: int):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def clock(self, max_clock=False) -> float:
        v = self.c.c_uint()
        fn = self.lib.nvmlDeviceGetMaxClockInfo if max_clock else self.lib.nvmlDeviceGetClockInfo
        if fn(self.h, self.CLOCK_SM, self.c.byref(v)) != 0:
            raise RuntimeError("clock query failed")
        return float(v.value)

    def reasons(self) -> int:
        v = self.c.c_ulonglong()
        if self._reasons(self.h, self.c.byref(v)) != 0:
            raise RuntimeError("reason query failed")
        return int(v.value)


class ClockSampler:
    """SM clock and throttle reasons sampled every 0.5 ms through NVML
    (read-only), so that even a short timed region gets dozens of samples (the
    host enqueues the timed steps ahead of the GPU, so the sampler's brief
    turns on the interpreter do not open gaps on the device)."""
    HW, HW_THERMAL, SW_THERMAL, SW_POWER = 0x8, 0x40, 0x20, 0x4

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = None
        self.error = None

    def __enter__(self):
        import threading
        try:
            self._nv = _Nvml(self.index)
            self.max_mhz = self._nv.clock(max_clock=True)
        except Exception as ex:  # no NVML: report why, keep going
            self._nv = None
            self.error = repr(ex)[:200]
            return self
        self._stop = threading.Event()

        def run():
            while not self._stop.is_set():
                try:
                    self.samples.append((self._nv.clock(), self._nv.reasons()))
                except Exception:
                    pass
                self._stop.wait(0.0005)

        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        if self._stop is not None:
            self._stop.set()
            self._t.join(timeout=2)

    def summary(self, sm_max_default):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": sm_max_default, "reasons": [], "samples": 0,
                    "error": self.error or "no samples"}
        names = {self.HW: "hw_slowdown", self.HW_THERMAL: "hw_thermal_slowdown",
                 self.SW_THERMAL: "sw_thermal_slowdown", self.SW_POWER: "sw_power_cap"}
        reasons = sorted({n for _, r in self.samples for bit, n in names.items() if r & bit})
        return {"sm_mhz": statistics.median(sm for sm, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples), "source": "NVML every 0.5 ms"}


# ---- synthetic frames ----------------------------------------------------------------------

def make_frames(seed: int, frames: int, hs, I, model, cam, device, W=W, H=H, traj=None, keep_device=True):
    """Render the ground-truth trajectory with the CUDA renderer (P = 1 debug
    output), corrupt it like a Kinect frame, return device observations."""
    import torch
    if traj is None:
        traj = I.trajectory(seed, frames).astype(np.float32)
    dummy = hs.Obs.from_numpy(np.zeros((H, W), np.uint16), np.zeros((H, W), np.uint8), device)
    hs.hs_obs_prepare(dummy)
    prims = torch.zeros(1, model.n_prims, 16, device=device)
    kc = torch.zeros(1, device=device)
    ws = hs.new_workspace(1, device)
    E = torch.zeros(1, device=device)
    dd = torch.zeros(1, H, W, device=device)
    dm = torch.zeros(1, H, W, dtype=torch.uint8, device=device)
    obs, host = [], []
    for f in range(frames):
        hs.pose_fk(model, torch.from_numpy(traj[f:f + 1]).to(device), cam, prims, kc)
        hs.render_score_batch(model, dummy, cam, prims, kc, hs.score_params(), ws, E, None, dd, dm)
        depth = dd[0].cpu().numpy().astype(np.float64)
        hit = (dm[0].cpu().numpy() & 1) > 0
        d16, skin = I.kinect_observation(depth, hit, seed * 100 + f)
        if keep_device:
            obs.append(hs.Obs.from_numpy(d16, skin, device))
        host.append((d16, skin))
    return traj, obs, host


def algorithmic_tests(box_words: np.ndarray, kinds: np.ndarray, Wp=W, Hp=H) -> np.ndarray:
    """Ray-primitive tests of one render launch, per primitive kind: for every
    particle and primitive, the pixels of its conservative box inside the ROI
    (pixel-exact box culling).  box_words: the last two words of every HsPrim
    record, [P, n_prims, 2] float32 holding int16 boxes.  Wp, Hp: the ROI size,
    or per-particle arrays [P] for a batch.  Returns [tests of kind 0, kind 1]."""
    box = np.ascontiguousarray(box_words).view(np.int16).reshape(box_words.shape[0], box_words.shape[1], 4)
    Wp = np.broadcast_to(np.asarray(Wp), (box.shape[0],))[:, None]
    Hp = np.broadcast_to(np.asarray(Hp), (box.shape[0],))[:, None]
    u0 = np.clip(box[..., 0], 0, Wp - 1)
    v0 = np.clip(box[..., 1], 0, Hp - 1)
    u1 = np.clip(box[..., 2], 0, Wp - 1)
    v1 = np.clip(box[..., 3], 0, Hp - 1)
    inside = (box[..., 2] >= 0) & (box[..., 3] >= 0) & (box[..., 0] < Wp) & (box[..., 1] < Hp)
    area = np.where(inside, (u1 - u0 + 1) * (v1 - v0 + 1), 0).astype(np.float64).sum(axis=0)
    kinds = np.asarray(kinds)
    return np.array([area[kinds == 0].sum(), area[kinds == 1].sum()])


def fp32_xu_peaks(dev, peaks):
    """FP32 and XU peaks from the unit counts and the measured maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or 2032.0)
    return {"sms": sms, "sm_max_mhz": sm_max,
            "fp32_tflops": sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12,
            "xu_tops": sms * XU_PER_SM_CLK * sm_max * 1e6 / 1e12}


def roofline_record(tests, launch_us, pk, kernel, timing, launches_timed, traffic=None, gens=1, note=None):
    """The roofline of a render launch: FP32 side and XU side of the tally;
    frac = the larger of the two fractions, and achieved / peak / unit are that
    side's (so frac = achieved / peak).  tests: [ellipsoid, cone] tests per
    generation; gens: generations per launch (the frame kernel)."""
    tests = np.asarray(tests, np.float64) * gens
    flop = float(tests[0] * FLOP_PER_TEST[0] + tests[1] * FLOP_PER_TEST[1])
    xu = float(tests[0] * XU_PER_TEST[0] + tests[1] * XU_PER_TEST[1])
    t = launch_us * 1e-6 if launch_us else float("inf")
    ach_f, ach_x = flop / t / 1e12, xu / t / 1e12
    frac_f, frac_x = ach_f / pk["fp32_tflops"], ach_x / pk["xu_tops"]
    xu_side = frac_x > frac_f
    rec = {"bound": "alu", "achieved": ach_x if xu_side else ach_f,
           "peak": pk["xu_tops"] if xu_side else pk["fp32_tflops"],
           "unit": "Top/s (XU)" if xu_side else "TFLOP/s", "frac": max(frac_f, frac_x),
           "frac_fp32": frac_f, "frac_xu": frac_x, "traffic": traffic, "kernel": kernel,
           "fp32": {"achieved_tflops": ach_f, "peak_tflops": pk["fp32_tflops"], "flop_per_launch": flop},
           "xu": {"achieved_tops": ach_x, "peak_tops": pk["xu_tops"], "ops_per_launch": xu},
           "tests_per_launch": float(tests.sum()),
           "peak_basis": (f"FP32: {pk['sms']} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x {pk['sm_max_mhz']:.0f} MHz; "
                          f"XU: {pk['sms']} SMs x {XU_PER_SM_CLK} x {pk['sm_max_mhz']:.0f} MHz (sm_max_mhz of "
                          f"measured)"),
           "flop_basis": TALLY_BASIS, "launch_us": launch_us, "launches_timed": launches_timed, "timing": timing}
    if note:
        rec["note"] = note
    return rec


# ---- the CPU oracle (baseline leg and reference arm) ----------------------------------------

def oracle_frame(seed: int):
    """Frame 0 of the same workload, rendered and corrupted on the CPU by the oracle."""
    import oracle
    from paper_2005_07068_b300 import inputs as I
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32).astype(np.float64) for a in I.search_limits())
    model = oracle.Model.from_geometry(g, lo, hi)
    cam = oracle.camera_tuple(I.kinect_camera(W, H))
    traj = I.trajectory(seed, 1)
    depth, hit, _, _ = oracle.render_pose(model, traj[0], cam, W, H, boundary=False)
    d16, skin = I.kinect_observation(depth, hit, seed * 100)
    return oracle, I, model, cam, traj[0], d16.astype(np.float64), skin


def time_oracle(seed: int, seconds: float, max_gens: int = GENS):
    """Oracle tracking on frame 0 for about `seconds`: (evals/s, generations, P, threads)."""
    oracle, I, model, cam, start, Od, S = oracle_frame(seed)
    sw = oracle.pso_init(PARTICLES, start, I.perturbation_scale(), model.lo, model.hi, seed, 0)
    t0 = time.perf_counter()
    gens = 0
    while gens < max_gens and (gens < 2 or time.perf_counter() - t0 < seconds):
        r = oracle.score_batch(model, sw.x, cam, Od, S)
        sw = oracle.pso_step(sw, r["E"], model.lo, model.hi, seed, 0, gens + 1)
        gens += 1
    dt = time.perf_counter() - t0
    return PARTICLES * gens / dt, gens, oracle.threads_used()


def run_reference(args, rank):
    if rank != 0:
        return 0
    seed = 2005070682
    oracle, I, model, cam, start, Od, S = oracle_frame(seed)
    sw = oracle.pso_init(PARTICLES, start, I.perturbation_scale(), model.lo, model.hi, seed, 0)
    g = 0
    for _ in range(args.warmup):
        r = oracle.score_batch(model, sw.x, cam, Od, S)
        g += 1
        sw = oracle.pso_step(sw, r["E"], model.lo, model.hi, seed, 0, g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.score_batch(model, sw.x, cam, Od, S)
        g += 1
        sw = oracle.pso_step(sw, r["E"], model.lo, model.hi, seed, 0, g)
    dt = time.perf_counter() - t0
    v = PARTICLES * args.steps / dt
    cores = oracle.threads_used()
    sample = (f"one step = one PSO generation of {PARTICLES} particles on a 320x240 frame (FP64 oracle: FK, "
              f"brute-force ray cast of every pixel x 37 primitives, Eq. 4-5, Eq. 6-7), OpenMP over particles")
    line = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "roi": [W, H], "particles": PARTICLES, "generations": GENS,
                       "frames": FRAMES, "parallelism": "replicas"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- many sequences at once -------------------------------------------------------------------

BATCH_SEQ, BATCH_FRAMES = 64, 8
BATCH_METRIC = "hypothesis evals/s (render+cost, 64 sequences, 48-256 px ROIs)"
BATCH_WORKLOAD = ("batched tracking: 64 independent sequences, square ROIs with sides uniform in [48, 256] px "
                  "(Kinect view scaled to the ROI), particles per sequence from {32, 64, 128, 256}, 40 generations, "
                  "uint16 depth with the Kinect-scale noise recipe")


def percentile(xs, q):
    xs = sorted(xs)
    k = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def batch_setup(hs, I, model, seed, frames, dev, render, ctas):
    """The batched workload: 64 sequences' frames resident in HBM (PackedObs
    each, with pinned twins), the staging buffers the batch is bound to, the
    batch and its tracker (render kernel autotuned on frame 0 when render is
    "tune")."""
    import torch
    from paper_2005_07068_b300.tracker import BatchTracker, PackedObs
    sizes, Ps, seq_seeds = I.batch_workload(seed, BATCH_SEQ)
    cams, trajs = [], []
    store = [PackedObs(sizes, device=dev) for _ in range(frames)]  # resident frames (+ pinned twins)
    for q, (Wq, Hq) in enumerate(sizes):
        ct = I.kinect_camera(Wq, Hq)
        cams.append(hs.camera(ct.fx, ct.fy, ct.cx, ct.cy))
        traj, _, host = make_frames(seq_seeds[q], frames, hs, I, model, cams[q], dev, W=Wq, H=Hq,
                                    keep_device=False)
        trajs.append(traj)
        for f in range(frames):
            store[f].write_host(q, *host[f])
    for st in store:
        st.upload(non_blocking=False)
    staging = PackedObs(sizes, device=dev, pinned=False)  # the buffers the batch is bound to
    batch = hs.Batch(model, staging.obs, cams, Ps, seq_seeds)
    score = hs.score_params(variant=hs.RENDER_VARIANTS.get(render, 0), ctas_per_particle=ctas)
    trk = BatchTracker(model, batch, GENS, device=dev, score=score)
    gt0 = torch.from_numpy(np.stack([t[0] for t in trajs])).to(dev)
    tune = None
    if render == "tune":
        staging.dev.copy_(store[0].dev)
        tune = trk.autotune(gt0)
    return sizes, Ps, store, staging, batch, trk, gt0, tune


def batch_render_roofline(hs, model, sizes, Ps, store, staging, batch, trk, gt0, kinds, pk, dev):
    """Roofline of render_score_multi on the batched workload: frame 0 of every
    sequence tracked step by step, the 40 render launches' inputs kept, then
    replayed back to back from one captured graph (CUDA events)."""
    import torch
    Pt = batch.P_total
    hist_p = torch.zeros(GENS, Pt, model.n_prims, 16, device=dev)
    hist_k = torch.zeros(GENS, Pt, device=dev)
    staging.dev.copy_(store[0].dev)
    cur, nxt = trk.x_buf
    trk.swarm.x = cur
    trk.seed_poses.copy_(gt0)
    hs.hs_obs_prepare_multi(batch)
    hs.pso_init_multi(model, batch, trk.swarm, trk.seed_poses, trk.scale, 0)
    hs.pose_fk_multi(model, batch, cur, trk.prims, trk.kc)
    for gen in range(1, GENS + 1):
        hist_p[gen - 1].copy_(trk.prims)
        hist_k[gen - 1].copy_(trk.kc)
        hs.render_score_multi(model, batch, trk.prims, trk.kc, trk.score, trk.ws, trk.swarm.E)
        trk.swarm.x = cur
        hs.pso_step_fk_multi(model, batch, trk.swarm, nxt, trk.pso, 0, gen, trk.prims, trk.kc)
        cur, nxt = nxt, cur
    trk.swarm.x = cur
    E_tmp = torch.zeros(Pt, device=dev)

    def renders():
        for q in range(GENS):
            hs.render_score_multi(model, batch, hist_p[q], hist_k[q], trk.score, trk.ws, E_tmp)
        return GENS

    render_us = replay_render_us(dev, renders)
    Wp = np.repeat([w for w, _ in sizes], Ps)
    Hp = np.repeat([h for _, h in sizes], Ps)
    tests = np.mean([algorithmic_tests(hist_p[q, :, :, 14:16].cpu().numpy(), kinds, Wp, Hp)
                     for q in range(0, GENS, 4)], axis=0)
    variant = hs.render_variant(trk.score, Pt)
    rec = roofline_record(tests, render_us, pk, f"render_score_multi ({variant})",
                          "CUDA events around a graph of one frame's 40 render_score_multi launches", 3 * GENS,
                          traffic=profile_traffic("batch", variant))
    rec.update({"workload": f"{batch.S} sequences, {Pt} particles, ROIs 48-256 px (one frame, 40 generations)",
                "ctas_per_particle": trk.score.ctas_per_particle})
    del hist_p, hist_k
    return rec


def batch_throughput(hs, bset, frames, steps, warmup, dev):
    """Tracking throughput of the batched workload: frames of every sequence
    replayed from their captured graphs (frame f's data copied into the bound
    buffers first), L2 flushed between steps, CUDA events around each step.
    Returns evals/s and the per-frame latency of every sequence (p50 / p99)."""
    import torch
    sizes, Ps, store, staging, batch, trk, gt0, _ = bset
    graphs = [trk.graph(f, gt0 if f == 0 else None) for f in range(frames)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        staging.dev.copy_(store[i % frames].dev)
        graphs[i % frames].replay()

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        step(warmup + i)
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in evs]
    return {"value": steps * trk.evals_per_frame() / (sum(ms) * 1e-3), "unit": "evals/s",
            "ms_per_frame": sum(ms) / steps, "latency_ms": {"p50": percentile(ms, 50), "p99": percentile(ms, 99)},
            "steps": steps, "warmup": warmup, "gpu_launches_per_step": trk.launches_per_frame(),
            "sequences": batch.S, "particles_total": batch.P_total,
            "step": "one frame of every sequence: one frame copy + one CUDA graph; L2 flushed between steps"}


def batch_frame_throughput(hs, bset, frames, steps, warmup, dev):
    """The same tracking with each frame of every sequence in one cooperative
    launch (track_frame_multi, after the two observation passes), bit for bit
    the graph path's swarms; timed like batch_throughput."""
    import torch
    from paper_2005_07068_b300.tracker import BatchFrameTracker
    sizes, Ps, store, staging, batch, trk, gt0, _ = bset
    ft = BatchFrameTracker(trk.model, batch, trk.gens, score=trk.score)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        f = i % frames
        staging.dev.copy_(store[f].dev)
        ft.run_frame(f, gt0 if f == 0 else None)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        step(warmup + i)
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in evs]
    out = {"value": steps * ft.evals_per_frame() / (sum(ms) * 1e-3), "unit": "evals/s",
           "ms_per_frame": sum(ms) / steps, "latency_ms": {"p50": percentile(ms, 50), "p99": percentile(ms, 99)},
           "steps": steps, "warmup": warmup, "gpu_launches_per_step": ft.launches_per_frame(),
           "ctas": hs.frame_multi_capacity(batch, trk.model),
           "kernel": "track_frame_multi: one cooperative launch per frame of every sequence (per-particle tasks)",
           "step": "one frame of every sequence: one frame copy + the observation passes + one launch; "
                   "L2 flushed between steps"}
    del ft
    return out


def run_batch(args, rank, world, local):
    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I
    from paper_2005_07068_b300 import replicas as R

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    peaks = measured_peaks()
    seed = R.replica_seed(I.CONFIG_SEED_BASE + 4, rank)
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    frames = 2 if args.profile else BATCH_FRAMES
    sizes, Ps, store, staging, batch, trk, gt0, tune = batch_setup(hs, I, model, seed, frames, dev, args.render,
                                                                    args.ctas)
    graphs = [trk.graph(f, gt0 if f == 0 else None) for f in range(frames)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    evals_frame = trk.evals_per_frame()

    def step(i):
        f = i % frames
        staging.dev.copy_(store[f].dev)  # this frame of every sequence into the bound buffers
        graphs[f].replay()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for i in range(K):
            flush.zero_()
            evs[i][0].record(stream)
            step(args.warmup + i)
            evs[i][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        wall = time.perf_counter() - w0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, t_dev, _ = R.aggregate(sum(step_ms) / 1e3, K * evals_frame, dev)

    clocks = clk.summary(peaks.get("sm_max_mhz", 2032.0))
    if args.profile or args.no_roofline:
        # the short form also runs two frames through the batch frame kernel
        fp = batch_frame_throughput(hs, (sizes, Ps, store, staging, batch, trk, gt0, tune), frames, 1, 1, dev)
        if rank == 0:
            print(json.dumps({"metric": BATCH_METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
                              "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / K,
                              "higher_is_better": True, "note": "short run (--profile / --no-roofline)",
                              "clocks": clocks, "gpu_launches": K * trk.launches_per_frame(),
                              "frame_path": fp}), flush=True)
        return 0

    # the same frames with each frame in one cooperative launch
    frame_path = batch_frame_throughput(hs, (sizes, Ps, store, staging, batch, trk, gt0, tune), frames, K,
                                        args.warmup, dev)

    # roofline: the render launches of one frame replayed back to back
    Pt = batch.P_total
    roofline = batch_render_roofline(hs, model, sizes, Ps, store, staging, batch, trk, gt0, g.prims_i[:, 1],
                                     fp32_xu_peaks(dev, peaks), dev)

    # end to end: one pinned copy of every sequence's frame, the graph, the results read back
    e2e = None
    if not args.no_e2e:
        out = torch.zeros(batch.S, 27, dtype=torch.float32).pin_memory()

        def track(i):
            f = i % frames
            staging.dev.copy_(store[f].host, non_blocking=True)
            graphs[f].replay()
            out[:, :26].copy_(trk.swarm.gbest, non_blocking=True)
            out[:, 26].copy_(trk.swarm.gbest_E, non_blocking=True)

        for i in range(args.warmup):
            track(i)
        torch.cuda.synchronize(dev)
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i in range(K):
            flush.zero_()
            ee[i][0].record(stream)
            track(args.warmup + i)
            ee[i][1].record(stream)
        torch.cuda.synchronize(dev)
        e2e_value, _, _ = R.aggregate(sum(a.elapsed_time(b) for a, b in ee) / 1e3, K * evals_frame, dev)
        e2e = {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": int(staging.nbytes),
               "d2h_bytes_per_step": int(out.numel() * out.element_size())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, gens, cores = time_oracle(seed, args.cpu_seconds)
        cpu = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"one 320x240 Kinect-scale frame (oracle-rendered), {PARTICLES} particles x {gens} "
                         f"generations of the FP64 oracle; its cost per evaluation grows with the ROI area "
                         f"(76800 px here, {np.mean([w * h for w, h in sizes]):.0f} px mean in this batch)"}
    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "sequences": batch.S, "particles_total": Pt,
                           "roi_px_mean": float(np.mean([w * h for w, h in sizes])), "generations": GENS,
                           "frames": frames, "step": f"one frame of every sequence = one CUDA graph "
                                                     f"({trk.launches_per_frame()} kernels) + one frame copy",
                           "l2": "flushed between steps (256 MiB write outside the step events)",
                           "parallelism": f"replicas x{world}", "wall_s": wall,
                           "render": {"kernel": hs.render_variant(trk.score, Pt),
                                      "ctas_per_particle": trk.score.ctas_per_particle, "autotune_us": tune}},
                "latency_ms": {"p50": percentile(step_ms, 50), "p99": percentile(step_ms, 99),
                               "what": "per-frame latency of every sequence (one step advances all of them)"},
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
                "gpu_launches": K * trk.launches_per_frame(), "frame_path": frame_path}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---- full frames: seconds per frame to <= 5 degrees -----------------------------------------

FULL_GENS = 50
FULL_METRIC = "s/frame to track within 5 deg mean joint error"
FULL_WORKLOAD = ("full-frame tracking: {W}x{H} uint16 depth + uint8 skin (Kinect noise recipe), seeded {F}-frame "
                 "trajectory (<= 5 deg / 5 mm per frame), frame 0 from the ground truth perturbed by U[+-10 deg, "
                 "+-10 mm], methods {M} x swarm sizes {P} x generation budgets {G} per frame")


def replay_render_us(dev, renders, reps: int = 3) -> float:
    """Average microseconds per render launch of `renders()` (n launches) replayed
    back to back from one captured graph, CUDA events on the launching stream."""
    import torch
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        n = renders()
    stream.wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        renders()
    g.replay()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) * 1e3 / (reps * n)


def record_frame_renders(hs, model, obs, cam, trk, seed_pose, seed, frame, gens, hist_p, hist_k, n=0):
    """One frame tracked step by step (init, FK, then gens x (render, fused
    step)), keeping the records and kc every render consumed in hist_p[n:],
    hist_k[n:]; returns the next free slot."""
    cur, nxt = trk.x_buf
    trk.swarm.x = cur
    trk.seed_pose.copy_(seed_pose)
    hs.hs_obs_prepare(obs)
    hs.pso_init(model, trk.swarm, trk.seed_pose, trk.scale, seed, frame)
    hs.pose_fk(model, cur, cam, trk.prims, trk.kc)
    for gen in range(1, gens + 1):
        hist_p[n].copy_(trk.prims)
        hist_k[n].copy_(trk.kc)
        n += 1
        hs.render_score_batch(model, obs, cam, trk.prims, trk.kc, trk.score, trk.ws, trk.swarm.E)
        trk.swarm.x = cur
        hs.pso_step_fk(model, trk.swarm, nxt, trk.pso, seed, frame, gen, cam, trk.prims, trk.kc)
        cur, nxt = nxt, cur
    trk.swarm.x = cur
    return n


FULL_ROOF_GENS = 10


def fullframe_render_roofline(hs, I, model, kinds, pk, dev, P, seed, Wf=640, Hf=480, obs=None, start=None,
                              render="tune", ctas=0, gens=FULL_ROOF_GENS, score=None):
    """Roofline of render_score_batch on full Kinect frames (Wf x Hf, P
    particles): frame 0 of the seeded sequence tracked from a perturbed start
    for `gens` generations, the render launches' inputs kept and replayed back
    to back from one captured graph (CUDA events)."""
    import torch
    from paper_2005_07068_b300.tracker import Tracker
    camt = I.kinect_camera(Wf, Hf)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    if obs is None:
        traj, obs_l, _ = make_frames(seed, 1, hs, I, model, cam, dev, W=Wf, H=Hf)
        obs = obs_l[0]
        rng = np.random.default_rng(seed)
        start_np = np.clip(traj[0] + rng.uniform(-1, 1, 26) * I.perturbation_scale(), lo, hi).astype(np.float32)
        start = torch.from_numpy(start_np).to(dev)
    tune = None
    if score is None:
        score = hs.score_params(variant=hs.RENDER_VARIANTS.get(render, 0), ctas_per_particle=ctas)
    elif render == "tune":
        render = "given"
    if render == "tune":
        tuner = Tracker(model, cam, P, 1, seed=seed, device=dev, score=score)
        tune = tuner.autotune(obs, start)
        score = tuner.score
        del tuner
    trk = Tracker(model, cam, P, gens, seed=seed, device=dev, score=score)
    hist_p = torch.zeros(gens, P, model.n_prims, 16, device=dev)
    hist_k = torch.zeros(gens, P, device=dev)
    record_frame_renders(hs, model, obs, cam, trk, start, seed, 0, gens, hist_p, hist_k)
    E_tmp = torch.zeros(P, device=dev)

    def renders():
        for q in range(gens):
            hs.render_score_batch(model, obs, cam, hist_p[q], hist_k[q], trk.score, trk.ws, E_tmp)
        return gens

    us = replay_render_us(dev, renders)
    tests = np.mean([algorithmic_tests(hist_p[q, :, :, 14:16].cpu().numpy(), kinds, Wf, Hf)
                     for q in range(0, gens, max(1, gens // 5))], axis=0)
    variant = hs.render_variant(trk.score, P)
    rec = roofline_record(tests, us, pk, f"render_score_batch ({variant})",
                          f"CUDA events around a graph of {gens} render_score_batch launches (generations 1-{gens} "
                          f"of a tracked frame)", 3 * gens, traffic=profile_traffic(f"fullframe{Wf}x{Hf}P{P}", variant))
    rec.update({"workload": f"{Wf}x{Hf} uint16 Kinect-style frame, {P} particles", "particles": P,
                "ctas_per_particle": trk.score.ctas_per_particle, "autotune_us": tune})
    del trk, hist_p, hist_k
    torch.cuda.empty_cache()
    return rec


WITHIN_FRAMES = 30
WITHIN_SETTINGS = (("plain", 1024, 50), ("hybrid", 4096, 20))  # the 640x480 sweep's fastest settings that track


def within_5deg_record(hs, I, model, dev, seed, render="tune", ctas=0, frames=WITHIN_FRAMES):
    """The headline metric's second half in the default line: seconds per frame
    to track within 5 deg (>= 90 % of frames end within 5 deg mean joint error
    over the 23 angular DOFs) on the first `frames` frames of the seeded
    640x480 sequence, for the full sweep's fastest plain and hybrid settings;
    CUDA events around each frame's graph."""
    import torch
    from paper_2005_07068_b300 import sweep as SW
    from paper_2005_07068_b300.tracker import HybridTracker, Tracker
    Wf, Hf = 640, 480
    camt = I.kinect_camera(Wf, Hf)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    traj, obs, _ = make_frames(seed, frames, hs, I, model, cam, dev, W=Wf, H=Hf)
    rng = np.random.default_rng(seed)
    start_np = np.clip(traj[0] + rng.uniform(-1, 1, 26) * I.perturbation_scale(), lo, hi).astype(np.float32)
    start = torch.from_numpy(start_np).to(dev)
    settings = []
    for method, P, G in WITHIN_SETTINGS:
        score = hs.score_params(variant=hs.RENDER_VARIANTS.get(render, 0), ctas_per_particle=ctas)
        if render == "tune":
            tuner = Tracker(model, cam, P, 1, seed=seed, device=dev, score=score)
            tuner.autotune(obs[0], start)
            score = tuner.score
            del tuner
        if method == "plain":
            trk = Tracker(model, cam, P, G, seed=seed, device=dev, score=score)
        else:
            trk = HybridTracker(model, cam, P, G, seed=seed, device=dev, score=score, k=8, steps=5)
        results = SW.track_sequence(trk, obs, traj, start, frames=frames)
        summ = SW.summarize(results)
        summ.update({"method": method, "particles": P, "generations": G,
                     "render": hs.render_variant(trk.score, P), "launches_per_frame": trk.launches_per_frame()})
        settings.append(summ)
        del trk
        torch.cuda.empty_cache()
    best = SW.fastest_within(settings, 0.9)
    return {"metric": f"{FULL_METRIC} ({Wf}x{Hf})", "value": best["frame_ms_mean"] * 1e-3 if best else None,
            "unit": "s/frame", "higher_is_better": False, "frames": frames, "threshold_deg": 5.0,
            "criterion": ">= 90 % of frames end within 5 deg mean joint error (23 angular DOFs)",
            "value_from": (f"{best['method']}: {best['particles']} particles x {best['generations']} generations"
                           if best else "no setting tracked within 5 deg on 90 % of frames"),
            "timing": "CUDA events around each frame's graph (observation totals, init, FK, G x (render, step))",
            "settings": settings}


def run_fullframe(args, rank, world, local):
    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I
    from paper_2005_07068_b300 import replicas as R
    from paper_2005_07068_b300 import sweep as SW
    from paper_2005_07068_b300.tracker import HybridTracker, Tracker

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measured_peaks()
    seed = R.replica_seed(I.CONFIG_SEED_BASE + 5, rank)
    FULL_W, FULL_H = (int(v) for v in args.roi.split(","))
    methods = [m for m in args.methods.split(",") if m]
    if any(m not in ("plain", "hybrid") for m in methods):
        raise SystemExit("--methods takes plain and/or hybrid")
    k_pol, steps_pol = (int(v) for v in args.polish.split(","))
    kc_var, kc_w = args.kc.split(",")
    kc_var, kc_w = int(kc_var), float(kc_w)
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    if kc_var != hs.HS_KC_ABDUCTION:
        model.set_kc(kc_var, kc_w)
    camt = I.kinect_camera(FULL_W, FULL_H)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    frames = max(2, args.frames)
    traj, obs, _ = make_frames(seed, frames, hs, I, model, cam, dev, W=FULL_W, H=FULL_H)
    rng = np.random.default_rng(seed)
    start_np = np.clip(traj[0] + rng.uniform(-1, 1, 26) * I.perturbation_scale(), lo, hi).astype(np.float32)
    start = torch.from_numpy(start_np).to(dev)
    kinds = g.prims_i[:, 1]
    pk = fp32_xu_peaks(dev, peaks)
    settings, per_p = [], []
    gen_budgets = [int(v) for v in args.gens.split(",") if v]
    log = None
    if args.log and rank == 0:
        from paper_2005_07068_b300.runlog import RunLog
        log = RunLog(args.log)
    with ClockSampler(local) as clk:
        for P in [int(v) for v in args.particles.split(",") if v]:
            score = hs.score_params(variant=hs.RENDER_VARIANTS.get(args.render, 0), ctas_per_particle=args.ctas)
            tune = None
            if args.render == "tune":
                tuner = Tracker(model, cam, P, 1, seed=seed, device=dev, score=score)
                tune = tuner.autotune(obs[0], start)
                score = tuner.score
                del tuner
            for method in methods:
                for G in gen_budgets:
                    hist = log is not None
                    if method == "plain":
                        trk = Tracker(model, cam, P, G, seed=seed, device=dev, score=score, record_history=hist)
                    else:
                        trk = HybridTracker(model, cam, P, G, seed=seed, device=dev, score=score,
                                            k=min(k_pol, P), steps=steps_pol, record_history=hist)
                    results = SW.track_sequence(trk, obs, traj, start, frames=frames, log=log, method=method,
                                                particles=P, generations=G)
                    summ = SW.summarize(results)
                    summ.update({"method": method, "particles": P, "generations": G,
                                 "evals_per_s": P * G * frames / (sum(r.frame_ms for r in results) * 1e-3),
                                 "launches_per_frame": trk.launches_per_frame()})
                    settings.append(summ)
                    if log is not None:
                        log.run(**summ)
                    del trk
            # render roofline at this P: generations of frame 0 replayed back to back
            rec = fullframe_render_roofline(hs, I, model, kinds, pk, dev, P, seed, FULL_W, FULL_H, obs=obs[0],
                                            start=start, score=score)
            rec["autotune_us"] = tune
            per_p.append(rec)
    clocks = clk.summary(peaks.get("sm_max_mhz", 2032.0))
    best = SW.fastest_within(settings, 0.9)
    if log is not None:
        for rec in per_p:
            log.run(record="render roofline", **{k: v for k, v in rec.items() if k != "autotune_us"})
        log.close()
    if rank == 0:
        work = FULL_WORKLOAD.format(W=FULL_W, H=FULL_H, F=frames, M=" / ".join(methods), P=args.particles,
                                    G=args.gens)
        line = {"metric": f"{FULL_METRIC} ({FULL_W}x{FULL_H})", "value": best["frame_ms_mean"] * 1e-3 if best else None,
                "unit": "s/frame", "n_gpus": world, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": work, "roi": [FULL_W, FULL_H], "frames": frames, "threshold_deg": 5.0,
                           "kc": {"variant": kc_var, "pen_weight_rad_per_mm": kc_w},
                           "polish": {"k": k_pol, "steps": steps_pol} if "hybrid" in methods else None,
                           "criterion": ">= 90 % of frames end within 5 deg mean joint error (23 angular DOFs)",
                           "value_from": (f"{best['method']}: {best['particles']} particles x {best['generations']} "
                                          f"generations" if best else
                                          "no setting tracked within 5 deg on 90 % of frames"),
                           "timing": "CUDA events around each frame's graph (observation totals, init, FK, "
                                     "G x (render, fused step))"},
                "settings": settings, "per_swarm_size": per_p, "clocks": clocks,
                "gpu_launches": sum(s_["launches_per_frame"] * s_["frames"] for s_ in settings)}
        print(json.dumps(line), flush=True)
    return 0


POLISH_METRIC = "gradient polish: one descent step of 8 particles (us)"


def run_polish(args, rank, world, local):
    """The gradient polish's kernels alone (Section III.B's hybrid, the
    smoothed objective E_s and its adjoint): 8 particles around the ground
    truth of a seeded Kinect-style frame at 320x240 and 640x480, each kernel
    and one whole descent step (FK, soft_score, soft_score_backward,
    pose_grad, polish_step) replayed from a captured graph, CUDA events."""
    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import grad as GR
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    P = 8
    scale = np.full(26, np.radians(10.0), np.float32)
    scale[:3] = 10.0
    out = {}
    with ClockSampler(local) as clk:
        for Wp, Hp in ((320, 240), (640, 480)):
            ct = I.kinect_camera(Wp, Hp)
            cam = hs.camera(ct.fx, ct.fy, ct.cx, ct.cy)
            traj, obs, _ = make_frames(I.CONFIG_SEED_BASE + 3, 1, hs, I, model, cam, dev, W=Wp, H=Hp)
            hs.hs_obs_prepare(obs[0])
            rng = np.random.default_rng(3)
            poses = torch.from_numpy(np.clip(traj[0][None] + 0.3 * rng.uniform(-1, 1, (P, 26)) *
                                             I.perturbation_scale(), lo, hi).astype(np.float32)).to(dev)
            sc = GR.SoftScorer(model, obs[0], cam, max_particles=P, device=dev)
            E = torch.empty(P, device=dev)
            x = poses.clone()
            sc.forward(x)
            sc.gradient(x)
            calls = {
                "soft_score": lambda: hs.soft_score(model, obs[0], cam, sc.prims, sc.kc, sc.params, sc.soft, sc.ws,
                                                    E, sc.sums),
                "soft_score_backward": lambda: hs.soft_score_backward(model, obs[0], cam, sc.prims, sc.params,
                                                                      sc.soft, sc.sums, sc.adj),
                "pose_grad": lambda: hs.pose_grad(model, x, cam, sc.params, sc.prims, sc.kc, sc.adj, sc.grad),
            }

            kernels = tuple(calls.values())

            def step():
                hs.pose_fk(model, x, cam, sc.prims, sc.kc)
                for fn in kernels:
                    fn()
                hs.polish_step(model, x, sc.grad, 0.5, scale)

            calls["descent_step"] = step
            rec = {}
            reps = max(1, args.steps)

            def repeat(fn):
                for _ in range(reps):
                    fn()
                return reps

            for name, fn in calls.items():
                rec[name + "_us"] = replay_render_us(dev, lambda: repeat(fn))
            out[f"{Wp}x{Hp}"] = rec
    clocks = clk.summary(measured_peaks().get("sm_max_mhz", 2032.0))
    if rank == 0:
        print(json.dumps({"metric": POLISH_METRIC, "value": out["320x240"]["descent_step_us"], "unit": "us",
                          "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "8 particles around the ground truth (0.3 of the tracking "
                                                 "perturbation) of a seeded Kinect-style frame; tau 0.5 px, "
                                                 "tau_mm 0.5 mm", "step": "pose_fk, soft_score, "
                                     "soft_score_backward, pose_grad, polish_step"},
                          "per_roi": out, "clocks": clocks}), flush=True)
    return 0


def run_render(args, rank, world, local):
    """render_score_batch alone: one seeded Kinect-style frame at --roi, the
    first swarm size of --particles spread around the ground truth (half the
    tracking perturbation), kernel --render (not tuned), --warmup untimed and
    --steps timed launches (CUDA events).  Few launches, small device
    footprint: the command profiling summaries capture one kernel with."""
    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    Wr, Hr = (int(v) for v in args.roi.split(","))
    P = int(args.particles.split(",")[0])
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    camt = I.kinect_camera(Wr, Hr)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    seed = I.CONFIG_SEED_BASE + 5
    traj, obs, _ = make_frames(seed, 1, hs, I, model, cam, dev, W=Wr, H=Hr)
    rng = np.random.default_rng(seed)
    poses = np.clip(traj[0][None] + 0.5 * rng.uniform(-1, 1, (P, 26)) * I.perturbation_scale(), lo, hi)
    prims = torch.zeros(P, model.n_prims, 16, device=dev)
    kc = torch.zeros(P, device=dev)
    hs.pose_fk(model, torch.from_numpy(poses.astype(np.float32)).to(dev), cam, prims, kc)
    hs.hs_obs_prepare(obs[0])
    ws = hs.new_workspace(P, dev)
    E = torch.zeros(P, device=dev)
    variant = "auto" if args.render == "tune" else args.render
    prm = hs.score_params(variant=hs.RENDER_VARIANTS[variant], ctas_per_particle=args.ctas)
    for _ in range(args.warmup):
        hs.render_score_batch(model, obs[0], cam, prims, kc, prm, ws, E)
    torch.cuda.synchronize(dev)
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record()
    for _ in range(args.steps):
        hs.render_score_batch(model, obs[0], cam, prims, kc, prm, ws, E)
    b_ev.record()
    torch.cuda.synchronize(dev)
    tests = algorithmic_tests(prims[:, :, 14:16].cpu().numpy(), g.prims_i[:, 1], Wr, Hr)
    us = a_ev.elapsed_time(b_ev) * 1e3 / max(args.steps, 1)
    rec = roofline_record(tests, us, fp32_xu_peaks(dev, measured_peaks()), f"render_score_batch ({variant})",
                          "CUDA events around back-to-back eager launches", args.steps)
    if rank == 0:
        print(json.dumps({"workload": f"render only: {Wr}x{Hr}, {P} particles", "launch_us": us,
                          "roofline": rec, "gpu_launches": args.warmup + args.steps}), flush=True)
    return 0


EQ_METRIC = "share of frames within 5 deg mean joint error at equal time per frame (320x240)"


def run_equal_time(args, rank, world, local):
    """Hybrid PSO (64 particles x 20 generations, every generation 5 descent
    steps of E_s on the 8 best) against plain PSO given the same wall time per
    frame, on the Kinect-scale sequence: plain with 64 particles and as many
    generations as fit, and plain with the swarm size (x 40 generations) whose
    frame time is nearest.  Every frame is one CUDA graph timed with events."""
    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I
    from paper_2005_07068_b300 import replicas as R
    from paper_2005_07068_b300 import sweep as SW
    from paper_2005_07068_b300.tracker import HybridTracker, Tracker

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measured_peaks()
    seed = R.replica_seed(I.CONFIG_SEED_BASE + 2, rank)
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    camt = I.kinect_camera(W, H)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    # the Kinect-scale sequence: its first 30 frames unless --frames asks for more (up to 300)
    frames = max(2, min(args.frames, 300)) if args.frames_given else FRAMES
    traj, obs, _ = make_frames(seed, frames, hs, I, model, cam, dev)
    rng = np.random.default_rng(seed)
    start = torch.from_numpy(np.clip(traj[0] + rng.uniform(-1, 1, 26) * I.perturbation_scale(), lo, hi)
                             .astype(np.float32)).to(dev)

    def run(trk, n=frames):
        summ = SW.summarize(SW.track_sequence(trk, obs, traj, start, frames=n))
        summ.update({"particles": trk.P, "generations": trk.gens, "launches_per_frame": trk.launches_per_frame()})
        return summ

    k_pol, steps_pol = (int(v) for v in args.polish.split(","))
    with ClockSampler(local) as clk:
        hyb = run(HybridTracker(model, cam, 64, 20, seed=seed, device=dev, k=k_pol, steps=steps_pol))
        hyb["method"] = "hybrid"
        t_h = hyb["frame_ms_mean"]
        # plain, 64 particles: generations that fill the hybrid's frame time
        cal = run(Tracker(model, cam, 64, 40, seed=seed, device=dev), n=min(4, frames))
        g_eq = max(40, int(round(40 * t_h / cal["frame_ms_mean"])))
        plain_g = run(Tracker(model, cam, 64, g_eq, seed=seed, device=dev))
        plain_g["method"] = "plain, more generations"
        # plain, 40 generations: the swarm size whose frame time is nearest
        best = None
        for P in (256, 512, 1024, 2048, 4096):
            c = run(Tracker(model, cam, P, 40, seed=seed, device=dev), n=min(4, frames))
            if best is None or abs(c["frame_ms_mean"] - t_h) < abs(best[1] - t_h):
                best = (P, c["frame_ms_mean"])
        plain_p = run(Tracker(model, cam, best[0], 40, seed=seed, device=dev))
        plain_p["method"] = "plain, larger swarm"
    clocks = clk.summary(peaks.get("sm_max_mhz", 2032.0))
    if rank == 0:
        rows = [hyb, plain_g, plain_p]
        print(json.dumps({"metric": EQ_METRIC, "value": hyb["within_fraction"], "unit": "fraction of frames",
                          "n_gpus": world, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                          "vs_baseline": None,
                          "config": {"workload": WORKLOAD, "frames": frames, "threshold_deg": 5.0,
                                     "hybrid": f"64 particles x 20 generations, every generation {steps_pol} descent "
                                               f"steps of E_s on the {k_pol} best",
                                     "value_from": "the hybrid's share; the plain rows get the same time per frame",
                                     "timing": "CUDA events around each frame's graph"},
                          "settings": rows, "clocks": clocks,
                          "gpu_launches": sum(r["frames"] * r["launches_per_frame"] for r in rows)}), flush=True)
    return 0


# ---- the native arm ------------------------------------------------------------------------

def main():
    args = parse()
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch":
        return run_batch(args, rank, world, local)
    if args.workload == "fullframe":
        return run_fullframe(args, rank, world, local)
    if args.workload == "render":
        return run_render(args, rank, world, local)
    if args.workload == "equaltime":
        return run_equal_time(args, rank, world, local)
    if args.workload == "polish":
        return run_polish(args, rank, world, local)

    import torch
    from paper_2005_07068_b300 import build as B
    from paper_2005_07068_b300 import handscore as hs
    from paper_2005_07068_b300 import inputs as I
    from paper_2005_07068_b300 import replicas as R
    from paper_2005_07068_b300.tracker import Tracker

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    peaks = measured_peaks()
    seed = R.replica_seed(I.CONFIG_SEED_BASE + 2, rank)
    g = I.hand_geometry()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    model = hs.Model.from_geometry(g, lo, hi)
    camt = I.kinect_camera(W, H)
    cam = hs.camera(camt.fx, camt.fy, camt.cx, camt.cy)
    frames = min(FRAMES, max(args.steps + args.warmup, 2)) if args.profile else FRAMES
    traj, obs, host = make_frames(seed, frames, hs, I, model, cam, dev)
    gt0 = torch.from_numpy(traj[0]).to(dev)
    score = hs.score_params(variant=hs.RENDER_VARIANTS.get(args.render, 0), ctas_per_particle=args.ctas)
    trk = Tracker(model, cam, PARTICLES, GENS, seed=seed, device=dev, score=score)
    tune = trk.autotune(obs[0], gt0) if args.render == "tune" else None
    graphs = [trk.graph(obs[f], f, gt0 if f == 0 else None) for f in range(frames)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        graphs[i % frames].replay()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)

    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for i in range(K):
            flush.zero_()  # evict the previous frame from the 126 MB L2 (outside the step events)
            evs[i][0].record(stream)
            step(args.warmup + i)
            evs[i][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        wall = time.perf_counter() - w0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, t_dev, evals_total = R.aggregate(sum(step_ms) / 1e3, K * PARTICLES * GENS, dev)

    # ---- the same frames, one cooperative launch per frame (track_frame) ----
    # The frame kernel keeps every particle's records and state on chip and
    # meets at one grid barrier per generation; it moves the swarm exactly as
    # the graph does.  Timed the same way (L2 flushed between steps).
    frame_path = None
    if not args.no_frame_path:
        from paper_2005_07068_b300.tracker import FrameTracker
        ft = FrameTracker(model, cam, PARTICLES, GENS, seed=seed, device=dev, score=trk.score)
        ftab = ft.autotune(obs[0], gt0)

        def fstep(i):
            f = i % frames
            ft.run_frame(obs[f], f, gt0 if f == 0 else None)

        for i in range(args.warmup):
            fstep(i)
        torch.cuda.synchronize(dev)
        fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        with ClockSampler(local) as fclk:
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            for i in range(K):
                flush.zero_()
                fev[i][0].record(stream)
                fstep(args.warmup + i)
                fev[i][1].record(stream)
            torch.cuda.synchronize(dev)
        f_value, f_t, _ = R.aggregate(sum(a.elapsed_time(b) for a, b in fev) / 1e3, K * PARTICLES * GENS, dev)
        fc = fclk.summary(peaks.get("sm_max_mhz", 2032.0))
        frame_path = {"value": f_value, "unit": "evals/s", "ms_per_step": 1e3 * f_t / K,
                      "kernel": "track_frame_kernel: one cooperative launch per frame",
                      "ctas": ft.ctas, "autotune_us_per_frame": ftab, "gpu_launches": K,
                      "clocks": fc}
    graph_ms = 1e3 * t_dev / K
    # the headline is the faster of the two paths (same frames, same swarm)
    use_frame = frame_path is not None and frame_path["ms_per_step"] < graph_ms

    # ---- roofline of render_score_batch ----
    # The timed frames are replayed generation by generation: the primitive
    # records and kc that each generation's render_score_batch consumed are
    # kept, then those launches run back to back in one captured graph, timed
    # with CUDA events on the launching stream (kernel time without host gaps).
    kinds = g.prims_i[:, 1]
    pk = fp32_xu_peaks(dev, peaks)
    clocks = clk.summary(peaks.get("sm_max_mhz", 2032.0))
    rf = min(3, frames) if not args.no_roofline else 0
    render_roofline, roofline, sub, within = None, None, {}, None
    if rf:
        hist_p = torch.zeros(rf * GENS, PARTICLES, model.n_prims, 16, device=dev)
        hist_k = torch.zeros(rf * GENS, PARTICLES, device=dev)
        n = 0
        for f in range(rf):
            n = record_frame_renders(hs, model, obs[f], cam, trk, gt0 if f == 0 else trk.swarm.gbest.clone(), seed,
                                     f, GENS, hist_p, hist_k, n)
        E_tmp = torch.zeros(PARTICLES, device=dev)

        def renders():
            for q in range(n):
                hs.render_score_batch(model, obs[q // GENS], cam, hist_p[q], hist_k[q], trk.score, trk.ws, E_tmp)
            return n

        render_us = replay_render_us(dev, renders, reps=5)
        hb = hist_p[:n, :, :, 14:16].cpu().numpy()
        tests = np.mean([algorithmic_tests(hb[q], kinds) for q in range(n)], axis=0)
        variant = hs.render_variant(trk.score, PARTICLES)
        render_roofline = roofline_record(tests, render_us, pk, f"render_score_batch ({variant})",
                                          "CUDA events around a graph of the timed frames' render_score_batch "
                                          "launches", n * 5, traffic=profile_traffic("kinect", variant))
        roofline = render_roofline
        if use_frame:
            # the frame kernel does all of a frame's renders (and its FK and steps,
            # whose work is not counted): the same algorithmic work per
            # generation, GENS generations per launch, over the launch's duration
            roofline = roofline_record(tests, frame_path["ms_per_step"] * 1e3, pk,
                                       "track_frame_kernel (one cooperative launch per frame)",
                                       "CUDA events around each timed frame's launch on the launching stream", K,
                                       traffic=profile_traffic("kinect", "frame"), gens=GENS,
                                       note=f"{GENS} generations x the render's algorithmic work; FK, cost finish "
                                            f"and swarm steps not counted")
        del hist_p, hist_k
        # the render roofline on the other two workloads the kernels are built
        # for: many sequences with uneven ROIs (render_score_multi) and full
        # 640x480 frames with 4096 particles (render_score_batch)
        if not args.no_sub_rooflines:
            bseed = R.replica_seed(I.CONFIG_SEED_BASE + 4, rank)
            bset = batch_setup(hs, I, model, bseed, 2, dev, args.render, args.ctas)
            thr = batch_throughput(hs, bset, 2, 8, 3, dev)
            thr_f = batch_frame_throughput(hs, bset, 2, 8, 3, dev)
            sub["batch_64seq"] = batch_render_roofline(hs, model, *bset[:7], kinds, pk, dev)
            sub["batch_64seq"]["autotune_us"] = bset[7]
            sub["batch_64seq"]["tracking"] = thr
            sub["batch_64seq"]["tracking_frame_kernel"] = thr_f
            del bset
            torch.cuda.empty_cache()
            fseed = R.replica_seed(I.CONFIG_SEED_BASE + 5, rank)
            sub["fullframe_640x480_P4096"] = fullframe_render_roofline(hs, I, model, kinds, pk, dev, 4096, fseed,
                                                                       render=args.render, ctas=args.ctas)
            within = within_5deg_record(hs, I, model, dev, fseed, render=args.render, ctas=args.ctas)

    # ---- end to end: pinned host frame -> device -> graph -> result on the host ----
    e2e = None
    if not args.no_e2e:
        staging = hs.Obs.from_numpy(host[0][0], host[0][1], dev)
        pin = []
        for d16, skin in host:
            from paper_2005_07068_b300.inputs import pitched
            pin.append((torch.from_numpy(pitched(d16)).pin_memory(), torch.from_numpy(pitched(skin)).pin_memory()))
        out = torch.zeros(27, dtype=torch.float32).pin_memory()
        etrk = ft if use_frame else trk
        if not use_frame:
            for f in range(frames):  # capture the staging graphs before timing
                trk.graph(staging, f, gt0 if f == 0 else None)
        for i in range(args.warmup):
            f = i % frames
            etrk.track(pin[f][0], pin[f][1], staging, f, out, gt0 if f == 0 else None)
        torch.cuda.synchronize(dev)
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if dist:
            dist.barrier()
        for i in range(K):
            f = (args.warmup + i) % frames
            flush.zero_()
            ee[i][0].record(stream)
            etrk.track(pin[f][0], pin[f][1], staging, f, out, gt0 if f == 0 else None)
            ee[i][1].record(stream)
        torch.cuda.synchronize(dev)
        e2e_value, _, _ = R.aggregate(sum(a.elapsed_time(b) for a, b in ee) / 1e3, K * PARTICLES * GENS, dev)
        e2e = {"value": e2e_value, "unit": "evals/s",
               "h2d_bytes_per_step": int(pin[0][0].numel() * pin[0][0].element_size() + pin[0][1].numel()),
               "d2h_bytes_per_step": int(out.numel() * out.element_size()),
               "timing": "CUDA events on the stream around each frame's copies in, tracking and result copy out "
                         "(L2 flushed between frames)"}
        # host wall clock: pinned host frame in -> pose on the host, one frame
        # at a time as a live camera delivers them (the host waits for each
        # frame's result before it submits the next; the binding's ctypes
        # calls and the launch are inside the interval; no L2 flush)
        n_wall = max(HOST_WALL_FRAMES, K)
        wall_ms = []
        with ClockSampler(local) as wclk:
            for i in range(n_wall):
                f = (args.warmup + K + i) % frames
                t0 = time.perf_counter()
                etrk.track(pin[f][0], pin[f][1], staging, f, out, gt0 if f == 0 else None)
                torch.cuda.current_stream(dev).synchronize()
                wall_ms.append((time.perf_counter() - t0) * 1e3)
        hw_value, _, _ = R.aggregate(sum(wall_ms) / 1e3, n_wall * PARTICLES * GENS, dev)
        e2e["host_wall"] = {"value": hw_value, "unit": "evals/s", "frames": n_wall,
                            "ms_per_frame_p50": percentile(wall_ms, 50), "ms_per_frame_p99": percentile(wall_ms, 99),
                            "timing": "host perf_counter from submitting a pinned frame to its pose on the host, "
                                      "a stream synchronisation per frame",
                            "clocks": wclk.summary(peaks.get("sm_max_mhz", 2032.0))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, gens, cores = time_oracle(seed, args.cpu_seconds)
        cpu = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"frame 0 of the same workload (oracle-rendered), {PARTICLES} particles x {gens} "
                         f"generations of FP64 FK + brute-force ray cast (all pixels x 37 primitives) + "
                         f"Eq. 4-5 + Eq. 6-7, OpenMP over particles"}

    graph_path = {"value": value, "unit": "evals/s", "ms_per_step": graph_ms,
                  "kernel": f"one CUDA graph of {trk.launches_per_frame()} launches per frame",
                  "gpu_launches": K * trk.launches_per_frame(), "clocks": clocks}
    if use_frame:
        value, step_ms_h, launches, clocks = frame_path["value"], frame_path["ms_per_step"], K, frame_path["clocks"]
        step_desc = (f"one frame = one cooperative launch of track_frame ({PARTICLES} particles, {ft.ctas} CTAs dealt "
                     f"evenly to them for the whole frame; "
                     f"the faster of it and the CUDA graph of the step-by-step calls)")
    else:
        step_ms_h, launches = graph_ms, K * trk.launches_per_frame()
        step_desc = (f"one frame = one CUDA graph ({trk.launches_per_frame()} kernels; the faster of it and the "
                     f"one-launch frame kernel)")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": step_ms_h, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "roi": [W, H], "particles": PARTICLES, "generations": GENS,
                           "frames": frames,
                           "step": step_desc,
                           "l2": "flushed between steps (256 MiB write outside the step events)",
                           "parallelism": f"replicas x{world}", "wall_s": wall,
                           "render": {"kernel": hs.render_variant(trk.score, PARTICLES),
                                      "ctas_per_particle": trk.score.ctas_per_particle, "autotune_us": tune}},
                "roofline": roofline, "render_roofline": render_roofline, "render_rooflines": sub,
                "cpu_baseline": cpu, "clocks": clocks,
                "e2e": e2e, "gpu_launches": launches, "frame_path": frame_path, "graph_path": graph_path,
                "s_per_frame_within_5deg": within}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
