#!/usr/bin/env python3
"""Benchmark of the GB300 DEM timestep library.

Workload: rotating drum, 1,000,000 spheres with radius uniform in [0.8, 1.2] mm
(rho 2500 kg/m^3, E 1 MPa, nu 0.3, e_n 0.5, mu 0.4/0.05/0.05) in a closed
cylinder of 4,096 triangles turning at 30 rpm about the horizontal x axis, 35 %
fill; synthetic seeded start (FCC lattice in the lower drum) settled on the
GPU before timing.  A step is one time step of the whole hot path: mesh pose,
rebuild check with the amortised cell binning / Verlet list / history remap,
contact forces, gather and integration.

Metric: particle-steps/s (Cundall number) of the whole job, headline in
DEM_MIXED (FP32 contact math, compensated state); the DEM_FP64 rate is
reported beside it.  One JSON line on rank 0.

`--impl reference` times the FP64 CPU oracle as it stands, on the host cores,
on a bounded sample of the same workload (a 2,000-sphere drum).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 1M spheres: FP64 vs mixed vs surrogate at stated error"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--settle", type=int, default=6000,
                    help="steps before timing: the lattice collapses into the dense "
                         "flowing bed (contacts per particle level off by ~6000 steps)")
    ap.add_argument("--frame", type=int, default=100, help="steps per state read-back (e2e)")
    ap.add_argument("--fp64-steps", type=int, default=0, help="0: steps // 20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-design", action="store_true",
                    help="skip the OpenMP paper-design CPU program")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble section")
    ap.add_argument("--batch-scenes", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-settle", type=int, default=3000)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--skin", type=float, default=0.0, help="Verlet skin (m); 0: 0.25 R_max")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """SM clock and throttle reasons sampled while the timed region runs.

    Polls NVML (libnvidia-ml, through ctypes) every millisecond from a thread,
    so even a region of a few milliseconds gets samples; falls back to
    `nvidia-smi -lms 100` when NVML cannot be loaded.  Reason bits are those
    of nvmlClocksEventReasons (nvml.h).
    """

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []  # (sm_mhz, max_mhz, reason bits)
        self.source = None
        self._stop = threading.Event()
        self.proc = None
        self.t = None

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(self.idx), "uuid", None)
            if u is not None:
                uuid = str(u)
                if not uuid.startswith("GPU-"):
                    uuid = "GPU-" + uuid
        except Exception:
            uuid = None
        rc = 1
        if uuid:
            rc = lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h))
        if rc != 0:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            ids = [c.strip() for c in vis.split(",") if c.strip()]
            phys = int(ids[self.idx]) if self.idx < len(ids) and ids[self.idx].isdigit() \
                else self.idx
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(phys), ctypes.byref(h))
        if rc != 0:
            raise OSError("no NVML handle")
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, get_reasons

    def _poll_nvml(self, lib, h, get_reasons):
        import ctypes
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while True:
            ok = (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
                  and lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0
                  and get_reasons(h, ctypes.byref(rs)) == 0)
            if ok:
                self.samples.append((float(clk.value), float(mx.value), int(rs.value)))
            if self._stop.wait(0.001):
                break

    def _read_smi(self):
        for line in self.proc.stdout:
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                bits = 0
                for b, val in zip((0x8, 0x40, 0x20, 0x4), f[5:9]):
                    if val.lower() in ("active", "0x1", "1"):
                        bits |= b
                self.samples.append((float(f[1]), float(f[2]), bits))
            except ValueError:
                continue

    def __enter__(self):
        try:
            lib, h, gr = self._nvml_handle()
            self.source = "nvml"
            self.t = threading.Thread(target=self._poll_nvml, args=(lib, h, gr), daemon=True)
            self.t.start()
        except (OSError, AttributeError):
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                     "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi"
                self.t = threading.Thread(target=self._read_smi, daemon=True)
                self.t.start()
            except (OSError, FileNotFoundError):
                self.proc = None
        # the timed region starts once the first sample is in
        t0 = time.time()
        while self.t is not None and not self.samples and time.time() - t0 < 5.0:
            time.sleep(0.001)
        self.n_before = len(self.samples)
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=5)

    def summary(self):
        # samples taken after the region started (the one before it as well
        # if the region was too short for its own)
        smp = self.samples[self.n_before:] or self.samples[-1:]
        if not smp:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "source": self.source}
        reasons = set()
        for _, _, bits in smp:
            for b, name in self.REASONS.items():
                if bits & b:
                    reasons.add(name)
        return {"sm_mhz": float(np.median([c for c, _, _ in smp])),
                "sm_max_mhz": float(max(m for _, m, _ in smp)), "reasons": sorted(reasons),
                "samples": len(smp), "source": self.source}


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """Largest value over the ranks of the process group (x itself if alone)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(n_per_rank: int, steps: int, elapsed_max: float, world: int) -> float:
    """Whole-job particle-steps/s of `world` replicas timed by the slowest."""
    return world * n_per_rank * steps / elapsed_max


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def drum_workload(n: int, seed: int = 5):
    from paper_2507_12610_gb300 import scenes
    # lattice pitch slightly above the mean diameter: the bed starts loose but
    # nearly touching and settles into a dense packing within the settle steps
    return scenes.drum_scene(n=n, seed=seed, nn_dist=2.15e-3, speed=0.02)


def algorithmic_bytes(n: int, st: dict, mixed: bool) -> int:
    """Bytes the method must move in one step-kernel launch, each byte once.

    Per particle: the state read, x, v, w (3 x 24 B), q (32 B) and R (4 B in
    mixed precision, 8 B in FP64), and the state written, x, v, w, q (104 B);
    4 B per candidate list entry; per touching pair (particle pair or
    particle-triangle): the friction history u_s, u_r, u_t read and written
    once (2 x 28 B mixed, 2 x 56 B FP64) and an 8 B pair key; 4 B per triangle
    candidate.  Neighbour gathers and the rebuild are not counted.
    """
    state = (108 if mixed else 112) + 104
    pair = 2 * (28 if mixed else 56) + 8
    return int(n * state + 4 * st["list_entries"] + 4 * st["mesh_candidates"]
               + pair * (st["pair_contacts"] + st["mesh_contacts"]))


# FP64 operations of one step, counted from the law as the library writes it
# (each +, -, *, /, sqrt one operation; static springs with history; the
# divisions and roots expand to several FP64-pipe instructions on the GPU):
# per touching particle pair the geometry (13), the unit normal (4), R*, m*,
# r_i, r_j (9), the rolling radius (3), relative velocities (15), stiffness
# and damping (11), contact velocities (41), normal force and its square (15),
# two vector springs (98), the twisting spring (8) and the torques (46) -- 263
# -- plus 6 additions into each of the two particles' sums: 275; per mesh
# contact about 330 (closest point, wall velocity, the law, one sum); per
# particle the integration, 190 (accelerations with drag 27, positions and
# velocities 12, two SPIRAL factors from their series 84 and the two
# quaternion products 56, spin 6, inertia and drag rates 5).
FP64_FLOPS_PER_PAIR = 275
FP64_FLOPS_PER_MESH_CONTACT = 330
FP64_FLOPS_PER_PARTICLE = 190
# GB300 double precision: 1.25 TFLOP/s nominal (2 FP64 FMAs per SM and clock
# at 2.07 GHz on 152 SMs)
NOMINAL_FP64_TFLOPS = 1.25


def fp64_algorithmic_flops(n: int, st: dict) -> int:
    """FP64 operations one DEM_FP64 step must do (counts of the last step)."""
    return int(FP64_FLOPS_PER_PAIR * st["pair_contacts"]
               + FP64_FLOPS_PER_MESH_CONTACT * st["mesh_contacts"]
               + FP64_FLOPS_PER_PARTICLE * n)


def kernel_sources_sha1() -> str:
    """Hash of the sources the step kernels are compiled from (their .cu files
    and the headers they include); a committed profile counts only while it
    matches."""
    import hashlib
    d = os.path.join(ROOT, "paper_2507_12610_gb300", "csrc")
    files = ["dem_step.cu", "dem_step_fp64.cu", "dem_step_warp.cuh", "dem_step_pairs.cuh",
             "dem_step_common.cuh", "dem_law.cuh", "dem_geom.cuh", "dem_math.cuh",
             "dem_internal.cuh"]
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def sphere_count(n: int) -> str:
    """1000000 -> '1M', 400000 -> '400k'."""
    if n % 1_000_000 == 0:
        return f"{n // 1_000_000}M"
    if n % 1000 == 0:
        return f"{n // 1000}k"
    return str(n)


def measured_traffic(n: int, mixed: bool):
    """DRAM bytes per step-kernel launch from the committed ncu summary.

    The summary (profiles/) records the DRAM bytes of one launch on a smaller
    drum per particle, with the hash of the kernel sources it was taken on; it
    is scaled to n particles (traffic grows in proportion) and reported only
    while the sources are unchanged.
    """
    name = "k_step_warp_mixed_drum400k.md" if mixed else "k_pairs_gather_fp64_drum400k.md"
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith("bench-traffic:"):
                    kv = dict(x.split("=", 1) for x in line.split()[1:])
                    if kv.get("sources_sha1") == kernel_sources_sha1():
                        return int(float(kv["bytes_per_particle"]) * n)
    except OSError:
        pass
    return None


def bench_ours(a):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    ge.build()
    from paper_2507_12610_gb300 import dem

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x: float) -> float:
        return max_over_ranks(x, world, "cuda")

    prec = dem.DEM_MIXED if a.precision == "mixed" else dem.DEM_FP64
    s = drum_workload(a.n, seed=5 + rank)
    n = a.n
    # every scene runs on this stream, so CUDA events recorded on it bracket
    # exactly the library's kernels
    strm = torch.cuda.Stream()
    # settle the bed (not timed), then keep its state as the job's input
    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(s, precision=dem.DEM_MIXED)
    sc.step(a.settle)
    assert sc.synchronize() == 0, "settle failed"
    settled = sc.state()
    sc.close()
    s_set = dict(s, x=settled["x"], v=settled["v"], w=settled["w"], q=settled["q"])

    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(s_set, precision=prec, skin=a.skin)
    sc.step(a.warmup)
    assert sc.synchronize() == 0, "warm-up failed"
    st0 = sc.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(strm)
        sc.step(a.steps)
        e1.record(strm)
        e1.synchronize()
    rc = sc.synchronize()
    barrier()
    assert rc == 0, f"timed run failed: {dem.status_string(rc)}"
    elapsed = rank_max(e0.elapsed_time(e1) / 1e3)
    st = sc.stats()
    value = aggregate_rate(n, a.steps, elapsed, world)
    ms_per_step = elapsed / a.steps * 1e3

    # per-phase device times with CUDA events on the scene stream
    k_phase = max(50, min(a.steps, 400))
    ph = sc.step_timed(k_phase)
    st2 = sc.stats()
    step_ms = ph[2] / k_phase
    bytes_launch = algorithmic_bytes(n, st2, prec == dem.DEM_MIXED)
    peaks, peak_src = measured_peaks()
    achieved = bytes_launch / (step_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": measured_traffic(n, prec == dem.DEM_MIXED),
                "peak_source": peak_src, "kernel": "k_step_warp<MixedPolicy>" if prec else "k_pairs+k_gather<Fp64Policy>",
                "kernel_ms": step_ms, "algorithmic_bytes_per_launch": bytes_launch,
                "phase_ms_per_step": {"mesh_pose": ph[0] / k_phase, "rebuild": ph[1] / k_phase,
                                      "step": ph[2] / k_phase, "advance": ph[3] / k_phase}}
    sc.close()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if prec == dem.DEM_MIXED else "f64", "data": "synthetic",
           "config": {"workload": f"rotating drum, {sphere_count(n)} spheres R~U[0.8,1.2] mm, 4096-triangle "
                                  "cylinder at 30 rpm, 35% fill, mu 0.4/0.05/0.05",
                      "n_particles": n, "n_triangles": int(s["tris"].shape[0]),
                      "precision": ("mixed: FP32 contact math, compensated double-float state"
                                    if prec == dem.DEM_MIXED else "fp64"),
                      "dt": s["params"]["dt"], "parallelism": f"replicas x{world}",
                      "l2": "working set > L2 (no flush needed)",
                      "settle_steps": a.settle, "seed": 5,
                      "rebuilds_in_timed": st["rebuilds"] - st0["rebuilds"],
                      "pair_contacts": st["pair_contacts"], "mesh_contacts": st["mesh_contacts"],
                      "list_entries": st["list_entries"],
                      "mesh_candidates": st["mesh_candidates"]},
           "gpu_launches": int(a.steps * st["launches_per_step"]
                               + (st["rebuilds"] - st0["rebuilds"]) * st["launches_per_rebuild"]),
           "roofline": roofline}
    out["clocks"] = clk.summary()

    # DEM_FP64 beside it
    if prec == dem.DEM_MIXED:
        k64 = a.fp64_steps or max(10, a.steps // 20)
        with torch.cuda.stream(strm):
            sd = dem.Scene.from_dict(s_set, precision=dem.DEM_FP64)
        sd.step(max(3, a.warmup // 10))
        sd.synchronize()
        barrier()
        e0.record(strm)
        sd.step(k64)
        e1.record(strm)
        e1.synchronize()
        rc64 = sd.synchronize()
        t64 = rank_max(e0.elapsed_time(e1) / 1e3)
        k_ph = max(5, k64 // 4)
        ph64 = sd.step_timed(k_ph)
        st64 = sd.stats()
        kms = ph64[2] / k_ph
        fma_rate = dem.probe_fp64_fma(stream=ctypes.c_void_p(strm.cuda_stream))
        peak_tf = 2.0 * fma_rate / 1e12
        flops = fp64_algorithmic_flops(n, st64)
        ach_tf = flops / (kms * 1e-3) / 1e12
        bytes64 = algorithmic_bytes(n, st64, False)
        ach_gb = bytes64 / (kms * 1e-3) / 1e9
        out["fp64"] = {"value": aggregate_rate(n, k64, t64, world), "ms_per_step": t64 / k64 * 1e3,
                       "steps": k64, "status": rc64, "step_kernel_ms": kms,
                       "roofline": {"bound": "alu", "achieved": ach_tf, "peak": peak_tf,
                                    "unit": "TFLOP/s", "frac": ach_tf / peak_tf,
                                    "traffic": measured_traffic(n, False),
                                    "kernel": "k_pairs+k_gather<Fp64Policy>",
                                    "peak_source": "measured: dem_probe_fp64_fma (FP64 FMA "
                                                   "rate x 2 flops) on this GPU",
                                    "nominal_peak_tflops": NOMINAL_FP64_TFLOPS,
                                    "algorithmic_flops_per_step": flops,
                                    "flop_counting": "FP64 operations of the law as written "
                                                     "(+, -, *, /, sqrt each 1): 275 per "
                                                     "touching pair (law and both sums), 330 "
                                                     "per mesh contact, 190 per particle "
                                                     "(integration)",
                                    "hbm": {"achieved": ach_gb, "peak": peaks["hbm_gbs"],
                                            "unit": "GB/s", "frac": ach_gb / peaks["hbm_gbs"],
                                            "algorithmic_bytes_per_launch": bytes64}},
                       "pair_contacts": st64["pair_contacts"],
                       "mesh_contacts": st64["mesh_contacts"]}
        sd.close()

    # DEM_MIXED64 beside it: the FP32 contact law with FP64 state
    if prec == dem.DEM_MIXED:
        k2 = max(20, a.steps)
        with torch.cuda.stream(strm):
            s2 = dem.Scene.from_dict(s_set, precision=dem.DEM_MIXED64, skin=a.skin)
        s2.step(max(3, a.warmup))
        s2.synchronize()
        barrier()
        e0.record(strm)
        s2.step(k2)
        e1.record(strm)
        e1.synchronize()
        rc2 = s2.synchronize()
        t2 = rank_max(e0.elapsed_time(e1) / 1e3)
        k_ph2 = max(10, k2 // 4)
        ph2 = s2.step_timed(k_ph2)
        st2b = s2.stats()
        kms2 = ph2[2] / k_ph2
        b2 = algorithmic_bytes(n, st2b, True) + 4 * n  # radius read as a double
        out["mixed64"] = {"value": aggregate_rate(n, k2, t2, world), "ms_per_step": t2 / k2 * 1e3,
                          "steps": k2, "status": rc2, "step_kernel_ms": kms2,
                          "precision": "FP32 contact law and springs, FP64 positions, "
                                       "velocities, spins and orientations",
                          "hbm": {"achieved": b2 / (kms2 * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                                  "unit": "GB/s",
                                  "frac": b2 / (kms2 * 1e-3) / 1e9 / peaks["hbm_gbs"]}}
        s2.close()

    # end to end through the C ABI with host buffers: create from host arrays
    # (H2D), step in frames, read the full state back after every frame (D2H)
    if not a.no_e2e:
        frames = max(1, a.steps // a.frame)
        # host buffers in pinned memory (inputs copied in before the clock starts)
        keep = []

        def pinned(arr):
            t = torch.empty(np.shape(arr), dtype=torch.float64, pin_memory=True)
            keep.append(t)
            out_ = t.numpy()
            out_[...] = arr
            return out_
        s_pin = dict(s_set)
        for key in ("R", "x", "v", "w", "q"):
            s_pin[key] = pinned(s_set[key])
        x, v, w = (pinned(np.zeros((n, 3))) for _ in range(3))
        q = pinned(np.zeros((n, 4)))
        barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(strm):
            se = dem.Scene.from_dict(s_pin, precision=prec)
        for _ in range(frames):
            se.step(a.frame)
            rce = se.read_state_into(x, v, w, q)
        t_e2e = rank_max(time.perf_counter() - t0)
        se.close()
        steps_e2e = frames * a.frame
        rec = 32
        out["e2e"] = {"value": aggregate_rate(n, steps_e2e, t_e2e, world), "unit": UNIT,
                      "h2d_bytes_per_step": int(n * 14 * 8 / steps_e2e),
                      "d2h_bytes_per_step": int(frames * n * (4 * rec + 4) / steps_e2e),
                      "status": rce, "frames": frames, "steps_per_frame": a.frame}

    out["contacts_per_s"] = (st["pair_contacts"] + st["mesh_contacts"]) * a.steps * world / elapsed

    # batched ensemble beside it: independent hopper scenes with per-scene
    # friction in one scene (one graph replay steps them all), autotuned
    if not a.no_batch:
        out["batched"] = bench_batch(a, dem, strm, barrier, rank_max, world)

    # the learned surrogate beside it: graph + network per stride of 10 steps
    # on a 100k drum, against 10 DEM steps on the same drum
    if not a.no_surrogate:
        out["surrogate"] = bench_surrogate(dem, strm)

    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(target_s=15.0)
        if not a.no_cpu_design:
            from paper_2507_12610_gb300 import scenes
            out["cpu_paper_design"] = cpu_paper_design(
                s_set, scenes.box_scene(n=1000, seed=1, speed=0.3))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_batch(a, dem, strm, barrier, rank_max, world):
    import torch
    from paper_2507_12610_gb300 import batch
    b = batch.combine(batch.ensemble(a.batch_scenes))
    n = len(b["R"])
    # settle the funnels' lattices into contact (not timed); the settled state
    # is the input of the tuning runs and of the timed run
    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(b, precision=dem.DEM_MIXED)
    sc.step(a.batch_settle)
    assert sc.synchronize() == 0, "batch settle failed"
    st = sc.state()
    sc.close()
    b = dict(b, x=st["x"], v=st["v"], w=st["w"], q=st["q"])
    best, table = batch.autotune(b, precision=dem.DEM_MIXED,
                                 skins=[0.2e-3, 0.3e-3, 0.45e-3, 0.6e-3], steps=100, warmup=20,
                                 dem=dem)
    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(b, precision=dem.DEM_MIXED, skin=best["skin"],
                                 step_warps=best["step_warps"])
    sc.step(max(3, a.warmup))
    sc.synchronize()
    st0 = sc.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = a.batch_steps
    barrier()
    e0.record(strm)
    sc.step(k)
    e1.record(strm)
    e1.synchronize()
    rc = sc.synchronize()
    t = rank_max(e0.elapsed_time(e1) / 1e3)
    st = sc.stats()
    f = batch.discharged(b, sc.state()["x"])
    # the step kernel's roofline on the batch (phase-timed steps after the run)
    k_ph = 50
    ph = sc.step_timed(k_ph)
    stb = sc.stats()
    kms = ph[2] / k_ph
    bytes_b = algorithmic_bytes(n, stb, True)
    peaks, _ = measured_peaks()
    sc.close()
    return {"value": aggregate_rate(n, k, t, world), "unit": UNIT, "ms_per_step": t / k * 1e3,
            "steps": k, "status": rc, "n_scenes": a.batch_scenes, "n_particles": n,
            "n_triangles": int(len(b["tris"])), "n_rectangles": int(len(b["elems"])),
            "workload": "hopper discharge, particles log-uniform in [500, 20000] per scene, "
                        "R~U[0.9,1.1] mm, 256-triangle funnel + 5-rectangle catch box, "
                        "mu_s~U[0.2,0.8], mu_r~U[0,0.2], mu_t~U[0,0.2] per scene",
            "precision": "mixed", "settle_steps": a.batch_settle,
            "autotuned": best, "autotune_table": table,
            "rebuilds_in_timed": st["rebuilds"] - st0["rebuilds"],
            "pair_contacts": st["pair_contacts"], "mesh_contacts": st["mesh_contacts"],
            "contacts_per_s": (st["pair_contacts"] + st["mesh_contacts"]) * k * world / t,
            "discharged_fraction_median": float(np.median(f)),
            "roofline": {"bound": "hbm", "kernel": "k_step_warp<MixedPolicy>",
                         "kernel_ms": kms, "algorithmic_bytes_per_launch": bytes_b,
                         "achieved": bytes_b / (kms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s",
                         "frac": bytes_b / (kms * 1e-3) / 1e9 / peaks["hbm_gbs"]}}


def bench_surrogate(dem, strm, n=100_000):
    """The learned surrogate on the 100,000-sphere drum: trained briefly on the
    DEM's own hopper trajectories, then timed per 10-step stride (cell-list
    graph + forward, device) against 10 DEM steps, with the position error of
    one network stride and of a 3-stride run with DEM fallback."""
    import torch
    from paper_2507_12610_gb300 import batch, scenes, surrogate
    rng = np.random.default_rng(3)
    b = batch.combine([batch.hopper_scene(int(m), 900 + k,
                                          (float(rng.uniform(0.2, 0.8)), 0.1, 0.1))
                       for k, m in enumerate((900, 1400, 2000, 2800))])
    t0 = time.perf_counter()
    pairs, Rb = surrogate.sample_pairs(b, 16, every=100, settle=2000)
    model = surrogate.MPNN(seed=0)
    surrogate.train(model, pairs, Rb, b["params"]["dt"], iters=400, lr=1e-3, lr_end=1e-4,
                    log_every=400)
    t_train = time.perf_counter() - t0
    d = scenes.drum_scene(n=n, seed=5, nn_dist=2.15e-3, speed=0.02,
                          radius=scenes.drum_geometry(n)[0])
    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(d, precision=dem.DEM_MIXED)
    sc.step(1500)
    st = sc.state()
    sc.step(20)
    sc.synchronize()
    t0 = time.perf_counter()
    sc.step(100)
    sc.synchronize()
    dem_ms = (time.perf_counter() - t0) * 1e3 / 10
    sc.close()
    surrogate.predict(model, st, d["R"])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 3
    for _ in range(k):
        surrogate.predict(model, st, d["R"])
    torch.cuda.synchronize()
    net_ms = (time.perf_counter() - t0) * 1e3 / k
    surrogate._mesh_kw.clear()
    surrogate._mesh_kw.update(verts=d["verts"], tris=d["tris"], tri_radius=d["tri_radius"])
    one = surrogate.rollout(model, st, d["R"], d["params"], 1, overlap_growth=1e9,
                            energy_limit=1e9)
    hyb = surrogate.rollout(model, st, d["R"], d["params"], 3)
    return {"value": n * 10 / (net_ms * 1e-3), "unit": UNIT, "n_particles": n,
            "stride_steps": 10, "ms_per_stride": net_ms, "dem_ms_per_stride": dem_ms,
            "gain": dem_ms / net_ms,
            "pos_error_one_stride_rms_over_rmax": one["pos_error_rms_over_rmax"][0][1],
            "hybrid_3_strides": {"fallbacks": hyb["fallbacks"],
                                 "pos_error_rms_over_rmax": [e for _, e, _ in
                                                             hyb["pos_error_rms_over_rmax"]]},
            "train_s": t_train, "train_pairs": 16, "train_iters": 400,
            "note": "trained network (cell-list graph + 3-round MPNN, bf16 weights, fp32 "
                    "accumulation) per 10-step stride against 10 DEM_MIXED steps"}


def oracle_sample(seed: int = 5):
    """A bounded sample of the drum workload the O(N^2) oracle can step."""
    from paper_2507_12610_gb300 import scenes
    return scenes.drum_scene(n=2000, seed=seed, n_theta=32, n_rings=4, nn_dist=2.15e-3,
                             speed=0.02)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_on_cores(steps: int | None = None, warmup: int = 3, target_s: float = 15.0,
                    cores: int | None = None):
    """The oracle as it stands on every host core: one independent 2,000-sphere
    drum sample per core (seeds 5, 6, ...), each stepped by its own thread
    (the oracle's ctypes calls release the GIL, so the threads run in
    parallel).  Returns (particle-steps/s over all cores, cores, steps, s)."""
    from oracle import oracle
    oracle.build()
    cores = cores or host_cores()
    ocs = []
    for k in range(cores):
        s = oracle_sample(seed=5 + k)
        ocs.append(oracle.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"],
                                      s["verts"], s["tris"], s["tri_radius"]))
    n = len(ocs[0].state()["x"])

    def run_all(k):
        th = [threading.Thread(target=oc.step, args=(k,)) for oc in ocs]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        return time.perf_counter() - t0

    per = run_all(warmup) / max(warmup, 1)
    k = steps or max(5, int(target_s / max(per, 1e-6)))
    el = run_all(k)
    return cores * n * k / el, cores, k, el, n


def cpu_baseline(target_s: float = 15.0):
    value, cores, k, el, n = oracle_on_cores(target_s=target_s)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent {n}-sphere drum samples (same radii, material, "
                      f"30 rpm; 320 triangles), one per host core, FP64 O(N^2) oracle, "
                      f"{k} steps each, {el:.1f} s"}


# The paper's own timings (Sec. 5): one step of N = 1,000 settled spheres in a
# cube took about 0.64 ms on a 3.6 GHz 8-core Intel Xeon Gold 6244; serial
# Cundall numbers (particle updates per second) from 3.5e6 down to 3.2e5 for
# N up to 10 million.
PAPER_TIMINGS = {
    "hardware": "Intel Xeon Gold 6244, 3.6 GHz, 8 cores (2019), GCC 11.2 -O3",
    "n1000_ms_per_step": 0.64,
    "n1000_particle_steps_per_s": 1000 / 0.64e-3,
    "serial_particle_steps_per_s_range": [3.5e6, 3.2e5],
    "source": "Sec. 5 (computational performance), settled spheres in a cube",
}


def cpu_paper_design(drum: dict, box: dict, target_s: float = 10.0):
    """The OpenMP cell-list program in the paper's design (baseline/dem_cpu.cpp)
    on all host cores: the 1,000-sphere box pour and the settled 1M-sphere
    drum (a few steps each, bounded by target_s)."""
    from baseline import dem_cpu
    from paper_2507_12610_gb300 import scenes
    out = {"kind": "OpenMP cell-list program in the paper's design (linked cells of edge "
                   "2 R_max rebuilt every step, one evaluation per pair, FP64)",
           "cores": dem_cpu.threads(), "cpu": dem_cpu.cpu_model(), "unit": UNIT,
           "paper": PAPER_TIMINGS}
    for name, s, warm in (("box_1000", box, 20), ("drum_1M", drum, 1)):
        V, El, rad = scenes.all_elements(s)
        cs = dem_cpu.CpuScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], V, El, rad)
        t0 = time.perf_counter()
        cs.step(warm)
        per = (time.perf_counter() - t0) / warm
        k = max(2, min(2000, int(target_s / 2 / max(per, 1e-6))))
        t0 = time.perf_counter()
        cs.step(k)
        el = time.perf_counter() - t0
        n = len(s["R"])
        out[name] = {"value": n * k / el, "ms_per_step": el / k * 1e3, "steps": k,
                     "n_particles": n}
        del cs
    return out


def bench_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each step of this arm is `cores` oracle steps (one per host core) on
    # independent 2,000-sphere samples of the drum workload
    value, cores, k, el, n = oracle_on_cores(steps=a.steps, warmup=a.warmup)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": el / a.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "rotating drum sample for the CPU oracle: 2,000 spheres "
                                  "R~U[0.8,1.2] mm, 320-triangle cylinder at 30 rpm, one "
                                  "independent sample per host core",
                      "n_particles": n * cores},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{cores} x {n}-sphere drum, {a.steps} steps, "
                                      f"one thread per core"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        bench_reference(a)
    else:
        bench_ours(a)


if __name__ == "__main__":
    main()
