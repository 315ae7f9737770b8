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
    ap.add_argument("--settle", type=int, default=1500)
    ap.add_argument("--frame", type=int, default=100, help="steps per state read-back (e2e)")
    ap.add_argument("--fp64-steps", type=int, default=0, help="0: steps // 20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [c.strip() for c in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


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
           "config": {"workload": "rotating drum, 1M spheres R~U[0.8,1.2] mm, 4096-triangle "
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
        ph64 = sd.step_timed(max(5, k64 // 4))
        out["fp64"] = {"value": aggregate_rate(n, k64, t64, world), "ms_per_step": t64 / k64 * 1e3,
                       "steps": k64, "status": rc64,
                       "step_kernel_ms": ph64[2] / max(5, k64 // 4),
                       "bound": "alu (FP64 pipe)"}
        sd.close()

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
    best, table = batch.autotune(b, precision=dem.DEM_MIXED, skins=[0.2e-3, 0.4e-3],
                                 steps=100, warmup=20, dem=dem)
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
            "discharged_fraction_median": float(np.median(f))}


def bench_surrogate(dem, strm, n=100_000):
    import torch
    from paper_2507_12610_gb300 import scenes, surrogate
    d = scenes.drum_scene(n=n, seed=5, nn_dist=2.15e-3, speed=0.02,
                          radius=scenes.drum_geometry(n)[0])
    with torch.cuda.stream(strm):
        sc = dem.Scene.from_dict(d, precision=dem.DEM_MIXED)
    sc.step(500)
    st = sc.state()
    sc.synchronize()
    t0 = time.perf_counter()
    sc.step(100)
    sc.synchronize()
    dem_ms = (time.perf_counter() - t0) * 1e3 / 10
    sc.close()
    model = surrogate.MPNN(seed=0)
    surrogate.predict(model, st, d["R"])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 3
    for _ in range(k):
        surrogate.predict(model, st, d["R"])
    torch.cuda.synchronize()
    net_ms = (time.perf_counter() - t0) * 1e3 / k
    return {"value": n * 10 / (net_ms * 1e-3), "unit": UNIT, "n_particles": n,
            "stride_steps": 10, "ms_per_stride": net_ms, "dem_ms_per_stride": dem_ms,
            "gain": dem_ms / net_ms,
            "note": "network time (all-pairs graph + 3-round MPNN, bf16) per 10-step stride; "
                    "its trajectory error is measured by paper_2507_12610_gb300.surrogate"}


def oracle_sample():
    """A bounded sample of the drum workload the O(N^2) oracle can step."""
    from paper_2507_12610_gb300 import scenes
    return scenes.drum_scene(n=2000, seed=5, n_theta=32, n_rings=4, nn_dist=2.15e-3, speed=0.02)


def cpu_baseline(target_s: float = 15.0, steps: int | None = None):
    from oracle import oracle
    s = oracle_sample()
    oc = oracle.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], s["verts"],
                            s["tris"], s["tri_radius"])
    t0 = time.perf_counter()
    oc.step(3)
    per = (time.perf_counter() - t0) / 3
    k = steps or max(5, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    oc.step(k)
    el = time.perf_counter() - t0
    n = len(s["R"])
    return {"value": n * k / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n}-sphere drum (same radii, material, 30 rpm; {len(s['tris'])} "
                      f"triangles), FP64 O(N^2) oracle, {k} steps, {el:.1f} s, 1 thread"}


def bench_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    s = oracle_sample()
    oc = oracle.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], s["verts"],
                            s["tris"], s["tri_radius"])
    n = len(s["R"])
    oc.step(a.warmup)
    t0 = time.perf_counter()
    oc.step(a.steps)
    el = time.perf_counter() - t0
    value = n * a.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": el / a.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "rotating drum sample for the CPU oracle: 2,000 spheres "
                                  "R~U[0.8,1.2] mm, 320-triangle cylinder at 30 rpm",
                      "n_particles": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{n}-sphere drum, {a.steps} steps, 1 thread"},
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
