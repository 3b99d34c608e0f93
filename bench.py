"""Benchmark: implicit MPM Lite time steps per second on one GB300 (or N replicas).

A step is one pass of the whole hot path through the C ABI: mpml_resample
(sort, P2Q, Q2N), mpml_newton_step (stretch reconstruction, Newton with
Jacobi-PCG to relative residual 1e-6 and line search), mpml_g2p (N2Q, Q2P,
advection, F update and the plastic return maps).

Workload (the largest single-GPU configuration): a von Mises slab (Hencky, E =
5e5 Pa, nu = 0.3, yield stress 2e3 Pa, rho = 1000) hitting a Drucker-Prager sand
box (Hencky, E = 1e6 Pa, nu = 0.3, friction angle 30 degrees, rho = 2000) on a
256^3 grid with 8 particles per cell (19,183,392 particles), dt = 2e-3 s, from
the moment of impact: the timed steps follow the trajectory after W warm-up
steps, with mixed slab / sand cells and plastic flow in both materials.  FP32
storage and arithmetic with FP64 reductions and FP64 Newton iterate / gradient.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on bounded samples of the same workload instead (see oracle_units).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton steps/s & HVP GB/s at rel resid 1e-6; learned-precond FP32 vs plain PCG"


def workload_text(n):
    return (f"von Mises slab (Hencky E=5e5, nu=0.3, yield 2e3) hitting a Drucker-Prager sand box (Hencky E=1e6, "
            f"nu=0.3, phi=30 deg) on a {n}^3 grid, 8 particles/cell, dt=2e-3, from the moment of impact "
            f"(slab one voxel row above the sand, falling at sqrt(2 g dh)); timed steps follow the trajectory")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid cells per axis of the headline workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner comparison")
    ap.add_argument("--hvp-probe", choices=["pressed_block_236", "slab_on_sand_256", "two_spheres_168"],
                    help="only build this workload, take one step, and time the standalone HVP (for profilers)")
    ap.add_argument("--pcg-probe", choices=["slab_on_sand_impact", "two_spheres_contact", "pressed_block"],
                    help="only build this workload at --n, take --warmup steps, then one solve (for profilers)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the extra measurements of the other workloads (batch, two spheres, large block)")
    ap.add_argument("--cg-forcing", type=float, default=0.3,
                    help="inexact-Newton forcing cap of the trajectory workloads' solves (solver option cg_forcing; "
                         "0: every CG solve to cg_rtol); Newton stops at 1e-6 of the initial FP64 gradient either way")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def host_cpu():
    """nproc and the CPU model of this host (lscpu), for the CPU legs."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return {"nproc": os.cpu_count(), "model": model}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_hash():
    """Hash of the persistent solver's source: the regions between the
    "[persistent-solver source: begin]" / "end" markers of k_newton.cu and
    mpml_internal.cuh (the kernel, its helpers and its host launch)."""
    h = hashlib.sha256()
    for f in ("k_newton.cu", "mpml_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2602_07853_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        pos = 0
        while True:
            a = text.find("[persistent-solver source: begin]", pos)
            if a < 0:
                break
            b = text.find("[persistent-solver source: end]", a)
            h.update(text[a:b].encode())
            pos = b + 1
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per CG iteration of the persistent solver on `workload`, from the committed ncu
    capture (profiles/pcg_traffic.json), or None when the capture was taken on another version of
    the kernel or on another workload."""
    path = os.path.join(ROOT, "profiles", "pcg_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e


# tangent bytes per active cell: 25 FP32 numbers (compressed, one elastic material) or 45 (packed)
CMP_TANGENT_BYTES = 100.0
PACKED_TANGENT_BYTES = 180.0


def pcg_bytes_per_iter(n_cells, n_nodes, tangent_bytes=CMP_TANGENT_BYTES):
    """Algorithmic bytes of one CG iteration (FP32) on the implemented representation: the HVP reads
    the stored tangent of every active cell and per DOF node p, m and writes q (28 B); the CG update
    makes about ten 12-byte vector passes per DOF node (x, r, p, q, D^-1 reads and writes)."""
    return tangent_bytes * n_cells + (28.0 + 120.0) * n_nodes


def pcg_kernel_name(k45, staging, ctas):
    """The persistent solver kernel a launch shape runs (staging 1 shared-memory block, 2 streamed
    rows, 3 column groups)."""
    fmt = "K45" if k45 else "compressed"
    if staging == 3:
        return f"k_pcg_groups<{fmt}> (half a brick per 64-thread group, {ctas} CTAs/SM)"
    kind = "staged" if staging == 1 else "streamed"
    return f"k_pcg_persistent<{fmt}, {kind}> ({ctas} CTAs/SM)"


def pcg_floor_bytes_per_iter(n_cells, n_nodes):
    """The same with the algorithmic floor of the HVP: the state that defines a cell's Hessian
    (F 9, S 6, V 1 numbers: 64 B per active cell, the tangent recomputed) instead of the stored one."""
    return 64.0 * n_cells + (28.0 + 120.0) * n_nodes


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def impact_scene(n):
    from paper_2602_07853_gb300 import scenes
    return scenes.slab_on_sand(n, impact=True)


def sample_arrays(sc, frac):
    """A bounded sample of the workload: the particles inside a vertical column over the impact
    zone (x, z in [0.35, 0.35 + w), full height, where slab and sand overlap), w chosen so that
    the column holds about `frac` of the particles.  Returned as the arrays the oracle reads."""
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles(np.float32).items()}
    if frac >= 1.0:
        return p
    x = p["x"]
    lo = 0.35
    w = 0.25
    for _ in range(40):  # bisection on the column width
        sel = (x[:, 0] >= lo) & (x[:, 0] < lo + w) & (x[:, 2] >= lo) & (x[:, 2] < lo + w)
        f = sel.mean()
        if abs(f - frac) <= 0.05 * frac:
            break
        w *= np.sqrt(frac / max(f, 1e-9))
        w = min(w, 0.6)
    return {k: np.ascontiguousarray(v[sel]) for k, v in p.items()}


def oracle_units(sc, arrays, cg_a=5, cg_b=15):
    """Per-unit costs of the oracle (single thread, FP64) measured on a bounded sample: unload and
    load per particle, stretch reconstruction per active cell, one Newton iteration's fixed work
    (linearisation, line search) per active cell and one Jacobi-PCG iteration per active cell, from
    two capped Newton iterations (cg_a and cg_b CG iterations) on the sample's own system."""
    import oracle

    o = oracle.Oracle(oracle.make_scene(sc.n, sc.dx, sc.dt, sc.gravity,
                                        [(m.model, m.E, m.nu, m.plastic, m.yield_stress, m.friction_angle)
                                         for m in sc.materials],
                                        wall_layers=sc.wall_layers, plate=sc.plate, inv_dx=sc.inv_dx))
    t0 = time.perf_counter()
    assert o.unload(**arrays) == 0
    t1 = time.perf_counter()
    assert o.stretch() == 0
    t2 = time.perf_counter()
    o.newton(oracle.default_solver(newton_max=1, cg_max=cg_a, cg_rtol=0.0))
    t3 = time.perf_counter()
    o.newton(oracle.default_solver(newton_max=1, cg_max=cg_b, cg_rtol=0.0))
    t4 = time.perf_counter()
    o.load()
    t5 = time.perf_counter()
    npart, ncell = len(arrays["x"]), o.count("cells")
    cg = max((t4 - t3) - (t3 - t2), 1e-9) / (cg_b - cg_a)
    return {"particle_s": ((t1 - t0) + (t5 - t4)) / npart, "stretch_cell_s": (t2 - t1) / ncell,
            "newton_cell_s": max((t3 - t2) - cg_a * cg, 0.0) / ncell, "cg_cell_s": cg / ncell,
            "sample_particles": npart, "sample_cells": ncell, "wall_s": t5 - t0}


def step_seconds(u, particles, cells, newton, cg):
    """Oracle seconds of one full step from per-unit costs and the step's counts."""
    return (u["particle_s"] * particles + u["stretch_cell_s"] * cells + u["newton_cell_s"] * cells * newton
            + u["cg_cell_s"] * cells * cg)


def _units_worker(args):
    path, n = args
    import oracle  # noqa: F401  (the child loads the oracle library itself)
    d = dict(np.load(path))
    t0 = time.perf_counter()
    u = oracle_units(impact_scene_desc(n), d)
    return u, time.perf_counter() - t0


def impact_scene_desc(n):
    """The workload's scene parameters without its particles (for sample workers)."""
    from paper_2602_07853_gb300 import scenes
    sc = scenes.slab_on_sand(8, impact=True)
    sc.n, sc.dx, sc.inv_dx = (n, n, n), 1.0 / n, float(n)
    return sc


def all_cores_units(arrays, n, procs):
    """The same sample timed in `procs` concurrent single-thread oracle processes (spawned): the
    host's aggregate rate when every core runs its own copy (the oracle itself is serial)."""
    import multiprocessing as mp

    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, **arrays)
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_units_worker, [(path, n)] * procs)
    finally:
        os.unlink(path)
    return res


def workload_counts(key):
    path = os.path.join(ROOT, "oracle", "bench_workload_counts.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get(key)
    return None


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on bounded samples of the workload (no reference code
    exists: the paper publishes none).  Each step times one sample (oracle_units) and scales it to a
    full step of the workload with the oracle's own iteration counts on it."""
    if rank != 0:
        return 0
    sc = impact_scene(args.n)
    frac = min(1.0, 600_000 / max(sc.num_particles, 1))
    arrays = sample_arrays(sc, frac)
    key = f"slab_on_sand_{args.n}_impact"
    cnt = workload_counts(key)
    if cnt is None:
        # no stored counts for this size: the oracle's own complete first step on the sample
        import oracle
        o = oracle.Oracle(oracle.make_scene(sc.n, sc.dx, sc.dt, sc.gravity,
                                            [(m.model, m.E, m.nu, m.plastic, m.yield_stress, m.friction_angle)
                                             for m in sc.materials], wall_layers=sc.wall_layers, inv_dx=sc.inv_dx))
        assert o.unload(**arrays) == 0 and o.stretch() == 0
        _, st = o.newton(oracle.default_solver())
        cnt = {"newton_iters_first_step": st.newton_iters, "cg_iters_first_step": st.cg_iters_total,
               "source": "the oracle's complete first step on the sample column"}
    else:
        cnt = dict(cnt, source="oracle/bench_workload_counts.json (the oracle's complete first step, "
                                "written by oracle/workload_counts.py)")
    # full-size counts of particles and active cells: the oracle's own unload of the whole workload
    # is too slow to repeat per step; the active-cell count scales with the sample's particle share
    full_p = sc.num_particles
    for _ in range(args.warmup):
        oracle_units(sc, arrays)
    walls, steps_s = [], []
    for _ in range(args.steps):
        u = oracle_units(sc, arrays)
        cells = cnt.get("cells") or u["sample_cells"] * full_p / u["sample_particles"]
        steps_s.append(step_seconds(u, full_p, cells, cnt["newton_iters_first_step"], cnt["cg_iters_first_step"]))
        walls.append(u["wall_s"])
    value = 1.0 / float(np.mean(steps_s))
    cpu = host_cpu()
    sample = (f"per step: one bounded sample of the workload timed (the {len(arrays['x'])} particles of a column "
              f"over the impact zone: unload, stretch, two capped Newton iterations with 5 and 15 Jacobi-PCG "
              f"iterations, load), giving the oracle's seconds per particle, per cell and stretch, per cell and "
              f"Newton iteration and per cell and CG iteration; scaled to a full step with {full_p} particles, "
              f"{int(cells)} active cells, {cnt['newton_iters_first_step']} Newton and "
              f"{cnt['cg_iters_first_step']} CG iterations ({cnt['source']}); single thread; "
              f"ms_per_step is the wall time of one sample, value the scaled full-step rate")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(args.n), "grid": args.n, "particles": full_p, "precision": "fp64",
                       "preconditioner": "jacobi", "cg_rtol": 1e-6, "newton_rtol": 1e-6,
                       "cg_forcing": 0.0},
            "extrapolated_ms_per_step": 1e3 / value,
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": cpu},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Multi-rank aggregation (replicas: one process per GPU, no data-path collective)
# ---------------------------------------------------------------------------
def max_over_ranks(value, dist, device):
    """The largest per-rank duration over all ranks (every rank receives it); `dist` is
    torch.distributed or None for a single process."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, seconds):
    """Whole-job steps/s: every rank runs `steps` steps of its own replica."""
    return world * steps / seconds


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def trajectory(m, sc, warmup, steps, peaks, opts=None, tangent_bytes=None):
    """W untimed then K timed steps of scene sc along its trajectory (one context on the current
    stream, device particles, CUDA events per step), with the persistent solver's own roofline."""
    import torch

    stream = torch.cuda.current_stream()
    ctx, p, pp = make_ctx(m, sc, stream)
    opts = opts if opts is not None else m.solver_opts()
    tb = tangent_bytes or (CMP_TANGENT_BYTES if len(sc.materials) == 1 and sc.materials[0].plastic == 0
                           else PACKED_TANGENT_BYTES)

    def one(s):
        m.mpml_set_time(ctx, s * sc.dt)
        m.mpml_resample(ctx, pp)
        rc, st = m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, pp)
        return st

    for s in range(warmup):
        one(s)
    tune_shape, tune_ms = m.mpml_autotune_pcg(ctx, 30, 2)
    torch.cuda.synchronize()
    m.mpml_set_profiling(ctx, 1)
    ms, newton, cg, fb, alg = [], 0, 0, 0, 0.0
    for i in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = one(warmup + i)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        newton += st.newton_iters
        cg += st.cg_iters_total
        fb += st.fcg_fallbacks
        cn = m.mpml_counts(ctx)
        alg += pcg_bytes_per_iter(cn["cells"], cn["nodes"], tb) * st.cg_iters_total
    pcg_n, pcg_iters, pcg_ms = m.mpml_pcg_timing(ctx)
    _, last_staging, last_ctas = m.mpml_get_pcg_config(ctx)
    cn = m.mpml_counts(ctx)
    m.mpml_destroy(ctx)
    del p
    torch.cuda.empty_cache()
    out = {"particles": int(cn["particles"]), "active_cells": int(cn["cells"]), "dof_nodes": int(cn["nodes"]),
           "steps_per_s": 1e3 * len(ms) / float(np.sum(ms)), "ms_per_step": float(np.mean(ms)),
           "newton_iters_per_step": newton / len(ms), "cg_iters_per_step": cg / len(ms),
           "steps_timed": f"trajectory steps {warmup}..{warmup + steps - 1}", "cg_forcing": opts.cg_forcing,
           "pcg_autotune": {"chosen": tune_shape,
                            "us_per_cg_iter": [round(1e3 * t / 30, 2) if t >= 0 else None for t in tune_ms]}}
    if fb:
        out["fcg_fallbacks_per_step"] = fb / len(ms)
    if pcg_n > 0 and pcg_iters > 0:
        gbs = alg / (pcg_ms / 1e3) / 1e9 if pcg_iters == cg else None
        out["pcg_kernel"] = {"shape": pcg_kernel_name(tb == PACKED_TANGENT_BYTES, last_staging, last_ctas),
                             "us_per_cg_iter": 1e3 * pcg_ms / pcg_iters, "launches": pcg_n,
                             "gbs": gbs, "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                             "bytes_rule": f"{int(tb)} B per active cell + 148 B per DOF node per CG iteration"}
    return out


def other_configs(m, args, peaks):
    """Secondary measurements (not the headline value), each with CUDA events, inputs resident,
    warm-up first: the 64-scene batch (config 4), the two-sphere collision at 168^3 (config 2b),
    the pressed block at dx = 1/236 (config 3-8M), the explicit integrator, PPC independence and
    the water dam break."""
    import torch

    from paper_2602_07853_gb300 import scenes

    out = {}
    # config 4: 64 scenes of uneven size, one context and stream each, batched solve; the shapes
    # start on the floor (lowest voxel row 1) so that every step solves a contact problem
    n_sc = 64
    scs = [scenes.batch_scene(i, row=1) for i in range(n_sc)]
    streams = [torch.cuda.Stream() for _ in scs]
    made = [make_ctx(m, sc, st) for sc, st in zip(scs, streams)]
    ctxs = [c for c, _, _ in made]
    parts = [pp for _, _, pp in made]
    torch.cuda.synchronize()

    def run_batch(k0, k):
        ms, newton, cg, alg = [], 0, 0, 0.0
        for s in range(k0, k0 + k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for c in ctxs:
                m.mpml_set_time(c, s * scs[0].dt)
            m.mpml_resample_batch(ctxs, parts)
            rc, st = m.mpml_newton_step_batch(ctxs, m.solver_opts(cg_forcing=args.cg_forcing))
            for c, pp in zip(ctxs, parts):
                m.mpml_g2p(c, pp)
            torch.cuda.synchronize()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            newton += sum(x.newton_iters for x in st)
            cg += sum(x.cg_iters_total for x in st)
            for c, x in zip(ctxs, st):
                cn = m.mpml_counts(c)
                alg += pcg_bytes_per_iter(cn["cells"], cn["nodes"]) * x.cg_iters_total
        return ms, newton, cg, alg

    run_batch(0, 3)  # warm-up: steps 0-2
    m.mpml_set_profiling(ctxs[0], 1)
    K = max(4, min(args.steps, 10))
    ms, newton, cg, alg = run_batch(3, K)
    pcg_n, pcg_iters, pcg_ms = m.mpml_pcg_timing(ctxs[0])
    m.mpml_set_profiling(ctxs[0], 0)
    gbs = alg / (pcg_ms / 1e3) / 1e9 if pcg_ms > 0 else None
    out["batch64"] = {"workload": "64 fixed-corotated scenes (box / sphere / torus, extents 8-48 voxels, E log-uniform "
                                  "1e4-1e7, nu 0.2-0.45) each on its own 64^3 grid, dropped at 1 m/s onto the floor "
                                  f"(lowest voxel row 1), dt = 1e-3, steps 3-{2 + K}",
                      "particles": int(sum(int(p["x"].shape[0]) for _, p, _ in made)),
                      "steps_per_s": 1e3 * len(ms) / float(np.sum(ms)), "ms_per_step": float(np.mean(ms)),
                      "newton_iters_per_step": newton / len(ms), "cg_iters_per_step": cg / len(ms),
                      "pcg_kernel": {"kernel": "k_pcg_batch", "launches": pcg_n, "ms": pcg_ms, "gbs": gbs,
                                     "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                                     "bytes_rule": "sum over scenes of (100 B per active cell + 148 B per DOF "
                                                   "node) x that scene's CG iterations, over the launches' time"},
                      "solver": "mpml_resample_batch + mpml_newton_step_batch (one persistent PCG launch per "
                                "Newton round over all scenes), one stream per scene",
                      "cg_forcing": args.cg_forcing}
    for c in ctxs:
        m.mpml_destroy(c)
    del made
    torch.cuda.empty_cache()

    # config 2b: the two-sphere collision at 168^3 along its trajectory from contact
    fo = m.solver_opts(cg_forcing=args.cg_forcing)
    out["two_spheres_168"] = trajectory(m, scenes.two_spheres(168, gap=1.0 / 168), 3, max(4, min(args.steps, 10)),
                                        peaks, fo)
    out["two_spheres_168"]["workload"] = ("two Neo-Hookean spheres (E=1e6, nu=0.4, r=0.15) colliding at 2 m/s on a "
                                          "168^3 grid, dt=2e-3, from contact")
    # config 3-8M: the pressed block at dx = 1/236
    out["pressed_block_236"] = trajectory(m, scenes.pressed_block(236), 2, max(3, min(args.steps, 5)), peaks, fo)
    out["pressed_block_236"]["workload"] = ("fixed-corotated block (E=1e8, nu=0.33) pressed by a plate at 0.1 m/s, "
                                            "dx=1/236, dt=1e-3")

    # the explicit integrator on the two-sphere workload (dt below the elastic CFL limit)
    sc = scenes.two_spheres(168, gap=1.0 / 168, dt=5e-5)
    stream = torch.cuda.current_stream()
    ctx, p, pp = make_ctx(m, sc, stream)
    ms = []
    for s in range(3 + 10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.mpml_set_time(ctx, s * sc.dt)
        m.mpml_resample(ctx, pp)
        m.mpml_explicit_step(ctx)
        m.mpml_g2p(ctx, pp)
        b.record(stream)
        torch.cuda.synchronize()
        if s >= 3:
            ms.append(a.elapsed_time(b))
    out["explicit_two_spheres_168"] = {"dt": sc.dt, "particles": int(sc.num_particles),
                                       "steps_per_s": 1e3 * len(ms) / float(np.sum(ms)),
                                       "ms_per_step": float(np.mean(ms)),
                                       "solver": "mpml_resample + mpml_explicit_step + mpml_g2p"}
    m.mpml_destroy(ctx)
    del p
    torch.cuda.empty_cache()

    # particles-per-cell independence (the paper's claim for integration without particles):
    # Newton time should stay flat over PPC 8 / 16 / 24 while P2Q and G2P grow with PPC
    ppc_rows = []
    for ppc in (8, 16, 24):
        sc = scenes.two_spheres(128, gap=1.0 / 128, ppc=ppc)
        ctx, p, pp = make_ctx(m, sc, stream)
        init = {k: v.clone() for k, v in p.items()}
        acc = {"unload": [], "integrate": [], "load": []}
        for s in range(1 + 3):
            for k in p:
                p[k].copy_(init[k])
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            m.mpml_resample(ctx, pp)
            ev[1].record(stream)
            rc, st = m.mpml_newton_step(ctx, m.solver_opts())
            ev[2].record(stream)
            m.mpml_g2p(ctx, pp)
            ev[3].record(stream)
            torch.cuda.synchronize()
            if s >= 1:
                acc["unload"].append(ev[0].elapsed_time(ev[1]))
                acc["integrate"].append(ev[1].elapsed_time(ev[2]))
                acc["load"].append(ev[2].elapsed_time(ev[3]))
        ppc_rows.append({"ppc": ppc, "particles": int(sc.num_particles),
                         "unload_ms": float(np.mean(acc["unload"])), "integrate_ms": float(np.mean(acc["integrate"])),
                         "load_ms": float(np.mean(acc["load"])), "newton_iters": int(st.newton_iters),
                         "cg_iters": int(st.cg_iters_total)})
        m.mpml_destroy(ctx)
        del p, init
        torch.cuda.empty_cache()
    out["ppc_independence_two_spheres_128"] = ppc_rows

    # water (Sec. "Water"): dam break with a solid cube in the flow, 128^3, implicit steps
    out["dam_break_water_128"] = trajectory(m, scenes.dam_break(128), 1, 3, peaks, fo)
    out["dam_break_water_128"]["workload"] = ("water column (bulk modulus 3.3e5 Pa) collapsing onto a fixed-corotated "
                                              "cube, steps 1-3 from rest")
    return out


def learned_comparison(m, args, stream, flush):
    """Config 3 (the pressed block at 128^3): the learned preconditioner trained on the first
    Newton system (untimed), then the same trajectory steps timed with it and with Jacobi-PCG."""
    from paper_2602_07853_gb300 import scenes

    peaks, _ = measured_peaks()
    sc = scenes.pressed_block(128)
    ctx, p, pp = make_ctx(m, sc, stream)
    m.mpml_resample(ctx, pp)
    m.mpml_nn_set_weights(ctx, m.nn_init_weights(0, gain=0.1))
    t0 = time.perf_counter()
    tr = m.mpml_nn_train(ctx, m.train_opts())
    train_s = time.perf_counter() - t0
    w = m.mpml_nn_get_weights(ctx)
    m.mpml_destroy(ctx)
    del p
    K = max(3, min(args.steps, 6))
    jac = trajectory(m, sc, 2, K, peaks)
    # the learned solve: a fresh context with the trained weights
    res = trajectory_learned(m, sc, 2, K, w)
    return {"workload": "config 3: fixed-corotated block (E=1e8) pressed by a plate, 128^3, trajectory steps 2.."
                        f"{1 + K}", "jacobi": jac, "learned": res, "train_s": train_s, "train_samples": tr.samples,
            "loss_first": tr.loss_first, "loss_last": tr.loss_last,
            "speedup": jac["ms_per_step"] / res["ms_per_step"]}


def trajectory_learned(m, sc, warmup, steps, weights):
    import torch

    stream = torch.cuda.current_stream()
    ctx, p, pp = make_ctx(m, sc, stream)
    opts = m.solver_opts(precond=m.PRECOND_LEARNED)
    ms, newton, cg, fb = [], 0, 0, 0
    for s in range(warmup + steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.mpml_set_time(ctx, s * sc.dt)
        m.mpml_resample(ctx, pp)
        if s == 0:
            m.mpml_nn_set_weights(ctx, weights)  # the weights need a resampled context
        rc, st = m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, pp)
        b.record(stream)
        torch.cuda.synchronize()
        if s >= warmup:
            ms.append(a.elapsed_time(b))
            newton += st.newton_iters
            cg += st.cg_iters_total
            fb += st.fcg_fallbacks
    m.mpml_destroy(ctx)
    del p
    return {"steps_per_s": 1e3 * len(ms) / float(np.sum(ms)), "ms_per_step": float(np.mean(ms)),
            "newton_iters_per_step": newton / len(ms), "cg_iters_per_step": cg / len(ms),
            "fcg_fallbacks_per_step": fb / len(ms)}


def make_ctx(m, sc, stream, host=False):
    """A context for scene sc on `stream` and its particles (device tensors, or pinned host
    tensors when host=True), plus a pristine copy of the initial particles."""
    import torch

    mats = [m.material(mt.model, *m.mpml_lame_parameters(mt.E, mt.nu), mt.plastic, mt.yield_stress,
                       mt.friction_angle) for mt in sc.materials]
    desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, m.FP32, sc.wall_layers, sc.plate, sc.inv_dx)
    ctx = m.mpml_create(desc, mats, stream.cuda_stream)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in sc.particles(np.float32).items()}
    p = {k: (v.pin_memory() if host else v.cuda()) for k, v in p.items()}
    parts = m.particles_from_tensors(p["x"], p["v"], p["F"], p["G"], p["mp"], p["Vp"], p["mat"])
    return ctx, p, parts


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2602_07853_gb300.mpml as m

    torch.cuda.set_device(local_rank)
    m.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    peaks, peak_kind = measured_peaks()
    sc = impact_scene(args.n)
    stream = torch.cuda.current_stream()
    ctx, cur, parts = make_ctx(m, sc, stream)
    init = {k: v.clone() for k, v in cur.items()}
    opts = m.solver_opts(cg_forcing=args.cg_forcing)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    W, K = args.warmup, args.steps

    def one_step(c, pp, s, o=None):
        m.mpml_set_time(c, s * sc.dt)
        m.mpml_resample(c, pp)
        rc, st = m.mpml_newton_step(c, o if o is not None else opts)
        m.mpml_g2p(c, pp)
        return st

    # warm-up: trajectory steps 0 .. W-1 from the moment of impact
    for s in range(W):
        one_step(ctx, parts, s)
    # the persistent solver's launch shape, autotuned on the last warm-up system (untimed; the
    # choice is cached for this tangent format and size class and used by the timed steps)
    tune_shape, tune_ms = m.mpml_autotune_pcg(ctx, 30, 2) if W > 0 else (None, [])
    barrier()
    m.mpml_set_profiling(ctx, 1)
    launches0 = m.mpml_kernel_launches(ctx)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    newton_its, cg_its, per_step = [], [], []
    alg_bytes = floor_bytes = 0.0
    barrier()
    for i in range(K):
        flush.zero_()  # L2 flush (256 MB > 129 MB L2) outside the timed events
        ev[i][0].record(stream)
        st = one_step(ctx, parts, W + i)
        ev[i][1].record(stream)
        newton_its.append(st.newton_iters)
        cg_its.append(st.cg_iters_total)
        # the step's algorithmic bytes of its CG iterations (the active set changes along the trajectory);
        # the counts are read after the step's end event, outside the timed region
        cn = m.mpml_counts(ctx)
        alg_bytes += pcg_bytes_per_iter(cn["cells"], cn["nodes"], PACKED_TANGENT_BYTES) * st.cg_iters_total
        floor_bytes += pcg_floor_bytes_per_iter(cn["cells"], cn["nodes"]) * st.cg_iters_total
        per_step.append({"step": W + i, "newton": st.newton_iters, "cg": st.cg_iters_total, "cells": cn["cells"],
                         "nodes": cn["nodes"], "status": st.status,
                         "g_rel": st.g_norm / st.g0_norm if st.g0_norm > 0 else 0.0,
                         "cg_per_newton": [int(st.cg_iters[k]) for k in range(min(st.newton_iters, 64))],
                         "alpha": [float(st.alpha[k]) for k in range(min(st.newton_iters, 64))]})
    barrier()
    clk = clocks.stop()
    launches = m.mpml_kernel_launches(ctx) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(np.sum(step_ms)), dist, "cuda")
    hvp_n, hvp_ms, hvp_bytes = m.mpml_hvp_timing(ctx)
    pcg_n, pcg_iters, pcg_ms = m.mpml_pcg_timing(ctx)
    _, last_staging, last_ctas = m.mpml_get_pcg_config(ctx)
    m.mpml_set_profiling(ctx, 0)
    counts = m.mpml_counts(ctx)
    value = job_throughput(world, K, total_ms / 1e3)

    # for comparison: the trajectory continued for three steps with every CG solve to cg_rtol
    exact = None
    if args.cg_forcing > 0:
        o0 = m.solver_opts()
        ms0, nw0, cg0, gr0 = [], [], [], []
        for i in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = one_step(ctx, parts, W + K + i, o0)
            e1.record(stream)
            e1.synchronize()
            ms0.append(e0.elapsed_time(e1))
            nw0.append(st.newton_iters)
            cg0.append(st.cg_iters_total)
            gr0.append(st.g_norm / st.g0_norm if st.g0_norm > 0 else 0.0)
        exact = {"cg_forcing": 0.0, "steps": f"trajectory steps {W + K}..{W + K + 2}",
                 "steps_per_s": 3e3 / float(np.sum(ms0)), "ms_per_step": float(np.mean(ms0)),
                 "newton_iters_per_step": float(np.mean(nw0)), "cg_iters_per_step": float(np.mean(cg0)),
                 "g_rel_max": float(np.max(gr0))}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region): the same
    # trajectory steps W .. W+K-1 after W untimed warm-up steps from the moment of impact
    e2e = None
    if not args.no_e2e:
        m.mpml_destroy(ctx)
        hctx, hcur, hparts = make_ctx(m, sc, stream, host=True)
        for s in range(W):
            one_step(hctx, hparts, s)
        barrier()
        t_e2e = 0.0
        for i in range(K):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            one_step(hctx, hparts, W + i)  # mpml_g2p synchronises after the device-to-host copies
            t_e2e += time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, dist, "cuda")
        per = 4 * (3 + 3 + 9 + 9 + 1 + 1) + 4
        e2e = {"value": job_throughput(world, K, t_e2e), "unit": "steps/s",
               "h2d_bytes_per_step": sc.num_particles * per, "d2h_bytes_per_step": sc.num_particles * per}
        ctx = hctx
        del hcur

    roof = None
    if pcg_n > 0:
        # the dominant kernel: one persistent cooperative launch runs a whole Jacobi-PCG solve
        mean_ms = pcg_ms / pcg_n
        achieved = alg_bytes / (pcg_ms / 1e3) / 1e9
        tr = ncu_traffic(f"slab_on_sand_{args.n}_impact") if last_staging == 3 else None
        if tr and tr.get("ctas_per_sm") != last_ctas:
            tr = None  # captured with another CTA count
        traffic = None
        if tr:
            # the captured smaller case's DRAM bytes per CG iteration, scaled by the active cells
            mean_cells = float(np.mean([r["cells"] for r in per_step]))
            traffic = tr["dram_bytes_per_cg_iter"] * mean_cells / tr["cells"] * (pcg_iters / pcg_n)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic,
                "algorithmic_bytes_per_launch": alg_bytes / pcg_n,
                "peak_kind": peak_kind + " (hbm_gbs of MEASURED_PEAKS.json)" if peak_kind == "measured" else peak_kind,
                "kernel": pcg_kernel_name(True, last_staging, last_ctas),
                "launches_timed": pcg_n, "mean_launch_ms": mean_ms, "cg_iters_per_launch": pcg_iters / pcg_n,
                "bytes_per_cg_iter_rule": "180 B per active cell (45-number tangent) + 28 B (HVP) + 120 B (CG "
                                          "vector passes) per DOF node",
                "us_per_cg_iter": 1e3 * pcg_ms / max(pcg_iters, 1),
                "floor_achieved": floor_bytes / (pcg_ms / 1e3) / 1e9,
                "floor_rule": "64 B per active cell (F, S, V: the state that defines the cell Hessian) + 148 B "
                              "per DOF node",
                "traffic_source": (tr["source"] + "; " + tr["scaling"]) if tr else None,
                "timing": "CUDA events around each cooperative launch on the context stream, timed steps"}
    hvp = None
    if hvp_n > 0:
        hvp_mean = hvp_ms / hvp_n
        hvp = {"gbs": hvp_bytes / (hvp_mean / 1e3) / 1e9, "frac": hvp_bytes / (hvp_mean / 1e3) / 1e9 / peaks["hbm_gbs"],
               "mean_us": 1e3 * hvp_mean, "phases_timed": hvp_n, "bytes_per_hvp": hvp_bytes,
               "timing": "device global timer, HVP phase of the persistent kernel (first block start to barrier), "
                         "last timed step's active set"}

    others = None
    if not args.no_other_configs and rank == 0:
        m.mpml_destroy(ctx)
        ctx = None
        del cur, init, parts
        torch.cuda.empty_cache()
        others = other_configs(m, args, peaks)
    learned = None
    if not args.no_learned and rank == 0:
        learned = learned_comparison(m, args, stream, flush)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        frac = min(1.0, 2_000_000 / sc.num_particles)
        arrays = sample_arrays(sc, frac)
        u = oracle_units(sc, arrays)
        nn, ncg = float(np.mean(newton_its)), float(np.mean(cg_its))
        cells = float(np.mean([r["cells"] for r in per_step]))
        t1 = step_seconds(u, sc.num_particles, cells, nn, ncg)
        hc = host_cpu()
        procs = max(1, min(hc["nproc"] or 1, 16))
        multi = all_cores_units(arrays, args.n, procs)
        t_all = [step_seconds(uu, sc.num_particles, cells, nn, ncg) for uu, _ in multi]
        cpu = {"value": 1.0 / t1, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": (f"FP64 oracle, single thread: a bounded sample of the workload (the {len(arrays['x'])} "
                          f"particles of a column over the impact zone: unload, stretch, two capped Newton "
                          f"iterations with 5 and 15 CG iterations, load; {u['wall_s']:.1f} s) gives its seconds "
                          f"per particle, per cell and stretch, per cell and Newton iteration and per cell and CG "
                          f"iteration, scaled to the timed steps' mean counts ({sc.num_particles} particles, "
                          f"{cells:.0f} active cells, {nn:.1f} Newton and {ncg:.0f} CG iterations per step)"),
               "host": hc,
               "all_cores": {"value": float(np.sum([1.0 / t for t in t_all])), "unit": "steps/s", "cores": procs,
                             "kind": "oracle",
                             "sample": f"the same sample in {procs} concurrent single-thread oracle processes "
                                       "(spawned), aggregate rate of independent copies (the oracle is serial)"}}
    if ctx is not None:
        m.mpml_destroy(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_text(args.n), "grid": args.n, "particles": int(counts["particles"]),
                           "active_cells": int(counts["cells"]), "dof_nodes": int(counts["nodes"]),
                           "materials": "2 (von Mises slab, Drucker-Prager sand; mixed cells)",
                           "precision": "fp32 storage and arithmetic, fp64 reductions and Newton iterate",
                           "preconditioner": "jacobi", "cg_rtol": 1e-6, "newton_rtol": 1e-6,
                           "cg_forcing": args.cg_forcing,
                           "steps_timed": f"trajectory steps {W}..{W + K - 1} after impact",
                           "l2": "inputs (2.1 GB of particles) larger than L2, and a 256 MB L2 flush between "
                                 "timed steps",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "newton_iters_per_step": float(np.mean(newton_its)),
                "cg_iters_per_step": float(np.mean(cg_its)),
                "newton_iters_per_s": float(np.sum(newton_its)) / (total_ms / 1e3),
                "per_step": per_step, "step_ms": step_ms, "without_forcing": exact,
                "pcg_autotune": {"chosen": tune_shape, "shapes": [list(sh) for sh in m.PCG_SHAPE_TABLE],
                                 "us_per_cg_iter": [round(1e3 * t / 30, 2) if t >= 0 else None for t in tune_ms],
                                 "rule": "30 CG iterations of the last warm-up Newton system per shape, best of 2; "
                                         "shape = (staging 1 staged / 2 streamed / 3 column groups, CTAs per SM)"},
                "hvp_gbs": hvp["gbs"] if hvp else None, "hvp": hvp, "learned_precond": learned,
                "other_configs": others,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def hvp_probe(args):
    """One workload, one implicit step, then a few standalone HVP launches on its tangent."""
    import torch

    import paper_2602_07853_gb300.mpml as m
    from paper_2602_07853_gb300 import scenes

    sc = {"pressed_block_236": lambda: scenes.pressed_block(236), "slab_on_sand_256": lambda: scenes.slab_on_sand(256),
          "two_spheres_168": lambda: scenes.two_spheres(168, gap=1.0 / 168)}[args.hvp_probe]()
    m.load()
    stream = torch.cuda.current_stream()
    mats = [m.material(mt.model, *m.lame_parameters(mt.E, mt.nu), mt.plastic, mt.yield_stress, mt.friction_angle)
            for mt in sc.materials]
    desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, m.FP32, sc.wall_layers, sc.plate, sc.inv_dx)
    ctx = m.mpml_create(desc, mats, stream.cuda_stream)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.particles(np.float32).items()}
    pp = m.particles_from_tensors(p["x"], p["v"], p["F"], p["G"], p["mp"], p["Vp"], p["mat"])
    m.mpml_resample(ctx, pp)
    rc, st = m.mpml_newton_step(ctx, m.solver_opts())
    counts = m.mpml_counts(ctx)
    m.mpml_stretch(ctx)
    m.mpml_linearize(ctx, m.mpml_get_field(ctx, m.F_NODE_VHAT))
    tile, tile_ms = m.mpml_autotune_hvp(ctx, 3)
    ms = m.mpml_hvp_bench(ctx, max(args.steps, 1))
    k_bytes = CMP_TANGENT_BYTES if len(sc.materials) == 1 else PACKED_TANGENT_BYTES
    alg = k_bytes * counts["cells"] + 28.0 * counts["nodes"]
    print(json.dumps({"probe": args.hvp_probe, "cells": counts["cells"], "nodes": counts["nodes"], "hvp_ms": ms,
                      "hvp_gbs": alg / (ms / 1e3) / 1e9, "tile": m.mpml_get_hvp_tile(ctx)[1], "tile_ms": tile_ms,
                      "newton_rc": rc}), flush=True)
    m.mpml_destroy(ctx)
    return 0


def pcg_probe(args):
    """One workload at --n, --warmup trajectory steps, then one more step (for profilers: its
    persistent solves are the launches after the warm-up's); prints the solve's counts."""
    import torch

    import paper_2602_07853_gb300.mpml as m
    from paper_2602_07853_gb300 import scenes

    sc = {"slab_on_sand_impact": lambda: scenes.slab_on_sand(args.n, impact=True),
          "two_spheres_contact": lambda: scenes.two_spheres(args.n, gap=1.0 / args.n),
          "pressed_block": lambda: scenes.pressed_block(args.n)}[args.pcg_probe]()
    m.load()
    stream = torch.cuda.current_stream()
    ctx, p, pp = make_ctx(m, sc, stream)
    launches = []
    for s in range(args.warmup + 1):
        if s == args.warmup:
            m.mpml_set_profiling(ctx, 1)  # the last step: solver launch and HVP-phase times
        m.mpml_set_time(ctx, s * sc.dt)
        m.mpml_resample(ctx, pp)
        rc, st = m.mpml_newton_step(ctx, m.solver_opts())
        m.mpml_g2p(ctx, pp)
        launches.append(st.newton_iters)
    cn = m.mpml_counts(ctx)
    _, staging, ctas = m.mpml_get_pcg_config(ctx)
    hn, hms, _ = m.mpml_hvp_timing(ctx)
    pn, pit, pms = m.mpml_pcg_timing(ctx)
    print(json.dumps({"probe": args.pcg_probe, "n": args.n, "particles": cn["particles"], "cells": cn["cells"],
                      "nodes": cn["nodes"], "newton_per_step": launches, "last_cg_iters":
                      [int(st.cg_iters[k]) for k in range(min(st.newton_iters, 64))], "staging": staging,
                      "ctas_per_sm": ctas, "us_per_cg_iter": 1e3 * pms / max(pit, 1),
                      "us_hvp_phase": 1e3 * hms / max(hn, 1), "rc": rc}), flush=True)
    m.mpml_destroy(ctx)
    return 0


def main():
    args = parse()
    if args.hvp_probe:
        return hvp_probe(args)
    if args.pcg_probe:
        return pcg_probe(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
