"""Benchmark: implicit MPM Lite time steps per second on one GB300 (or N replicas).

A step is one pass of the whole hot path through the C ABI: mpml_resample
(sort, P2Q, Q2N), mpml_newton_step (stretch reconstruction, Newton with
Jacobi-PCG to relative residual 1e-6 and line search), mpml_g2p.

Workload: two Neo-Hookean spheres (E = 1e6 Pa, nu = 0.4, r = 0.15 m, rho =
1000) approaching at 2 m/s relative velocity on a 168^3 grid with 8
particles per cell (1,073,088 particles), dt = 2e-3 s, starting at contact so
that every step solves a nonlinear system; FP32 with FP64 reductions.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded sample, see cpu_baseline).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton steps/s & HVP GB/s at rel resid 1e-6; learned-precond FP32 vs plain PCG"
WORKLOAD = ("two Neo-Hookean spheres (E=1e6, nu=0.4, r=0.15) colliding at 2 m/s on a 168^3 grid, "
            "8 particles/cell (1,073,088 particles), dt=2e-3, starting at contact")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=168, help="grid cells per axis")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--check-every", type=int, default=16)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner comparison")
    ap.add_argument("--hvp-probe", choices=["pressed_block_236", "slab_on_sand_256", "two_spheres_168"],
                    help="only build this workload, take one step, and time the standalone HVP (for profilers)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the extra measurements of the other workloads (batch, plasticity, large block)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


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


def ncu_traffic():
    """DRAM bytes of one persistent-PCG launch from the committed ncu capture (cold cache; the CG
    working set then stays in L2), or None when the capture was taken on another version of the
    kernel."""
    path = os.path.join(ROOT, "profiles", "pcg_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d["dram_bytes_per_launch"]


# tangent bytes per active cell: 25 FP32 numbers (compressed, one material) or 45 (packed)
CMP_TANGENT_BYTES = 100.0
PACKED_TANGENT_BYTES = 180.0


def pcg_bytes_per_iter(n_cells, n_nodes):
    """Algorithmic bytes of one CG iteration (FP32): the HVP reads the compressed tangent of every
    active cell (25 numbers, 100 B) and per DOF node p, m and writes q (28 B); the CG update makes
    about ten 12-byte vector passes per DOF node (x, r, p, q, D^-1 reads and writes)."""
    return CMP_TANGENT_BYTES * n_cells + (28.0 + 120.0) * n_nodes


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(sc, newton_iters_per_step):
    """Oracle on the full workload, bounded: unload, stretch, ONE Newton iteration
    (full Jacobi-PCG to 1e-6), load.  Step time = fixed part + newton_iters_per_step
    x one Newton iteration."""
    import oracle

    o = oracle.Oracle(oracle.make_scene(sc.n, sc.dx, sc.dt, sc.gravity,
                                        [(m.model, m.E, m.nu) for m in sc.materials],
                                        wall_layers=sc.wall_layers, inv_dx=sc.inv_dx))
    p = sc.particles(np.float32)
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in p.items()}
    t0 = time.perf_counter()
    o.unload(**p)
    o.stretch()
    t1 = time.perf_counter()
    o.newton(oracle.default_solver(newton_max=1))
    t2 = time.perf_counter()
    o.load()
    t3 = time.perf_counter()
    fixed = (t1 - t0) + (t3 - t2)
    per_newton = t2 - t1
    return fixed + newton_iters_per_step * per_newton, fixed, per_newton


def oracle_newton_count(n):
    path = os.path.join(ROOT, "oracle", "bench_workload_counts.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        if str(n) in d:
            return d[str(n)]["newton_iters_first_step"]
    return 8


def run_reference(args, rank, world):
    from paper_2602_07853_gb300 import scenes

    if rank != 0:
        return 0
    sc = scenes.two_spheres(args.n, gap=1.0 / args.n)
    nnewton = oracle_newton_count(args.n)
    for _ in range(args.warmup):
        oracle_sample(sc, nnewton)
    times = []
    for _ in range(args.steps):
        t, fixed, per_newton = oracle_sample(sc, nnewton)
        times.append(t)
    total = float(np.sum(times))
    value = args.steps / total
    sample = (f"full workload, per step: unload+stretch+load plus ONE Newton iteration (Jacobi-PCG to 1e-6) "
              f"timed, step time = fixed + {nnewton} x Newton iteration ({nnewton} = the oracle's own Newton "
              f"count on this workload's first step); single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": args.n, "precision": "fp64", "preconditioner": "jacobi",
                       "cg_rtol": 1e-6, "newton_rtol": 1e-6},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample},
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
def other_configs(m, scenes, args, peaks):
    """Secondary measurements (not the headline value): the 64-scene batch (config 4), the
    von Mises / Drucker-Prager slab on sand at 256^3 (config 5) and the HVP of the 3-8M pressed
    block, each with CUDA events, inputs resident, warm-up first."""
    import torch

    out = {}
    steps = max(2, min(args.steps, 4))

    def make(sc, stream):
        mats = [m.material(mt.model, *m.lame_parameters(mt.E, mt.nu), mt.plastic, mt.yield_stress,
                           mt.friction_angle) for mt in sc.materials]
        desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, m.FP32, sc.wall_layers, sc.plate, sc.inv_dx)
        ctx = m.mpml_create(desc, mats, stream.cuda_stream)
        p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.particles(np.float32).items()}
        parts = m.particles_from_tensors(p["x"], p["v"], p["F"], p["G"], p["mp"], p["Vp"], p["mat"])
        return ctx, p, parts

    # config 4: 64 scenes of uneven size, one context and stream each, batched solve
    n_sc = 64
    scs = [scenes.batch_scene(i) for i in range(n_sc)]
    streams = [torch.cuda.Stream() for _ in scs]
    made = [make(sc, st) for sc, st in zip(scs, streams)]
    ctxs = [c for c, _, _ in made]
    parts = [pp for _, _, pp in made]
    init = [{k: v.clone() for k, v in p.items()} for _, p, _ in made]
    torch.cuda.synchronize()

    def run_batch(k0, k):
        ms, newton, cg = [], 0, 0
        for s in range(k0, k0 + k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for c in ctxs:
                m.mpml_set_time(c, s * scs[0].dt)
            m.mpml_resample_batch(ctxs, parts)
            rc, st = m.mpml_newton_step_batch(ctxs)
            for c, pp in zip(ctxs, parts):
                m.mpml_g2p(c, pp)
            torch.cuda.synchronize()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            newton += sum(x.newton_iters for x in st)
            cg += sum(x.cg_iters_total for x in st)
        return ms, newton, cg

    run_batch(0, 3)  # warm-up
    for (_, p, _), q in zip(made, init):
        for key in p:
            p[key].copy_(q[key])
    torch.cuda.synchronize()
    ms, newton, cg = run_batch(0, 8)
    out["batch64"] = {"workload": "64 fixed-corotated scenes (box / sphere / torus, extents 8-48 voxels, E log-uniform "
                                  "1e4-1e7, nu 0.2-0.45) each on its own 64^3 grid, dropped at 1 m/s, dt = 1e-3, "
                                  "steps 0-7 from rest above the floor",
                      "particles": int(sum(int(p["x"].shape[0]) for _, p, _ in made)),
                      "steps_per_s": 1e3 * len(ms) / float(np.sum(ms)), "ms_per_step": float(np.mean(ms)),
                      "newton_iters_per_step": newton / len(ms), "cg_iters_per_step": cg / len(ms),
                      "solver": "mpml_resample_batch + mpml_newton_step_batch (one persistent PCG launch per "
                                "Newton round over all scenes), one stream per scene"}
    for c in ctxs:
        m.mpml_destroy(c)
    del made, init
    torch.cuda.empty_cache()

    # the explicit integrator on the two-sphere workload (dt below the elastic CFL limit)
    sc = scenes.two_spheres(168, gap=1.0 / 168, dt=5e-5)
    stream = torch.cuda.current_stream()
    ctx, p, pp = make(sc, stream)
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
        stream = torch.cuda.current_stream()
        ctx, p, pp = make(sc, stream)
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
    sc = scenes.dam_break(128)
    stream = torch.cuda.current_stream()
    ctx, p, pp = make(sc, stream)
    times, newton, cg = [], 0, 0
    for s in range(1 + 3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.mpml_set_time(ctx, s * sc.dt)
        m.mpml_resample(ctx, pp)
        rc, st = m.mpml_newton_step(ctx, m.solver_opts())
        m.mpml_g2p(ctx, pp)
        b.record(stream)
        torch.cuda.synchronize()
        if s > 0:
            times.append(a.elapsed_time(b))
            newton += st.newton_iters
            cg += st.cg_iters_total
    out["dam_break_water_128"] = {"particles": int(sc.num_particles), "dt": sc.dt,
                                  "steps_per_s": 1e3 * len(times) / float(np.sum(times)),
                                  "ms_per_step": float(np.mean(times)), "newton_iters_per_step": newton / len(times),
                                  "cg_iters_per_step": cg / len(times),
                                  "workload": "water column (bulk modulus 3.3e5 Pa) collapsing onto a fixed-corotated "
                                              "cube, steps 1-3 from rest"}
    m.mpml_destroy(ctx)
    del p
    torch.cuda.empty_cache()

    # config 5 at full size and the 3-8M pressed block: step time and HVP bandwidth
    for key, sc, nstep in (("slab_on_sand_256", scenes.slab_on_sand(256), 2),
                           ("pressed_block_236", scenes.pressed_block(236), 2)):
        stream = torch.cuda.current_stream()
        ctx, p, pp = make(sc, stream)
        times, newton, cg = [], 0, 0
        for s in range(nstep + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.mpml_set_time(ctx, s * sc.dt)
            m.mpml_resample(ctx, pp)
            rc, st = m.mpml_newton_step(ctx, m.solver_opts())
            m.mpml_g2p(ctx, pp)
            b.record(stream)
            torch.cuda.synchronize()
            if s > 0:  # the first step is the warm-up
                times.append(a.elapsed_time(b))
                newton += st.newton_iters
                cg += st.cg_iters_total
        counts = m.mpml_counts(ctx)
        vhat = m.mpml_get_field(ctx, m.F_NODE_VHAT)
        m.mpml_stretch(ctx)
        m.mpml_linearize(ctx, vhat)
        tile, tile_ms = m.mpml_autotune_hvp(ctx, 5)  # the standalone HVP's fastest launch shape
        hvp_ms = m.mpml_hvp_bench(ctx, 20)
        k_bytes = CMP_TANGENT_BYTES if len(sc.materials) == 1 else PACKED_TANGENT_BYTES
        alg = k_bytes * counts["cells"] + 28.0 * counts["nodes"]
        gbs = alg / (hvp_ms / 1e3) / 1e9
        out[key] = {"particles": int(counts["particles"]), "active_cells": int(counts["cells"]),
                    "dof_nodes": int(counts["nodes"]), "steps_per_s": 1e3 * len(times) / float(np.sum(times)),
                    "ms_per_step": float(np.mean(times)), "newton_iters_per_step": newton / len(times),
                    "cg_iters_per_step": cg / len(times),
                    "hvp": {"kernel": m.mpml_get_hvp_tile(ctx)[1], "tile_ms": tile_ms,
                            "mean_ms": hvp_ms, "bytes": alg, "gbs": gbs, "frac": gbs / peaks["hbm_gbs"],
                            "bytes_rule": f"{int(k_bytes)} B per active cell + 28 B per DOF node, working set "
                                          f"{alg / 1e6:.0f} MB vs 129 MB L2"}}
        m.mpml_destroy(ctx)
        del p
        torch.cuda.empty_cache()
    return out


def learned_comparison(m, ctx, parts, reset, one_step, args, stream, flush):
    """Trains the learned preconditioner on the workload's first Newton system (untimed), then
    times the same steps with flexible CG (CUDA events, L2 flushed as for the main number)."""
    import torch

    reset()
    m.mpml_set_time(ctx, 0.0)
    m.mpml_resample(ctx, parts)
    m.mpml_nn_set_weights(ctx, m.nn_init_weights(0, gain=0.1))
    t0 = time.perf_counter()
    tr = m.mpml_nn_train(ctx, m.train_opts())
    train_s = time.perf_counter() - t0
    opts = m.solver_opts(precond=m.PRECOND_LEARNED)
    for _ in range(max(1, args.warmup)):
        reset()
        m.mpml_set_time(ctx, 0.0)
        m.mpml_resample(ctx, parts)
        m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, parts)
    torch.cuda.synchronize()
    ms, cg, fb, nw = [], [], [], []
    for _ in range(args.steps):
        reset()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.mpml_set_time(ctx, 0.0)
        m.mpml_resample(ctx, parts)
        rc, st = m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, parts)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        cg.append(st.cg_iters_total)
        fb.append(st.fcg_fallbacks)
        nw.append(st.newton_iters)
    # direction quality on a Newton system the network was not trained on (one step later):
    # mean 1 - cos_H(z(r), e) of the trained network and of Jacobi (zero network)
    trained = m.mpml_nn_get_weights(ctx)
    reset()
    m.mpml_set_time(ctx, 0.0)
    m.mpml_resample(ctx, parts)
    m.mpml_newton_step(ctx, m.solver_opts())
    m.mpml_g2p(ctx, parts)
    m.mpml_set_time(ctx, 2e-3)
    m.mpml_resample(ctx, parts)
    ev = m.mpml_nn_train(ctx, m.train_opts(samples=16, epochs=1, batch=4, lr=0.0))
    m.mpml_nn_set_weights(ctx, [np.zeros(s) for s in m.NN_SHAPES])
    ev0 = m.mpml_nn_train(ctx, m.train_opts(samples=16, epochs=1, batch=4, lr=0.0))
    m.mpml_nn_set_weights(ctx, trained)
    return {"steps_per_s": 1e3 * len(ms) / float(np.sum(ms)), "ms_per_step": float(np.mean(ms)),
            "unseen_system_loss": {"learned": ev.loss_first, "jacobi": ev0.loss_first,
                                   "definition": "mean 1 - cos_H(z(r), e) over 16 (r, e) pairs of the next "
                                                 "step's first Newton system"},
            "cg_iters_per_step": float(np.mean(cg)), "newton_iters_per_step": float(np.mean(nw)),
            "fcg_fallbacks_per_step": float(np.mean(fb)), "train_s": train_s, "train_samples": tr.samples,
            "loss_first": tr.loss_first, "loss_last": tr.loss_last,
            "solver": "flexible CG with the trained 3-layer 16-channel BF16 network, Jacobi-PCG fallback"}


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2602_07853_gb300.mpml as m
    from paper_2602_07853_gb300 import scenes

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

    sc = scenes.two_spheres(args.n, gap=1.0 / args.n)
    mats = [m.material(mt.model, *m.lame_parameters(mt.E, mt.nu)) for mt in sc.materials]
    desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, m.FP32, sc.wall_layers, sc.plate, sc.inv_dx)
    stream = torch.cuda.current_stream()
    ctx = m.mpml_create(desc, mats, stream.cuda_stream)
    p32 = sc.particles(np.float32)
    init = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in p32.items()}
    cur = {k: v.clone() for k, v in init.items()}
    parts = m.particles_from_tensors(cur["x"], cur["v"], cur["F"], cur["G"], cur["mp"], cur["Vp"], cur["mat"])
    opts = m.solver_opts(check_every=args.check_every)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def reset():
        for k in cur:
            cur[k].copy_(init[k])

    def one_step(t):
        m.mpml_set_time(ctx, t)
        m.mpml_resample(ctx, parts)
        rc, st = m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, parts)
        return st

    # warm-up (each step restarts from the contact state so all steps do equal work)
    for _ in range(args.warmup):
        reset()
        one_step(0.0)
    barrier()
    m.mpml_set_profiling(ctx, 1)
    launches0 = m.mpml_kernel_launches(ctx)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    newton_its, cg_its, last_cg = [], [], []
    barrier()
    for i in range(args.steps):
        reset()
        flush.zero_()  # L2 flush (256 MB > 129 MB L2) outside the timed events
        ev[i][0].record(stream)
        st = one_step(0.0)
        ev[i][1].record(stream)
        newton_its.append(st.newton_iters)
        cg_its.append(st.cg_iters_total)
        last_cg = [int(st.cg_iters[k]) for k in range(min(st.newton_iters, 64))]
    barrier()
    clk = clocks.stop()
    launches = m.mpml_kernel_launches(ctx) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(np.sum(step_ms)), dist, "cuda")
    hvp_n, hvp_ms, hvp_bytes = m.mpml_hvp_timing(ctx)
    pcg_n, pcg_iters, pcg_ms = m.mpml_pcg_timing(ctx)
    m.mpml_set_profiling(ctx, 0)
    counts = m.mpml_counts(ctx)
    value = job_throughput(world, args.steps, total_ms / 1e3)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in init.items()}
        hcur = {k: v.clone().pin_memory() for k, v in host.items()}
        hparts = m.particles_from_tensors(hcur["x"], hcur["v"], hcur["F"], hcur["G"], hcur["mp"], hcur["Vp"],
                                          hcur["mat"])
        for k in hcur:
            hcur[k].copy_(host[k])
        m.mpml_resample(ctx, hparts)
        m.mpml_newton_step(ctx, opts)
        m.mpml_g2p(ctx, hparts)
        barrier()
        t_e2e = 0.0
        for i in range(args.steps):
            for k in hcur:
                hcur[k].copy_(host[k])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.mpml_set_time(ctx, 0.0)
            m.mpml_resample(ctx, hparts)
            m.mpml_newton_step(ctx, opts)
            m.mpml_g2p(ctx, hparts)  # synchronises after the device-to-host copies
            t_e2e += time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, dist, "cuda")
        n = sc.num_particles
        per = 4 * (3 + 3 + 9 + 9 + 1 + 1) + 4
        e2e = {"value": job_throughput(world, args.steps, t_e2e), "unit": "steps/s", "h2d_bytes_per_step": n * per,
               "d2h_bytes_per_step": n * per}

    peaks, peak_kind = measured_peaks()
    roof = None
    if pcg_n > 0:
        # the dominant kernel: one persistent cooperative launch runs a whole Jacobi-PCG solve
        per_iter = pcg_bytes_per_iter(counts["cells"], counts["nodes"])
        mean_ms = pcg_ms / pcg_n
        iters_per_launch = pcg_iters / pcg_n
        achieved = per_iter * iters_per_launch / (mean_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(),
                "peak_kind": peak_kind, "kernel": "k_pcg_persistent", "launches_timed": pcg_n,
                "mean_launch_ms": mean_ms, "cg_iters_per_launch": iters_per_launch,
                "bytes_per_cg_iter": per_iter, "us_per_cg_iter": 1e3 * pcg_ms / max(pcg_iters, 1),
                "timing": "CUDA events around each launch on the context stream"}
    hvp = None
    if hvp_n > 0:
        hvp_mean = hvp_ms / hvp_n
        hvp = {"gbs": hvp_bytes / (hvp_mean / 1e3) / 1e9, "frac": hvp_bytes / (hvp_mean / 1e3) / 1e9 / peaks["hbm_gbs"],
               "mean_us": 1e3 * hvp_mean, "phases_timed": hvp_n, "bytes_per_hvp": hvp_bytes,
               "timing": "device global timer, HVP phase of the persistent kernel (first block start to barrier)"}

    learned = None
    if not args.no_learned:
        learned = learned_comparison(m, ctx, parts, reset, one_step, args, stream, flush)
    others = None
    if not args.no_other_configs and rank == 0:
        others = other_configs(m, scenes, args, peaks)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        nn = float(np.mean(newton_its)) if newton_its else 8.0
        t_step, fixed, per_newton = oracle_sample(sc, nn)
        cpu = {"value": 1.0 / t_step, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": (f"full workload: unload+stretch+load ({fixed:.1f} s) plus ONE Newton iteration with "
                          f"Jacobi-PCG to 1e-6 ({per_newton:.1f} s), scaled to {nn:.1f} Newton iterations per "
                          "step (the GPU run's mean); single thread")}
    m.mpml_destroy(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": args.n, "particles": int(counts["particles"]),
                           "active_cells": int(counts["cells"]), "dof_nodes": int(counts["nodes"]),
                           "precision": "fp32 storage and arithmetic, fp64 reductions",
                           "preconditioner": "jacobi", "cg_rtol": 1e-6, "newton_rtol": 1e-6,
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "newton_iters_per_step": float(np.mean(newton_its)),
                "cg_iters_per_step": float(np.mean(cg_its)),
                "newton_iters_per_s": float(np.sum(newton_its)) / (total_ms / 1e3),
                "cg_iters_last_step": last_cg,
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


def main():
    args = parse()
    if args.hvp_probe:
        return hvp_probe(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
