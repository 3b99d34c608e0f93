"""Writes oracle/bench_workload_counts.json: the oracle's own Newton and Jacobi-PCG
iteration counts on the first time step of the benchmark workloads (test and benchmark
infrastructure; it calls only the oracle).

The CPU timing legs of the benchmark cannot run whole steps of the large workloads within
minutes; they time bounded samples of the oracle's work per particle, per cell, per Newton
iteration and per CG iteration, and scale those to a full step with these counts.

Usage: python oracle/workload_counts.py [workload ...]   (hours of CPU time for the
256^3 slab on sand; each workload is merged into the file as it finishes).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2602_07853_gb300 import scenes  # noqa: E402

WORKLOADS = {
    "slab_on_sand_256_impact": lambda: scenes.slab_on_sand(256, impact=True),
    "two_spheres_168_contact": lambda: scenes.two_spheres(168, gap=1.0 / 168),
}
OUT = os.path.join(HERE, "bench_workload_counts.json")


def counts(name):
    sc = WORKLOADS[name]()
    o = oracle.Oracle(oracle.make_scene(sc.n, sc.dx, sc.dt, sc.gravity,
                                        [(m.model, m.E, m.nu, m.plastic, m.yield_stress, m.friction_angle)
                                         for m in sc.materials],
                                        wall_layers=sc.wall_layers, plate=sc.plate, inv_dx=sc.inv_dx))
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles(np.float32).items()}
    t0 = time.perf_counter()
    rc, _, st = o.step(p)
    assert rc >= 0, rc
    return {"newton_iters_first_step": int(st.newton_iters), "cg_iters_first_step": int(st.cg_iters_total),
            "cg_iters": [int(st.cg_iters[k]) for k in range(min(st.newton_iters, 64))],
            "particles": int(sc.num_particles), "cells": o.count("cells"), "nodes": o.count("nodes"),
            "oracle_seconds_single_thread": time.perf_counter() - t0}


def main(names):
    for name in names:
        r = counts(name)
        d = {}
        if os.path.exists(OUT):
            with open(OUT) as fh:
                d = json.load(fh)
        d[name] = r
        with open(OUT, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        print(name, r, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
