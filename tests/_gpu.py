"""GPU test harness: drives the CUDA library through the C ABI (mpml.py binding)."""
import numpy as np
import torch

import paper_2602_07853_gb300.mpml as m

NP_DTYPE = {m.FP32: np.float32, m.FP64: np.float64}
TORCH_DTYPE = {m.FP32: torch.float32, m.FP64: torch.float64}


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class GpuSim:
    """One library context on cuda:0 for a seeded scene."""

    def __init__(self, sc, precision=m.FP32):
        m.load()
        self.sc = sc
        self.prec = precision
        self.npdt = NP_DTYPE[precision]
        desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, precision, sc.wall_layers, sc.plate, sc.inv_dx)
        self.mats = [m.material(mt.model, *m.lame_parameters(mt.E, mt.nu), mt.plastic, mt.yield_stress,
                                mt.friction_angle) for mt in sc.materials]
        self.stream = torch.cuda.current_stream()
        self.ctx = m.mpml_create(desc, self.mats, self.stream.cuda_stream)
        self.t = None

    def close(self):
        if self.ctx is not None:
            m.mpml_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def inputs(self):
        """The particle arrays in the precision of the context (what both sides see), as float64/int32."""
        p = self.sc.particles(self.npdt)
        return {k: (v.astype(np.float64) if k != "mat" else v) for k, v in p.items()}

    def set_particles(self, p=None, host=False):
        p = p if p is not None else self.sc.particles(self.npdt)
        dev = "cpu" if host else "cuda"
        self.t = {}
        for k, v in p.items():
            arr = np.ascontiguousarray(v.astype(np.int32) if k == "mat" else v.astype(self.npdt))
            t = torch.from_numpy(arr)
            self.t[k] = t.pin_memory() if host else t.to(dev)
        n = self.t["x"].shape[0]
        self.t["perm"] = torch.zeros(n, dtype=torch.int32, device=dev)
        if host:
            self.t["perm"] = self.t["perm"].pin_memory()
        t = self.t
        self.parts = m.particles_from_tensors(t["x"], t["v"], t["F"], t["G"], t["mp"], t["Vp"], t["mat"], t["perm"])

    def resample(self):
        return m.mpml_resample(self.ctx, self.parts)

    def newton(self, opts=None):
        return m.mpml_newton_step(self.ctx, opts if opts is not None else m.solver_opts())

    def g2p(self):
        m.mpml_g2p(self.ctx, self.parts)
        m.mpml_sync(self.ctx)

    def step(self, t=0.0, opts=None):
        m.mpml_set_time(self.ctx, t)
        self.resample()
        rc, st = self.newton(opts)
        self.g2p()
        return rc, st

    def particles(self):
        return {k: (v.cpu().numpy().astype(np.float64) if k not in ("mat", "perm") else v.cpu().numpy())
                for k, v in self.t.items()}

    def field(self, f):
        return m.mpml_get_field(self.ctx, f, len(self.mats))

    def keys(self, what):
        return m.mpml_get_keys(self.ctx, what)
