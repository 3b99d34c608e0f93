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


def max_err(a, b):
    """Largest element error relative to the reference's largest element."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    sb = np.abs(b).max()
    return float(np.abs(a - b).max() / (sb if sb > 0 else 1.0))


# every check of the session: (test, field, norm-relative error, max-relative error, tolerance);
# written out by conftest.py when MPML_PRECISION_REPORT names a file
REPORT = []


def record(name, value, tol):
    """A scalar error measured by a test (e.g. positions in units of dx) into the report."""
    import os
    REPORT.append((os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], str(name), float(value), float(value), tol))
    assert value <= tol, f"{name}: {value:.3e} > {tol}"


def check(got, want, tol, name="", elem_tol=None):
    """Element-by-element parity of a floating-point field: the norm-relative error
    ||a - b|| / ||b|| and the largest element error max|a - b| / max|b| are both within tol
    (elem_tol for the second if given)."""
    import os
    a, b = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    assert np.isfinite(a).all(), (name, "non-finite values")
    nrel, mrel = rel_err(a, b), max_err(a, b)
    REPORT.append((os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], str(name), nrel, mrel, tol))
    et = tol if elem_tol is None else elem_tol
    assert nrel <= tol and mrel <= et, f"{name}: norm-relative {nrel:.3e}, max-relative {mrel:.3e} (tol {tol}, {et})"
    return nrel, mrel


def by_identity(p, ids):
    """Particle arrays reordered by original particle index: ids[s] is the original index of
    the s-th particle in the (sorted) order the arrays are in.  After a few steps the GPU and
    the oracle sort a particle that sits within rounding of a cell boundary into different
    cells (their positions differ at the FP32 / FP64 rounding level), so trajectories are
    compared particle by particle through the identities both sides report (perm)."""
    out = {}
    for k, v in p.items():
        a = np.empty_like(v)
        a[ids] = v
        out[k] = a
    return out


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
        self.ids = np.arange(n, dtype=np.int64)

    def resample(self):
        rc = m.mpml_resample(self.ctx, self.parts)
        # identities of the sorted particles (perm[s] = index before the call)
        self.ids = self.ids[self.t["perm"].cpu().numpy().astype(np.int64)]
        return rc

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

    def particles_by_identity(self):
        p = self.particles()
        p.pop("perm")
        return by_identity(p, self.ids)


    def field(self, f):
        return m.mpml_get_field(self.ctx, f, len(self.mats))

    def keys(self, what):
        return m.mpml_get_keys(self.ctx, what)


class OracleSim:
    """The FP64 oracle stepping the same scene, tracking particle identities like GpuSim."""

    def __init__(self, o, particles):
        self.o = o
        self.p = particles
        self.ids = np.arange(len(particles["x"]), dtype=np.int64)

    def step(self, t, solver=None, explicit=False):
        self.o.set_time(t)
        if explicit:
            rc, out = self.o.explicit_step(self.p)
            st = None
        else:
            rc, out, st = self.o.step(self.p, solver)
        if rc >= 0:
            self.ids = self.ids[self.o.perm()]
            self.p = out
        return rc, st

    def particles_by_identity(self):
        return by_identity(self.p, self.ids)
