// C ABI of the library (declared in include/mpml.h): context lifecycle, the
// three calls of one MPM Lite time step (Algorithm 1: Unload, Integrate,
// Load), and the synchronising introspection / operator entry points.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "mpml_internal.cuh"

using namespace mpml;

namespace mpml {

namespace {
constexpr int LF_MAX_DEVICES = 64;
std::mutex g_lf_mu;
int g_lf_fit[LF_MAX_DEVICES][LS_COUNT];
bool g_lf_init = false;
}  // namespace

int launch_fit(const void* fn, int threads, size_t smem, int slot, int* nsm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || slot < 0 || slot >= LS_COUNT) {
    cudaGetLastError();
    return 0;
  }
  if (nsm) {
    *nsm = 0;
    if (cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  if (dev < 0 || dev >= LF_MAX_DEVICES) return 0;
  std::lock_guard<std::mutex> lk(g_lf_mu);
  if (!g_lf_init) {
    for (auto& row : g_lf_fit)
      for (int& v : row) v = -1;
    g_lf_init = true;
  }
  int& fit = g_lf_fit[dev][slot];
  if (fit < 0) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
    fit = per_sm;
  }
  return fit;
}

}  // namespace mpml

namespace {

bool bad_desc(const mpml_scene_desc* d, const mpml_material* mats, int n_mats) {
  if (!d || !mats || n_mats < 1 || n_mats > MPML_MAX_MATS) return true;
  for (int a = 0; a < 3; ++a)
    if (d->n[a] < 2 || d->n[a] > (1 << 16)) return true;
  if (!(d->dx > 0) || !(d->inv_dx > 0) || !(d->dt > 0)) return true;
  if (d->precision != MPML_FP32 && d->precision != MPML_FP64) return true;
  if (d->wall_layers < 0) return true;
  for (int k = 0; k < n_mats; ++k) {
    if (mats[k].model < 0 || mats[k].model > MPML_WATER) return true;
    if (mats[k].model == MPML_WATER) {
      if (!(mats[k].mu >= 0) || !(mats[k].lambda + 2.0 / 3.0 * mats[k].mu > 0)) return true;
      if (mats[k].plastic != MPML_ELASTIC) return true;
    } else if (!(mats[k].mu > 0)) {
      return true;
    }
    if (mats[k].plastic < MPML_ELASTIC || mats[k].plastic > MPML_DRUCKER_PRAGER) return true;
    if (mats[k].plastic == MPML_VON_MISES && !(mats[k].yield_stress >= 0)) return true;
    if (mats[k].plastic == MPML_DRUCKER_PRAGER && !(mats[k].friction_angle >= 0 && mats[k].friction_angle < 1.5707963))
      return true;
  }
  // P2Q shared-memory accumulators: 729 centres x (13 + 7 n_mats) fields
  const size_t es = d->precision == MPML_FP64 ? 8 : 4;
  if (729 * (size_t)(13 + 7 * n_mats) * es > 227 * 1024) return true;
  return false;
}

int latched(mpml_ctx_s* c) {
  int st = *c->hstatus;
  if (st & ST_NONFINITE) return MPML_ERR_NONFINITE;
  if (st & ST_OUT_OF_DOMAIN) return MPML_ERR_OUT_OF_DOMAIN;
  if (st & ST_STRETCH) return MPML_ERR_STRETCH;
  if (st & ST_BADMAT) return MPML_ERR_ARG;
  if (st & ST_TIMEOUT) return MPML_ERR_TIMEOUT;
  return MPML_OK;
}

int sync_status(mpml_ctx_s* c) {
  cudaMemcpyAsync(c->hstatus, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->s);
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  return latched(c);
}

bool bad_particles(const mpml_particles* p) {
  if (!p || p->n < 0 || p->n > (int64_t)INT32_MAX - 1) return true;
  if (p->n > 0 && (!p->x || !p->v || !p->F || !p->G || !p->mass || !p->volume || !p->mat)) return true;
  return p->mem != MPML_MEM_DEVICE && p->mem != MPML_MEM_HOST;
}

// host-side compaction: copy a brick-layout array and keep the slots whose
// flag is set, in brick-list (= key) order.
template <typename T>
int export_slots(mpml_ctx_s* c, const void* dev, int width, const mpml::Buf& flag, uint8_t mask, double* out) {
  const int64_t ns = c->nb * BV;
  std::vector<T> h((size_t)ns * width);
  std::vector<uint8_t> f((size_t)ns);
  if (ns == 0) return MPML_OK;
  cudaMemcpyAsync(h.data(), dev, sizeof(T) * ns * width, cudaMemcpyDeviceToHost, c->s);
  cudaMemcpyAsync(f.data(), flag.p, ns, cudaMemcpyDeviceToHost, c->s);
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  int64_t q = 0;
  for (int64_t b = 0; b < c->nb; ++b)
    for (int l = 0; l < BV; ++l) {
      if (!(f[b * BV + l] & mask)) continue;
      for (int w = 0; w < width; ++w) out[q * width + w] = (double)h[(b * width + w) * BV + l];
      ++q;
    }
  return MPML_OK;
}

// host-side scatter of a DOF-ordered node vector (n*3 doubles) into the brick layout
template <typename T>
int import_nodes(mpml_ctx_s* c, const double* in, void* dev) {
  const int64_t ns = c->nb * BV;
  std::vector<T> h((size_t)ns * 3, T(0));
  std::vector<uint8_t> f((size_t)ns);
  if (ns == 0) return MPML_OK;
  cudaMemcpyAsync(f.data(), c->nflag.p, ns, cudaMemcpyDeviceToHost, c->s);
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  int64_t q = 0;
  for (int64_t b = 0; b < c->nb; ++b)
    for (int l = 0; l < BV; ++l) {
      if (!(f[b * BV + l] & NF_DOF)) continue;
      for (int a = 0; a < 3; ++a) h[(b * 3 + a) * BV + l] = (T)in[q * 3 + a];
      ++q;
    }
  cudaMemcpyAsync(dev, h.data(), sizeof(T) * ns * 3, cudaMemcpyHostToDevice, c->s);
  return cuda_status(cudaStreamSynchronize(c->s));
}

template <typename T>
int get_field_t(mpml_ctx_s* c, int field, double* out) {
  const int nm = c->nm, nf = acc_fields(nm);
  const int64_t ns = c->nb * BV;
  switch (field) {
    case MPML_F_CELL_MASS:
    case MPML_F_CELL_VEL:
    case MPML_F_CELL_VGRAD:
    case MPML_F_CELL_VOL:
    case MPML_F_CELL_TAU: {
      std::vector<double> a((size_t)c->nb * 0 + 1);
      int64_t ncell = 0;
      // export all accumulator fields, then normalise on the host
      std::vector<uint8_t> f((size_t)ns);
      cudaMemcpyAsync(f.data(), c->cflag.p, ns ? ns : 1, cudaMemcpyDeviceToHost, c->s);
      int rc = cuda_status(cudaStreamSynchronize(c->s));
      if (rc) return rc;
      for (auto v : f) ncell += v ? 1 : 0;
      std::vector<double> acc((size_t)ncell * nf);
      if ((rc = export_slots<T>(c, c->cacc.p, nf, c->cflag, 1, acc.data()))) return rc;
      for (int64_t i = 0; i < ncell; ++i) {
        const double* r = &acc[i * nf];
        const double m = r[0];
        if (field == MPML_F_CELL_MASS) out[i] = m;
        if (field == MPML_F_CELL_VEL)
          for (int a2 = 0; a2 < 3; ++a2) out[i * 3 + a2] = m != 0 ? r[1 + a2] / m : 0;
        if (field == MPML_F_CELL_VGRAD)
          for (int q = 0; q < 9; ++q) out[i * 9 + q] = m != 0 ? r[4 + q] / m : 0;
        if (field == MPML_F_CELL_VOL)
          for (int k = 0; k < nm; ++k) out[i * nm + k] = r[acc_V(k)];
        if (field == MPML_F_CELL_TAU)
          for (int k = 0; k < nm; ++k) {
            const double V = r[acc_V(k)];
            const int ra[6] = {0, 1, 2, 0, 0, 1}, rb[6] = {0, 1, 2, 1, 2, 2};
            for (int q = 0; q < 6; ++q) {
              double t = V != 0 ? r[acc_tau(k) + q] / V : 0;
              out[(i * nm + k) * 9 + 3 * ra[q] + rb[q]] = t;
              out[(i * nm + k) * 9 + 3 * rb[q] + ra[q]] = t;
            }
          }
      }
      return MPML_OK;
    }
    case MPML_F_CELL_STRETCH: {
      std::vector<uint8_t> f((size_t)ns);
      cudaMemcpyAsync(f.data(), c->cflag.p, ns ? ns : 1, cudaMemcpyDeviceToHost, c->s);
      int rc = cuda_status(cudaStreamSynchronize(c->s));
      if (rc) return rc;
      int64_t ncell = 0;
      for (auto v : f) ncell += v ? 1 : 0;
      std::vector<double> s6((size_t)ncell * 6 * nm);
      if ((rc = export_slots<double>(c, c->cs.p, 6 * nm, c->cflag, 1, s6.data()))) return rc;
      const int ra[6] = {0, 1, 2, 0, 0, 1}, rb[6] = {0, 1, 2, 1, 2, 2};
      for (int64_t i = 0; i < ncell; ++i)
        for (int k = 0; k < nm; ++k)
          for (int q = 0; q < 6; ++q) {
            double v = s6[i * 6 * nm + k * 6 + q] + (q < 3 ? 1.0 : 0.0);
            out[(i * nm + k) * 9 + 3 * ra[q] + rb[q]] = v;
            out[(i * nm + k) * 9 + 3 * rb[q] + ra[q]] = v;
          }
      return MPML_OK;
    }
    case MPML_F_CELL_VEL_NEW:
    case MPML_F_CELL_VGRAD_NEW: {
      std::vector<uint8_t> f((size_t)ns);
      cudaMemcpyAsync(f.data(), c->cflag.p, ns ? ns : 1, cudaMemcpyDeviceToHost, c->s);
      int rc = cuda_status(cudaStreamSynchronize(c->s));
      if (rc) return rc;
      int64_t ncell = 0;
      for (auto v : f) ncell += v ? 1 : 0;
      std::vector<double> a12((size_t)ncell * 12);
      if ((rc = export_slots<T>(c, c->cnew.p, 12, c->cflag, 1, a12.data()))) return rc;
      for (int64_t i = 0; i < ncell; ++i) {
        if (field == MPML_F_CELL_VEL_NEW)
          for (int a2 = 0; a2 < 3; ++a2) out[i * 3 + a2] = a12[i * 12 + a2];
        else
          for (int q = 0; q < 9; ++q) out[i * 9 + q] = a12[i * 12 + 3 + q];
      }
      return MPML_OK;
    }
    case MPML_F_NODE_MASS: return export_slots<T>(c, c->nmass.p, 1, c->nflag, NF_DOF, out);
    case MPML_F_NODE_VEL: return export_slots<double>(c, c->nv.p, 3, c->nflag, NF_DOF, out);
    case MPML_F_NODE_VHAT: return export_slots<double>(c, c->nvhat.p, 3, c->nflag, NF_DOF, out);
    case MPML_F_NODE_VNEW: return export_slots<double>(c, c->nvnew.p, 3, c->nflag, NF_DOF, out);
    case MPML_F_NODE_FIXED: {
      std::vector<uint8_t> f((size_t)ns);
      cudaMemcpyAsync(f.data(), c->nflag.p, ns ? ns : 1, cudaMemcpyDeviceToHost, c->s);
      int rc = cuda_status(cudaStreamSynchronize(c->s));
      if (rc) return rc;
      int64_t q = 0;
      for (int64_t i = 0; i < ns; ++i)
        if (f[i] & NF_DOF) out[q++] = (f[i] & NF_FIXED) ? 1.0 : 0.0;
      return MPML_OK;
    }
    default: return MPML_ERR_ARG;
  }
}

template <typename T>
int node_vector_op(mpml_ctx_s* c, int op, const double* in, double* phi, double* out) {
  // op 0: eval (in = v, out = grad); 1: linearize (in = v); 2: hvp (in = p, out = y)
  const int64_t ns = c->nb * BV;
  mpml::Buf tmp_in, tmp_out;
  int rc;
  if ((rc = ensure(tmp_in, sizeof(T) * 3 * (ns ? ns : 1))) || (rc = ensure(tmp_out, sizeof(T) * 3 * (ns ? ns : 1)))) {
    free_buf(tmp_in);
    free_buf(tmp_out);
    return rc;
  }
  rc = import_nodes<T>(c, in, tmp_in.p);
  if (!rc) {
    if (op == 0) rc = eval_device(c, tmp_in.p, phi, out ? tmp_out.p : nullptr);
    if (op == 1) rc = linearize_device(c, tmp_in.p);
    if (op == 2) rc = hvp_device(c, tmp_in.p, tmp_out.p);
  }
  if (!rc && out) {
    rc = export_slots<T>(c, tmp_out.p, 3, c->nflag, NF_DOF, out);
    if (!rc && op == 2) {
      // mask rows of fixed DOFs
      std::vector<double> fixed((size_t)c->nb * BV);
      std::vector<uint8_t> f((size_t)ns);
      cudaMemcpy(f.data(), c->nflag.p, ns, cudaMemcpyDeviceToHost);
      int64_t q = 0;
      for (int64_t i = 0; i < ns; ++i)
        if (f[i] & NF_DOF) {
          if (f[i] & NF_FIXED) out[3 * q] = out[3 * q + 1] = out[3 * q + 2] = 0;
          ++q;
        }
    }
  }
  cudaStreamSynchronize(c->s);
  free_buf(tmp_in);
  free_buf(tmp_out);
  return rc;
}

}  // namespace

extern "C" {

int mpml_create(const mpml_scene_desc* desc, const mpml_material* mats, int n_mats, void* stream, mpml_ctx* out) {
  if (!out) return MPML_ERR_ARG;
  *out = nullptr;
  if (bad_desc(desc, mats, n_mats)) return MPML_ERR_ARG;
  mpml_ctx_s* c = new mpml_ctx_s();
  c->d = *desc;
  for (int k = 0; k < n_mats; ++k) c->mats[k] = mats[k];
  c->nm = n_mats;
  c->s = (cudaStream_t)stream;
  c->fp64 = desc->precision == MPML_FP64;
  c->esz = c->fp64 ? 8 : 4;
  // the compressed tangent serves elastic single-material FP32 contexts (plastic ones, whose
  // fixed-point solve may change the base, keep the 45-number form)
  c->compressed = (!c->fp64 && n_mats == 1 && mats[0].plastic == MPML_ELASTIC) ? 1 : 0;
  for (int a = 0; a < 3; ++a) c->NB[a] = (desc->n[a] >> 3) + 1;
  c->NBT = (int64_t)c->NB[0] * c->NB[1] * c->NB[2];
  cudaGetDevice(&c->device);
  int rc;
  if ((rc = ensure(c->scal, sizeof(DevScalars))) || (rc = ensure(c->status, sizeof(int)))) {
    mpml_destroy(c);
    return rc;
  }
  if (cudaMallocHost(&c->hscal, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&c->hstatus, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    mpml_destroy(c);
    return MPML_ERR_NOMEM;
  }
  memset(c->hscal, 0, sizeof(DevScalars));
  *c->hstatus = 0;
  cudaMemsetAsync(c->scal.p, 0, sizeof(DevScalars), c->s);
  cudaMemsetAsync(c->status.p, 0, sizeof(int), c->s);
  if ((rc = cuda_status(cudaStreamSynchronize(c->s)))) {
    mpml_destroy(c);
    return rc;
  }
  *out = c;
  return MPML_OK;
}

int mpml_destroy(mpml_ctx c) {
  if (!c) return MPML_ERR_ARG;
  if (c->s || true) cudaStreamSynchronize(c->s);
  Buf* bufs[] = {&c->bflag_c, &c->bflag_n, &c->bmap, &c->blist, &c->cblist, &c->nbr, &c->px, &c->pv, &c->pF,
                 &c->pG, &c->pm, &c->pV, &c->pmat, &c->pperm, &c->pkey, &c->prank, &c->pbase, &c->ux, &c->uv,
                 &c->uF, &c->uG, &c->um, &c->uV, &c->umat, &c->cnt, &c->start, &c->scan_tmp, &c->cflag,
                 &c->cacc, &c->cs, &c->cK, &c->cnew, &c->nflag, &c->nmass, &c->nv, &c->nvhat, &c->nvfix,
                 &c->nvnew, &c->nvtry, &c->ng, &c->ndinv, &c->nx, &c->nr, &c->np, &c->nq, &c->np2, &c->scal, &c->status, &c->prof, &c->part, &c->gbar, &c->bbatch, &c->nolist,
                 &c->nnw, &c->nnact, &c->nny, &c->nnpart, &c->nz, &c->nns_r, &c->nns_e, &c->nnhd, &c->tuneq, &c->cB};
  for (Buf* b : bufs) free_buf(*b);
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->hstatus) cudaFreeHost(c->hstatus);
  if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaEvent_t e : c->pcg_ev)
    if (e) cudaEventDestroy(e);
  if (c->bev) cudaEventDestroy(c->bev);
  delete c;
  return MPML_OK;
}

const char* mpml_status_str(int s) {
  switch (s) {
    case MPML_OK: return "ok";
    case MPML_WARN_NOT_CONVERGED: return "warning: Newton did not converge";
    case MPML_ERR_ARG: return "invalid argument";
    case MPML_ERR_OUT_OF_DOMAIN: return "particle stencil outside the grid";
    case MPML_ERR_NONFINITE: return "non-finite value";
    case MPML_ERR_STRETCH: return "stress-to-stretch inversion failed";
    case MPML_ERR_TIMEOUT: return "bounded device wait timed out";
    case MPML_ERR_CUDA: return "CUDA runtime error";
    case MPML_ERR_NOMEM: return "out of device memory";
    case MPML_ERR_TOO_LARGE: return "size above the fixed scratch capacity";
    default: return "unknown status";
  }
}

int mpml_set_time(mpml_ctx c, double t) {
  if (!c) return MPML_ERR_ARG;
  c->time = t;
  return MPML_OK;
}

int mpml_sync(mpml_ctx c) {
  if (!c) return MPML_ERR_ARG;
  return sync_status(c);
}

int mpml_resample(mpml_ctx c, const mpml_particles* p) {
  if (!c || bad_particles(p)) return MPML_ERR_ARG;
  cudaMemsetAsync(c->status.p, 0, sizeof(int), c->s);
  c->np_count = p->n;
  const void *x = p->x, *v = p->v, *F = p->F, *G = p->G, *m = p->mass, *V = p->volume;
  const int32_t* mat = p->mat;
  int32_t* perm = p->perm;
  const int64_t n = p->n;
  const size_t es = c->esz;
  int rc;
  Buf perm_stage;
  if (p->mem == MPML_MEM_HOST) {
    if ((rc = ensure(c->ux, es * 3 * n)) || (rc = ensure(c->uv, es * 3 * n)) || (rc = ensure(c->uF, es * 9 * n)) ||
        (rc = ensure(c->uG, es * 9 * n)) || (rc = ensure(c->um, es * n)) || (rc = ensure(c->uV, es * n)) ||
        (rc = ensure(c->umat, sizeof(int32_t) * n)))
      return rc;
    cudaMemcpyAsync(c->ux.p, x, es * 3 * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->uv.p, v, es * 3 * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->uF.p, F, es * 9 * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->uG.p, G, es * 9 * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->um.p, m, es * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->uV.p, V, es * n, cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(c->umat.p, mat, sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->s);
    x = c->ux.p; v = c->uv.p; F = c->uF.p; G = c->uG.p; m = c->um.p; V = c->uV.p;
    mat = (const int32_t*)c->umat.p;
    if (perm) {
      if ((rc = ensure(perm_stage, sizeof(int32_t) * n))) return rc;
    }
  }
  int32_t* perm_dev = (p->mem == MPML_MEM_HOST) ? (perm ? (int32_t*)perm_stage.p : nullptr) : perm;
  rc = resample_device(c, x, v, F, G, m, V, mat, perm_dev);
  if (!rc) rc = p2q_q2n(c);
  if (!rc && p->mem == MPML_MEM_HOST && perm)
    cudaMemcpyAsync(perm, perm_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->s);
  if (perm_stage.p) {
    cudaStreamSynchronize(c->s);
    free_buf(perm_stage);
  }
  if (rc) return rc;
  c->stage = 1;
  c->have_lin = 0;
  return MPML_OK;
}

int mpml_stretch(mpml_ctx c) {
  if (!c || c->stage < 1) return MPML_ERR_ARG;
  int rc = stretch_all(c);
  if (rc) return rc;
  rc = sync_status(c);
  if (rc) return rc;
  c->stage = 2;
  return MPML_OK;
}

int mpml_newton_step(mpml_ctx c, const mpml_solver_opts* o, mpml_solve_stats* st) {
  if (!c || c->stage < 1) return MPML_ERR_ARG;
  mpml_solver_opts def = {1e-6, 10000, 1e-6, 0.0, 50, 1e-4, 30, MPML_PRECOND_JACOBI, 16, 2, 0, 0.0};
  if (!o) o = &def;
  if (!(o->cg_forcing >= 0.0 && o->cg_forcing <= 0.5)) return MPML_ERR_ARG;
  mpml_solve_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  int rc = stretch_all(c);
  if (rc) return rc;
  if ((rc = sync_status(c))) return rc;
  rc = newton_solve(c, o, st);
  st->n_particles = c->np_count;
  st->n_bricks = c->nb;
  if (rc < 0) return rc;
  c->have_lin = 1;
  int rc2 = sync_status(c);
  if (rc2) return rc2;
  c->stage = 3;
  return rc;
}

int mpml_resample_batch(mpml_ctx* ctxs, const mpml_particles* parts, int n) {
  if (!ctxs || !parts || n < 1 || n > MPML_BATCH_MAX) return MPML_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || bad_particles(&parts[i]) || parts[i].mem != MPML_MEM_DEVICE) return MPML_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return MPML_ERR_ARG;
  }
  int rc;
  // first halves on every stream, one wait per context, then the second halves
  for (int i = 0; i < n; ++i) {
    mpml_ctx c = ctxs[i];
    cudaMemsetAsync(c->status.p, 0, sizeof(int), c->s);
    c->np_count = parts[i].n;
    if ((rc = resample_device_begin(c, parts[i].x))) return rc;
  }
  for (int i = 0; i < n; ++i)
    if ((rc = cuda_status(cudaStreamSynchronize(ctxs[i]->s)))) return rc;
  for (int i = 0; i < n; ++i) {
    mpml_ctx c = ctxs[i];
    const mpml_particles& p = parts[i];
    if ((rc = resample_device_end(c, p.x, p.v, p.F, p.G, p.mass, p.volume, p.mat, p.perm))) return rc;
    if ((rc = p2q_q2n(c))) return rc;
    c->stage = 1;
    c->have_lin = 0;
  }
  return MPML_OK;
}

int mpml_newton_step_batch(mpml_ctx* ctxs, int n, const mpml_solver_opts* o, mpml_solve_stats* stats) {
  if (!ctxs || n < 1 || n > MPML_BATCH_MAX) return MPML_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    mpml_ctx c = ctxs[i];
    if (!c || c->stage < 1 || c->fp64 || !c->compressed || c->device != ctxs[0]->device) return MPML_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return MPML_ERR_ARG;
  }
  mpml_solver_opts def = {1e-6, 10000, 1e-6, 0.0, 50, 1e-4, 30, MPML_PRECOND_JACOBI, 16, 2, 0, 0.0};
  if (!o) o = &def;
  if (o->plastic_fixed_point) return MPML_ERR_ARG;  // single-scene solver only
  if (!(o->cg_forcing >= 0.0 && o->cg_forcing <= 0.5)) return MPML_ERR_ARG;
  std::vector<mpml_solve_stats> local;
  if (!stats) {
    local.resize(n);
    stats = local.data();
  }
  int rc;
  for (int i = 0; i < n; ++i)
    if ((rc = stretch_all(ctxs[i]))) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = sync_status(ctxs[i]))) return rc;
  rc = newton_batch(ctxs, n, o, stats);
  if (rc < 0) return rc;
  for (int i = 0; i < n; ++i) {
    ctxs[i]->have_lin = 1;
    int rc2 = sync_status(ctxs[i]);
    if (rc2) return rc2;
    ctxs[i]->stage = 3;
  }
  return rc;
}

int mpml_explicit_step(mpml_ctx c) {
  if (!c || c->stage < 1) return MPML_ERR_ARG;
  int rc = explicit_solve(c);
  if (rc) return rc;
  c->stage = 3;
  c->have_lin = 0;
  return MPML_OK;
}

int mpml_g2p(mpml_ctx c, const mpml_particles* p) {
  if (!c || bad_particles(p) || c->stage < 1 || p->n != c->np_count) return MPML_ERR_ARG;
  const int64_t n = p->n;
  const size_t es = c->esz;
  int rc;
  if (p->mem == MPML_MEM_DEVICE) {
    rc = g2p_device(c, p->x, p->v, p->F, p->G, p->mass, p->volume, p->mat);
    if (rc) return rc;
  } else {
    if ((rc = ensure(c->ux, es * 3 * n)) || (rc = ensure(c->uv, es * 3 * n)) || (rc = ensure(c->uF, es * 9 * n)) ||
        (rc = ensure(c->uG, es * 9 * n)) || (rc = ensure(c->um, es * n)) || (rc = ensure(c->uV, es * n)) ||
        (rc = ensure(c->umat, sizeof(int32_t) * n)))
      return rc;
    rc = g2p_device(c, c->ux.p, c->uv.p, c->uF.p, c->uG.p, c->um.p, c->uV.p, (int32_t*)c->umat.p);
    if (rc) return rc;
    cudaMemcpyAsync(p->x, c->ux.p, es * 3 * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->v, c->uv.p, es * 3 * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->F, c->uF.p, es * 9 * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->G, c->uG.p, es * 9 * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->mass, c->um.p, es * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->volume, c->uV.p, es * n, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(p->mat, c->umat.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->s);
    if ((rc = sync_status(c))) return rc;
  }
  c->stage = 4;
  return MPML_OK;
}

int mpml_counts(mpml_ctx c, int64_t out[4]) {
  if (!c || !out) return MPML_ERR_ARG;
  const int64_t ns = c->nb * BV;
  std::vector<uint8_t> cf((size_t)ns), nf((size_t)ns);
  if (ns) {
    cudaMemcpyAsync(cf.data(), c->cflag.p, ns, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(nf.data(), c->nflag.p, ns, cudaMemcpyDeviceToHost, c->s);
  }
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  int64_t ncell = 0, nnode = 0;
  for (int64_t i = 0; i < ns; ++i) {
    ncell += cf[i] ? 1 : 0;
    nnode += (nf[i] & NF_DOF) ? 1 : 0;
  }
  out[0] = c->np_count;
  out[1] = ncell;
  out[2] = nnode;
  out[3] = c->nb;
  return MPML_OK;
}

int mpml_get_keys(mpml_ctx c, int what, int64_t* out) {
  if (!c || !out) return MPML_ERR_ARG;
  if (what == MPML_KEYS_PARTICLES) {
    // compact key -> brick-major key via the brick list
    std::vector<int> k((size_t)c->np_count), bl((size_t)c->nb);
    if (c->np_count) cudaMemcpyAsync(k.data(), c->pkey.p, sizeof(int) * c->np_count, cudaMemcpyDeviceToHost, c->s);
    if (c->nb) cudaMemcpyAsync(bl.data(), c->blist.p, sizeof(int) * c->nb, cudaMemcpyDeviceToHost, c->s);
    int rc = cuda_status(cudaStreamSynchronize(c->s));
    if (rc) return rc;
    for (int64_t i = 0; i < c->np_count; ++i) out[i] = (int64_t)bl[k[i] / BV] * BV + (k[i] % BV);
    return MPML_OK;
  }
  if (what != MPML_KEYS_CELLS && what != MPML_KEYS_NODES) return MPML_ERR_ARG;
  const int64_t ns = c->nb * BV;
  std::vector<uint8_t> f((size_t)ns);
  std::vector<int> bl((size_t)c->nb);
  if (ns) {
    cudaMemcpyAsync(f.data(), what == MPML_KEYS_CELLS ? c->cflag.p : c->nflag.p, ns, cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(bl.data(), c->blist.p, sizeof(int) * c->nb, cudaMemcpyDeviceToHost, c->s);
  }
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  int64_t q = 0;
  const uint8_t mask = what == MPML_KEYS_CELLS ? 1 : NF_DOF;
  for (int64_t b = 0; b < c->nb; ++b)
    for (int l = 0; l < BV; ++l)
      if (f[b * BV + l] & mask) out[q++] = (int64_t)bl[b] * BV + l;
  return MPML_OK;
}

int mpml_get_field(mpml_ctx c, int field, double* out) {
  if (!c || !out || c->stage < 1) return MPML_ERR_ARG;
  return c->fp64 ? get_field_t<double>(c, field, out) : get_field_t<float>(c, field, out);
}

int mpml_set_node_velocity(mpml_ctx c, const double* v) {
  if (!c || !v || c->stage < 1) return MPML_ERR_ARG;
  return import_nodes<double>(c, v, c->nvnew.p);
}

int mpml_eval(mpml_ctx c, const double* v, double* phi, double* grad) {
  if (!c || !v || !phi || c->stage < 2) return MPML_ERR_ARG;
  int rc = node_vector_op<double>(c, 0, v, phi, grad);  // the Newton iterate and gradient are FP64
  if (!rc) c->have_lin = 1;
  return rc;
}

int mpml_linearize(mpml_ctx c, const double* v) {
  if (!c || !v || c->stage < 2) return MPML_ERR_ARG;
  int rc = node_vector_op<double>(c, 1, v, nullptr, nullptr);
  if (!rc) c->have_lin = 1;
  return rc;
}

int mpml_hvp(mpml_ctx c, const double* p, double* y) {
  if (!c || !p || !y || !c->have_lin) return MPML_ERR_ARG;
  return c->fp64 ? node_vector_op<double>(c, 2, p, nullptr, y) : node_vector_op<float>(c, 2, p, nullptr, y);
}

int mpml_set_profiling(mpml_ctx c, int enable) {
  if (!c) return MPML_ERR_ARG;
  int rc = ensure(c->prof, sizeof(DevProf));
  if (rc) return rc;
  DevProf init = {~0ull, 0ull, 0ull, 0, 0};
  cudaMemcpyAsync(c->prof.p, &init, sizeof init, cudaMemcpyHostToDevice, c->s);
  rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  for (int k = 0; k < 2; ++k)
    if (!c->pcg_ev[k] && cudaEventCreate(&c->pcg_ev[k]) != cudaSuccess) return MPML_ERR_CUDA;
  c->pcg_launches = c->pcg_iters = 0;
  c->pcg_ms = 0.0;
  c->profiling = enable ? 1 : 0;
  return MPML_OK;
}

int mpml_pcg_timing(mpml_ctx c, int64_t* launches, int64_t* cg_iters, double* total_ms) {
  if (!c) return MPML_ERR_ARG;
  if (launches) *launches = c->pcg_launches;
  if (cg_iters) *cg_iters = c->pcg_iters;
  if (total_ms) *total_ms = c->pcg_ms;
  return MPML_OK;
}

int mpml_hvp_timing(mpml_ctx c, int64_t* launches, double* total_ms, double* bytes_per_launch) {
  if (!c) return MPML_ERR_ARG;
  DevProf pf = {~0ull, 0ull, 0ull, 0, 0};
  if (c->prof.p) {
    cudaMemcpyAsync(&pf, c->prof.p, sizeof pf, cudaMemcpyDeviceToHost, c->s);
    int rc = cuda_status(cudaStreamSynchronize(c->s));
    if (rc) return rc;
  }
  if (launches) *launches = (int64_t)pf.count;
  if (total_ms) *total_ms = (double)pf.ns * 1e-6;
  if (bytes_per_launch) {
    // per cell brick: K (45/cell) read, p (3/node) read, m read, q (3/node) written
    const double e = (double)c->esz;
    const double kf = c->compressed ? (double)NQC : 45.0;  // tangent numbers per cell
    *bytes_per_launch = (double)c->ncb * BV * (kf * e + 3 * e + e + 3 * e);
  }
  return MPML_OK;
}

int mpml_hvp_bench(mpml_ctx c, int iters, double* mean_ms) {
  if (!c || !mean_ms || !c->have_lin) return MPML_ERR_ARG;
  return hvp_bench(c, iters, mean_ms);
}

int64_t mpml_kernel_launches(mpml_ctx c) { return c ? c->launches : -1; }

int mpml_autotune_hvp(mpml_ctx c, int reps, int* tile, float* ms) {
  if (!c || !c->have_lin || c->fp64) return MPML_ERR_ARG;
  return hvp_autotune(c, reps, tile, ms);
}

int mpml_set_hvp_tile(mpml_ctx c, int tile) {
  if (!c || c->fp64 || tile < -1 || tile >= HVP_TILES) return MPML_ERR_ARG;
  c->hvp_tile = tile;
  c->hvp_tile_fixed = tile >= 0 ? 1 : 0;
  return MPML_OK;
}

int mpml_get_hvp_tile(mpml_ctx c, int* tile, const char** description) {
  if (!c || c->fp64) return MPML_ERR_ARG;
  if (tile) *tile = c->hvp_tile;
  if (description) *description = c->hvp_tile >= 0 ? hvp_tile_name(c->compressed, c->hvp_tile) : "";
  return MPML_OK;
}

int mpml_set_pcg_config(mpml_ctx c, const mpml_pcg_config* cfg) {
  if (!c || !cfg) return MPML_ERR_ARG;
  if (cfg->tangent_staging < MPML_PCG_AUTO || cfg->tangent_staging > MPML_PCG_COLUMNS) return MPML_ERR_ARG;
  if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 4) return MPML_ERR_ARG;
  c->pcg_cfg = *cfg;
  return MPML_OK;
}

int mpml_get_pcg_config(mpml_ctx c, mpml_pcg_config* cfg, int* last_staging, int* last_ctas_per_sm) {
  if (!c || !cfg) return MPML_ERR_ARG;
  *cfg = c->pcg_cfg;
  if (last_staging) *last_staging = c->pcg_last_staging;
  if (last_ctas_per_sm) *last_ctas_per_sm = c->pcg_last_ctas;
  return MPML_OK;
}

int mpml_autotune_pcg(mpml_ctx c, int iters, int reps, int* shape, float* ms) {
  if (!c || c->stage < 2) return MPML_ERR_ARG;
  return pcg_autotune(c, iters, reps, shape, ms);
}

int mpml_lame_parameters(double E, double nu, double* mu, double* lambda) {
  if (!mu || !lambda || !(E > 0) || !(nu > -1.0 && nu < 0.5)) return MPML_ERR_ARG;
  *mu = E / (2.0 * (1.0 + nu));
  *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  return MPML_OK;
}

int mpml_tile_cache_save(const char* path) { return tile_cache_save(path); }
int mpml_tile_cache_load(const char* path) { return tile_cache_load(path); }
void mpml_tile_cache_clear(void) { tile_cache_clear(); }

int mpml_nn_weight_count(void) { return nn_weight_count(); }

int mpml_nn_set_weights(mpml_ctx c, const float* w) {
  if (!c || !w || c->stage < 1) return MPML_ERR_ARG;
  if (c->fp64 || !c->compressed) return MPML_ERR_ARG;  // FP32 single-material contexts
  int rc = nn_set_weights(c, w);
  if (!rc) c->nn_ready = 1;
  return rc;
}

int mpml_nn_get_weights(mpml_ctx c, float* w) {
  if (!c || !w || !c->nn_ready) return MPML_ERR_ARG;
  return nn_get_weights(c, w, 0);
}

int mpml_nn_get_grad(mpml_ctx c, float* g) {
  if (!c || !g || !c->nn_ready) return MPML_ERR_ARG;
  return nn_get_weights(c, g, 1);
}

int mpml_nn_apply(mpml_ctx c, const double* r, double* z) {
  if (!c || !r || !z || !c->nn_ready || !c->have_lin) return MPML_ERR_ARG;
  const int64_t ns = c->nb * BV;
  mpml::Buf rin, zout;
  int rc;
  if ((rc = ensure(rin, sizeof(float) * 3 * (ns ? ns : 1))) || (rc = ensure(zout, sizeof(float) * 3 * (ns ? ns : 1))) ||
      (rc = nn_ensure(c))) {
    free_buf(rin);
    free_buf(zout);
    return rc;
  }
  rc = import_nodes<float>(c, r, rin.p);
  if (!rc) rc = nn_apply_host(c, rin.p, zout.p);
  if (!rc) rc = export_slots<float>(c, zout.p, 3, c->nflag, NF_DOF, z);
  cudaStreamSynchronize(c->s);
  free_buf(rin);
  free_buf(zout);
  return rc;
}

int mpml_nn_adam_step(mpml_ctx c, float lr) {
  if (!c || !c->nn_ready || !(lr > 0.f)) return MPML_ERR_ARG;
  int rc = nn_ensure(c);
  if (rc) return rc;
  nn_adam(c, lr, ++c->nn_adam_step);
  if ((rc = nn_refresh_weights(c))) return rc;
  return cuda_status(cudaStreamSynchronize(c->s));
}

int mpml_nn_loss_grad(mpml_ctx c, const double* r, const double* e, double* loss) {
  if (!c || !r || !e || !loss || !c->nn_ready || !c->have_lin) return MPML_ERR_ARG;
  const int64_t ns = c->nb * BV;
  mpml::Buf rin, ein;
  int rc;
  if ((rc = ensure(rin, sizeof(float) * 3 * (ns ? ns : 1))) || (rc = ensure(ein, sizeof(float) * 3 * (ns ? ns : 1))) ||
      (rc = nn_ensure(c))) {
    free_buf(rin);
    free_buf(ein);
    return rc;
  }
  rc = import_nodes<float>(c, r, rin.p);
  if (!rc) rc = import_nodes<float>(c, e, ein.p);
  if (!rc) {
    // zero the gradient accumulator (it follows the master weights)
    cudaMemsetAsync((float*)c->nnw.p + 3 * 27 * 256, 0, sizeof(float) * 3 * 27 * 256, c->s);
    rc = nn_loss_grad_host(c, rin.p, ein.p, loss);
  }
  cudaStreamSynchronize(c->s);
  free_buf(rin);
  free_buf(ein);
  return rc;
}

int mpml_nn_train(mpml_ctx c, const mpml_train_opts* o, mpml_train_stats* st) {
  if (!c || !o || c->stage < 1 || !c->nn_ready) return MPML_ERR_ARG;
  if (o->samples < 1 || o->epochs < 0 || o->batch < 1 || !(o->lr >= 0)) return MPML_ERR_ARG;
  int rc = nn_collect(c, o->samples, o->rtol, o->cg_max);
  if (rc) return rc;
  double l0 = 0, l1 = 0;
  rc = nn_train(c, o->epochs, o->batch, o->lr, &l0, &l1);
  if (rc) return rc;
  c->have_lin = 1;
  if (st) {
    st->samples = c->nn_nsamples;
    st->loss_first = l0;
    st->loss_last = l1;
  }
  return sync_status(c);
}

}  // extern "C"
