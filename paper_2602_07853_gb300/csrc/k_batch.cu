// Batched implicit solve: the Newton iterations of many independent scenes
// (one library context each, FP32 single-material, on one device; each on its
// own stream or a shared one) run in lockstep, and every round of their
// Jacobi-PCG solves is ONE persistent cooperative launch over the union of the
// scenes' bricks.  The per-scene kernels (prep, energy, update) stay on each
// context's stream, so scenes on different streams overlap; events order
// them against the shared launch, which runs on the first context's stream.
//
// Each scene keeps its own scalars (alpha, beta, r.z, tolerance, iteration
// count, convergence flag): a CTA looks the scene up per work item (cell brick,
// node-only brick, node brick), the per-scene sums of every phase are added
// atomically into per-scene FP64 accumulators, and after each bounded grid
// barrier every CTA updates the scalars of all scenes identically.  Scenes that
// converged skip their bricks; the launch ends when every scene has.  The
// Newton logic per scene (convergence test, Armijo line search, update) is the
// one of mpml_newton_step, evaluated for all active scenes with one host
// synchronisation per stage instead of one per scene.
#include <algorithm>
#include <vector>

#include "mpml_internal.cuh"

namespace mpml {

// pieces of the single-scene solver (k_newton.cu)
int batch_alloc_solver(mpml_ctx_s* c);
int batch_prep(mpml_ctx_s* c, double cg_rtol, int cg_max);
void batch_slope_launch(mpml_ctx_s* c);
void batch_energy_launch(mpml_ctx_s* c, double alpha);
void batch_axpy_launch(mpml_ctx_s* c, double alpha);
int batch_trial_launch(mpml_ctx_s* c, double cg_rtol, int cg_max);
void batch_trial_revert(mpml_ctx_s* c);
int batch_cg_start(mpml_ctx_s* c, double cg_rtol, int cg_max);

struct BScene {
  const int* cblist;
  const int* nolist;
  const int* nbr;
  const uint8_t* cflag;
  const float* C;
  const float* m;
  const float* dinv;
  float* x;
  float* r;
  float* pa;
  float* pb;
  float* q;
  DevScalars* sc;
  int ncb, nnob, nb, pad;
};

constexpr int BATCH_MAX = MPML_BATCH_MAX;
// dynamic shared memory: the 9^3 p halo of a brick and the column walk's
// exchange buffers (the compressed tangent is streamed from global memory)
constexpr size_t BC_SMEM = sizeof(float) * (3 * 729 + HVP_X_FLOATS + HVP_R_FLOATS);

// warp sum of FP32 values in float-float arithmetic (error-free two-sum at every
// level, the rounding errors carried in lo); FP64 only where lane 0 converts the pair
__device__ __forceinline__ void bwarp_sum_ff(float v, float& hi_out, float& lo_out) {
  float hi = v, lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_down_sync(0xffffffffu, hi, o), bl = __shfl_down_sync(0xffffffffu, lo, o);
    const float s = hi + bh;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (bh - bp);
    lo = lo + bl + e;
    hi = s;
  }
  hi_out = hi;
  lo_out = lo;
}

// block sums of (a, b) added atomically to acc[0..1] (thread 0); FP64 only on
// lane 0 and thread 0 (FP64 instructions are slow on this part)
__device__ __forceinline__ void bblock_atomic2(float a_, float b_, double* acc) {
  __shared__ double red[2][32];
  float ah, al, bh, bl;
  bwarp_sum_ff(a_, ah, al);
  bwarp_sum_ff(b_, bh, bl);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = (double)ah + (double)al;
    red[1][wid] = (double)bh + (double)bl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    if (sa != 0.0) atomicAdd(acc, sa);
    if (sb != 0.0) atomicAdd(acc + 1, sb);
  }
  __syncthreads();
}

struct BatchArgs {
  const BScene* scenes;
  const int2* cw;  // (scene, cell brick index) work items
  const int2* nw;  // (scene, node-only brick index)
  const int2* aw;  // (scene, brick) for the vector update
  int ncw, nnw, naw, nsc;
  double* acc;     // [4][nsc][2] rotating per-scene accumulators
  unsigned* gbar;
  int cg_max;
  unsigned spins;  // bound on the polls of one grid-barrier wait
  int* status;
};

__global__ void __launch_bounds__(256, 2) k_pcg_batch(BatchArgs A) {
  extern __shared__ __align__(128) unsigned char psm[];
  float (*sv)[729] = reinterpret_cast<float (*)[729]>(psm);
  float* Xs = reinterpret_cast<float*>(psm + sizeof(float) * 3 * 729);
  __shared__ int s_nbr[NBR];
  __shared__ int s_flag, s_alldone;
  __shared__ double s_rz[BATCH_MAX], s_tol2[BATCH_MAX], s_rr[BATCH_MAX];
  __shared__ float s_alpha[BATCH_MAX], s_beta[BATCH_MAX];
  __shared__ int s_done[BATCH_MAX], s_it[BATCH_MAX];
  __shared__ unsigned char s_flip[BATCH_MAX];  // p ping-pong parity per scene
  const int S = A.nsc, G = gridDim.x;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const DevScalars* d = A.scenes[s].sc;
    s_rz[s] = d->rz;
    s_tol2[s] = d->tol2;
    s_rr[s] = d->rr_last;
    s_done[s] = d->done;
    s_it[s] = 0;
    s_alpha[s] = 0.f;
    s_beta[s] = 0.f;
    s_flip[s] = 0;
  }
  __syncthreads();
  bool alive = true;
  int round = 0;
  while (alive) {
    if (threadIdx.x == 0) {
      int all = 1;
      for (int s = 0; s < S; ++s) all &= s_done[s];
      s_alldone = all;
    }
    __syncthreads();
    if (s_alldone) break;
    double* accH = A.acc + (size_t)2 * S * ((2 * round) & 3);
    double* accA = A.acc + (size_t)2 * S * ((2 * round + 1) & 3);
    if (blockIdx.x == 0) {  // slot of phase 2 round + 2, last read two barriers ago
      double* z = A.acc + (size_t)2 * S * ((2 * round + 2) & 3);
      for (int i = threadIdx.x; i < 2 * S; i += blockDim.x) z[i] = 0.0;
    }
    // ---------------- phase H: p update (staged) and HVP ----------------
    for (int w = blockIdx.x; w < A.ncw; w += G) {
      const int2 item = A.cw[w];
      const int s = item.x;
      if (s_done[s]) continue;
      const BScene& B = A.scenes[s];
      const float beta = s_beta[s];
      const float* pold = s_flip[s] ? B.pb : B.pa;
      float* pnext = s_flip[s] ? B.pa : B.pb;
      const int id = B.cblist[item.y];
      if (threadIdx.x < NBR) s_nbr[threadIdx.x] = B.nbr[id * NBR + threadIdx.x];
      __syncthreads();
      float pmp = 0.f;
      {
        // every thread owns at most 3 of the 729 halo slots: issue all loads first
        int tt[3], ll[3];
        float dv[3][3], rv[3][3], pv[3][3], mv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i = threadIdx.x + k * 256;
          tt[k] = -1;
          ll[k] = 0;
          mv[k] = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a) dv[k][a] = rv[k][a] = pv[k][a] = 0.f;
          if (i < 729) {
            const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
            const int t = (nx < 8 && ny < 8 && nz < 8) ? id : s_nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
            const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
            tt[k] = t;
            ll[k] = l;
            if (t >= 0) {
              const int64_t o = (int64_t)t * 3 * BV + l;
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                dv[k][a] = __ldcg(B.dinv + o + a * BV);
                rv[k][a] = __ldcg(B.r + o + a * BV);
                pv[k][a] = __ldcg(pold + o + a * BV);
              }
              if (t == id) mv[k] = __ldcg(B.m + (int64_t)id * BV + l);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i = threadIdx.x + k * 256;
          if (i >= 729) continue;
          float v[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) v[a] = dv[k][a] > 0.f ? dv[k][a] * rv[k][a] + beta * pv[k][a] : 0.f;
          if (tt[k] == id) {
            const int64_t o = (int64_t)id * 3 * BV + ll[k];
            pnext[o] = v[0];
            pnext[o + BV] = v[1];
            pnext[o + 2 * BV] = v[2];
            pmp += mv[k] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          }
          sv[0][i] = v[0];
          sv[1][i] = v[1];
          sv[2][i] = v[2];
        }
      }
      __syncthreads();
      // the column walk of the single-scene persistent solver, tangent rows streamed
      const float pkp = phase_h_col<false, true>(id, s_nbr, sv, B.C + (int64_t)id * NQC * BV, B.cflag, B.m, B.q, Xs,
                                                 Xs + HVP_X_FLOATS, true);
      bblock_atomic2(pmp, pkp, accH + 2 * s);  // ends with a barrier: sv / s_nbr / exchange buffers free
    }
    // node-only bricks: p_new and the mass term, dealt from the last CTA down (the
    // CTAs with the fewest cell work items)
    for (int w = G - 1 - (int)blockIdx.x; w < A.nnw; w += G) {
      const int2 item = A.nw[w];
      const int s = item.x;
      if (s_done[s]) continue;
      const BScene& B = A.scenes[s];
      const float beta = s_beta[s];
      const float* pold = s_flip[s] ? B.pb : B.pa;
      float* pnext = s_flip[s] ? B.pa : B.pb;
      const int id = B.nolist[item.y];
      float pmp = 0.f;
      for (int l = threadIdx.x; l < BV; l += blockDim.x) {
        const int64_t o = (int64_t)id * 3 * BV + l;
        const float mi = B.m[(int64_t)id * BV + l];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float di = B.dinv[o + a * BV];
          const float v = di > 0.f ? di * B.r[o + a * BV] + beta * pold[o + a * BV] : 0.f;
          pnext[o + a * BV] = v;
          pmp += mi * v * v;
          if (v != 0.f) atomicAdd(B.q + o + a * BV, mi * v);
        }
      }
      bblock_atomic2(pmp, 0.f, accH + 2 * s);
    }
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      if (s_done[s]) continue;
      const double pq = __ldcg(accH + 2 * s) + __ldcg(accH + 2 * s + 1);
      if (!(pq > 0.0)) {
        s_done[s] = 1;  // breakdown: keep the current iterate
        s_alpha[s] = 0.f;
      } else {
        s_alpha[s] = (float)(s_rz[s] / pq);
      }
    }
    __syncthreads();
    // ---------------- phase A: x, r update and the new dots ----------------
    // slot of phase 2 round + 3 was last read before the barrier just passed
    if (blockIdx.x == 0) {
      double* z = A.acc + (size_t)2 * S * ((2 * round + 3) & 3);
      for (int i = threadIdx.x; i < 2 * S; i += blockDim.x) z[i] = 0.0;
    }
    for (int w = blockIdx.x; w < A.naw; w += G) {
      const int2 item = A.aw[w];
      const int s = item.x;
      if (s_done[s]) continue;
      const BScene& B = A.scenes[s];
      const float alpha = s_alpha[s];
      const float* pn = s_flip[s] ? B.pa : B.pb;
      float rzl = 0.f, rrl = 0.f;
      for (int l = threadIdx.x; l < BV; l += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int64_t o = ((int64_t)item.y * 3 + a) * BV + l;
          const float d = __ldcg(B.dinv + o);
          float x = __ldcg(B.x + o), r = __ldcg(B.r + o);
          if (d > 0.f) {
            x += alpha * __ldcg(pn + o);
            r -= alpha * __ldcg(B.q + o);
            rzl += r * d * r;
            rrl += r * r;
          }
          B.x[o] = x;
          B.r[o] = r;
          B.q[o] = 0.f;
        }
      }
      bblock_atomic2(rzl, rrl, accA + 2 * s);
    }
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      if (s_done[s]) continue;
      const double rzn = __ldcg(accA + 2 * s), rrn = __ldcg(accA + 2 * s + 1);
      const int it = ++s_it[s];
      s_rr[s] = rrn;
      if (rrn <= s_tol2[s] || it >= A.cg_max || !(rrn == rrn)) s_done[s] = 1;
      s_beta[s] = (float)(rzn / s_rz[s]);
      s_rz[s] = rzn;
      s_flip[s] ^= 1;
    }
    __syncthreads();
    ++round;
  }
  if (!alive && threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
  if (blockIdx.x == 0)
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      DevScalars* d = A.scenes[s].sc;
      d->iters = s_it[s];
      d->rr_last = s_rr[s];
      d->rz = s_rz[s];
      d->done = 1;
    }
}

namespace {

// the scalars and status of every context, each copied on its own stream,
// then one wait per distinct stream
int read_all(const std::vector<mpml_ctx_s*>& cs) {
  std::vector<cudaStream_t> streams;
  for (mpml_ctx_s* c : cs) {
    cudaMemcpyAsync(c->hscal, c->scal.p, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(c->hstatus, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (std::find(streams.begin(), streams.end(), c->s) == streams.end()) streams.push_back(c->s);
  }
  for (cudaStream_t s : streams) {
    const int rc = cuda_status(cudaStreamSynchronize(s));
    if (rc) return rc;
  }
  return MPML_OK;
}

int ensure_event(mpml_ctx_s* c) {
  if (c->bev) return MPML_OK;
  if (cudaEventCreateWithFlags(&c->bev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return MPML_ERR_CUDA;
  }
  return MPML_OK;
}

int pcg_batch(mpml_ctx_s* owner, const std::vector<mpml_ctx_s*>& cs, int cg_max) {
  // CTAs per SM: the first context's mpml_pcg_config, else as many as fit
  int nsm = 0;
  const int fit = launch_fit((const void*)k_pcg_batch, 256, BC_SMEM, LS_BATCH, &nsm);
  if (fit <= 0) return MPML_ERR_CUDA;
  const int per_sm = owner->pcg_cfg.ctas_per_sm > 0 ? owner->pcg_cfg.ctas_per_sm : fit;
  if (per_sm > fit) return MPML_ERR_ARG;
  const int max_blocks = per_sm * nsm;
  const int S = (int)cs.size();
  std::vector<BScene> sc(S);
  std::vector<int2> cw, nw, aw;
  for (int i = 0; i < S; ++i) {
    mpml_ctx_s* c = cs[i];
    BScene& b = sc[i];
    b.cblist = (const int*)c->cblist.p;
    b.nolist = (const int*)c->nolist.p;
    b.nbr = (const int*)c->nbr.p;
    b.cflag = (const uint8_t*)c->cflag.p;
    b.C = (const float*)c->cK.p;
    b.m = (const float*)c->nmass.p;
    b.dinv = (const float*)c->ndinv.p;
    b.x = (float*)c->nx.p;
    b.r = (float*)c->nr.p;
    b.pa = (float*)c->np.p;
    b.pb = (float*)c->np2.p;
    b.q = (float*)c->nq.p;
    b.sc = (DevScalars*)c->scal.p;
    b.ncb = (int)c->ncb;
    b.nnob = (int)c->nnob;
    b.nb = (int)c->nb;
    b.pad = 0;
    for (int j = 0; j < (int)c->ncb; ++j) cw.push_back(make_int2(i, j));
    for (int j = 0; j < (int)c->nnob; ++j) nw.push_back(make_int2(i, j));
    for (int j = 0; j < (int)c->nb; ++j) aw.push_back(make_int2(i, j));
  }
  // interleave the scenes' cell bricks so that uneven scenes spread over all CTAs
  std::stable_sort(cw.begin(), cw.end(), [&](const int2& a, const int2& b) { return a.y < b.y; });
  const size_t bytes_sc = sizeof(BScene) * S, bytes_w = sizeof(int2) * (cw.size() + nw.size() + aw.size());
  const size_t acc_bytes = sizeof(double) * 8 * S;
  const size_t off_w = (bytes_sc + 255) & ~size_t(255);
  const size_t off_acc = (off_w + bytes_w + 255) & ~size_t(255);
  const size_t off_bar = off_acc + acc_bytes;
  int rc;
  if ((rc = ensure(owner->bbatch, off_bar + 16))) return rc;
  char* base = (char*)owner->bbatch.p;
  std::vector<char> host(off_acc);
  memcpy(host.data(), sc.data(), bytes_sc);
  int2* hw = reinterpret_cast<int2*>(host.data() + off_w);
  std::copy(cw.begin(), cw.end(), hw);
  std::copy(nw.begin(), nw.end(), hw + cw.size());
  std::copy(aw.begin(), aw.end(), hw + cw.size() + nw.size());
  cudaStream_t s = owner->s;
  // the shared launch runs on the first context's stream after every scene's prep
  if ((rc = ensure_event(owner))) return rc;
  for (mpml_ctx_s* c : cs) {
    if (c->s == s) continue;
    if ((rc = ensure_event(c))) return rc;
    cudaEventRecord(c->bev, c->s);
    cudaStreamWaitEvent(s, c->bev, 0);
  }
  cudaMemcpyAsync(base, host.data(), off_acc, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(base + off_acc, 0, acc_bytes + 16, s);
  for (mpml_ctx_s* c : cs) {
    // q starts at zero (phase A zeroes it after each use)
    cudaMemsetAsync(c->nq.p, 0, sizeof(float) * 3 * c->nb * BV, s);
  }
  BatchArgs a;
  a.scenes = reinterpret_cast<const BScene*>(base);
  a.cw = reinterpret_cast<const int2*>(base + off_w);
  a.nw = a.cw + cw.size();
  a.aw = a.nw + nw.size();
  a.ncw = (int)cw.size();
  a.nnw = (int)nw.size();
  a.naw = (int)aw.size();
  a.nsc = S;
  a.acc = reinterpret_cast<double*>(base + off_acc);
  a.gbar = reinterpret_cast<unsigned*>(base + off_bar);
  a.cg_max = cg_max;
  a.spins = owner->pcg_cfg.barrier_spins ? owner->pcg_cfg.barrier_spins : BARRIER_SPINS_DEFAULT;
  a.status = (int*)owner->status.p;
  void* args[] = {&a};
  // with profiling enabled on the first context: CUDA events around the launch (mpml_pcg_timing)
  const bool timed = owner->profiling && owner->pcg_ev[0] && owner->pcg_ev[1];
  if (timed) cudaEventRecord(owner->pcg_ev[0], s);
  rc = cuda_status(cudaLaunchCooperativeKernel((const void*)k_pcg_batch, dim3(max_blocks), dim3(256), args, BC_SMEM, s));
  if (timed) cudaEventRecord(owner->pcg_ev[1], s);
  owner->launches++;
  owner->pcg_last_ctas = per_sm;
  if (rc) return rc;
  // every scene's stream continues after the shared launch
  cudaEventRecord(owner->bev, s);
  for (mpml_ctx_s* c : cs)
    if (c->s != s) cudaStreamWaitEvent(c->s, owner->bev, 0);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int newton_batch(mpml_ctx_s** ctxs, int n, const mpml_solver_opts* o, mpml_solve_stats* st) {
  int rc;
  std::vector<mpml_ctx_s*> all(ctxs, ctxs + n);
  std::vector<int> it(n, 0), status(n, MPML_OK), active(n, 0);
  std::vector<double> g0(n, 0.0), gn(n, 0.0), phi(n, 0.0), phi_el(n, 0.0), gfloor(n, 0.0);
  std::vector<double> gprev(n, 0.0), eta(n, 0.0);  // inexact Newton (opts.cg_forcing > 0)
  mpml_ctx_s* owner = ctxs[0];
  std::vector<mpml_ctx_s*> work;
  for (int i = 0; i < n; ++i) {
    memset(&st[i], 0, sizeof(mpml_solve_stats));
    mpml_ctx_s* c = ctxs[i];
    st[i].n_particles = c->np_count;
    st[i].n_bricks = c->nb;
    if ((rc = batch_alloc_solver(c))) return rc;
    if (c->nb == 0) continue;
    if ((rc = batch_prep(c, o->cg_rtol, o->cg_max))) return rc;
    work.push_back(c);
    active[i] = 1;
  }
  if ((rc = read_all(work))) return rc;
  for (int i = 0; i < n; ++i) {
    if (!active[i]) continue;
    mpml_ctx_s* c = ctxs[i];
    if (*c->hstatus & ST_NONFINITE) return MPML_ERR_NONFINITE;
    g0[i] = gn[i] = sqrt(c->hscal->gg);
    gfloor[i] = 1e-12 * sqrt(c->hscal->mv2);
    phi[i] = c->hscal->phi_in + c->hscal->phi_el;
    phi_el[i] = c->hscal->phi_el;
    st[i].g0_norm = g0[i];
    st[i].phi0 = phi[i];
  }
  while (true) {
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      if (gn[i] <= o->newton_rtol * g0[i] || gn[i] <= o->newton_atol || gn[i] <= gfloor[i]) {
        active[i] = 0;
        continue;
      }
      if (it[i] >= o->newton_max) {
        status[i] = MPML_WARN_NOT_CONVERGED;
        active[i] = 0;
        continue;
      }
      idx.push_back(i);
    }
    if (idx.empty()) break;
    std::vector<mpml_ctx_s*> cs;
    for (int i : idx) cs.push_back(ctxs[i]);
    if (o->cg_forcing > 0.0) {
      // each scene's solve stops at its own forcing term (written on the launch's stream)
      for (int i : idx) {
        eta[i] = newton_forcing(o, it[i], gn[i], gprev[i], eta[i], fmax(o->newton_rtol * g0[i], o->newton_atol));
        gprev[i] = gn[i];
        if ((rc = set_cg_tol2(ctxs[i], owner->s, eta[i] * eta[i] * gn[i] * gn[i]))) return rc;
      }
    }
    // one cooperative launch for every active scene's Jacobi-PCG solve
    if ((rc = pcg_batch(owner, cs, o->cg_max))) return rc;
    if ((rc = read_all(cs))) return rc;
    if (owner->profiling && owner->pcg_ev[0] && owner->pcg_ev[1]) {
      // the launch's time, and as its CG iterations the largest count of its scenes
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, owner->pcg_ev[0], owner->pcg_ev[1]) == cudaSuccess) {
        int mx = 0;
        for (mpml_ctx_s* c : cs) mx = std::max(mx, c->hscal->iters);
        owner->pcg_ms += ms;
        owner->pcg_launches += 1;
        owner->pcg_iters += mx;
      } else {
        cudaGetLastError();
      }
    }
    for (int i : idx) {
      mpml_ctx_s* c = ctxs[i];
      const int k = it[i];
      const double rr0 = c->hscal->rr0;
      if (k < 64) {
        st[i].cg_iters[k] = c->hscal->iters;
        st[i].cg_rel_resid[k] = rr0 > 0 ? sqrt(c->hscal->rr_last / rr0) : 0.0;
      }
      st[i].cg_iters_total += c->hscal->iters;
      batch_slope_launch(c);
    }
    if ((rc = read_all(cs))) return rc;
    std::vector<double> slope(n), lsA(n), lsB(n), alpha(n, 1.0), phit_el(n, 0.0);
    std::vector<int> accepted(n, 0), lin(n, 0);
    for (int i : idx) {
      slope[i] = ctxs[i]->hscal->slope;
      lsA[i] = ctxs[i]->hscal->ls_a;
      lsB[i] = ctxs[i]->hscal->ls_b;
    }
    // the full step first, by each scene's prep at its trial iterate (as the single-scene
    // solver): accepted, it is the next round's linearisation (CG start added); rejected,
    // the scene goes back to v and halves from 1/2 with the line-search energy
    for (int i : idx)
      if ((rc = batch_trial_launch(ctxs[i], o->cg_rtol, o->cg_max))) return rc;
    if ((rc = read_all(cs))) return rc;
    for (int i : idx) {
      const mpml_ctx_s* c = ctxs[i];
      const double pel = c->hscal->phi_el, gg = c->hscal->gg;
      const double dphi = lsA[i] + 0.5 * lsB[i] + (pel - phi_el[i]);
      if (c->hscal->infeasible == 0 && dphi <= o->ls_c1 * slope[i] && gg == gg) {
        accepted[i] = lin[i] = 1;
        if ((rc = batch_cg_start(ctxs[i], o->cg_rtol, o->cg_max))) return rc;
      } else {
        batch_trial_revert(ctxs[i]);
        alpha[i] = 0.5;
      }
    }
    for (int ls = 1; ls <= o->ls_max; ++ls) {
      std::vector<mpml_ctx_s*> pend;
      std::vector<int> pidx;
      for (int i : idx)
        if (!accepted[i]) {
          batch_energy_launch(ctxs[i], alpha[i]);
          pend.push_back(ctxs[i]);
          pidx.push_back(i);
        }
      if (pend.empty()) break;
      if ((rc = read_all(pend))) return rc;
      for (int i : pidx) {
        const mpml_ctx_s* c = ctxs[i];
        // Armijo on the energy change (inertia part in closed form, elastic part as a
        // difference of elastic sums), as in the single-scene solver
        phit_el[i] = c->hscal->phi_el;
        const double dphi = alpha[i] * lsA[i] + 0.5 * alpha[i] * alpha[i] * lsB[i] + (phit_el[i] - phi_el[i]);
        if (c->hscal->infeasible == 0 && dphi <= o->ls_c1 * alpha[i] * slope[i])
          accepted[i] = 1;
        else
          alpha[i] *= 0.5;
      }
    }
    std::vector<mpml_ctx_s*> upd;
    for (int i : idx) {
      const int k = it[i]++;
      if (k < 64) st[i].alpha[k] = accepted[i] ? alpha[i] : 0.0;
      if (!accepted[i]) {
        status[i] = MPML_WARN_NOT_CONVERGED;
        active[i] = 0;
        continue;
      }
      if (lin[i]) {  // linearised at the trial iterate already
        upd.push_back(ctxs[i]);
        continue;
      }
      batch_axpy_launch(ctxs[i], alpha[i]);
      if ((rc = batch_prep(ctxs[i], o->cg_rtol, o->cg_max))) return rc;
      upd.push_back(ctxs[i]);
    }
    if ((rc = read_all(upd))) return rc;
    for (int i : idx) {
      if (!active[i]) continue;
      const mpml_ctx_s* c = ctxs[i];
      gn[i] = sqrt(c->hscal->gg);
      phi[i] = c->hscal->phi_in + c->hscal->phi_el;
      phi_el[i] = c->hscal->phi_el;
    }
  }
  int worst = MPML_OK;
  for (int i = 0; i < n; ++i) {
    st[i].newton_iters = it[i];
    st[i].g_norm = gn[i];
    st[i].phi = phi[i];
    st[i].status = status[i];
    if (status[i] != MPML_OK) worst = status[i];
  }
  // device-side errors (timeouts, non-finite values) latched in any context
  for (int i = 0; i < n; ++i) {
    const int sw = *ctxs[i]->hstatus | *owner->hstatus;
    if (sw & ST_TIMEOUT) return MPML_ERR_TIMEOUT;
    if (sw & ST_NONFINITE) return MPML_ERR_NONFINITE;
  }
  return worst;
}

}  // namespace mpml
