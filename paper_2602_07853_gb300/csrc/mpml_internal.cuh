// Internal declarations of the sm_103a MPM Lite library: the context, the
// brick layout, device status bits, and the per-cell constitutive math
// shared by the kernels (stretch reconstruction, Newton prep, line search).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mpml.h"

namespace mpml {

// ---------------------------------------------------------------------------
// Brick layout: 8x8x8 cells (or nodes) per brick, brick-major keys.
// Cell data is stored per brick as [brick][field][512] so that the 512
// threads of a brick read each field coalesced; node vectors as
// [brick][component][512].
// ---------------------------------------------------------------------------
constexpr int BR = 8;
constexpr int BV = 512;
constexpr int NBR = 27;  // neighbour table entries per brick (offsets -1..1)

__host__ __device__ inline int nbr_index(int dx, int dy, int dz) {
  return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}

// device status bits (latched, OR-ed)
enum : int {
  ST_OUT_OF_DOMAIN = 1,
  ST_NONFINITE = 2,
  ST_STRETCH = 4,
  ST_TIMEOUT = 8,
  ST_BADMAT = 16,
};

// node flags
enum : uint8_t { NF_DOF = 1, NF_FIXED = 2 };

// Per-cell accumulators of the unload (Algorithm 2), per brick-field plane:
//   0: m   1-3: m v   4-12: m G   then per material k: V_k, (V tau)_k (6 sym)
__host__ __device__ inline int acc_fields(int nm) { return 13 + 7 * nm; }
__host__ __device__ inline int acc_V(int k) { return 13 + 7 * k; }
__host__ __device__ inline int acc_tau(int k) { return 14 + 7 * k; }

// symmetric 3x3 packing: xx yy zz xy xz yz
__host__ __device__ inline int sym_idx(int a, int b) {
  if (a == b) return a;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// symmetric 9x9 packed upper triangle, row-major: index of (r, c), r <= c
__host__ __device__ inline int k45(int r, int c) { return r * 9 - r * (r - 1) / 2 + (c - r); }

// Device-side solver scalars (one struct per context, in device memory).
struct DevScalars {
  double pMp;      // sum m |p|^2 of the current direction (update kernel)
  double pKp;      // sum_c D^T K D (HVP kernel)
  double rz;       // r^T z
  double rz_new;
  double rr;       // r^T r
  double rr0;
  double alpha, beta;
  double gg;       // |g|^2
  double phi_el;   // elastic energy sum
  double phi_in;   // inertia sum
  double slope;    // g^T dx
  double ls_a;     // sum m (v - vhat) . dx over DOF nodes (line search, inertia)
  double ls_b;     // sum m |dx|^2 over DOF nodes
  double tol2;     // (cg_rtol)^2 rr0
  double rr_last;  // r^T r at the last CG update
  double pq;       // p^T H p of the current direction
  double nn_s;     // RMS of D^-1/2 r (network input scale)
  double nn_a, nn_b;  // training: z^T r and z^T H z of the current pair
  double mv2;      // sum over free DOFs of (m vhat)^2 (Newton's rounding floor)
  double nfree;    // number of free DOF components
  double rzj;      // r^T D^-1 r (Jacobi) of the current residual
  double rr_ring[32];  // r^T r history (stall test of flexible CG)
  int fallback;    // flexible CG stalled: continue with Jacobi-PCG
  int infeasible;  // cells where the energy is undefined (line search)
  int done;
  int iters;
  int cg_max;
  int bodies;      // executed bodies of the graph-driven CG loop
  int nproj;       // fixed-point plasticity: slots whose base a projection changed
  int counter[8];  // last-block tickets per kernel kind
  int pad;
};

// Device-side launch timing of the HVP (globaltimer ns), enabled by profiling.
struct DevProf {
  unsigned long long t0;     // earliest block start of the running launch
  unsigned long long ns;     // accumulated launch durations
  unsigned long long count;  // timed launches
  int counter;               // last-block ticket
  int pad;
};

template <typename T>
struct MatParams {
  int model;
  T mu, lam;
};

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace mpml

struct mpml_ctx_s {
  mpml_scene_desc d;
  mpml_material mats[MPML_MAX_MATS];
  int nm = 1;
  cudaStream_t s = nullptr;
  int fp64 = 0;
  int compressed = 0;  // FP32, single material: HVP on the compressed (NQC-number) tangent
  // launch shape ("tile") of the standalone FP32 HVP, an index into the table of
  // hvp_tile_name(); -1: chosen by the autotuner (or its cache) at the first solve
  int hvp_tile = -1;
  int hvp_tile_fixed = 0;  // set by mpml_set_hvp_tile: never re-tuned
  mpml::Buf tuneq;         // scratch output of the autotuner's timed launches
  // fixed-point plastic solve: general bases B - I of every slot (9 numbers), used
  // by the energy / gradient / tangent kernels while fp_active is set
  mpml::Buf cB;
  int fp_active = 0;
  size_t esz = 4;
  int NB[3] = {0, 0, 0};
  int64_t NBT = 0;
  double time = 0;
  int device = 0;

  // brick bookkeeping
  mpml::Buf bflag_c, bflag_n, bmap, blist, cblist, nolist, nbr;
  // particles (sorted library copies and temporaries)
  mpml::Buf px, pv, pF, pG, pm, pV, pmat, pperm, pkey, prank, pbase;
  // staging of unsorted input (host mode)
  mpml::Buf ux, uv, uF, uG, um, uV, umat;
  // counting sort
  mpml::Buf cnt, start, scan_tmp;
  // cells
  mpml::Buf cflag, cacc, cs, cK, cnew;
  // nodes
  mpml::Buf nflag, nmass, nv, nvhat, nvfix, nvnew, ng, ndinv, nx, nr, np, np2, nq;
  mpml::Buf nvtry;  // the line search's trial iterate v + x (swapped with nvnew when accepted)
  // scalars and status
  mpml::Buf scal, status, prof, part, gbar;
  mpml::Buf bbatch;  // batched solver: scene table, work lists, accumulators (first context of a batch)
  cudaEvent_t bev = nullptr;  // batched solver: orders this context's stream against the shared launch
  // learned preconditioner: weights/grads/Adam + bf16 copies, activations,
  // network output, wgrad partials, z, training samples
  mpml::Buf nnw, nnact, nny, nnpart, nz, nns_r, nns_e, nnhd;
  int nn_ready = 0;        // weights set
  int nn_nsamples = 0;     // stored training pairs
  int nn_adam_step = 0;
  int last_fcg_fallback = 0;  // the last learned solve fell back to Jacobi-PCG
  mpml::DevScalars* hscal = nullptr;  // pinned mirror
  int* hstatus = nullptr;             // pinned

  int64_t np_count = 0, nb = 0, ncb = 0, nnob = 0;  // bricks: all, with cells, node-only
  int stage = 0;  // 0 nothing, 1 unloaded, 2 stretched, 3 solved, 4 loaded
  int have_lin = 0;

  // graph-driven CG loop (conditional WHILE node), rebuilt when its key changes
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  uintptr_t cg_key[17] = {};

  // profiling of HVP launches
  int profiling = 0;
  int64_t launches = 0;
  // CUDA-event timing of the persistent PCG kernel (profiling): launches,
  // their CG iterations and total milliseconds
  cudaEvent_t pcg_ev[2] = {nullptr, nullptr};
  int64_t pcg_launches = 0, pcg_iters = 0;
  double pcg_ms = 0.0;
  // persistent-solver launch controls (mpml_set_pcg_config) and the shape the
  // last launch used (staging 1 = shared-memory block, 2 = streamed rows)
  mpml_pcg_config pcg_cfg = {0, 0, 0u};
  int pcg_last_staging = 0, pcg_last_ctas = 0;
};

namespace mpml {

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
int ensure(Buf& b, size_t bytes);
void free_buf(Buf& b);
int cuda_status(cudaError_t e);

int resample_device(mpml_ctx_s* c, const void* x, const void* v, const void* F, const void* G,
                    const void* m, const void* V, const int32_t* mat, int32_t* perm_out);
int resample_device_begin(mpml_ctx_s* c, const void* x);
int resample_device_end(mpml_ctx_s* c, const void* x, const void* v, const void* F, const void* G,
                        const void* m, const void* V, const int32_t* mat, int32_t* perm_out);
int p2q_q2n(mpml_ctx_s* c);
int stretch_all(mpml_ctx_s* c);
int newton_solve(mpml_ctx_s* c, const mpml_solver_opts* o, mpml_solve_stats* st);
// inexact Newton (opts.cg_forcing > 0): the forcing term of Newton iteration k, and the
// device write of the next CG solve's threshold |r|^2 <= tol2 on stream s
double newton_forcing(const mpml_solver_opts* o, int k, double gn, double gprev, double eta_prev, double target);
int set_cg_tol2(mpml_ctx_s* c, cudaStream_t s, double tol2);
int explicit_solve(mpml_ctx_s* c);
int newton_batch(mpml_ctx_s** ctxs, int n, const mpml_solver_opts* o, mpml_solve_stats* st);
int g2p_device(mpml_ctx_s* c, void* x, void* v, void* F, void* G, void* m, void* V, int32_t* mat);

// operator-level helpers used by the introspection API
int eval_device(mpml_ctx_s* c, const void* v_nodes, double* phi, void* grad_nodes);
int linearize_device(mpml_ctx_s* c, const void* v_nodes);
int hvp_device(mpml_ctx_s* c, const void* p_nodes, void* y_nodes);
int hvp_bench(mpml_ctx_s* c, int iters, double* mean_ms);
// standalone FP32 HVP launch shapes and their autotuner
constexpr int HVP_TILES = 3;
const char* hvp_tile_name(int compressed, int tile);
int hvp_autotune(mpml_ctx_s* c, int reps, int* choice, float* ms);
// process-wide cache of autotuned tiles, keyed by tangent format and brick count
int tile_cache_lookup(int compressed, int64_t ncb);
void tile_cache_store(int compressed, int64_t ncb, int tile, float ms);
int tile_cache_lookup_fmt(int fmt, int64_t ncb);
void tile_cache_store_fmt(int fmt, int64_t ncb, int tile, float ms);
// persistent-solver autotuner (mpml_autotune_pcg)
int pcg_autotune(mpml_ctx_s* c, int iters, int reps, int* choice, float* ms);
int tile_cache_save(const char* path);
int tile_cache_load(const char* path);
void tile_cache_clear();
int n2q_device(mpml_ctx_s* c);

// learned preconditioner (k_nn.cu)
int nn_ensure(mpml_ctx_s* c);
int nn_refresh_weights(mpml_ctx_s* c);
void nn_forward(mpml_ctx_s* c);
void nn_apply(mpml_ctx_s* c, const double* s_ptr, const float* q, double* part);
void nn_backward(mpml_ctx_s* c, const float* gy, float scale);
void nn_adam(mpml_ctx_s* c, float lr, int step);
int nn_set_weights(mpml_ctx_s* c, const float* w);
int nn_get_weights(mpml_ctx_s* c, float* w, int grad);
int nn_weight_count();
float* nn_output(mpml_ctx_s* c);  // y, fp32 [brick][3][512]
// learned preconditioner drivers (k_newton.cu)
int nn_apply_host(mpml_ctx_s* c, const void* r_nodes, void* z_nodes);
int nn_loss_grad_host(mpml_ctx_s* c, const void* r_nodes, const void* e_nodes, double* loss);
int nn_collect(mpml_ctx_s* c, int nsamples, double rtol, int cg_max);
int nn_train(mpml_ctx_s* c, int epochs, int batch, float lr, double* loss_first, double* loss_last);

inline unsigned div_up(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Per-device launch facts, looked up once per (current device, slot): the
// first call sets fn's dynamic shared-memory limit to smem on that device and
// queries how many CTAs of `threads` threads fit on one SM; returns that count
// (0 when the query fails) and, if nsm is not null, the device's SM count.
enum LaunchSlot : int {
  LS_PCG = 0,       // 10 persistent-solver builds (tangent format x form x CTAs per SM)
  LS_BATCH = 10,
  LS_HVP64 = 11,
  LS_CONV = 12,     // 4 convolution kernels of the learned preconditioner
  LS_COUNT = 16
};
int launch_fit(const void* fn, int threads, size_t smem, int slot, int* nsm);

// ---------------------------------------------------------------------------
// Device math
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }
template <>
__device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 (row-major A);
// eigenvectors in the columns of Q.
template <typename T>
__device__ void jacobi3(const T Ain[9], T ev[3], T Q[9]) {
  T A[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) A[i] = Ain[i];
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? T(1) : T(0);
  T fro = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) fro += A[i] * A[i];
  const T tol = eps_of<T>() * eps_of<T>() * fro * T(1e-2);
  for (int sweep = 0; sweep < 12; ++sweep) {
    T off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (!(off > tol)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      T apq = A[3 * p + q];
      if (apq == T(0)) continue;
      T theta = (A[3 * q + q] - A[3 * p + p]) / (T(2) * apq);
      T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + dsqrt(theta * theta + T(1)));
      T cc = T(1) / dsqrt(t * t + T(1)), ss = t * cc;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = cc * akp - ss * akq;
        A[3 * k + q] = ss * akp + cc * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = cc * apk - ss * aqk;
        A[3 * q + k] = ss * apk + cc * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T vkp = Q[3 * k + p], vkq = Q[3 * k + q];
        Q[3 * k + p] = cc * vkp - ss * vkq;
        Q[3 * k + q] = ss * vkp + cc * vkq;
      }
    }
  }
  ev[0] = A[0];
  ev[1] = A[4];
  ev[2] = A[8];
}

// Eigen-decomposition of a symmetric 3x3 to FP64 accuracy with most of the
// work off the (slow) FP64 pipe: cyclic Jacobi in FP32 on the matrix scaled
// by a power of two, the FP32 eigenvectors made orthonormal in FP64 by two
// Newton-Schulz steps Q <- Q (3I - Q^T Q) / 2, then Jacobi sweeps in FP64 on
// Q^T A Q with rotation angles formed in FP32 and cosines refined to FP64 by
// two Newton steps of 1/sqrt(1 + t^2) (every rotation orthogonal to FP64
// rounding; an inexact angle only slows the annihilation to a factor ~1e-7
// per sweep).  Same output convention as jacobi3; FP64 divisions: none.
__device__ inline void jacobi3_mixed(const double Ain[9], double ev[3], double Q[9]) {
  double amax = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) amax = fmax(amax, fabs(Ain[i]));
  if (!(amax > 0.0) || !(amax < 1e300)) {  // zero or non-finite: the plain FP64 sweeps
    jacobi3<double>(Ain, ev, Q);
    return;
  }
  const int ex = ilogb(amax);
  const double sc = scalbn(1.0, -ex), isc = scalbn(1.0, ex);
  double A[9];
  float Af[9], evf[3], Qf[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    A[i] = Ain[i] * sc;
    Af[i] = (float)A[i];
  }
  jacobi3<float>(Af, evf, Qf);
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (double)Qf[i];
#pragma unroll
  for (int ns = 0; ns < 2; ++ns) {
    double X[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) X[3 * a + b] = Q[a] * Q[b] + Q[3 + a] * Q[3 + b] + Q[6 + a] * Q[6 + b];
    double Y[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double acc = 1.5 * Q[3 * a + b];
#pragma unroll
        for (int k = 0; k < 3; ++k) acc -= 0.5 * Q[3 * a + k] * X[3 * k + b];
        Y[3 * a + b] = acc;
      }
#pragma unroll
    for (int i = 0; i < 9; ++i) Q[i] = Y[i];
  }
  // B = Q^T A Q (symmetric: upper part, mirrored)
  double AQ[9], B[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) AQ[3 * a + b] = A[3 * a] * Q[b] + A[3 * a + 1] * Q[3 + b] + A[3 * a + 2] * Q[6 + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const double v = Q[a] * AQ[b] + Q[3 + a] * AQ[3 + b] + Q[6 + a] * AQ[6 + b];
      B[3 * a + b] = v;
      B[3 * b + a] = v;
    }
  double fro = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) fro += B[i] * B[i];
  const double tol = 4.930380657631324e-32 * fro * 1e-2;  // eps^2 fro / 100, as jacobi3
  for (int sweep = 0; sweep < 8; ++sweep) {
    const double off = B[1] * B[1] + B[2] * B[2] + B[5] * B[5];
    if (!(off > tol)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const float apq = (float)B[3 * p + q];
      if (apq == 0.f) continue;
      const float theta = (float)(B[3 * q + q] - B[3 * p + p]) / (2.f * apq);
      const float tf = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const double t = (double)tf, x = 1.0 + t * t;
      double y = (double)rsqrtf((float)x);
      y = y * (1.5 - 0.5 * x * y * y);
      y = y * (1.5 - 0.5 * x * y * y);
      const double cc = y, ss = t * y;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double bkp = B[3 * k + p], bkq = B[3 * k + q];
        B[3 * k + p] = cc * bkp - ss * bkq;
        B[3 * k + q] = ss * bkp + cc * bkq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double bpk = B[3 * p + k], bqk = B[3 * q + k];
        B[3 * p + k] = cc * bpk - ss * bqk;
        B[3 * q + k] = ss * bpk + cc * bqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double vkp = Q[3 * k + p], vkq = Q[3 * k + q];
        Q[3 * k + p] = cc * vkp - ss * vkq;
        Q[3 * k + q] = ss * vkp + cc * vkq;
      }
    }
  }
  ev[0] = B[0] * isc;
  ev[1] = B[4] * isc;
  ev[2] = B[8] * isc;
}

// 1/sqrt(x) and 1/x (x > 0, finite, within the FP32 range) from the FP32 rsqrt
// approximation refined by Newton-Raphson steps in FP64: y <- y (3 - x y^2) / 2 for
// the reciprocal square root, y <- y (2 - x y) for the reciprocal (each step squares
// the relative error: 1e-7 -> 1e-14 -> rounding).  A few FP64 multiply-adds in place
// of the longer FP64 division and square-root sequences.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  return y * (1.5 - 0.5 * x * y * y);
}
__device__ __forceinline__ double rcp_nr(double x) {
  const double r = (double)rsqrtf((float)x);
  double y = r * r;
  y = y + y * (1.0 - x * y);
  return y + y * (1.0 - x * y);
}

// Eigen-decomposition of a symmetric 3x3 to about 1e-14 of its norm (eigenvalues)
// with the least FP64 work, for the FP64 stress, gradient and energy of FP32
// contexts: cyclic Jacobi in FP32 on the matrix scaled by a power of two; the
// first two FP32 eigenvectors made orthonormal in FP64 by Gram-Schmidt, the third
// their cross product; B = Q^T A Q in FP64; then one FP64 Jacobi sweep on B with
// FP32-formed angles and the symmetric update (b_pp -= t b_pq, b_qq += t b_pq,
// b_pq := 0).  After the FP32 stage the off-diagonal of B is ~1e-7 of the norm;
// the sweep's angles are good to FP32 rounding, so what it leaves is ~1e-14 of
// the norm, and the eigenvalues (diagonal of B) carry its square over the gap.
// Same output convention as jacobi3.
__device__ inline void jacobi3_lite(const double Ain[9], double ev[3], double Q[9]) {
  double amax = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) amax = fmax(amax, fabs(Ain[i]));
  if (!(amax > 0.0) || !(amax < 1e300)) {  // zero or non-finite: the plain FP64 sweeps
    jacobi3<double>(Ain, ev, Q);
    return;
  }
  const int ex = ilogb(amax);
  const double sc = scalbn(1.0, -ex), isc = scalbn(1.0, ex);
  double A[9];
  float Af[9], evf[3], Qf[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    A[i] = Ain[i] * sc;
    Af[i] = (float)A[i];
  }
  jacobi3<float>(Af, evf, Qf);
  // Gram-Schmidt on columns 0 and 1, column 2 = column 0 x column 1
  double q0[3] = {(double)Qf[0], (double)Qf[3], (double)Qf[6]};
  double q1[3] = {(double)Qf[1], (double)Qf[4], (double)Qf[7]};
  const double i0 = rsqrt_nr(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2]);
#pragma unroll
  for (int r = 0; r < 3; ++r) q0[r] *= i0;
  const double d01 = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2];
#pragma unroll
  for (int r = 0; r < 3; ++r) q1[r] -= d01 * q0[r];
  const double i1 = rsqrt_nr(q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2]);
#pragma unroll
  for (int r = 0; r < 3; ++r) q1[r] *= i1;
  const double q2[3] = {q0[1] * q1[2] - q0[2] * q1[1], q0[2] * q1[0] - q0[0] * q1[2], q0[0] * q1[1] - q0[1] * q1[0]};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Q[3 * r] = q0[r];
    Q[3 * r + 1] = q1[r];
    Q[3 * r + 2] = q2[r];
  }
  // B = Q^T A Q (upper part, mirrored)
  double AQ[9], B[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) AQ[3 * a + b] = A[3 * a] * Q[b] + A[3 * a + 1] * Q[3 + b] + A[3 * a + 2] * Q[6 + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const double v = Q[a] * AQ[b] + Q[3 + a] * AQ[3 + b] + Q[6 + a] * AQ[6 + b];
      B[3 * a + b] = v;
      B[3 * b + a] = v;
    }
#pragma unroll
  for (int pq = 0; pq < 3; ++pq) {
    const int p = pq == 2 ? 1 : 0;
    const int q = pq == 0 ? 1 : 2;
    const int r = 3 - p - q;
    const double bpq = B[3 * p + q];
    const float apq = (float)bpq;
    if (apq == 0.f) continue;
    const float theta = (float)(B[3 * q + q] - B[3 * p + p]) / (2.f * apq);
    const float tf = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
    const double t = (double)tf;
    const double cc = rsqrt_nr(1.0 + t * t), ss = t * cc;
    B[3 * p + p] -= t * bpq;
    B[3 * q + q] += t * bpq;
    B[3 * p + q] = B[3 * q + p] = 0.0;
    const double brp = B[3 * r + p], brq = B[3 * r + q];
    B[3 * r + p] = B[3 * p + r] = cc * brp - ss * brq;
    B[3 * r + q] = B[3 * q + r] = ss * brp + cc * brq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double vkp = Q[3 * k + p], vkq = Q[3 * k + q];
      Q[3 * k + p] = cc * vkp - ss * vkq;
      Q[3 * k + q] = ss * vkp + cc * vkq;
    }
  }
  ev[0] = B[0] * isc;
  ev[1] = B[4] * isc;
  ev[2] = B[8] * isc;
}

// jacobi3 in the type's precision; FP64 through jacobi3_mixed (to FP64 rounding) or
// jacobi3_lite (to about 1e-14)
template <typename T, bool LITE = false>
__device__ __forceinline__ void jacobi3_fast(const T A[9], T ev[3], T Q[9]) {
  if constexpr (sizeof(T) == 8) {
    if constexpr (LITE)
      jacobi3_lite(A, ev, Q);
    else
      jacobi3_mixed(A, ev, Q);
  } else {
    jacobi3<T>(A, ev, Q);
  }
}

// [persistent-solver source: begin]
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded grid barrier (all CTAs co-resident: cooperative launch) on one
// counter that starts at zero: CTA 0 adds 2^31 - (G - 1), every other CTA adds
// 1, so the top bit flips exactly when the last CTA of a round arrives (no
// proper subset of the adds crosses 2^31) and the low bits return to zero.
// The last arrival learns it from its own add; the others poll the top bit.
// `limit` bounds the polls of one wait (each after a 32 ns sleep).
constexpr unsigned BARRIER_SPINS_DEFAULT = 1u << 25;
__device__ __forceinline__ bool grid_barrier(unsigned* gbar, int* s_flag, unsigned limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(gbar, add);
    int ok = 1;
    if ((((old + add) ^ old) & 0x80000000u) == 0u) {
      unsigned spins = 0;
      while (((ld_acquire_gpu(gbar) ^ old) & 0x80000000u) == 0u) {
        if (++spins > limit) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// rotation matrix (row-major) of a unit quaternion (w, x, y, z)
template <typename T>
__device__ __forceinline__ void quat_to_rot(T w, T x, T y, T z, T R[9]) {
  R[0] = T(1) - T(2) * (y * y + z * z);
  R[1] = T(2) * (x * y - z * w);
  R[2] = T(2) * (x * z + y * w);
  R[3] = T(2) * (x * y + z * w);
  R[4] = T(1) - T(2) * (x * x + z * z);
  R[5] = T(2) * (y * z - x * w);
  R[6] = T(2) * (x * z - y * w);
  R[7] = T(2) * (y * z + x * w);
  R[8] = T(1) - T(2) * (x * x + y * y);
}

// Numbers per cell of the compressed tangent (single material, FP32):
//   [0, 4)   unit quaternion of U
//   [4, 13)  W = S V (row-major; S the symmetric stretch base, V the right
//            singular vectors of the trial deformation)
//   [13, 19) A = Q diag(lambda+) Q^T (xx, yy, zz, xy, xz, yz): the clamped 3x3
//            block of the isotropic tangent acting on the diagonal of M
//   [19, 22) flip moduli / 2 of the pairs (0,1), (0,2), (1,2)
//   [22, 25) twist moduli / 2 of the same pairs
constexpr int NQC = 25;

// FP32 HVP of one cell on the compressed tangent:
// K D' = U Mt W^T with M = U^T D' W, and Mt the clamped eigen-modes of the
// isotropic tangent applied to M (the block A on the diagonal of M, flip /
// twist modes on its off-diagonal pairs).
__device__ __forceinline__ void apply_cmp(const float c[NQC], const float D[9], float KD[9]) {
  float U[9];
  quat_to_rot<float>(c[0], c[1], c[2], c[3], U);
  const float* W = c + 4;
  // M = U^T D W
  float T1[9], M[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int b = 0; b < 3; ++b) T1[3 * i + b] = U[i] * D[b] + U[3 + i] * D[3 + b] + U[6 + i] * D[6 + b];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[3 * i + j] = T1[3 * i] * W[j] + T1[3 * i + 1] * W[3 + j] + T1[3 * i + 2] * W[6 + j];
  float Mt[9];
  // diagonal block
  Mt[0] = c[13] * M[0] + c[16] * M[4] + c[17] * M[8];
  Mt[4] = c[16] * M[0] + c[14] * M[4] + c[18] * M[8];
  Mt[8] = c[17] * M[0] + c[18] * M[4] + c[15] * M[8];
  // pairs (0,1), (0,2), (1,2): flip (M_ij + M_ji)/sqrt2, twist (M_ij - M_ji)/sqrt2
  const int PI[3] = {0, 0, 1}, PJ[3] = {1, 2, 2};
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int i = PI[p], j = PJ[p];
    const float f = c[19 + p] * (M[3 * i + j] + M[3 * j + i]);
    const float t = c[22 + p] * (M[3 * i + j] - M[3 * j + i]);
    Mt[3 * i + j] = f + t;
    Mt[3 * j + i] = f - t;
  }
  // K D' = U Mt W^T
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j) T1[3 * a + j] = U[3 * a] * Mt[j] + U[3 * a + 1] * Mt[3 + j] + U[3 * a + 2] * Mt[6 + j];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) KD[3 * a + b] = T1[3 * a] * W[3 * b] + T1[3 * a + 1] * W[3 * b + 1] + T1[3 * a + 2] * W[3 * b + 2];
}

// streamed read-only load: no L1 allocation, L2 fetches in 256-byte sectors
// (the tangent block is read once per launch, in 128-byte rows per warp)
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ int hidx(int nx, int ny, int nz) { return (nz * 9 + ny) * 9 + nx; }

// the column-walk phase H adds the z-exchange of the four 64-thread groups
// (12 floats per thread) and their row 3 -> 4 partials (3 layers x 2 x 3 x 8)
constexpr size_t HVP_X_FLOATS = 4 * 12 * 64, HVP_R_FLOATS = 4 * 3 * 2 * 3 * 8;

// node (nx, ny, nz) of the 9^3 halo of brick id receives y[3] inside the
// persistent solvers (one scene or a batch), where q starts at zero: own nodes take the mass term too
// (plain store where only this brick contributes, atomic add elsewhere).
__device__ __forceinline__ void col_emit_m(int id, const int* s_nbr, const float (*sv)[729],
                                          const float* __restrict__ m, float* q, int nx, int ny, int nz,
                                          const float y[3]) {
  if (nx < 8 && ny < 8 && nz < 8) {
    const int l = (nz * 8 + ny) * 8 + nx;
    float* dst = q + (int64_t)id * 3 * BV + l;
    const float mi = __ldcg(m + (int64_t)id * BV + l);
    const int i = hidx(nx, ny, nz);
    if (nx >= 1 && ny >= 1 && nz >= 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) dst[a * BV] = y[a] + mi * sv[a][i];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float val = y[a] + mi * sv[a][i];
        if (val != 0.f) atomicAdd(dst + a * BV, val);
      }
    }
  } else {
    const int t = s_nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
    if (t < 0) return;
    const int l = ((nz & 7) * 8 + (ny & 7)) * 8 + (nx & 7);
    float* dst = q + (int64_t)t * 3 * BV + l;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (y[a] != 0.f) atomicAdd(dst + a * BV, y[a]);
  }
}

// corner contributions of one cell: lower-z corners into N (added), upper-z
// corners returned in U; node (x + ox, y + oy, z + oz) gets
// (2ox-1) X + (2oy-1) Y + (2oz-1) Z of the cell's K D' rows (X, Y, Z)
__device__ __forceinline__ void col_corners(const float KD[9], float N[2][2][3], float U[2][2][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float X = KD[3 * a], Yv = KD[3 * a + 1], Z = KD[3 * a + 2];
    const float Ap = X + Yv, B = X - Yv;
    N[1][1][a] += Ap - Z;
    N[0][0][a] -= Ap + Z;
    N[1][0][a] += B - Z;
    N[0][1][a] -= B + Z;
    U[1][1][a] = Ap + Z;
    U[0][0][a] = Z - Ap;
    U[1][0][a] = B + Z;
    U[0][1][a] = Z - B;
  }
}

// D' = sum_o p_o (x) sgn_o from the lower (P0) and upper (P1) node layers of a cell
__device__ __forceinline__ void col_D(const float P0[2][2][3], const float P1[2][2][3], float D[9]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float s00 = P0[0][0][a] + P1[0][0][a], s10 = P0[1][0][a] + P1[1][0][a];
    const float s01 = P0[0][1][a] + P1[0][1][a], s11 = P0[1][1][a] + P1[1][1][a];
    D[3 * a + 0] = (s10 + s11) - (s00 + s01);
    D[3 * a + 1] = (s01 + s11) - (s00 + s10);
    D[3 * a + 2] = (P1[0][0][a] - P0[0][0][a]) + (P1[1][0][a] - P0[1][0][a]) + (P1[0][1][a] - P0[0][1][a]) +
                   (P1[1][1][a] - P0[1][1][a]);
  }
}

// Phase H of one brick in the column walk: the CTA's four 64-thread groups take
// two z-layers of cells each (group g: cells z = 2g, 2g + 1 of column (x, y));
// node layers are summed along z in registers, across groups through shared
// memory (layer 2g gets group g-1's upper corners), along x by warp shuffles and
// along y by shuffles of eight lanes (rows 3 -> 4 through shared memory).
// Returns the thread's sum of D' . K D'.
template <bool K45, bool GLOBAL = false>
__device__ __forceinline__ float phase_h_col(int id, const int* s_nbr, const float (*sv)[729], const float* Cs,
                                             const uint8_t* __restrict__ cflag, const float* __restrict__ m, float* q,
                                             float* X, float* R, bool ok) {
  constexpr unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, g = t >> 6, x = t & 7, y = (t >> 3) & 7, row = y & 3, c64 = t & 63;
  float pkp = 0.f;
  float Pa[2][2][3], Pb[2][2][3];
  float Na[2][2][3], Nb[2][2][3], Nc[2][2][3];
#pragma unroll
  for (int ox = 0; ox < 2; ++ox)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Pa[ox][oy][a] = sv[a][hidx(x + ox, y + oy, 2 * g)];
        Pb[ox][oy][a] = sv[a][hidx(x + ox, y + oy, 2 * g + 1)];
        Na[ox][oy][a] = 0.f;
      }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = (2 * g + h) * 64 + c64;
    float KD[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) KD[r] = 0.f;
    if (ok && cflag[(int64_t)id * BV + l]) {
      float D[9];
      col_D(Pa, Pb, D);
      if (K45) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          KD[r] += (GLOBAL ? ld_stream(Cs + k45(r, r) * BV + l) : Cs[k45(r, r) * BV + l]) * D[r];
#pragma unroll
          for (int cc = r + 1; cc < 9; ++cc) {
            const float kv = GLOBAL ? ld_stream(Cs + k45(r, cc) * BV + l) : Cs[k45(r, cc) * BV + l];
            KD[r] += kv * D[cc];
            KD[cc] += kv * D[r];
          }
        }
      } else {
        float c[NQC];
#pragma unroll
        for (int qq = 0; qq < NQC; ++qq) c[qq] = GLOBAL ? ld_stream(Cs + qq * BV + l) : Cs[qq * BV + l];
        apply_cmp(c, D, KD);
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) pkp += D[r] * KD[r];
    }
    if (h == 0) {
      col_corners(KD, Na, Nb);  // Nb <- upper corners of cell 2g (lower of cell 2g+1 added next)
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            Pa[ox][oy][a] = Pb[ox][oy][a];
            Pb[ox][oy][a] = sv[a][hidx(x + ox, y + oy, 2 * g + 2)];
          }
    } else {
      col_corners(KD, Nb, Nc);
    }
  }
  // across groups: node layer 2g + 2 = this group's Nc + group g+1's Na
  if (K45 && !GLOBAL) __syncthreads();  // X overlays the tangent block: every cell has been applied
  if (g < 3) {
    float* Xg = X + g * 12 * 64;
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int a = 0; a < 3; ++a) Xg[((ox * 2 + oy) * 3 + a) * 64 + c64] = Nc[ox][oy][a];
  }
  __syncthreads();
  if (g > 0) {
    const float* Xg = X + (g - 1) * 12 * 64;
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int a = 0; a < 3; ++a) Na[ox][oy][a] += Xg[((ox * 2 + oy) * 3 + a) * 64 + c64];
  }
  // along x (shuffles), then the row-3 partials of every layer into shared memory
  const int nl = g == 3 ? 3 : 2;
  float E[3][2][3], E8[3][2][3];
#pragma unroll
  for (int L = 0; L < 3; ++L) {
    if (L == 2 && nl < 3) break;
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float n0 = L == 0 ? Na[0][oy][a] : (L == 1 ? Nb[0][oy][a] : Nc[0][oy][a]);
        const float n1 = L == 0 ? Na[1][oy][a] : (L == 1 ? Nb[1][oy][a] : Nc[1][oy][a]);
        const float left = __shfl_up_sync(FULL, n1, 1);
        E[L][oy][a] = n0 + (x > 0 ? left : 0.f);
        E8[L][oy][a] = n1;
      }
    if (y == 3) {
      float* Rg = R + (g * 3 + L) * 48;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Rg[a * 8 + x] = E[L][1][a];
        Rg[24 + a * 8 + x] = E8[L][1][a];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int L = 0; L < 3; ++L) {
    if (L == 2 && nl < 3) break;
    const int nz = L == 2 ? 8 : 2 * g + L;
    const float* Rg = R + (g * 3 + L) * 48;
    float T[3], T8[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float up = __shfl_up_sync(FULL, E[L][1][a], 8), up8 = __shfl_up_sync(FULL, E8[L][1][a], 8);
      float prev = 0.f, prev8 = 0.f;
      if (row > 0) {
        prev = up;
        prev8 = up8;
      } else if (y == 4) {
        prev = Rg[a * 8 + x];
        prev8 = Rg[24 + a * 8 + x];
      }
      T[a] = E[L][0][a] + prev;
      T8[a] = E8[L][0][a] + prev8;
    }
    col_emit_m(id, s_nbr, sv, m, q, x, y, nz, T);
    if (x == 7) col_emit_m(id, s_nbr, sv, m, q, 8, y, nz, T8);
    if (y == 7) {
      col_emit_m(id, s_nbr, sv, m, q, x, 8, nz, E[L][1]);
      if (x == 7) col_emit_m(id, s_nbr, sv, m, q, 8, 8, nz, E8[L][1]);
    }
  }
  return pkp;
}

// [persistent-solver source: end]

// 1 / sqrt(nn): FP64 LITE builds take rsqrt_nr within the FP32 range
template <typename T, bool LITE>
__device__ __forceinline__ T inv_sqrt_t(T nn) {
  if constexpr (LITE && sizeof(T) == 8) {
    if (nn > T(1e-36) && nn < T(1e36)) return rsqrt_nr(nn);
  }
  return T(1) / dsqrt(nn);
}

// Signed SVD of F = I + H from the eigen-decomposition of F^T F - I =
// H + H^T + H^T H, returning s = singular values (s0 >= s1 >= |s2|, s2 < 0
// when det F < 0), e = s - 1 computed without cancellation, J - 1 likewise.
// LITE (FP64): the eigen-decomposition by jacobi3_lite and the square roots and
// reciprocals by rsqrt_nr / rcp_nr -- results to about 1e-14 instead of FP64 rounding.
template <typename T, bool LITE = false>
__device__ void svd_from_h(const T H[9], T U[9], T s[3], T e[3], T V[9], T& Jm1) {
  T E[9];  // symmetric: the upper triangle, mirrored
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      T acc = H[3 * a + b] + H[3 * b + a];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += H[3 * k + a] * H[3 * k + b];
      E[3 * a + b] = acc;
      E[3 * b + a] = acc;
    }
  T lam[3], W[9];
  jacobi3_fast<T, LITE>(E, lam, W);
  int i0 = 0, i1 = 1, i2 = 2;
  if (lam[i1] > lam[i0]) { int t = i0; i0 = i1; i1 = t; }
  if (lam[i2] > lam[i0]) { int t = i0; i0 = i2; i2 = t; }
  if (lam[i2] > lam[i1]) { int t = i1; i1 = i2; i2 = t; }
  const int id[3] = {i0, i1, i2};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) V[3 * r + c] = W[3 * r + id[c]];
  T detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
           V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (detV < T(0)) {
    V[2] = -V[2];
    V[5] = -V[5];
    V[8] = -V[8];
  }
  T l[3] = {lam[i0], lam[i1], lam[i2]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T li = l[i] > T(-1) ? l[i] : T(-1);
    const T x = T(1) + li;
    if constexpr (LITE && sizeof(T) == 8) {
      if (x > T(1e-30) && x < T(1e30)) {
        s[i] = x * rsqrt_nr(x);
        e[i] = li * rcp_nr(T(1) + s[i]);
        continue;
      }
    }
    s[i] = dsqrt(x);
    e[i] = li / (T(1) + s[i]);
  }
  // b_j = F v_j
  T b[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      T acc = V[3 * r + j];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += H[3 * r + k] * V[3 * k + j];
      b[j][r] = acc;
    }
  T u0[3], u1[3], u2[3];
  const T nn0 = b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2];
  if (nn0 > T(1e-60)) {
    const T in0 = inv_sqrt_t<T, LITE>(nn0);  // three products (divisions are costly in FP64)
#pragma unroll
    for (int r = 0; r < 3; ++r) u0[r] = b[0][r] * in0;
  } else {
    u0[0] = 1; u0[1] = 0; u0[2] = 0;
  }
  T dd = u0[0] * b[1][0] + u0[1] * b[1][1] + u0[2] * b[1][2];
#pragma unroll
  for (int r = 0; r < 3; ++r) u1[r] = b[1][r] - dd * u0[r];
  const T nn1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
  if (nn1 > T(1e-60)) {
    const T in1 = inv_sqrt_t<T, LITE>(nn1);
#pragma unroll
    for (int r = 0; r < 3; ++r) u1[r] *= in1;
  } else {
    T a0 = fabs(u0[0]) > T(0.9) ? T(0) : T(1), a1 = fabs(u0[0]) > T(0.9) ? T(1) : T(0);
    T ee = a0 * u0[0] + a1 * u0[1];
    u1[0] = a0 - ee * u0[0];
    u1[1] = a1 - ee * u0[1];
    u1[2] = -ee * u0[2];
    T nn = dsqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) u1[r] /= nn;
  }
  u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
  u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
  u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
  T d2 = u2[0] * b[2][0] + u2[1] * b[2][1] + u2[2] * b[2][2];
  if (d2 < T(0)) {
    s[2] = -s[2];
    e[2] = s[2] - T(1);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    U[3 * r + 0] = u0[r];
    U[3 * r + 1] = u1[r];
    U[3 * r + 2] = u2[r];
  }
  Jm1 = e[0] + e[1] + e[2] + e[0] * e[1] + e[0] * e[2] + e[1] * e[2] + e[0] * e[1] * e[2];
}

// Spectral data of an isotropic energy at principal stretches s (e = s - 1,
// Jm1 = J - 1 given accurately): psi, d1 = dpsi/ds, d2 = Hessian in s, and
// per pair (0,1),(0,2),(1,2): pp = (d1_i - d1_j)/(s_i - s_j),
// pm = (d1_i + d1_j)/(s_i + s_j), in closed forms finite at s_i = s_j.
template <typename T>
struct Spec {
  T psi, d1[3], d2[9], pp[3], pm[3];
};

template <typename T>
__device__ __forceinline__ T log1p_t(T x);
template <>
__device__ __forceinline__ float log1p_t<float>(float x) { return log1pf(x); }
template <>
__device__ __forceinline__ double log1p_t<double>(double x) { return log1p(x); }
template <typename T>
__device__ __forceinline__ T expm1_t(T x);
template <>
__device__ __forceinline__ float expm1_t<float>(float x) { return expm1f(x); }
template <>
__device__ __forceinline__ double expm1_t<double>(double x) { return expm1(x); }
template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// x - log(1 + x) without cancellation near 0
template <typename T>
__device__ __forceinline__ T x_minus_log1p(T x) {
  if (fabs(x) < T(0.05)) {
    // Taylor series of x - log(1 + x) = sum_{k>=2} (-1)^k x^k / k to k = 13 (error < 0.05^14 / 14),
    // in Horner form with the coefficients as constants: multiplications, no divisions
    // (FP64 divisions are slow on this part)
    T acc = T(-1.0 / 13);
    acc = acc * x + T(1.0 / 12);
    acc = acc * x - T(1.0 / 11);
    acc = acc * x + T(1.0 / 10);
    acc = acc * x - T(1.0 / 9);
    acc = acc * x + T(1.0 / 8);
    acc = acc * x - T(1.0 / 7);
    acc = acc * x + T(1.0 / 6);
    acc = acc * x - T(1.0 / 5);
    acc = acc * x + T(1.0 / 4);
    acc = acc * x - T(1.0 / 3);
    acc = acc * x + T(1.0 / 2);
    return acc * x * x;
  }
  return x - log1p_t(x);
}

// (1 + x)^(-2/3) - 1: for |x| < 0.05 the binomial series sum_{k=1..12} C(-2/3, k) x^k
// (remainder below 4e-18), in Horner form with the exact rational coefficients;
// otherwise expm1(-2/3 log1p(x)).  Saves two FP64 transcendentals per cell.
template <typename T>
__device__ __forceinline__ T jpow_m23_m1(T x) {
  if (fabs(x) < T(0.05)) {
    T acc = T(41273960.0 / 129140163.0);
    acc = acc * x - T(4717024.0 / 14348907.0);
    acc = acc * x + T(1621477.0 / 4782969.0);
    acc = acc * x - T(559130.0 / 1594323.0);
    acc = acc * x + T(21505.0 / 59049.0);
    acc = acc * x - T(7480.0 / 19683.0);
    acc = acc * x + T(2618.0 / 6561.0);
    acc = acc * x - T(308.0 / 729.0);
    acc = acc * x + T(110.0 / 243.0);
    acc = acc * x - T(40.0 / 81.0);
    acc = acc * x + T(5.0 / 9.0);
    acc = acc * x - T(2.0 / 3.0);
    return acc * x;
  }
  return expm1_t(T(-2) / T(3) * log1p_t(x));
}

// 3 ((1 + x)^(-2/3) - 1) + 2 x, which is second order in x: for |x| < 0.05 from the
// binomial series without its linear term (so the first-order parts cancel exactly),
// otherwise from jpow_m23_m1 directly.
template <typename T>
__device__ __forceinline__ T nh_a2(T x) {
  if (fabs(x) < T(0.05)) {
    T acc = T(41273960.0 / 129140163.0);
    acc = acc * x - T(4717024.0 / 14348907.0);
    acc = acc * x + T(1621477.0 / 4782969.0);
    acc = acc * x - T(559130.0 / 1594323.0);
    acc = acc * x + T(21505.0 / 59049.0);
    acc = acc * x - T(7480.0 / 19683.0);
    acc = acc * x + T(2618.0 / 6561.0);
    acc = acc * x - T(308.0 / 729.0);
    acc = acc * x + T(110.0 / 243.0);
    acc = acc * x - T(40.0 / 81.0);
    acc = acc * x + T(5.0 / 9.0);
    return T(3) * acc * x * x;
  }
  return T(3) * jpow_m23_m1(x) + T(2) * x;
}

// Split Neo-Hookean energy (Sec. 4.3.2) mu/2 (J^(-2/3) I1 - 3) + kappa/4 (J^2 - 1 - 2 log J)
// from second-order quantities only, so that small strains keep their relative
// accuracy (the first-order parts of J^(-2/3) I1 - 3 cancel analytically):
//   J^(-2/3) I1 - 3 = [3 cm1 + 2 (J-1)] + [I1 - 3 - 2 (J-1)] + cm1 (I1 - 3),
//   cm1 = J^(-2/3) - 1, with b2 = I1 - 3 - 2 (J-1) supplied by the caller as a sum of
//   second-order terms; J^2 - 1 - 2 log J = (J-1)^2 + 2 ((J-1) - log(1 + (J-1))).
template <typename T>
__device__ __forceinline__ T nh_psi(T mu, T kap, T Jm1, T I1m3, T b2) {
  const T cm1 = jpow_m23_m1(Jm1);
  return T(0.5) * mu * (nh_a2(Jm1) + b2 + cm1 * I1m3) + T(0.25) * kap * (T(2) * x_minus_log1p(Jm1) + Jm1 * Jm1);
}

__device__ __forceinline__ int pair_i(int p) { return p == 2 ? 1 : 0; }
__device__ __forceinline__ int pair_j(int p) { return p == 0 ? 1 : 2; }
__device__ __forceinline__ int pair_k(int p) { return 2 - p; }

// log(1 + x): for |x| < 0.05 as x minus the series of x - log(1 + x) (about one
// rounding error, multiply-adds only), otherwise the library function
template <typename T>
__device__ __forceinline__ T log1p_series(T x) {
  return fabs(x) < T(0.05) ? x - x_minus_log1p(x) : log1p_t(x);
}

// Symmetric 3x3 as (xx, yy, zz, xy, xz, yz); sym_mul is the product of two that commute
// (so that the product is symmetric again)
template <typename T>
struct Sym3 {
  T xx, yy, zz, xy, xz, yz;
};
template <typename T>
__device__ __forceinline__ Sym3<T> sym_mul(const Sym3<T>& A, const Sym3<T>& B) {
  return {A.xx * B.xx + A.xy * B.xy + A.xz * B.xz, A.xy * B.xy + A.yy * B.yy + A.yz * B.yz,
          A.xz * B.xz + A.yz * B.yz + A.zz * B.zz, A.xx * B.xy + A.xy * B.yy + A.xz * B.yz,
          A.xx * B.xz + A.xy * B.yz + A.xz * B.zz, A.xy * B.xz + A.yy * B.yz + A.yz * B.zz};
}

// log(I + E) of a symmetric E near zero without an eigen-decomposition: 2 atanh(Z) with
// Z = E (2I + E)^-1 (symmetric; commutes with E), as the odd series 2 (Z + Z^3/3 + ...)
// in Horner form in Z^2 -- to Z^11 in FP64, Z^5 in FP32.  Only where every |E_ij| <= 0.03
// (then |Z| <= 0.047 and the first omitted term is below the type's rounding of |Z|):
// returns false elsewhere.  Multiply-adds and one reciprocal (Newton-refined in FP64).
template <typename T>
__device__ bool log_spd_series(const Sym3<T>& E, Sym3<T>& L) {
  const T mx = fmax(fmax(fmax(fabs(E.xx), fabs(E.yy)), fmax(fabs(E.zz), fabs(E.xy))), fmax(fabs(E.xz), fabs(E.yz)));
  if (!(mx <= T(0.03))) return false;
  // (2I + E)^-1 by cofactors (symmetric); its determinant is within [6.2, 10]
  const T a00 = T(2) + E.xx, a11 = T(2) + E.yy, a22 = T(2) + E.zz;
  const T c00 = a11 * a22 - E.yz * E.yz, c11 = a00 * a22 - E.xz * E.xz, c22 = a00 * a11 - E.xy * E.xy;
  const T c01 = E.xz * E.yz - E.xy * a22, c02 = E.xy * E.yz - E.xz * a11, c12 = E.xy * E.xz - a00 * E.yz;
  const T det = a00 * c00 + E.xy * c01 + E.xz * c02;
  T id;
  if constexpr (sizeof(T) == 8)
    id = rcp_nr(det);
  else
    id = T(1) / det;
  const Sym3<T> Ai = {c00 * id, c11 * id, c22 * id, c01 * id, c02 * id, c12 * id};
  const Sym3<T> Z = sym_mul(E, Ai), Y = sym_mul(Z, Z);
  // S = 1 + Y/3 + Y^2/5 + ... (to Y^5/11 in FP64, Y^2/5 in FP32)
  constexpr int NT = sizeof(T) == 8 ? 5 : 2;
  const T cl = T(1) / T(2 * NT + 1), cn = T(1) / T(2 * NT - 1);
  Sym3<T> S = {Y.xx * cl + cn, Y.yy * cl + cn, Y.zz * cl + cn, Y.xy * cl, Y.xz * cl, Y.yz * cl};
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) {
    const T ck = T(1) / T(2 * k + 1);
    S = sym_mul(Y, S);
    S.xx += ck;
    S.yy += ck;
    S.zz += ck;
  }
  const Sym3<T> Tz = sym_mul(Z, S);
  L = {T(2) * Tz.xx, T(2) * Tz.yy, T(2) * Tz.zz, T(2) * Tz.xy, T(2) * Tz.xz, T(2) * Tz.yz};
  return true;
}

// returns false where the energy is undefined (J <= 0 for NH / Hencky)
// The isotropic eigen-data of psi at the signed singular values s (e = s - 1,
// Jm1 = J - 1): PARTS bit 1 the energy and the principal stresses d1 (what the
// gradient needs), bit 2 the projected-tangent moduli d2 (3x3 block), pp (flip)
// and pm (twist).  The two parts can be evaluated in different precisions.
// Bit 4 (with the FP64 energy and stresses of FP32 contexts): the Hencky
// logarithms by log1p_series and the reciprocals of s by rcp_nr.
template <typename T, int PARTS = 3>
__device__ bool spectral(const MatParams<T>& M, const T s[3], const T e[3], T Jm1, Spec<T>& o) {
  constexpr bool P1 = (PARTS & 1) != 0, P2 = (PARTS & 2) != 0;
  constexpr bool LITE = (PARTS & 4) != 0 && sizeof(T) == 8;
  const T mu = M.mu, lam = M.lam;
  const T J = T(1) + Jm1;
  if (M.model == MPML_FIXED_COROTATED) {
    if (P1) o.psi = mu * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) + T(0.5) * lam * Jm1 * Jm1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      if (P1) o.d1[i] = T(2) * mu * e[i] + lam * Jm1 * s[j] * s[k];
      if (P2) o.d2[4 * i] = T(2) * mu + lam * (s[j] * s[k]) * (s[j] * s[k]);
    }
    if (P2) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int i = pair_i(p), j = pair_j(p), k = pair_k(p);
        o.d2[3 * i + j] = o.d2[3 * j + i] = lam * s[k] * (T(2) * J - T(1));
        o.pp[p] = T(2) * mu - lam * Jm1 * s[k];
        o.pm[p] = T(2) * mu * (e[i] + e[j]) / (s[i] + s[j]) + lam * Jm1 * s[k];
      }
    }
    return true;
  }
  if (M.model == MPML_NEO_HOOKEAN) {
    if (!(J > T(0))) return false;
    const T kap = T(2) / T(3) * mu + lam;
    const T cm1 = jpow_m23_m1(Jm1);  // J^{-2/3} - 1
    const T c = T(1) + cm1;
    const T I1m3 = e[0] * (T(2) + e[0]) + e[1] * (T(2) + e[1]) + e[2] * (T(2) + e[2]);
    const T I1 = T(3) + I1m3;
    const T J2m1 = Jm1 * (T(2) + Jm1);
    if (P1) {
      // I1 - 3 - 2 (J - 1) = sum e_i^2 - 2 (e0 e1 + e0 e2 + e1 e2) - 2 e0 e1 e2
      const T b2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] - T(2) * (e[0] * e[1] + e[0] * e[2] + e[1] * e[2]) -
                   T(2) * e[0] * e[1] * e[2];
      o.psi = nh_psi(mu, kap, Jm1, I1m3, b2);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      if (P1) {
        // s_i - I1/(3 s_i) = ((s_i^2 - s_j^2) + (s_i^2 - s_k^2)) / (3 s_i)
        const T dij = (e[i] - e[j]) * (T(2) + e[i] + e[j]);
        const T dik = (e[i] - e[k]) * (T(2) + e[i] + e[k]);
        o.d1[i] = mu * c * (dij + dik) / (T(3) * s[i]) + T(0.5) * kap * J2m1 / s[i];
      }
      if (P2)
        o.d2[4 * i] = mu * c * (T(-1) / T(3) + T(5) * I1 / (T(9) * s[i] * s[i])) +
                      T(0.5) * kap * (J * J + T(1)) / (s[i] * s[i]);
    }
    if (P2) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int i = pair_i(p), j = pair_j(p);
        const T sij = s[i] * s[j];
        o.d2[3 * i + j] = o.d2[3 * j + i] =
            mu * c / sij * (T(-2) / T(3) * s[i] * s[i] - T(2) / T(3) * s[j] * s[j] + T(2) / T(9) * I1) +
            kap * J * J / sij;
        o.pp[p] = mu * c * (T(1) + I1 / (T(3) * sij)) - T(0.5) * kap * J2m1 / sij;
        o.pm[p] = mu * c * (T(1) - I1 / (T(3) * sij)) + T(0.5) * kap * J2m1 / sij;
      }
    }
    return true;
  }
  if (M.model == MPML_WATER) {
    // Sec. "Water": psi = kappa/2 (J - 1)^2, kappa = lam + 2/3 mu; no inverted fluid
    if (!(J > T(0))) return false;
    const T kap = lam + T(2) / T(3) * mu;
    if (P1) o.psi = T(0.5) * kap * Jm1 * Jm1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      if (P1) o.d1[i] = kap * Jm1 * s[j] * s[k];
      if (P2) o.d2[4 * i] = kap * (s[j] * s[k]) * (s[j] * s[k]);
    }
    if (P2) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int i = pair_i(p), j = pair_j(p), k = pair_k(p);
        o.d2[3 * i + j] = o.d2[3 * j + i] = kap * s[k] * (T(2) * J - T(1));
        o.pp[p] = -kap * Jm1 * s[k];
        o.pm[p] = kap * Jm1 * s[k];
      }
    }
    return true;
  }
  if (M.model == MPML_HENCKY) {
    if (!(s[0] > T(0) && s[1] > T(0) && s[2] > T(0))) return false;
    T l[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) l[i] = LITE ? log1p_series(e[i]) : log1p_t(e[i]);
    const T tr = l[0] + l[1] + l[2];
    if (P1) o.psi = mu * (l[0] * l[0] + l[1] * l[1] + l[2] * l[2]) + T(0.5) * lam * tr * tr;
    T t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      t[i] = T(2) * mu * l[i] + lam * tr;
      if (P1) {
        if constexpr (LITE) {
          o.d1[i] = (s[i] > T(1e-30) && s[i] < T(1e30)) ? t[i] * rcp_nr(s[i]) : t[i] / s[i];
        } else {
          o.d1[i] = t[i] / s[i];
        }
      }
      if (P2) o.d2[4 * i] = (T(2) * mu + lam - t[i]) / (s[i] * s[i]);
    }
    if (P2) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int i = pair_i(p), j = pair_j(p);
        o.d2[3 * i + j] = o.d2[3 * j + i] = lam / (s[i] * s[j]);
        const T z = (s[i] - s[j]) / s[j];
        const T L = fabs(z) < T(1e-4) ? T(1) - T(0.5) * z + z * z / T(3) : log1p_t(z) / z;
        o.pp[p] = (T(2) * mu * (L - l[j]) - lam * tr) / (s[i] * s[j]);
        o.pm[p] = (t[i] * s[j] + t[j] * s[i]) / (s[i] * s[j] * (s[i] + s[j]));
      }
    }
    return true;
  }
  return false;
}

// Plastic return map of one particle's elastic F (in place), in the Hencky
// strain eps = log(s) of F = U diag(s) V^T with U, V kept; tau = 2 mu eps +
// lam tr(eps) I.  Von Mises: |dev eps| beyond sqrt(2/3) ys / (2 mu) is scaled
// back to it.  Drucker-Prager (cohesionless): tr(eps) > 0 -> eps = 0;
// otherwise dgamma = |dev eps| + (3 lam + 2 mu) / (2 mu) alpha tr(eps) > 0 is
// removed from |dev eps| along dev eps.  F with a non-positive singular value
// is left unchanged.  Returns whether F was changed.
template <typename T>
__device__ bool return_map(int kind, double mu_, double lam_, double ys, double alpha_, T F[9]) {
  T H[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) H[i] = F[i] - ((i % 4 == 0) ? T(1) : T(0));
  T U[9], s[3], e[3], V[9], Jm1;
  svd_from_h<T>(H, U, s, e, V, Jm1);
  if (!(s[0] > T(0) && s[1] > T(0) && s[2] > T(0))) return false;
  T eps[3] = {log1p(e[0]), log1p(e[1]), log1p(e[2])};
  const T mu = (T)mu_, lam = (T)lam_;
  const T tr = eps[0] + eps[1] + eps[2];
  const T d[3] = {eps[0] - tr / T(3), eps[1] - tr / T(3), eps[2] - tr / T(3)};
  const T dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (kind == MPML_VON_MISES) {
    const T lim = (T)(sqrt(2.0 / 3.0) * ys / (2.0 * mu_));
    if (dn <= lim) return false;
#pragma unroll
    for (int i = 0; i < 3; ++i) eps[i] = tr / T(3) + d[i] * (lim / dn);
  } else if (kind == MPML_DRUCKER_PRAGER) {
    if (tr > T(0)) {
      eps[0] = eps[1] = eps[2] = T(0);
    } else {
      const T dg = dn + (T(3) * lam + T(2) * mu) / (T(2) * mu) * tr * (T)alpha_;
      if (dg <= T(0)) return false;
#pragma unroll
      for (int i = 0; i < 3; ++i) eps[i] -= dg * d[i] / dn;
    }
  } else {
    return false;
  }
  const T ex[3] = {exp(eps[0]), exp(eps[1]), exp(eps[2])};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) F[3 * r + c] = U[3 * r] * ex[0] * V[3 * c] + U[3 * r + 1] * ex[1] * V[3 * c + 1] +
                                               U[3 * r + 2] * ex[2] * V[3 * c + 2];
  return true;
}


}  // namespace mpml
