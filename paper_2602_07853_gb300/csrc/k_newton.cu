// Algorithm 3 (Integrate, implicit branch) on the voxel hex mesh.
//
// Stretch reconstruction (Sec. 4.2, 4.3): per active centre and material,
//   tau = (V tau)/V, tau = Q diag(t) Q^T, s_i from the principal relation of
//   the material, S = Q diag(s) Q^T (FP64 on the device); stored as S - I.
// Incremental potential (Sec. 4.2, Algorithm 3 line 12):
//   Phi(v) = sum_i 1/2 m_i |v_i - vhat_i|^2 + sum_c sum_k V_ck psi_k(F_ck(v)),
//   F_ck(v) = (I + dt G_c(v)) S_ck, G_c(v) = sum_i v_i (x) grad w_ic.
// Newton prep (per Newton iteration): per cell the gradient contribution
//   dt V P S^T grad w_ic, and the PSD-projected tangent on D = G_c(p):
//   K_c = dt^2 sum_k V_ck L_S^T A_k^+ L_S, built from the analytic eigensystem
//   of isotropic energies in the signed-SVD frame (3x3 block of psi's Hessian
//   in the principal stretches, and the twist/flip pairs), eigenvalues
//   clamped at 0.  Stored as 45 packed floats per cell.
// HVP (the hot loop): y = M p + sum_c B_c^T K_c B_c p; one CTA per 8^3 brick,
//   the 9^3 node block of p staged once in shared memory, K_c streamed
//   coalesced, per-node sums of the 8 neighbouring cells formed in shared
//   memory, interior nodes stored once, brick-face nodes added atomically.
//   p^T H p = sum m |p|^2 + sum_c D^T K D is accumulated on the fly (FP64).
// Jacobi-PCG with FP64 dot products; scalars updated by the last block of
// each kernel (no host round trip inside an iteration).
#include "mpml_internal.cuh"

#include <utility>

namespace mpml {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of N doubles; thread 0 atomically adds them to dst[i]
template <int N>
__device__ __forceinline__ void block_add(double (&v)[N], double* const (&dst)[N]) {
  __shared__ double sh[N][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sh[i][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = lane < nw ? sh[i][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0 && s != 0.0) atomicAdd(dst[i], s);
    }
  }
}

// true in exactly one block: the last one to arrive (after a fence)
// (what must be visible before the ticket is written by thread 0 only)
__device__ __forceinline__ bool arrive_last(int* counter) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int t = atomicAdd(counter, 1);
    last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  return last != 0;
}

// block-wide sums of N doubles stored by thread 0 to part[blockIdx.x * N + i]
template <int N>
__device__ __forceinline__ void block_store(double (&v)[N], double* part) {
  __shared__ double sh[N][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sh[i][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = lane < nw ? sh[i][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[(int64_t)blockIdx.x * N + i] = s;
    }
  }
}

// sums of the per-block partials in a fixed order (deterministic); result in
// thread 0.  Called by every thread of the last block.
template <int N>
__device__ __forceinline__ void block_sum_parts(const double* part, int nblk, double (&out)[N]) {
  __shared__ double sh[N][32];
  double acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += __ldcg(&part[(int64_t)b * N + i]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = warp_sum(acc[i]);
    if (lane == 0) sh[i][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[i][w];
      out[i] = s;
    }
  }
}

__device__ __forceinline__ double vload(const double* p) { return *(volatile const double*)p; }

enum { CNT_FIN = 0, CNT_HVP = 1, CNT_A = 2, CNT_B = 3, CNT_MISC = 4 };

template <typename T>
__global__ void k_init_faces(const T* __restrict__ p, const T* __restrict__ m, T* q);

// ---------------------------------------------------------------------------
// stretch reconstruction (FP64)
// ---------------------------------------------------------------------------
// fixed-corotated principal stretches for a given J: 2 mu s (s - 1) = t - lam J (J - 1)
// (i2mu = 1 / (2 mu))
__device__ bool fc_sigma(double i2mu, double lam, const double t[3], double J, double s[3]) {
  double c = lam * J * (J - 1);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double disc = 0.25 + (t[i] - c) * i2mu;
    if (disc < -1e-12) ok = false;
    s[i] = 0.5 + sqrt(disc > 0 ? disc : 0);
  }
  return ok;
}
__device__ double fc_h(double i2mu, double lam, const double t[3], double J) {
  double s[3];
  fc_sigma(i2mu, lam, t, J, s);
  return s[0] * s[1] * s[2] - J;
}
__device__ double cbrt_signed(double z) { return z >= 0 ? cbrt(z) : -cbrt(-z); }

// principal stretches from principal Kirchhoff stresses; false if none admissible
__device__ bool invert_principal(int model, double mu, double lam, const double t[3], double s[3]) {
  if (model == MPML_WATER) {
    // Sec. "Water": pi = tr(tau)/3 = kappa J (J - 1), root J >= 1/2; S = J^(1/3) I
    const double kap = lam + 2.0 / 3.0 * mu;
    if (!(kap > 0)) return false;
    const double d = 1.0 + 4.0 * ((t[0] + t[1] + t[2]) / 3.0) / kap;
    if (!(d >= 0)) return false;
    const double c = cbrt(0.5 * (1.0 + sqrt(d)));
    s[0] = s[1] = s[2] = c;
    return true;
  }
  if (model == MPML_HENCKY) {
    // Sec. 4.3.1 closed form
    if (!(mu > 0 && lam > -2 * mu / 3)) return false;
    double tr = t[0] + t[1] + t[2];
    double ls = tr / (2 * mu + 3 * lam);
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = exp((t[i] - lam * ls) / (2 * mu));
    return true;
  }
  if (model == MPML_NEO_HOOKEAN) {
    // Sec. 4.3.2 / App. C; the one-real-root branch of Cardano uses u v = -p/3
    double kap = 2.0 / 3.0 * mu + lam;
    double alpha = (t[0] + t[1] + t[2]) / 3;
    double arg = 1 + 2 * alpha / kap;
    if (!(arg > 0)) return false;
    double J = sqrt(arg);
    double sc = mu * pow(J, -2.0 / 3.0);
    double dl[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dl[i] = (t[i] - alpha) / sc;
    double p = dl[0] * dl[1] + dl[1] * dl[2] + dl[2] * dl[0];
    double q = dl[0] * dl[1] * dl[2] - J * J;
    double disc = (q / 2) * (q / 2) + (p / 3) * (p / 3) * (p / 3);
    double m;
    if (disc >= 0) {
      double sd = sqrt(disc);
      double u = cbrt_signed(-q / 2 + (q <= 0 ? sd : -sd));
      double v = (u != 0) ? -p / (3 * u) : 0;
      m = u + v;
    } else {
      double r = 2 * sqrt(-p / 3);
      double a = 3 * q / (2 * p) * sqrt(-3 / p);
      a = a > 1 ? 1 : (a < -1 ? -1 : a);
      m = r * cos(acos(a) / 3);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double beta = m + dl[i];
      if (!(beta > 0)) return false;
      s[i] = sqrt(beta);
    }
    return true;
  }
  if (model == MPML_FIXED_COROTATED) {
    // library's inverse: unique root of prod_i s_i(J) = J on J >= 1/2
    if (!(mu > 0) || lam < 0) return false;
    const double i2mu = 0.5 / mu;
    if (lam == 0) return fc_sigma(i2mu, lam, t, 1.0, s);
    double tmin = fmin(t[0], fmin(t[1], t[2]));
    double d = 0.25 + (tmin + 0.5 * mu) / lam;
    if (d < 0) return false;
    double lo = 0.5, hi = 0.5 + sqrt(d);
    if (fc_h(i2mu, lam, t, lo) < 0 || fc_h(i2mu, lam, t, hi) > 0) return false;
    // starting point: Newton on h(J) = prod s_i(J) - J in FP32 (GB300's FP64 pipe
    // is slow), kept inside the bracket; the FP64 iteration below then needs a
    // couple of steps
    double J;
    {
      const float fl = (float)lam, fi = (float)i2mu, flo = (float)lo, fhi = (float)hi;
      const float ft[3] = {(float)t[0], (float)t[1], (float)t[2]};
      float Jf = __expf((ft[0] + ft[1] + ft[2]) / (float)(2 * mu + 3 * lam));
      if (!(Jf > flo && Jf < fhi)) Jf = 0.5f * (flo + fhi);
      for (int it = 0; it < 8; ++it) {
        const float cJ = fl * Jf * (Jf - 1.f), dc = fl * (2.f * Jf - 1.f);
        float sv[3], ir[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float disc = fmaxf(0.25f + (ft[i] - cJ) * fi, 1e-30f);
          ir[i] = rsqrtf(disc);
          sv[i] = 0.5f + disc * ir[i];
        }
        const float h = sv[0] * sv[1] * sv[2] - Jf;
        // d s_i / dJ = -dc i2mu / (2 sqrt(disc_i))
        const float dh = -0.5f * dc * fi * (ir[0] * sv[1] * sv[2] + ir[1] * sv[0] * sv[2] + ir[2] * sv[0] * sv[1]) - 1.f;
        if (!(dh < 0.f)) break;
        const float Jn = Jf - h / dh;
        if (!(Jn > flo && Jn < fhi)) break;
        const bool small = fabsf(Jn - Jf) <= 2e-6f * Jf;
        Jf = Jn;
        if (small) break;
      }
      J = (double)Jf;
      if (!(J > lo && J < hi)) J = 0.5 * (lo + hi);
    }
    // safeguarded Newton in FP64 (decreasing h on the bracket): a step that
    // leaves the bracket is replaced by bisection
    for (int it = 0; it < 100; ++it) {
      const double cJ = lam * J * (J - 1), dc = lam * (2 * J - 1);
      double sv[3], ir[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double disc = 0.25 + (t[i] - cJ) * i2mu;
        if (disc > 0) {
          ir[i] = rsqrt(disc);
          sv[i] = 0.5 + disc * ir[i];
        } else {
          ir[i] = 0;
          sv[i] = 0.5;
        }
      }
      const double prod = sv[0] * sv[1] * sv[2];
      const double h = prod - J;
      if (h > 0) lo = J; else hi = J;
      if (h == 0) break;
      const double dh = -0.5 * dc * i2mu * (ir[0] * sv[1] * sv[2] + ir[1] * sv[0] * sv[2] + ir[2] * sv[0] * sv[1]) - 1;
      double Jn = (dh < 0) ? J - h / dh : 0.5 * (lo + hi);
      if (!(Jn > lo && Jn < hi)) Jn = 0.5 * (lo + hi);
      if (fabs(Jn - J) <= 4e-16 * J || hi - lo <= 2e-16 * hi) {
        J = Jn;
        break;
      }
      J = Jn;
    }
    return fc_sigma(i2mu, lam, t, J, s);
  }
  return false;
}

struct SolveInfo {
  double dt, dx;
  int nm, nf;
  MatParams<double> mat[MPML_MAX_MATS];
  int b9;  // the base is the general 9-number one (fixed-point plastic solve)
  int plastic[MPML_MAX_MATS];
  double ys[MPML_MAX_MATS], alpha[MPML_MAX_MATS];
};

template <typename T>
__global__ void __launch_bounds__(256) k_stretch(const int* __restrict__ cblist, const uint8_t* __restrict__ cflag,
                                                 const T* __restrict__ acc, SolveInfo si, double* __restrict__ cs,
                                                 int* status) {
  const int id = cblist[blockIdx.x];
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    if (!cflag[(int64_t)id * BV + l]) continue;
    for (int k = 0; k < si.nm; ++k) {
      double* so = cs + ((int64_t)id * si.nm + k) * 6 * BV + l;
      const T* a = acc + (int64_t)id * si.nf * BV + l;
      const double V = (double)a[acc_V(k) * BV];
      if (V == 0.0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) so[q * BV] = 0.0;
        continue;
      }
      double tau[9];
      const int ra[6] = {0, 1, 2, 0, 0, 1}, rb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        double tq = (double)a[(acc_tau(k) + q) * BV] / V;
        tau[3 * ra[q] + rb[q]] = tau[3 * rb[q] + ra[q]] = tq;
      }
      if (si.mat[k].model == MPML_HENCKY) {
        // Hencky inverts in closed form: eps = (tau - lam tr(eps) I) / (2 mu) with
        // tr(eps) = tr(tau) / (2 mu + 3 lam), and S - I = expm1(eps); at small strain
        // (every |eps_ij| <= 0.03) by the series to eps^9 / 9! (remainder below 1e-16 of
        // |eps|) instead of the eigen-decomposition
        const double mu = si.mat[k].mu, lam = si.mat[k].lam;
        const double i2m = 1.0 / (2.0 * mu), lt = lam * (tau[0] + tau[4] + tau[8]) / (2.0 * mu + 3.0 * lam);
        const Sym3<double> E = {(tau[0] - lt) * i2m, (tau[4] - lt) * i2m, (tau[8] - lt) * i2m,
                                tau[1] * i2m,        tau[2] * i2m,        tau[5] * i2m};
        const double mx = fmax(fmax(fmax(fabs(E.xx), fabs(E.yy)), fmax(fabs(E.zz), fabs(E.xy))),
                               fmax(fabs(E.xz), fabs(E.yz)));
        if (sizeof(T) == 4 && mu > 0.0 && mx <= 0.01) {
          // FP32 contexts, |eps| <= 0.03: E + E^2/2 in FP64 and the remainder E^3 (1/6 + E/24 +
          // E^2/120 + E^3/720 + E^4/5040) in FP32 (at most 1.5e-4 of S - I: its rounding stays
          // near 1e-11 of it)
          const Sym3<double> E2 = sym_mul(E, E);
          const Sym3<float> Ef = {(float)E.xx, (float)E.yy, (float)E.zz, (float)E.xy, (float)E.xz, (float)E.yz};
          const float cs[5] = {1.f / 6.f, 1.f / 24.f, 1.f / 120.f, 1.f / 720.f, 1.f / 5040.f};
          Sym3<float> Pf = {cs[4], cs[4], cs[4], 0.f, 0.f, 0.f};
#pragma unroll
          for (int kk = 3; kk >= 0; --kk) {
            Pf = sym_mul(Ef, Pf);
            Pf.xx += cs[kk];
            Pf.yy += cs[kk];
            Pf.zz += cs[kk];
          }
          const Sym3<float> R = sym_mul(sym_mul(sym_mul(Ef, Ef), Ef), Pf);
          so[0] = E.xx + 0.5 * E2.xx + (double)R.xx;
          so[BV] = E.yy + 0.5 * E2.yy + (double)R.yy;
          so[2 * BV] = E.zz + 0.5 * E2.zz + (double)R.zz;
          so[3 * BV] = E.xy + 0.5 * E2.xy + (double)R.xy;
          so[4 * BV] = E.xz + 0.5 * E2.xz + (double)R.xz;
          so[5 * BV] = E.yz + 0.5 * E2.yz + (double)R.yz;
          continue;
        }
        if (mu > 0.0 && mx <= 0.03) {
          Sym3<double> P = {1.0 + E.xx / 9.0, 1.0 + E.yy / 9.0, 1.0 + E.zz / 9.0, E.xy / 9.0, E.xz / 9.0, E.yz / 9.0};
#pragma unroll
          for (int kk = 8; kk >= 2; --kk) {
            const double ik = 1.0 / kk;
            const Sym3<double> EP = sym_mul(E, P);
            P = {1.0 + EP.xx * ik, 1.0 + EP.yy * ik, 1.0 + EP.zz * ik, EP.xy * ik, EP.xz * ik, EP.yz * ik};
          }
          const Sym3<double> Sm = sym_mul(E, P);
          so[0] = Sm.xx;
          so[BV] = Sm.yy;
          so[2 * BV] = Sm.zz;
          so[3 * BV] = Sm.xy;
          so[4 * BV] = Sm.xz;
          so[5 * BV] = Sm.yz;
          continue;
        }
      }
      double ev[3], Q[9], s[3];
      jacobi3_mixed(tau, ev, Q);
      if (!invert_principal(si.mat[k].model, si.mat[k].mu, si.mat[k].lam, ev, s)) {
        atomicOr(status, ST_STRETCH);
#pragma unroll
        for (int q = 0; q < 6; ++q) so[q * BV] = 0.0;
        continue;
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        double acc2 = 0;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) acc2 += Q[3 * ra[q] + kk] * (s[kk] - 1.0) * Q[3 * rb[q] + kk];
        so[q * BV] = acc2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// node-block staging: the 9^3 nodes of a cell brick (own 8^3 + upper halo)
// ---------------------------------------------------------------------------
template <typename S, typename A, typename B>
__device__ __forceinline__ void stage_nodes(int id, const int* __restrict__ nbr, const A* __restrict__ a,
                                            const B* __restrict__ b, double beta, S (*sv)[729]) {
  // sv[r][i] = a + beta * b (b may be null)
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    const int t = (nx < 8 && ny < 8 && nz < 8) ? id : __ldg(&nbr[id * NBR + nbr_index(nx >> 3, ny >> 3, nz >> 3)]);
    const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      S val = S(0);
      if (t >= 0) {
        const int64_t o = (int64_t)t * 3 * BV + r * BV + l;
        val = (S)a[o];
        if (b) val += (S)(beta * (double)b[o]);
      }
      sv[r][i] = val;
    }
  }
}

// same, with the brick's 27-entry neighbour row already in shared memory
template <typename S, typename A>
__device__ __forceinline__ void stage_nodes_sn(int id, const int* s_nbr, const A* __restrict__ a, S (*sv)[729]) {
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    const int t = (nx < 8 && ny < 8 && nz < 8) ? id : s_nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
    const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
    S v0 = S(0), v1 = S(0), v2 = S(0);
    if (t >= 0) {
      const int64_t o = (int64_t)t * 3 * BV + l;
      v0 = (S)a[o];
      v1 = (S)a[o + BV];
      v2 = (S)a[o + 2 * BV];
    }
    sv[0][i] = v0;
    sv[1][i] = v1;
    sv[2][i] = v2;
  }
}

__device__ __forceinline__ int node_of(int l, int o) {
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  return ((lz + ((o >> 2) & 1)) * 9 + (ly + ((o >> 1) & 1))) * 9 + (lx + (o & 1));
}

// D' = sum_o p_o (x) sgn_o (the 1/(4 dx) scale is folded into K)
template <typename T>
__device__ __forceinline__ void gather_D(int l, const T (*sv)[729], T D[9]) {
  // per component: the x differences and sums of the four corner pairs, then the
  // y and z combinations of those (17 additions instead of 24)
  const int i0 = node_of(l, 0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T c[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) c[o] = sv[a][i0 + ((o >> 2) & 1) * 81 + ((o >> 1) & 1) * 9 + (o & 1)];
    const T d0 = c[1] - c[0], d1 = c[3] - c[2], d2 = c[5] - c[4], d3 = c[7] - c[6];
    const T e0 = c[0] + c[1], e1 = c[2] + c[3], e2 = c[4] + c[5], e3 = c[6] + c[7];
    D[3 * a + 0] = (d0 + d1) + (d2 + d3);
    D[3 * a + 1] = (e1 - e0) + (e3 - e2);
    D[3 * a + 2] = (e2 + e3) - (e0 + e1);
  }
}

// ---------------------------------------------------------------------------
// Per-cell constitutive work.  The stress, gradient and energy are formed in
// FP64 (they decide where Newton stops and whether the line search accepts);
// the projected tangent K only sets the CG convergence rate and is built in
// the storage precision T from the FP64 decomposition.
// ---------------------------------------------------------------------------
template <typename T>
struct CellOut {
  double Q[9];  // dt V P S^T / (4 dx)   (gradient, node contribution = Q sgn)
  T K[45];      // dt^2 V L^T A+ L / (16 dx^2)
  // the same tangent as NQC numbers (single material): quaternion of U, W = S V,
  // the clamped 3x3 block, flip and twist moduli (layout at apply_cmp)
  T C[NQC];
  double psi;
  bool ok;
};

// unit quaternion (w, x, y, z) of a rotation matrix (row-major), Shepperd's method
template <typename T>
__device__ __forceinline__ void rot_to_quat(const T R[9], T q[4]) {
  const T tr = R[0] + R[4] + R[8];
  if (tr > 0) {
    const T s = T(2) * sqrt(tr + T(1));
    q[0] = T(0.25) * s;
    q[1] = (R[7] - R[5]) / s;
    q[2] = (R[2] - R[6]) / s;
    q[3] = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const T s = T(2) * sqrt(T(1) + R[0] - R[4] - R[8]);
    q[0] = (R[7] - R[5]) / s;
    q[1] = T(0.25) * s;
    q[2] = (R[1] + R[3]) / s;
    q[3] = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const T s = T(2) * sqrt(T(1) + R[4] - R[0] - R[8]);
    q[0] = (R[2] - R[6]) / s;
    q[1] = (R[1] + R[3]) / s;
    q[2] = T(0.25) * s;
    q[3] = (R[5] + R[7]) / s;
  } else {
    const T s = T(2) * sqrt(T(1) + R[8] - R[0] - R[4]);
    q[0] = (R[3] - R[1]) / s;
    q[1] = (R[2] + R[6]) / s;
    q[2] = (R[5] + R[7]) / s;
    q[3] = T(0.25) * s;
  }
  const T n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] /= n;
}


// F - I = dt G + s + dt G s with S = I + s (symmetric, packed xx yy zz xy xz yz)
// the base B - I (row-major) of slot k of a cell: the symmetric stretch S - I (6
// numbers) of the stretch step, or, during a fixed-point plastic solve, the
// general base (9 numbers) its projections leave
__device__ __forceinline__ void load_base(const double* __restrict__ cs, int b9, int64_t id, int nm, int k, int l,
                                          double bm[9]) {
  if (b9) {
#pragma unroll
    for (int q = 0; q < 9; ++q) bm[q] = cs[(((int64_t)id * nm + k) * 9 + q) * BV + l];
    return;
  }
  double s6[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) s6[q] = cs[(((int64_t)id * nm + k) * 6 + q) * BV + l];
  bm[0] = s6[0]; bm[1] = s6[3]; bm[2] = s6[4];
  bm[3] = s6[3]; bm[4] = s6[1]; bm[5] = s6[5];
  bm[6] = s6[4]; bm[7] = s6[5]; bm[8] = s6[2];
}

// H = (I + Gd)(I + bm) - I with bm = B - I
__device__ __forceinline__ void trial_h(const double Gd[9], const double bm[9], double sm[9], double H[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) sm[q] = bm[q];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double acc = Gd[3 * a + b] + sm[3 * a + b];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += Gd[3 * a + k] * sm[3 * k + b];
      H[3 * a + b] = acc;
    }
}

// Eigenvalues of a symmetric 3x3 matrix (row-major), closed form by the
// trigonometric solution of the characteristic cubic (FP64).
__device__ __forceinline__ void sym3_eigenvalues(const double A[9], double w[3]) {
  const double p1 = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
  const double q = (A[0] + A[4] + A[8]) / 3.0;
  const double d0 = A[0] - q, d1 = A[4] - q, d2 = A[8] - q;
  const double p2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1;
  if (!(p2 > 0.0)) {
    w[0] = w[1] = w[2] = q;
    return;
  }
  const double p = sqrt(p2 / 6.0), ip = 1.0 / p;
  const double b0 = d0 * ip, b1 = d1 * ip, b2 = d2 * ip, b01 = A[1] * ip, b02 = A[2] * ip, b12 = A[5] * ip;
  double r = 0.5 * (b0 * (b1 * b2 - b12 * b12) - b01 * (b01 * b2 - b12 * b02) + b02 * (b01 * b12 - b1 * b02));
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  w[0] = q + 2.0 * p * cos(phi);
  w[2] = q + 2.0 * p * cos(phi + 2.0943951023931954923);
  w[1] = 3.0 * q - w[0] - w[2];
}

// J - 1 of F = I + H from the invariants of H, without cancellation
__device__ __forceinline__ double jm1_of_h(const double H[9]) {
  const double trH = H[0] + H[4] + H[8];
  double trH2 = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) trH2 += H[3 * a + b] * H[3 * b + a];
  const double detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                      H[2] * (H[3] * H[7] - H[4] * H[6]);
  return trH + 0.5 * (trH * trH - trH2) + detH;
}

// L = log(b) of b = F F^T = I + E, E = H + H^T + H H^T, without an eigen-decomposition
// (log_spd_series; with mixed, for the FP64 stress of FP32 contexts, the split below at the
// smallest strains); false where some |E_ij| > 0.03 (the caller takes the eigen-decomposition)
__device__ bool hencky_log_b(const double H[9], Sym3<double>& L, bool mixed) {
  double e[6];
  const int I[6] = {0, 1, 2, 0, 0, 1}, Jx[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int a = I[q], b = Jx[q];
    double acc = H[3 * a + b] + H[3 * b + a];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc += H[3 * a + k] * H[3 * b + k];
    e[q] = acc;
  }
  const Sym3<double> E = {e[0], e[1], e[2], e[3], e[4], e[5]};
  const double mx = fmax(fmax(fmax(fabs(E.xx), fabs(E.yy)), fmax(fabs(E.zz), fabs(E.xy))), fmax(fabs(E.xz), fabs(E.yz)));
  if (mixed && mx <= 0.01) {
    // (FP32 contexts) |E| <= 0.03: log(I + E) = E - E^2/2 + R with the first two terms in FP64 and the
    // remainder R = E^3 (1/3 - E/4 + E^2/5 - E^3/6 + E^4/7) (next term below 1e-7 of R) in
    // FP32: R is at most 3e-4 of the logarithm, so its FP32 rounding stays below 1e-10 of it
    const Sym3<double> E2 = sym_mul(E, E);
    const Sym3<float> Ef = {(float)E.xx, (float)E.yy, (float)E.zz, (float)E.xy, (float)E.xz, (float)E.yz};
    const float cs[5] = {1.f / 3.f, -1.f / 4.f, 1.f / 5.f, -1.f / 6.f, 1.f / 7.f};
    Sym3<float> P = {cs[4], cs[4], cs[4], 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 3; k >= 0; --k) {
      P = sym_mul(Ef, P);
      P.xx += cs[k];
      P.yy += cs[k];
      P.zz += cs[k];
    }
    const Sym3<float> R = sym_mul(sym_mul(sym_mul(Ef, Ef), Ef), P);
    L = {E.xx - 0.5 * E2.xx + (double)R.xx, E.yy - 0.5 * E2.yy + (double)R.yy, E.zz - 0.5 * E2.zz + (double)R.zz,
         E.xy - 0.5 * E2.xy + (double)R.xy, E.xz - 0.5 * E2.xz + (double)R.xz, E.yz - 0.5 * E2.yz + (double)R.yz};
    return true;
  }
  return log_spd_series(E, L);
}

// Hencky energy from L = log(F F^T): mu/4 tr(L^2) + lam/8 (tr L)^2 (= mu |log s|^2 +
// lam/2 (sum log s)^2 over the singular values s)
__device__ __forceinline__ double hencky_psi(const MatParams<double>& M, const Sym3<double>& L) {
  const double tr = L.xx + L.yy + L.zz;
  const double tr2 = L.xx * L.xx + L.yy * L.yy + L.zz * L.zz + 2.0 * (L.xy * L.xy + L.xz * L.xz + L.yz * L.yz);
  return 0.25 * M.mu * tr2 + 0.125 * M.lam * tr * tr;
}

// Hencky P S^T of F = (I + dt G) B = I + H in FP64 without an SVD, at small strain:
// the Kirchhoff stress tau = mu L + lam/2 tr(L) I with L = log(F F^T), and P S^T =
// tau F^{-T} B^T = tau (I + dt G)^{-T}.  Returns false outside hencky_log_b's range
// or for J <= 0; psi is the energy by hencky_psi; mixed as for hencky_log_b.
// det(I + H) > 0 where hencky_log_b accepted H: there F F^T is within 0.1 of I, so |det F| is
// near 1 and its sign is safe in FP32
__device__ __forceinline__ bool det_positive_near_rotation(const double H[9]) {
  float f[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) f[q] = (float)H[q] + ((q % 4 == 0) ? 1.f : 0.f);
  return f[0] * (f[4] * f[8] - f[5] * f[7]) - f[1] * (f[3] * f[8] - f[5] * f[6]) + f[2] * (f[3] * f[7] - f[4] * f[6]) >
         0.f;
}

__device__ bool hencky_closed_form(const MatParams<double>& M, const double Gd[9], const double H[9], double PSt[9],
                                   double& psi, bool mixed) {
  Sym3<double> L;
  if (!hencky_log_b(H, L, mixed) || !det_positive_near_rotation(H)) return false;
  psi = hencky_psi(M, L);
  const double hl = 0.5 * M.lam * (L.xx + L.yy + L.zz);
  const double tau[9] = {M.mu * L.xx + hl, M.mu * L.xy, M.mu * L.xz, M.mu * L.xy, M.mu * L.yy + hl,
                         M.mu * L.yz, M.mu * L.xz, M.mu * L.yz, M.mu * L.zz + hl};
  const double a0 = 1.0 + Gd[0], a1 = Gd[1], a2 = Gd[2], a3 = Gd[3], a4 = 1.0 + Gd[4], a5 = Gd[5], a6 = Gd[6],
               a7 = Gd[7], a8 = 1.0 + Gd[8];
  const double cof[9] = {a4 * a8 - a5 * a7, a5 * a6 - a3 * a8, a3 * a7 - a4 * a6,
                         a2 * a7 - a1 * a8, a0 * a8 - a2 * a6, a1 * a6 - a0 * a7,
                         a1 * a5 - a2 * a4, a2 * a3 - a0 * a5, a0 * a4 - a1 * a3};
  const double idet = rcp_nr(a0 * cof[0] + a1 * cof[1] + a2 * cof[2]);  // det(I + dt G) near 1
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      PSt[3 * a + b] = (tau[3 * a] * cof[b] + tau[3 * a + 1] * cof[3 + b] + tau[3 * a + 2] * cof[6 + b]) * idet;
  return true;
}

// Split Neo-Hookean P S^T of F = (I + dt G)(I + s) = I + H in FP64 without an
// SVD: tau = mu J^{-2/3} dev(b) + kappa/2 (J^2 - 1) I with b - I = H + H^T +
// H H^T, and P S^T = tau (I + dt G)^{-T}.  Returns false for J <= 0.
__device__ bool nh_closed_form(const MatParams<double>& M, const double Gd[9], const double H[9], double PSt[9]) {
  const double Jm1 = jm1_of_h(H);
  if (!(Jm1 > -1.0)) return false;
  double B[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double acc = H[3 * a + b] + H[3 * b + a];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += H[3 * a + k] * H[3 * b + k];
      B[3 * a + b] = acc;
    }
  const double I1m3 = B[0] + B[4] + B[8];
  const double kap = 2.0 / 3.0 * M.mu + M.lam;
  const double cm1 = jpow_m23_m1(Jm1);  // J^{-2/3} - 1
  const double c = 1.0 + cm1;
  const double iso = 0.5 * kap * Jm1 * (2.0 + Jm1), mc = M.mu * c;
  double tau[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) tau[q] = mc * B[q];
  tau[0] += iso - mc * I1m3 / 3.0;
  tau[4] += iso - mc * I1m3 / 3.0;
  tau[8] += iso - mc * I1m3 / 3.0;
  // A = I + dt G; A^{-T} = cof(A) / det(A)
  const double a0 = 1.0 + Gd[0], a1 = Gd[1], a2 = Gd[2], a3 = Gd[3], a4 = 1.0 + Gd[4], a5 = Gd[5], a6 = Gd[6],
               a7 = Gd[7], a8 = 1.0 + Gd[8];
  double cof[9] = {a4 * a8 - a5 * a7, a5 * a6 - a3 * a8, a3 * a7 - a4 * a6,
                   a2 * a7 - a1 * a8, a0 * a8 - a2 * a6, a1 * a6 - a0 * a7,
                   a1 * a5 - a2 * a4, a2 * a3 - a0 * a5, a0 * a4 - a1 * a3};
  const double det = a0 * cof[0] + a1 * cof[1] + a2 * cof[2];
  const double idet = 1.0 / det;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      PSt[3 * a + b] = (tau[3 * a] * cof[b] + tau[3 * a + 1] * cof[3 + b] + tau[3 * a + 2] * cof[6 + b]) * idet;
  return true;
}

// Fixed-corotated P S^T of F = (I + dt G)(I + s) = I + H in FP64 without an
// SVD: the rotation R of the polar decomposition by Newton's iteration
// X <- (X + X^-T) / 2 from X = F (quadratic convergence; F is near a
// rotation), then P S^T = 2 mu (F - R) S + lam (J - 1) J (I + dt G)^{-T}.
// Returns false for J <= 0 (inverted cells keep the signed-SVD path).
__device__ bool fc_closed_form(const MatParams<double>& M, const double Gd[9], const double H[9], const double sm[9],
                               double PSt[9]) {
  const double Jm1 = jm1_of_h(H);
  if (!(Jm1 > -1.0)) return false;
  double X[9] = {1.0 + H[0], H[1], H[2], H[3], 1.0 + H[4], H[5], H[6], H[7], 1.0 + H[8]};
  for (int it = 0; it < 12; ++it) {
    const double c0 = X[4] * X[8] - X[5] * X[7], c1 = X[5] * X[6] - X[3] * X[8], c2 = X[3] * X[7] - X[4] * X[6];
    const double c3 = X[2] * X[7] - X[1] * X[8], c4 = X[0] * X[8] - X[2] * X[6], c5 = X[1] * X[6] - X[0] * X[7];
    const double c6 = X[1] * X[5] - X[2] * X[4], c7 = X[2] * X[3] - X[0] * X[5], c8 = X[0] * X[4] - X[1] * X[3];
    const double idet = 1.0 / (X[0] * c0 + X[1] * c1 + X[2] * c2);
    const double cof[9] = {c0, c1, c2, c3, c4, c5, c6, c7, c8};  // X^{-T} = cof / det
    double diff = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double xn = 0.5 * (X[q] + cof[q] * idet);
      diff = fmax(diff, fabs(xn - X[q]));
      X[q] = xn;
    }
    if (diff <= 4e-16) break;
  }
  // F - R with F = I + H
  double FR[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) FR[q] = ((q % 4 == 0) ? 1.0 : 0.0) + H[q] - X[q];
  const double J = 1.0 + Jm1;
  const double kJ = M.lam * Jm1 * J;
  const double a0 = 1.0 + Gd[0], a1 = Gd[1], a2 = Gd[2], a3 = Gd[3], a4 = 1.0 + Gd[4], a5 = Gd[5], a6 = Gd[6],
               a7 = Gd[7], a8 = 1.0 + Gd[8];
  const double cof[9] = {a4 * a8 - a5 * a7, a5 * a6 - a3 * a8, a3 * a7 - a4 * a6,
                         a2 * a7 - a1 * a8, a0 * a8 - a2 * a6, a1 * a6 - a0 * a7,
                         a1 * a5 - a2 * a4, a2 * a3 - a0 * a5, a0 * a4 - a1 * a3};
  const double idet = 1.0 / (a0 * cof[0] + a1 * cof[1] + a2 * cof[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // (F - R) B^T with B = I + sm (= (F - R) S for the stretch step's symmetric S)
      double fs = FR[3 * a + b];
#pragma unroll
      for (int k = 0; k < 3; ++k) fs += FR[3 * a + k] * sm[3 * b + k];  // (F - R) B^T
      PSt[3 * a + b] = 2.0 * M.mu * fs + kJ * cof[3 * a + b] * idet;
    }
  return true;
}

// Energy density of F = I + H (FP64) from the eigenvalues of F^T F - I only;
// returns false when it is undefined.  Fixed-corotated with J <= 0 (an inverted
// cell, where the signed SVD is needed) reports `need_svd`.
__device__ bool psi_from_h(const MatParams<double>& M, const double H[9], double& psi, bool& need_svd,
                           bool mixed = false) {
  need_svd = false;
  if (M.model == MPML_HENCKY) {
    Sym3<double> L;
    if (hencky_log_b(H, L, mixed) && det_positive_near_rotation(H)) {  // small strain (as hencky_closed_form)
      psi = hencky_psi(M, L);
      return true;
    }
  }
  const double Jm1 = jm1_of_h(H);
  if (M.model == MPML_NEO_HOOKEAN) {
    if (!(Jm1 > -1.0)) return false;
    const double trH = H[0] + H[4] + H[8];
    double hF2 = 0, trH2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        hF2 += H[3 * a + b] * H[3 * a + b];
        trH2 += H[3 * a + b] * H[3 * b + a];
      }
    const double detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                        H[2] * (H[3] * H[7] - H[4] * H[6]);
    const double I1m3 = 2.0 * trH + hF2;
    // I1 - 3 - 2 (J - 1) with J - 1 = tr H + ((tr H)^2 - tr H^2)/2 + det H: second order only
    const double b2 = hF2 + trH2 - trH * trH - 2.0 * detH;
    psi = nh_psi(M.mu, 2.0 / 3.0 * M.mu + M.lam, Jm1, I1m3, b2);
    return true;
  }
  if (M.model == MPML_FIXED_COROTATED && !(Jm1 > -1.0)) {
    need_svd = true;
    return true;
  }
  if (M.model == MPML_WATER) {
    if (!(Jm1 > -1.0)) return false;
    psi = 0.5 * (M.lam + 2.0 / 3.0 * M.mu) * Jm1 * Jm1;
    return true;
  }
  double E[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double acc = H[3 * a + b] + H[3 * b + a];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += H[3 * k + a] * H[3 * k + b];
      E[3 * a + b] = acc;
    }
  double w[3], e[3];
  sym3_eigenvalues(E, w);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double li = w[i] > -1.0 ? w[i] : -1.0;
    e[i] = li / (1.0 + sqrt(1.0 + li));  // singular value - 1
  }
  if (M.model == MPML_FIXED_COROTATED) {
    psi = M.mu * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) + 0.5 * M.lam * Jm1 * Jm1;
    return true;
  }
  // Hencky
  if (!(Jm1 > -1.0) || !(e[0] > -1.0 && e[1] > -1.0 && e[2] > -1.0)) return false;
  const double l0 = log1p(e[0]), l1 = log1p(e[1]), l2 = log1p(e[2]), tr = l0 + l1 + l2;
  psi = M.mu * (l0 * l0 + l1 * l1 + l2 * l2) + 0.5 * M.lam * tr * tr;
  return true;
}

// The projected tangent of one cell in the storage precision T from the signed
// SVD (U, V, W = S V) and the isotropic eigen-data of psi: the 45-number
// packed form and the NQC-number compressed form (layout at apply_cmp).
// want_k: 1 the packed 45-number form, 2 also the compressed form (the packed one
// gives the Jacobi diagonal in both cases).
template <typename T>
__device__ void build_tangent(const T Ut[9], const T Vt[9], const T Wt[9], T d2[9], const T pp[3], const T pm[3], T kv,
                              const double bm[9], int want_k, CellOut<T>& out) {
  // diagonal block: eigen-decomposition of d2, clamp
  T ev[3], Qd[9];
  jacobi3<T>(d2, ev, Qd);
  if (want_k == 2) {
    // compressed record (valid for single-material cells; bm = B - I, the
    // stretch step's base S - I in elastic contexts)
    double Ud[9], q[4];
#pragma unroll
    for (int i = 0; i < 9; ++i) Ud[i] = (double)Ut[i];
    rot_to_quat<double>(Ud, q);
#pragma unroll
    for (int i = 0; i < 4; ++i) out.C[i] = (T)q[i];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double w = (double)Vt[3 * a + b];
#pragma unroll
        for (int k = 0; k < 3; ++k) w += bm[3 * a + k] * (double)Vt[3 * k + b];
        out.C[4 + 3 * a + b] = (T)w;
      }
    double lp[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) lp[m] = ev[m] > T(0) ? (double)kv * (double)ev[m] : 0.0;
    const int AI[6] = {0, 1, 2, 0, 0, 1}, AJ[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m) acc += (double)Qd[3 * AI[e] + m] * lp[m] * (double)Qd[3 * AJ[e] + m];
      out.C[13 + e] = (T)acc;
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      out.C[19 + p] = pp[p] > T(0) ? T(0.5) * kv * pp[p] : T(0);
      out.C[22 + p] = pm[p] > T(0) ? T(0.5) * kv * pm[p] : T(0);
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    if (!(ev[m] > T(0))) continue;
    T d[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T acc = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) acc += Qd[3 * i + m] * Ut[3 * a + i] * Wt[3 * b + i];
        d[3 * a + b] = acc;
      }
    const T lam = kv * ev[m];
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int cc = r; cc < 9; ++cc) out.K[k45(r, cc)] += lam * d[r] * d[cc];
  }
  // twist (pm, E_ij - E_ji) and flip (pp, E_ij + E_ji) pairs
  const T rs2 = T(0.70710678118654752440);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int i = pair_i(p), j = pair_j(p);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const T lamv = sg == 0 ? pp[p] : pm[p];
      if (!(lamv > T(0))) continue;
      const T sgn = sg == 0 ? T(1) : T(-1);
      T d[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          d[3 * a + b] = rs2 * (Ut[3 * a + i] * Wt[3 * b + j] + sgn * Ut[3 * a + j] * Wt[3 * b + i]);
      const T lam = kv * lamv;
#pragma unroll
      for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int cc = r; cc < 9; ++cc) out.K[k45(r, cc)] += lam * d[r] * d[cc];
    }
  }
}


template <typename T>
__device__ void cell_material(const MatParams<double>& M, double V, const double Gd[9] /* dt*G */,
                              const double bm[9] /* B - I */, double kq, double kk, int want_k, CellOut<T>& out,
                              bool want_psi = true) {
  double sm[9], H[9];
  trial_h(Gd, bm, sm, H);
  if constexpr (sizeof(T) == 4) {
    double PSt[9], psi_h = 0.0;
    const bool hencky = M.model == MPML_HENCKY && hencky_closed_form(M, Gd, H, PSt, psi_h, true);
    const bool closed = hencky || (M.model == MPML_NEO_HOOKEAN && nh_closed_form(M, Gd, H, PSt)) ||
                        (M.model == MPML_FIXED_COROTATED && fc_closed_form(M, Gd, H, sm, PSt));
    if (M.model == MPML_NEO_HOOKEAN && !closed) {
      out.ok = false;
      return;
    }
    if (closed) {
      // stress and energy without an FP64 SVD; the tangent from an FP32 SVD.  The
      // energy is skipped when the caller has it already (the accepted line-search
      // value at this iterate): its FP64 transcendentals dominate this kernel.
      if (want_psi) {
        double psi = psi_h;  // Hencky: from the same L (psi_from_h's small-strain branch)
        bool need_svd;
        if (!hencky && (!psi_from_h(M, H, psi, need_svd, true) || need_svd)) {
          out.ok = false;
          return;
        }
        out.psi += V * psi;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) out.Q[q] += kq * V * PSt[q];
      if (!want_k) return;
      float Hf[9], Uf[9], sf[3], ef[3], Vf[9], Jm1f, Wf[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) Hf[q] = (float)H[q];
      svd_from_h<float>(Hf, Uf, sf, ef, Vf, Jm1f);
      MatParams<float> Mf;
      Mf.model = M.model;
      Mf.mu = (float)M.mu;
      Mf.lam = (float)M.lam;
      Spec<float> spf;
      if (!spectral<float>(Mf, sf, ef, Jm1f, spf)) {
        out.ok = false;
        return;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          float acc = Vf[3 * a + b];
#pragma unroll
          for (int k = 0; k < 3; ++k) acc += (float)sm[3 * a + k] * Vf[3 * k + b];
          Wf[3 * a + b] = acc;
        }
      build_tangent<T>(Uf, Vf, Wf, spf.d2, spf.pp, spf.pm, (float)(kk * V), bm, want_k, out);
      return;
    }
  }
  // FP32 contexts: the FP64 stress and energy to about 1e-14 (LITE: jacobi3_lite, Newton-
  // refined reciprocals, series logarithms; the FP64 pipe bounds this kernel), the tangent
  // moduli, stored in FP32, evaluated in FP32
  constexpr bool LITE = sizeof(T) == 4;
  double U[9], s[3], e[3], Vv[9], Jm1;
  svd_from_h<double, LITE>(H, U, s, e, Vv, Jm1);
  Spec<double> sp;
  if (!spectral<double, LITE ? 5 : 3>(M, s, e, Jm1, sp)) {
    out.ok = false;
    return;
  }
  if (want_psi) {
    // the energy by the same formula as the line search (k_energy_cells)
    double psi;
    bool need_svd;
    if (!psi_from_h(M, H, psi, need_svd, sizeof(T) == 4)) {
      out.ok = false;
      return;
    }
    out.psi += V * (need_svd ? sp.psi : psi);
  }
  // W = S V = V + s V
  double W[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double acc = Vv[3 * a + b];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += sm[3 * a + k] * Vv[3 * k + b];
      W[3 * a + b] = acc;
    }
  // Q += kq V U diag(d1) W^T   (P S^T = U diag(d1) V^T S = U diag(d1) W^T)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += U[3 * a + k] * sp.d1[k] * W[3 * b + k];
      out.Q[3 * a + b] += kq * V * acc;
    }
  if (!want_k) return;
  T Ut[9], Wt[9], Vt[9], d2[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    Ut[i] = (T)U[i];
    Wt[i] = (T)W[i];
    Vt[i] = (T)Vv[i];
  }
  T pp[3], pm[3];
  if constexpr (sizeof(T) == 4) {
    MatParams<float> Mf;
    Mf.model = M.model;
    Mf.mu = (float)M.mu;
    Mf.lam = (float)M.lam;
    const float sf[3] = {(float)s[0], (float)s[1], (float)s[2]}, ef[3] = {(float)e[0], (float)e[1], (float)e[2]};
    Spec<float> spf;
    if (!spectral<float, 2>(Mf, sf, ef, (float)Jm1, spf)) {
      out.ok = false;
      return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) d2[i] = spf.d2[i];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      pp[p] = spf.pp[p];
      pm[p] = spf.pm[p];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) d2[i] = (T)sp.d2[i];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      pp[p] = (T)sp.pp[p];
      pm[p] = (T)sp.pm[p];
    }
  }
  build_tangent<T>(Ut, Vt, Wt, d2, pp, pm, (T)(kk * V), bm, want_k, out);
}

// node init: g = m (v - vhat) (FP64), diag = m, inertia energy (all bricks, 512 thr)
template <typename T>
__global__ void __launch_bounds__(512) k_node_init(const uint8_t* __restrict__ nflag, const T* __restrict__ m,
                                                   const double* __restrict__ v, const double* __restrict__ vhat,
                                                   double* g, T* diag, DevScalars* sc, int nb) {
  const int l = threadIdx.x;
  double ein = 0, mv2 = 0;
  // several bricks per block: the FP64 block sums (slow on this part) once per block
  for (int id = blockIdx.x; id < nb; id += gridDim.x) {
    const int64_t slot = (int64_t)id * BV + l;
    const bool dof = nflag[slot] & NF_DOF;
    const bool free_ = dof && !(nflag[slot] & NF_FIXED);
    const double mi = dof ? (double)m[slot] : 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int64_t o = (int64_t)id * 3 * BV + r * BV + l;
      double d = dof ? v[o] - vhat[o] : 0.0;
      g[o] = mi * d;
      diag[o] = (T)mi;
      ein += 0.5 * mi * d * d;
      if (free_) mv2 += (mi * vhat[o]) * (mi * vhat[o]);
    }
  }
  double vals[2] = {ein, mv2};
  double* const dst[2] = {&sc->phi_in, &sc->mv2};
  block_add<2>(vals, dst);
}

// pointer to a node slot addressed from a cell brick (local node 0..8 per axis)
template <typename T>
__device__ __forceinline__ T* node_ptr(T* base, int id, const int* __restrict__ nbr, int nx, int ny, int nz, int r) {
  const int t = (nx < 8 && ny < 8 && nz < 8) ? id : __ldg(&nbr[id * NBR + nbr_index(nx >> 3, ny >> 3, nz >> 3)]);
  if (t < 0) return nullptr;
  return base + (int64_t)t * 3 * BV + r * BV + (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
}

// Newton prep over cell bricks (256 threads, 2 cells each).
template <typename T>
__global__ void __launch_bounds__(256, 1) k_prep(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                 const uint8_t* __restrict__ cflag, const T* __restrict__ acc,
                                                 const double* __restrict__ cs, const double* __restrict__ v,
                                                 SolveInfo si, int want_k, T* __restrict__ K, double* g, T* diag,
                                                 DevScalars* sc, int* status, int want_psi, int trial) {
  __shared__ double sv[3][729];
  const int id = cblist[blockIdx.x];
  stage_nodes<double, double, double>(id, nbr, v, nullptr, 0.0, sv);
  __syncthreads();
  const double gw = 0.25 / si.dx;
  const double kq = si.dt * 0.25 / si.dx;
  const double kk = si.dt * si.dt / (16.0 * si.dx * si.dx);
  double esum = 0;
  int bad = 0;
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    if (!cflag[(int64_t)id * BV + l]) continue;
    double D[9];
    gather_D<double>(l, sv, D);
    double Gd[9];
    const double sgd = si.dt * gw;
#pragma unroll
    for (int q = 0; q < 9; ++q) Gd[q] = sgd * D[q];
    CellOut<T> co;
#pragma unroll
    for (int q = 0; q < 9; ++q) co.Q[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 45; ++q) co.K[q] = T(0);
#pragma unroll
    for (int q = 0; q < NQC; ++q) co.C[q] = T(0);
    co.psi = 0;
    co.ok = true;
    for (int k = 0; k < si.nm; ++k) {
      const double V = (double)acc[((int64_t)id * si.nf + acc_V(k)) * BV + l];
      if (V == 0.0) continue;
      double bm[9];
      load_base(cs, si.b9, id, si.nm, k, l, bm);
      cell_material<T>(si.mat[k], V, Gd, bm, kq, kk, want_k, co, want_psi != 0);
    }
    if (!co.ok) {
      bad = 1;
      continue;
    }
    esum += co.psi;
    if (want_k == 2) {  // compressed tangent (single material, FP32)
      T* Kd = K + (int64_t)id * NQC * BV + l;
#pragma unroll
      for (int q = 0; q < NQC; ++q) Kd[q * BV] = co.C[q];
    } else if (want_k) {
      T* Kd = K + (int64_t)id * 45 * BV + l;
#pragma unroll
      for (int q = 0; q < 45; ++q) Kd[q * BV] = co.K[q];
    }
    // scatter gradient (FP64) and Jacobi diagonal to the 8 corners; the corner values
    // +-Q0 +-Q1 +-Q2 are four sums and their negatives
    double qs[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double sp = co.Q[3 * a] + co.Q[3 * a + 1], sm = co.Q[3 * a] - co.Q[3 * a + 1];
      qs[a][0] = sp + co.Q[3 * a + 2];  // corner o = 7 (+,+,+); o = 0 is its negative
      qs[a][1] = sm + co.Q[3 * a + 2];  // o = 5 (+,-,+); o = 2 negated
      qs[a][2] = sm - co.Q[3 * a + 2];  // o = 1 (+,-,-); o = 6 negated
      qs[a][3] = sp - co.Q[3 * a + 2];  // o = 3 (+,+,-); o = 4 negated
    }
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const double sg[3] = {(o & 1) ? 1.0 : -1.0, (o & 2) ? 1.0 : -1.0, (o & 4) ? 1.0 : -1.0};
      const int nx = lx + (o & 1), ny = ly + ((o >> 1) & 1), nz = lz + ((o >> 2) & 1);
      // corner o's sign pattern -> (which sum, sign): o = 7,5,1,3 direct; 0,2,6,4 negated
      constexpr int WHICH[8] = {0, 2, 1, 3, 3, 1, 2, 0};
      const bool neg = (o == 0 || o == 2 || o == 6 || o == 4);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double* gp = node_ptr(g, id, nbr, nx, ny, nz, a);
        if (!gp) continue;
        const double gv = neg ? -qs[a][WHICH[o]] : qs[a][WHICH[o]];
        atomicAdd(gp, gv);
        if (want_k) {
          T dv = 0;
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              const int r = 3 * a + b, cc = 3 * a + bb;
              dv += co.K[r <= cc ? k45(r, cc) : k45(cc, r)] * (T)sg[b] * (T)sg[bb];
            }
          atomicAdd(node_ptr(diag, id, nbr, nx, ny, nz, a), dv);
        }
      }
    }
  }
  // a trial iterate of the line search reports cells where the energy is undefined as
  // infeasible (the step is rejected); elsewhere they are an error
  if (bad) {
    if (trial)
      atomicAdd(&sc->infeasible, 1);
    else
      atomicOr(status, ST_NONFINITE);
  }
  double vals[1] = {esum};
  double* const dst[1] = {&sc->phi_el};
  block_add<1>(vals, dst);
}

// finalize the gradient (mask), Jacobi inverse, |g|^2 and the CG start:
// x = 0, r = -g, z = D^-1 r, p = z, q(face) = 0.
// mode 0: mask, inverse and |g|^2 only; 1: all; 2: the CG start only (g masked and the
// diagonal inverted by an earlier mode-0 launch).
template <typename T>
__global__ void __launch_bounds__(512) k_finalize(const uint8_t* __restrict__ nflag, const T* __restrict__ m,
                                                  double* g, T* diag_dinv, T* x, T* r, T* p, T* q, int mode,
                                                  double rtol2, int cg_max, DevScalars* sc, double* part, int nb) {
  const int l = threadIdx.x;
  const bool face = (l & 7) == 0 || ((l >> 3) & 7) == 0 || (l >> 6) == 0;
  double gg = 0, rz = 0, rr = 0, pmp = 0, nfr = 0;
  // several bricks per block: the FP64 block sums (slow on this part) once per block
  for (int id = blockIdx.x; id < nb; id += gridDim.x) {
  const int64_t slot = (int64_t)id * BV + l;
  const uint8_t f = nflag[slot];
  const bool free_ = (f & NF_DOF) && !(f & NF_FIXED);
  nfr += free_ ? 3.0 : 0.0;
  const T mi = free_ ? m[slot] : T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    double gv = free_ ? g[o] : 0.0;
    T di;
    if (mode == 2) {
      di = free_ ? diag_dinv[o] : T(0);
    } else {
      g[o] = gv;
      di = free_ ? T(1) / diag_dinv[o] : T(0);
      diag_dinv[o] = di;
    }
    gg += gv * gv;
    if (mode != 0) {
      T rv = (T)(-gv), zv = di * rv;
      x[o] = T(0);
      r[o] = rv;
      p[o] = zv;
      if (face) q[o] = mi * zv;  // mass term of brick-face nodes (HVP adds the rest)
      rz += (double)rv * (double)zv;
      rr += (double)rv * (double)rv;
      pmp += (double)mi * (double)zv * (double)zv;
    }
  }
  }
  double vals[5] = {gg, rz, rr, pmp, nfr};
  block_store<5>(vals, part);
  if (arrive_last(&sc->counter[CNT_FIN])) {
    double tot[5];
    block_sum_parts<5>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    sc->gg = tot[0];
    sc->rz = tot[1];
    sc->rzj = tot[1];
    sc->rr0 = tot[2];
    sc->pMp = tot[3];
    sc->nfree = tot[4];
    double rr0 = tot[2];
    sc->tol2 = rtol2 * rr0;
    sc->done = (rr0 == 0.0) ? 1 : 0;
    sc->iters = 0;
    sc->cg_max = cg_max;
    sc->rr = 0;
    sc->rr_last = rr0;
    sc->rz_new = 0;
    sc->pKp = 0;
    sc->counter[CNT_FIN] = 0;
  }
}

// ---------------------------------------------------------------------------
// device-side launch timing (globaltimer): first block start .. last block end
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void prof_begin(DevProf* pf) {
  if (pf && threadIdx.x == 0) atomicMin(&pf->t0, gtimer());
}
__device__ __forceinline__ void prof_end(DevProf* pf) {
  if (!pf) return;
  if (arrive_last(&pf->counter) && threadIdx.x == 0) {
    const unsigned long long t1 = gtimer(), t0 = *(volatile unsigned long long*)&pf->t0;
    pf->ns += t1 - t0;
    pf->count += 1;
    pf->t0 = ~0ull;
    pf->counter = 0;
  }
}

// ---------------------------------------------------------------------------
// The regions between the persistent-solver markers (here and in mpml_internal.cuh)
// are hashed by bench.py to tie an ncu capture to the solver version it measured.
// [persistent-solver source: begin]
// TMA bulk copy + mbarrier helpers (sm_90+ PTX, used on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> shared, completion counted on the mbarrier (16-byte
// aligned addresses, size a multiple of 16)
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false on timeout (the caller flags ST_TIMEOUT)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 24); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// [persistent-solver source: end]

// Standalone FP32 HVP of one cell brick per CTA on the compressed tangent (the
// 45-number form runs in k_hvp_col), read straight from global memory (read-only during the kernel, coalesced per tangent entry; measured faster
// than a TMA copy into shared memory: 27 KB of shared memory per CTA lets
// three CTAs share an SM with more loads in flight).
constexpr size_t HVP_G_SMEM = sizeof(float) * 3 * 729 + 4 + sizeof(float) * 9 * BV;
template <bool CMP>
__global__ void __launch_bounds__(256, 3) k_hvp_glob(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                     const uint8_t* __restrict__ cflag, const float* __restrict__ K,
                                                     const float* __restrict__ p, const float* __restrict__ m,
                                                     float* q, DevScalars* sc, int finalize, DevProf* pf,
                                                     int* status, double* part) {
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = finalize ? sc->done : 0;
  __syncthreads();
  if (s_done) return;
  prof_begin(pf);
  extern __shared__ __align__(128) unsigned char gsm[];
  float (*sv)[729] = reinterpret_cast<float (*)[729]>(gsm);
  float (*skd)[BV] = reinterpret_cast<float (*)[BV]>(gsm + sizeof(float) * 3 * 729 + 4);
  __shared__ int s_nbr[NBR];
  const int id = cblist[blockIdx.x];
  if (threadIdx.x < NBR) s_nbr[threadIdx.x] = nbr[id * NBR + threadIdx.x];
  __syncthreads();
  stage_nodes_sn<float, float>(id, s_nbr, p, sv);
  __syncthreads();
  float pkp = 0.f;
  const float* Kb = K + (int64_t)id * (CMP ? NQC : 45) * BV;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = threadIdx.x + h * 256;
    float KD[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) KD[r] = 0.f;
    if (cflag[(int64_t)id * BV + l]) {
      float D[9];
      gather_D<float>(l, sv, D);
      if (CMP) {
        float c[NQC];
#pragma unroll
        for (int qq = 0; qq < NQC; ++qq) c[qq] = ld_stream(Kb + qq * BV + l);
        apply_cmp(c, D, KD);
      } else
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        KD[r] += ld_stream(Kb + k45(r, r) * BV + l) * D[r];
#pragma unroll
        for (int cc = r + 1; cc < 9; ++cc) {
          const float kv = ld_stream(Kb + k45(r, cc) * BV + l);
          KD[r] += kv * D[cc];
          KD[cc] += kv * D[r];
        }
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) pkp += D[r] * KD[r];
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) skd[r][l] = KD[r];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    float y[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int cx = nx - (o & 1), cy = ny - ((o >> 1) & 1), cz = nz - ((o >> 2) & 1);
      if (cx < 0 || cy < 0 || cz < 0 || cx > 7 || cy > 7 || cz > 7) continue;
      const int c = (cz * 8 + cy) * 8 + cx;
      const float s0 = (o & 1) ? 1.f : -1.f, s1 = (o & 2) ? 1.f : -1.f, s2 = (o & 4) ? 1.f : -1.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] += skd[3 * a][c] * s0 + skd[3 * a + 1][c] * s1 + skd[3 * a + 2][c] * s2;
    }
    const bool own = nx < 8 && ny < 8 && nz < 8;
    const bool excl = nx >= 1 && nx <= 7 && ny >= 1 && ny <= 7 && nz >= 1 && nz <= 7;
    if (own) {
      const int l = nz * 64 + ny * 8 + nx;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float* dst = q + (int64_t)id * 3 * BV + a * BV + l;
        if (excl) *dst = y[a] + m[(int64_t)id * BV + l] * sv[a][i];
        else if (y[a] != 0.f) atomicAdd(dst, y[a]);
      }
    } else {
      const int t = s_nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
      if (t < 0) continue;
      const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (y[a] != 0.f) atomicAdd(q + (int64_t)t * 3 * BV + a * BV + l, y[a]);
    }
  }
  double vals[1] = {(double)pkp};
  block_store<1>(vals, part);
  if (finalize && arrive_last(&sc->counter[CNT_HVP])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    double pq = sc->pMp + tot[0];
    if (threadIdx.x != 0) {
      // only thread 0 updates the scalars
    } else if (!(pq > 0.0)) {
      sc->done = 1;
      sc->alpha = 0;
    } else {
      sc->alpha = sc->rz / pq;
    }
    sc->pq = pq;
    sc->counter[CNT_HVP] = 0;
  }
  prof_end(pf);
}

// ---------------------------------------------------------------------------
// Column-walk FP32 HVP: one cell brick per 64-thread CTA, thread (x, y) walks
// the brick's z-column of cells (x, y, 0..7).  Every cell's eight corner
// contributions K D' sgn_o are summed into node values without a shared-memory
// scatter: along z in registers (the upper-z corners of cell z are carried to
// the node layer z + 1), along x by a warp shuffle (the eight cells of a row
// are eight adjacent lanes) and along y by a shuffle of eight lanes (rows 0-3
// and 4-7 are the two warps; the row 3 -> 4 step goes through shared memory).
// D' is formed from the p halo in shared memory, reusing the upper node layer
// of cell z as the lower layer of cell z + 1.
// ---------------------------------------------------------------------------

// node (nx, ny, nz) of the 9^3 halo of brick id receives the in-brick sum y[3]:
// a plain store (with the mass term) where only this brick contributes, an
// atomic add elsewhere (the mass term of those slots is written beforehand)
__device__ __forceinline__ void col_emit(int id, const int* s_nbr, const float (*sv)[729],
                                        const float* __restrict__ m, float* q, int nx, int ny, int nz,
                                        const float y[3]) {
  if (nx < 8 && ny < 8 && nz < 8) {
    const int l = (nz * 8 + ny) * 8 + nx;
    float* dst = q + (int64_t)id * 3 * BV + l;
    if (nx >= 1 && ny >= 1 && nz >= 1) {
      const float mi = m[(int64_t)id * BV + l];
      const int i = hidx(nx, ny, nz);
#pragma unroll
      for (int a = 0; a < 3; ++a) dst[a * BV] = y[a] + mi * sv[a][i];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (y[a] != 0.f) atomicAdd(dst + a * BV, y[a]);
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

// K45 by default: 64 registers, 16 CTAs (32 warps) per SM, which measured
// faster than the 256-thread brick kernel at 3 CTAs per SM on the 45-number
// tangent (latency-bound: more loads in flight per SM).
template <bool CMP, int MINB>
__global__ void __launch_bounds__(64, MINB) k_hvp_col(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                    const uint8_t* __restrict__ cflag, const float* __restrict__ K,
                                                    const float* __restrict__ p, const float* __restrict__ m,
                                                    float* q, DevScalars* sc, int finalize, DevProf* pf,
                                                    double* part) {
  constexpr int NQ = CMP ? NQC : 45;
  __shared__ float sv[3][729];
  __shared__ int s_nbr[NBR];
  __shared__ float sxr[2][2][3][8];  // [z parity][E, E8 of row 3][a][x]
  __shared__ int s_done;
  const int t = threadIdx.x, x = t & 7, y = t >> 3, row = y & 3;
  const int id = cblist[blockIdx.x];
  if (t == 0) s_done = finalize ? sc->done : 0;
  if (t < NBR) s_nbr[t] = nbr[id * NBR + t];
  __syncthreads();
  if (s_done) return;
  prof_begin(pf);
  for (int i = t; i < 729; i += 64) {  // the 9^3 p halo, streamed (read once per brick)
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    const int tb = (nx < 8 && ny < 8 && nz < 8) ? id : s_nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
    const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    if (tb >= 0) {
      const float* src = p + (int64_t)tb * 3 * BV + l;
      v0 = ld_stream(src);
      v1 = ld_stream(src + BV);
      v2 = ld_stream(src + 2 * BV);
    }
    sv[0][i] = v0;
    sv[1][i] = v1;
    sv[2][i] = v2;
  }
  __syncthreads();
  const float* Kb = K + (int64_t)id * NQ * BV;
  const uint8_t* cf = cflag + (int64_t)id * BV;
  constexpr unsigned FULL = 0xffffffffu;
  // lower node layer of the current cell: P0[ox][oy][a]; carried upper-z corners: Cz
  float P0[2][2][3], Cz[2][2][3];
#pragma unroll
  for (int ox = 0; ox < 2; ++ox)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        P0[ox][oy][a] = sv[a][hidx(x + ox, y + oy, 0)];
        Cz[ox][oy][a] = 0.f;
      }
  float pkp = 0.f;
#pragma unroll 1
  for (int z = 0; z <= 8; ++z) {
    float N[2][2][3];
    if (z < 8) {
      float P1[2][2][3];
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) P1[ox][oy][a] = sv[a][hidx(x + ox, y + oy, z + 1)];
      const int l = (z * 8 + y) * 8 + x;
      float KD[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) KD[r] = 0.f;
      if (cf[l]) {
        // D' = sum_o p_o (x) sgn_o
        float D[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float s00 = P0[0][0][a] + P1[0][0][a], s10 = P0[1][0][a] + P1[1][0][a];
          const float s01 = P0[0][1][a] + P1[0][1][a], s11 = P0[1][1][a] + P1[1][1][a];
          D[3 * a + 0] = (s10 + s11) - (s00 + s01);
          D[3 * a + 1] = (s01 + s11) - (s00 + s10);
          D[3 * a + 2] = (P1[0][0][a] - P0[0][0][a]) + (P1[1][0][a] - P0[1][0][a]) + (P1[0][1][a] - P0[0][1][a]) +
                         (P1[1][1][a] - P0[1][1][a]);
        }
        if (CMP) {
          float c[NQC];
#pragma unroll
          for (int qq = 0; qq < NQC; ++qq) c[qq] = ld_stream(Kb + qq * BV + l);
          apply_cmp(c, D, KD);
        } else {
          float k[45];
#pragma unroll
          for (int qq = 0; qq < 45; ++qq) k[qq] = ld_stream(Kb + qq * BV + l);
#pragma unroll
          for (int r = 0; r < 9; ++r) {
            KD[r] += k[k45(r, r)] * D[r];
#pragma unroll
            for (int cc = r + 1; cc < 9; ++cc) {
              KD[r] += k[k45(r, cc)] * D[cc];
              KD[cc] += k[k45(r, cc)] * D[r];
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) pkp += D[r] * KD[r];
      }
      // corner values: node (x + ox, y + oy, z + oz) gets (2ox-1) X + (2oy-1) Y + (2oz-1) Z
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float X = KD[3 * a], Yv = KD[3 * a + 1], Z = KD[3 * a + 2];
        const float A = X + Yv, B = X - Yv;
        N[1][1][a] = Cz[1][1][a] + (A - Z);
        N[0][0][a] = Cz[0][0][a] - (A + Z);
        N[1][0][a] = Cz[1][0][a] + (B - Z);
        N[0][1][a] = Cz[0][1][a] - (B + Z);
        Cz[1][1][a] = A + Z;
        Cz[0][0][a] = Z - A;
        Cz[1][0][a] = B + Z;
        Cz[0][1][a] = Z - B;
      }
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) P0[ox][oy][a] = P1[ox][oy][a];
    } else {
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) N[ox][oy][a] = Cz[ox][oy][a];
    }
    // along x: node (x, y + oy) gets N[0][oy] of this lane and N[1][oy] of lane x - 1;
    // E8 = N[1] is the node (8, y + oy) of the x = 7 lanes
    float E[2][3], E8[2][3];
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float left = __shfl_up_sync(FULL, N[1][oy][a], 1);
        E[oy][a] = N[0][oy][a] + (x > 0 ? left : 0.f);
        E8[oy][a] = N[1][oy][a];
      }
    // along y: node row y gets E[0] of row y and E[1] of row y - 1 (row 3 -> 4 through
    // shared memory, double-buffered by z parity so one barrier per layer suffices)
    const int buf = z & 1;
    if (y == 3) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sxr[buf][0][a][x] = E[1][a];
        sxr[buf][1][a][x] = E8[1][a];
      }
    }
    __syncthreads();
    float T[3], T8[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float up = __shfl_up_sync(FULL, E[1][a], 8), up8 = __shfl_up_sync(FULL, E8[1][a], 8);
      float prev = 0.f, prev8 = 0.f;
      if (row > 0) {
        prev = up;
        prev8 = up8;
      } else if (y == 4) {
        prev = sxr[buf][0][a][x];
        prev8 = sxr[buf][1][a][x];
      }
      T[a] = E[0][a] + prev;
      T8[a] = E8[0][a] + prev8;
    }
    col_emit(id, s_nbr, sv, m, q, x, y, z, T);
    if (x == 7) col_emit(id, s_nbr, sv, m, q, 8, y, z, T8);
    if (y == 7) {
      col_emit(id, s_nbr, sv, m, q, x, 8, z, E[1]);
      if (x == 7) col_emit(id, s_nbr, sv, m, q, 8, 8, z, E8[1]);
    }
  }
  double vals[1] = {(double)pkp};
  block_store<1>(vals, part);
  if (finalize && arrive_last(&sc->counter[CNT_HVP])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
      const double pq = sc->pMp + tot[0];
      if (!(pq > 0.0)) {
        sc->done = 1;
        sc->alpha = 0;
      } else {
        sc->alpha = sc->rz / pq;
      }
      sc->pq = pq;
      sc->counter[CNT_HVP] = 0;
    }
  }
  prof_end(pf);
}

// [persistent-solver source: begin]
// Shared memory of the persistent solver's HVP phase: the brick's compressed
// tangents (NQC x 512 floats, one TMA bulk copy), the 9^3 p halo and the
// mbarrier.
constexpr unsigned HVP_C_BYTES = (unsigned)NQC * BV * 4u;
constexpr size_t HVP_C_SMEM = HVP_C_BYTES + sizeof(float) * 3 * 729 + 16 + 16;
constexpr size_t HVP_C_SMEM_COL = HVP_C_SMEM + sizeof(float) * (HVP_X_FLOATS + HVP_R_FLOATS);
// 45-number tangent in the persistent solver: the brick's 45 x 512 floats by one
// bulk copy; the exchange buffers overlay the tangent block once it is used
constexpr unsigned HVP_K_BYTES45 = 45u * BV * 4u;
constexpr size_t HVP_K_SMEM45 = HVP_K_BYTES45 + sizeof(float) * 3 * 729 + 16 + 16;

// [persistent-solver source: end]
__device__ __forceinline__ void apply_compressed(const float* __restrict__ Cs, int l, const float D[9], float KD[9]) {
  float c[NQC];
#pragma unroll
  for (int q = 0; q < NQC; ++q) c[q] = Cs[q * BV + l];
  apply_cmp(c, D, KD);
}


// HVP over cell bricks: q = M p + sum_c B^T K B p (faces atomically).
template <typename T>
__global__ void __launch_bounds__(256) k_hvp(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                             const uint8_t* __restrict__ cflag, const T* __restrict__ K,
                                             const T* __restrict__ p, const T* __restrict__ m, T* q,
                                             DevScalars* sc, int finalize, DevProf* pf, double* part) {
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = finalize ? sc->done : 0;
  __syncthreads();
  if (s_done) return;
  prof_begin(pf);
  extern __shared__ __align__(16) unsigned char hvp_smem[];
  T (*sv)[729] = reinterpret_cast<T (*)[729]>(hvp_smem);
  T (*skd)[BV] = reinterpret_cast<T (*)[BV]>(hvp_smem + sizeof(T) * 3 * 729 + (16 - (sizeof(T) * 3 * 729) % 16) % 16);
  const int id = cblist[blockIdx.x];
  stage_nodes<T, T, T>(id, nbr, p, (const T*)nullptr, 0.0, sv);
  __syncthreads();
  double pkp = 0;
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    T KD[9];
    if (cflag[(int64_t)id * BV + l]) {
      T D[9];
      gather_D<T>(l, sv, D);
      const T* Kc = K + (int64_t)id * 45 * BV + l;
      T Kv[45];
#pragma unroll
      for (int j = 0; j < 45; ++j) Kv[j] = __ldg(&Kc[j * BV]);
#pragma unroll
      for (int r = 0; r < 9; ++r) KD[r] = T(0);
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        KD[r] += Kv[k45(r, r)] * D[r];
#pragma unroll
        for (int cc = r + 1; cc < 9; ++cc) {
          KD[r] += Kv[k45(r, cc)] * D[cc];
          KD[cc] += Kv[k45(r, cc)] * D[r];
        }
      }
      T dkd = 0;
#pragma unroll
      for (int r = 0; r < 9; ++r) dkd += D[r] * KD[r];
      pkp += (double)dkd;
    } else {
#pragma unroll
      for (int r = 0; r < 9; ++r) KD[r] = T(0);
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) skd[r][l] = KD[r];
  }
  __syncthreads();
  // node sums over the 9^3 block
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    T y[3] = {0, 0, 0};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int cx = nx - (o & 1), cy = ny - ((o >> 1) & 1), cz = nz - ((o >> 2) & 1);
      if (cx < 0 || cy < 0 || cz < 0 || cx > 7 || cy > 7 || cz > 7) continue;
      const int c = (cz * 8 + cy) * 8 + cx;
      const T s0 = (o & 1) ? T(1) : T(-1), s1 = (o & 2) ? T(1) : T(-1), s2 = (o & 4) ? T(1) : T(-1);
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] += skd[3 * a][c] * s0 + skd[3 * a + 1][c] * s1 + skd[3 * a + 2][c] * s2;
    }
    const bool own = nx < 8 && ny < 8 && nz < 8;
    const bool excl = nx >= 1 && nx <= 7 && ny >= 1 && ny <= 7 && nz >= 1 && nz <= 7;
    if (own) {
      // brick-face nodes arrive here with q = m p already (set by the kernel
      // that produced p, for every brick including those without cells)
      const int l = nz * 64 + ny * 8 + nx;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T* dst = q + (int64_t)id * 3 * BV + a * BV + l;
        if (excl) *dst = y[a] + m[(int64_t)id * BV + l] * sv[a][i];
        else if (y[a] != T(0)) atomicAdd(dst, y[a]);
      }
    } else {
      const int t = __ldg(&nbr[id * NBR + nbr_index(nx >> 3, ny >> 3, nz >> 3)]);
      if (t < 0) continue;
      const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (y[a] != T(0)) atomicAdd(q + (int64_t)t * 3 * BV + a * BV + l, y[a]);
    }
  }
  double vals[1] = {pkp};
  block_store<1>(vals, part);
  if (finalize && arrive_last(&sc->counter[CNT_HVP])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    double pq = sc->pMp + tot[0];
    if (threadIdx.x != 0) {
      // only thread 0 updates the scalars
    } else if (!(pq > 0.0)) {
      sc->done = 1;  // breakdown (zero direction)
      sc->alpha = 0;
    } else {
      sc->alpha = sc->rz / pq;
    }
    sc->pq = pq;
    sc->counter[CNT_HVP] = 0;
  }
  prof_end(pf);
}

// CG update A: x += alpha p, r -= alpha q, z = D^-1 r, r^T z, r^T r; the last
// block tests convergence and forms beta.  Generic version (any T).
template <typename T>
__global__ void __launch_bounds__(512) k_cg_a(const T* __restrict__ dinv, const T* __restrict__ p,
                                              const T* __restrict__ q, T* x, T* r, DevScalars* sc, double* part) {
  __shared__ int s_done;
  __shared__ double s_alpha;
  if (threadIdx.x == 0) {
    s_done = sc->done;
    s_alpha = sc->alpha;
  }
  __syncthreads();
  if (s_done) return;
  const int id = blockIdx.x, l = threadIdx.x;
  const T al = (T)s_alpha;
  double rz = 0, rr = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    const T di = dinv[o];
    if (di > T(0)) {
      T xv = x[o] + al * p[o];
      T rv = r[o] - al * q[o];
      x[o] = xv;
      r[o] = rv;
      rz += (double)rv * (double)(di * rv);
      rr += (double)rv * (double)rv;
    }
  }
  double vals[2] = {rz, rr};
  block_store<2>(vals, part);
  if (arrive_last(&sc->counter[CNT_A])) {
    double tot[2];
    block_sum_parts<2>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    const double rzn = tot[0], rrv = tot[1];
    const int it = sc->iters + 1;
    sc->iters = it;
    sc->rr_last = rrv;
    if (rrv <= sc->tol2 || it >= sc->cg_max || !(rrv == rrv)) sc->done = 1;
    sc->beta = rzn / sc->rz;
    sc->rz = rzn;
    sc->counter[CNT_A] = 0;
  }
}

// FP32 version: 128 threads per brick, 4 consecutive slots per thread with
// 16-byte loads; products and per-thread sums in FP32, accumulation across
// threads and blocks in FP64 (FP64 arithmetic is scarce on this GPU).
__global__ void __launch_bounds__(128) k_cg_a4(const float* __restrict__ dinv, const float* __restrict__ p,
                                               const float* __restrict__ q, float* x, float* r, DevScalars* sc,
                                               double* part, int fcg) {
  __shared__ int s_done;
  __shared__ float s_alpha;
  if (threadIdx.x == 0) {
    s_done = sc->done;
    s_alpha = (float)sc->alpha;
  }
  __syncthreads();
  if (s_done) return;
  const float al = s_alpha;
  double rz = 0, rr = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = ((int64_t)blockIdx.x * 3 + a) * BV + 4 * threadIdx.x;
    const float4 d4 = *reinterpret_cast<const float4*>(dinv + o);
    const float4 p4 = *reinterpret_cast<const float4*>(p + o);
    const float4 q4 = *reinterpret_cast<const float4*>(q + o);
    float4 x4 = *reinterpret_cast<const float4*>(x + o);
    float4 r4 = *reinterpret_cast<const float4*>(r + o);
    const float dd[4] = {d4.x, d4.y, d4.z, d4.w}, pp[4] = {p4.x, p4.y, p4.z, p4.w}, qq[4] = {q4.x, q4.y, q4.z, q4.w};
    float xx[4] = {x4.x, x4.y, x4.z, x4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
    float srz = 0.f, srr = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool f = dd[j] > 0.f;
      xx[j] = f ? xx[j] + al * pp[j] : xx[j];
      rv[j] = f ? rv[j] - al * qq[j] : rv[j];
      srz += f ? rv[j] * dd[j] * rv[j] : 0.f;
      srr += f ? rv[j] * rv[j] : 0.f;
    }
    *reinterpret_cast<float4*>(x + o) = make_float4(xx[0], xx[1], xx[2], xx[3]);
    *reinterpret_cast<float4*>(r + o) = make_float4(rv[0], rv[1], rv[2], rv[3]);
    rz += (double)srz;
    rr += (double)srr;
  }
  double vals[2] = {rz, rr};
  block_store<2>(vals, part);
  if (arrive_last(&sc->counter[CNT_A])) {
    double tot[2];
    block_sum_parts<2>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    const double rzn = tot[0], rrv = tot[1];
    const int it = sc->iters + 1;
    sc->iters = it;
    sc->rr_last = rrv;
    if (rrv <= sc->tol2 || it >= sc->cg_max || !(rrv == rrv)) sc->done = 1;
    if (fcg) {
      // flexible CG: beta and r^T z come later (after the network); here the
      // network input scale and the stall test (no progress in 20 iterations)
      sc->rzj = rzn;
      sc->nn_s = sc->nfree > 0 ? sqrt(rzn / sc->nfree) : 0.0;
      if (it > 20 && rrv >= sc->rr_ring[(it - 20) & 31]) {
        sc->fallback = 1;
        sc->done = 1;
      }
      sc->rr_ring[it & 31] = rrv;
    } else {
      sc->beta = rzn / sc->rz;
      sc->rz = rzn;
    }
    sc->counter[CNT_A] = 0;
  }
}

// CG update B: p = D^-1 r + beta p, q(face) = m p, sum m |p|^2
template <typename T>
__global__ void __launch_bounds__(512) k_cg_b(const T* __restrict__ dinv, const T* __restrict__ m,
                                              const T* __restrict__ r, T* p, T* q, DevScalars* sc, double* part) {
  __shared__ int s_done;
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    s_done = sc->done;
    s_beta = sc->beta;
  }
  __syncthreads();
  if (s_done) return;
  const int id = blockIdx.x, l = threadIdx.x;
  const T be = (T)s_beta;
  const bool face = (l & 7) == 0 || ((l >> 3) & 7) == 0 || (l >> 6) == 0;
  const T mi = m[(int64_t)id * BV + l];
  double pmp = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    const T di = dinv[o];
    T pv = T(0);
    if (di > T(0)) pv = di * r[o] + be * p[o];
    p[o] = pv;
    if (face) q[o] = mi * pv;  // mass term of brick-face nodes (HVP adds the rest)
    pmp += (double)mi * (double)pv * (double)pv;
  }
  double vals[1] = {pmp};
  block_store<1>(vals, part);
  if (arrive_last(&sc->counter[CNT_B])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    sc->pMp = tot[0];
    sc->counter[CNT_B] = 0;
  }
}

// FP32 version of B (4 slots per thread, 16-byte accesses)
__global__ void __launch_bounds__(128) k_cg_b4(const float* __restrict__ dinv, const float* __restrict__ m,
                                               const float* __restrict__ r, float* p, float* q, DevScalars* sc,
                                               double* part) {
  __shared__ int s_done;
  __shared__ float s_beta;
  if (threadIdx.x == 0) {
    s_done = sc->done;
    s_beta = (float)sc->beta;
  }
  __syncthreads();
  if (s_done) return;
  const float be = s_beta;
  const int l0 = 4 * threadIdx.x;
  // slots l0..l0+3 share (ly, lz); lx = l0 & 7 is 0 or 4
  const bool face_yz = ((l0 >> 3) & 7) == 0 || (l0 >> 6) == 0;
  const bool face0 = face_yz || (l0 & 7) == 0;
  const float4 m4 = *reinterpret_cast<const float4*>(m + (int64_t)blockIdx.x * BV + l0);
  const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
  float spmp = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = ((int64_t)blockIdx.x * 3 + a) * BV + l0;
    const float4 d4 = *reinterpret_cast<const float4*>(dinv + o);
    const float4 r4 = *reinterpret_cast<const float4*>(r + o);
    const float4 p4 = *reinterpret_cast<const float4*>(p + o);
    const float dd[4] = {d4.x, d4.y, d4.z, d4.w}, rr4[4] = {r4.x, r4.y, r4.z, r4.w}, po[4] = {p4.x, p4.y, p4.z, p4.w};
    float pv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pv[j] = dd[j] > 0.f ? dd[j] * rr4[j] + be * po[j] : 0.f;
      spmp += mm[j] * pv[j] * pv[j];
    }
    *reinterpret_cast<float4*>(p + o) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    if (face_yz) {
      *reinterpret_cast<float4*>(q + o) = make_float4(mm[0] * pv[0], mm[1] * pv[1], mm[2] * pv[2], mm[3] * pv[3]);
    } else if (face0) {
      q[o] = mm[0] * pv[0];
    }
  }
  double vals[1] = {(double)spmp};
  block_store<1>(vals, part);
  if (arrive_last(&sc->counter[CNT_B])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    sc->pMp = tot[0];
    sc->counter[CNT_B] = 0;
  }
}

// g^T x over free DOFs
template <typename T>
__global__ void __launch_bounds__(512) k_dot(const double* __restrict__ a, const T* __restrict__ b, double* out) {
  const int id = blockIdx.x, l = threadIdx.x;
  double s = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t o = (int64_t)id * 3 * BV + c * BV + l;
    s += a[o] * (double)b[o];
  }
  double vals[1] = {s};
  double* const dst[1] = {out};
  block_add<1>(vals, dst);
}

// Line-search set-up for the direction x: slope g^T x and the coefficients of the
// exact inertia change along it, sum_i m_i/2 |v_i + a x_i - vhat_i|^2 - (the same at
// a = 0) = a A + a^2 B / 2 with A = sum m (v - vhat).x, B = sum m |x|^2.  Evaluating
// the change this way avoids subtracting two nearly equal inertia sums whose
// terms carry the rounding of v + a x (relative to |v|, not to |v - vhat|).
template <typename T>
__global__ void __launch_bounds__(512) k_ls_setup(const uint8_t* __restrict__ nflag, const T* __restrict__ m,
                                                  const double* __restrict__ g, const double* __restrict__ v,
                                                  const double* __restrict__ vhat, const T* __restrict__ x,
                                                  DevScalars* sc, int nb) {
  const int l = threadIdx.x;
  double sl = 0, A = 0, B = 0;
  // several bricks per block: the FP64 block sums (slow on this part) once per block
  for (int id = blockIdx.x; id < nb; id += gridDim.x) {
    const int64_t slot = (int64_t)id * BV + l;
    const bool dof = (nflag[slot] & NF_DOF) != 0;
    const double mi = (double)m[slot];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
      const double xv = (double)x[o];
      sl += g[o] * xv;
      if (dof) {
        A += mi * (v[o] - vhat[o]) * xv;
        B += mi * xv * xv;
      }
    }
  }
  double vals[3] = {sl, A, B};
  double* const dst[3] = {&sc->slope, &sc->ls_a, &sc->ls_b};
  block_add<3>(vals, dst);
}

// line-search energy at v + alpha x: inertia over all bricks
template <typename T>
__global__ void __launch_bounds__(512) k_energy_nodes(const uint8_t* __restrict__ nflag, const T* __restrict__ m,
                                                      const double* __restrict__ v, const T* __restrict__ x,
                                                      const double* __restrict__ vhat, double alpha, DevScalars* sc,
                                                      int nb) {
  const int l = threadIdx.x;
  double e = 0;
  for (int id = blockIdx.x; id < nb; id += gridDim.x) {
    const int64_t slot = (int64_t)id * BV + l;
    if (nflag[slot] & NF_DOF) {
      const double mi = (double)m[slot];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
        const double d = v[o] + alpha * (double)x[o] - vhat[o];
        e += 0.5 * mi * d * d;
      }
    }
  }
  double vals[1] = {e};
  double* const dst[1] = {&sc->phi_in};
  block_add<1>(vals, dst);
}

template <typename T>
__global__ void __launch_bounds__(256) k_energy_cells(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                      const uint8_t* __restrict__ cflag, const T* __restrict__ acc,
                                                      const double* __restrict__ cs, const double* __restrict__ v,
                                                      const T* __restrict__ x, double alpha, SolveInfo si,
                                                      DevScalars* sc) {
  __shared__ double sv[3][729];
  const int id = cblist[blockIdx.x];
  stage_nodes<double, double, T>(id, nbr, v, x, alpha, sv);
  __syncthreads();
  const double gw = 0.25 / si.dx;
  double esum = 0;
  int bad = 0;
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    if (!cflag[(int64_t)id * BV + l]) continue;
    double D[9];
    gather_D<double>(l, sv, D);
    double Gd[9];
    const double sgd = si.dt * gw;
#pragma unroll
    for (int q = 0; q < 9; ++q) Gd[q] = sgd * D[q];
    for (int k = 0; k < si.nm; ++k) {
      const double V = (double)acc[((int64_t)id * si.nf + acc_V(k)) * BV + l];
      if (V == 0.0) continue;
      double bm[9], sm[9], H[9];
      load_base(cs, si.b9, id, si.nm, k, l, bm);
      trial_h(Gd, bm, sm, H);
      double psi;
      bool need_svd;
      if (!psi_from_h(si.mat[k], H, psi, need_svd, sizeof(T) == 4)) {
        bad = 1;
        continue;
      }
      if (need_svd) {
        // FP32 contexts: the same LITE evaluation as the Newton prep's energy
        double U[9], s[3], e[3], Vv[9], Jm1;
        svd_from_h<double, sizeof(T) == 4>(H, U, s, e, Vv, Jm1);
        Spec<double> sp;
        if (!spectral<double, sizeof(T) == 4 ? 5 : 1>(si.mat[k], s, e, Jm1, sp)) {  // the energy only
          bad = 1;
          continue;
        }
        psi = sp.psi;
      }
      esum += V * psi;
    }
  }
  if (bad) atomicAdd(&sc->infeasible, 1);
  double vals[1] = {esum};
  double* const dst[1] = {&sc->phi_el};
  block_add<1>(vals, dst);
}

// v += alpha x on free DOFs
template <typename T>
__global__ void __launch_bounds__(512) k_axpy(const T* __restrict__ dinv, const T* __restrict__ x, double alpha,
                                              double* v) {
  const int id = blockIdx.x, l = threadIdx.x;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    if (dinv[o] > T(0)) v[o] += alpha * (double)x[o];
  }
}

// v_out = v + alpha x on free DOFs, v elsewhere (the line search's trial iterate)
template <typename T>
__global__ void __launch_bounds__(512) k_axpy_out(const T* __restrict__ dinv, const T* __restrict__ x, double alpha,
                                                  const double* __restrict__ v, double* vout) {
  const int id = blockIdx.x, l = threadIdx.x;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    const double vo = v[o];
    vout[o] = dinv[o] > T(0) ? vo + alpha * (double)x[o] : vo;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static SolveInfo solve_info(mpml_ctx_s* c) {
  SolveInfo si;
  si.dt = c->d.dt;
  si.dx = c->d.dx;
  si.nm = c->nm;
  si.nf = acc_fields(c->nm);
  si.b9 = c->fp_active;
  for (int k = 0; k < MPML_MAX_MATS; ++k) {
    const mpml_material& m = c->mats[k < c->nm ? k : 0];
    si.mat[k].model = m.model;
    si.mat[k].mu = m.mu;
    si.mat[k].lam = m.lambda;
    si.plastic[k] = k < c->nm ? m.plastic : MPML_ELASTIC;
    si.ys[k] = m.yield_stress;
    const double sp = sin(m.friction_angle);
    si.alpha[k] = sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp);
  }
  return si;
}

template <typename T>
static int alloc_solver(mpml_ctx_s* c) {
  const int64_t ns = c->nb * BV;
  const size_t es = sizeof(T);
  int rc;
  if ((rc = ensure(c->cs, sizeof(double) * 6 * c->nm * ns)) || (rc = ensure(c->cK, es * 45 * ns)) ||
      (rc = ensure(c->ng, sizeof(double) * 3 * ns)) || (rc = ensure(c->ndinv, es * 3 * ns)) || (rc = ensure(c->nx, es * 3 * ns)) ||
      (rc = ensure(c->nr, es * 3 * ns)) || (rc = ensure(c->np, es * 3 * ns)) || (rc = ensure(c->nq, es * 3 * ns)) ||
      (rc = ensure(c->part, sizeof(double) * 10 * (c->nb ? c->nb : 1))) ||
      (rc = ensure(c->nvtry, sizeof(double) * 3 * ns)))
    return rc;
  return MPML_OK;
}

template <typename T>
static int stretch_t(mpml_ctx_s* c) {
  int rc = alloc_solver<T>(c);
  if (rc) return rc;
  SolveInfo si = solve_info(c);
  if (c->ncb > 0) {
    k_stretch<T><<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const uint8_t*)c->cflag.p,
                                                    (const T*)c->cacc.p, si, (double*)c->cs.p, (int*)c->status.p);
    c->launches++;
  }
  return cuda_status(cudaGetLastError());
}

int stretch_all(mpml_ctx_s* c) { return c->fp64 ? stretch_t<double>(c) : stretch_t<float>(c); }

static DevScalars* dscal(mpml_ctx_s* c) { return (DevScalars*)c->scal.p; }
// per-block partial sums of the reductions (8 doubles per brick)
static double* part_fin(mpml_ctx_s* c) { return (double*)c->part.p; }
static double* part_hvp(mpml_ctx_s* c) { return (double*)c->part.p + 5 * c->nb; }
static double* part_a(mpml_ctx_s* c) { return (double*)c->part.p + 6 * c->nb; }
static double* part_b(mpml_ctx_s* c) { return (double*)c->part.p + 8 * c->nb; }

static int read_scalars(mpml_ctx_s* c) {
  cudaMemcpyAsync(c->hscal, c->scal.p, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s);
  cudaMemcpyAsync(c->hstatus, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->s);
  return cuda_status(cudaStreamSynchronize(c->s));
}

// blocks of the node-wise kernels: eight node bricks per block (their FP64 block sums once
// per block)
static unsigned node_blocks(int64_t nb) { return (unsigned)((nb + 7) / 8); }

// prep at the current iterate (c->nvnew): gradient, energy, K (optional), CG start
template <typename T>
static int prep_t(mpml_ctx_s* c, int want_k, int init_cg, double cg_rtol, int cg_max, int want_psi = 1,
                  int trial = 0) {
  SolveInfo si = solve_info(c);
  cudaMemsetAsync(c->scal.p, 0, sizeof(DevScalars), c->s);
  const unsigned nb = (unsigned)c->nb, ncb = (unsigned)c->ncb;
  if (nb == 0) return MPML_OK;
  k_node_init<T><<<node_blocks(nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p, (const double*)c->nvnew.p,
                                     (const double*)c->nvhat.p, (double*)c->ng.p, (T*)c->ndinv.p, dscal(c), (int)nb);
  if (ncb > 0)
    k_prep<T><<<ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p, (const uint8_t*)c->cflag.p,
                                    (const T*)c->cacc.p, (const double*)(c->fp_active ? c->cB.p : c->cs.p), (const double*)c->nvnew.p, si,
                                    want_k ? (c->compressed ? 2 : 1) : 0, (T*)c->cK.p, (double*)c->ng.p,
                                    (T*)c->ndinv.p, dscal(c),
                                    (int*)c->status.p, want_psi, trial);
  k_finalize<T><<<node_blocks(nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p, (double*)c->ng.p,
                                    (T*)c->ndinv.p, (T*)c->nx.p, (T*)c->nr.p, (T*)c->np.p, (T*)c->nq.p,
                                    init_cg ? 1 : 0, cg_rtol * cg_rtol, cg_max, dscal(c), part_fin(c), (int)nb);
  c->launches += ncb > 0 ? 3 : 2;
  return cuda_status(cudaGetLastError());
}

// the CG start (x = 0, r = -g, ...) after a prep without it
template <typename T>
static int cg_start_t(mpml_ctx_s* c, double cg_rtol, int cg_max) {
  if (c->nb == 0) return MPML_OK;
  k_finalize<T><<<node_blocks(c->nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p,
                                                 (double*)c->ng.p, (T*)c->ndinv.p, (T*)c->nx.p, (T*)c->nr.p,
                                                 (T*)c->np.p, (T*)c->nq.p, 2, cg_rtol * cg_rtol, cg_max, dscal(c),
                                                 part_fin(c), (int)c->nb);
  c->launches++;
  return cuda_status(cudaGetLastError());
}

template <typename T>
constexpr size_t hvp_smem_bytes() {
  return sizeof(T) * 3 * 729 + (16 - (sizeof(T) * 3 * 729) % 16) % 16 + sizeof(T) * 9 * BV;
}

// The launch shapes ("tiles") of the standalone FP32 HVP, per tangent format.
// Entry 0 is the default before (or without) autotuning.
const char* hvp_tile_name(int compressed, int tile) {
  static const char* cmp[HVP_TILES] = {"z-column: 64 threads, 8 cells each, 12 CTAs/SM (k_hvp_col)",
                                       "brick: 256 threads, 2 cells each, 3 CTAs/SM (k_hvp_glob)",
                                       "z-column: 64 threads, 8 cells each, 8 CTAs/SM (k_hvp_col)"};
  static const char* k45[HVP_TILES] = {"z-column: 64 threads, 8 cells each, 16 CTAs/SM (k_hvp_col)",
                                       "z-column: 64 threads, 8 cells each, 12 CTAs/SM (k_hvp_col)",
                                       "brick: 256 threads, 2 cells each, 3 CTAs/SM (k_hvp_glob)"};
  if (tile < 0 || tile >= HVP_TILES) return "";
  return compressed ? cmp[tile] : k45[tile];
}

static void launch_hvp_f32(mpml_ctx_s* c, int tile, const float* p, float* q, int finalize) {
  DevProf* pf = c->profiling ? (DevProf*)c->prof.p : nullptr;
  const unsigned g = (unsigned)c->ncb;
#define HVP_IN (const int*)c->cblist.p, (const int*)c->nbr.p, (const uint8_t*)c->cflag.p, (const float*)c->cK.p, p, \
               (const float*)c->nmass.p, q, dscal(c), finalize, pf
  if (c->compressed) {
    if (tile == 1) k_hvp_glob<true><<<g, 256, HVP_G_SMEM, c->s>>>(HVP_IN, (int*)c->status.p, part_hvp(c));
    else if (tile == 2) k_hvp_col<true, 8><<<g, 64, 0, c->s>>>(HVP_IN, part_hvp(c));
    else k_hvp_col<true, 12><<<g, 64, 0, c->s>>>(HVP_IN, part_hvp(c));
  } else {
    if (tile == 1) k_hvp_col<false, 12><<<g, 64, 0, c->s>>>(HVP_IN, part_hvp(c));
    else if (tile == 2) k_hvp_glob<false><<<g, 256, HVP_G_SMEM, c->s>>>(HVP_IN, (int*)c->status.p, part_hvp(c));
    else k_hvp_col<false, 16><<<g, 64, 0, c->s>>>(HVP_IN, part_hvp(c));
  }
#undef HVP_IN
}

template <typename T>
static void launch_hvp(mpml_ctx_s* c, const T* p, T* q, int finalize) {
  DevProf* pf = c->profiling ? (DevProf*)c->prof.p : nullptr;
  if (sizeof(T) == 4) {
    launch_hvp_f32(c, c->hvp_tile >= 0 ? c->hvp_tile : 0, (const float*)p, (float*)q, finalize);
  } else {
    launch_fit((const void*)k_hvp<T>, 256, hvp_smem_bytes<T>(), LS_HVP64, nullptr);
    k_hvp<T><<<(unsigned)c->ncb, 256, hvp_smem_bytes<T>(), c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                                 (const uint8_t*)c->cflag.p, (const T*)c->cK.p, p,
                                                                 (const T*)c->nmass.p, q, dscal(c), finalize, pf,
                                                                 part_hvp(c));
  }
  c->launches++;
}

template <typename T>
static void cg_iteration(mpml_ctx_s* c) {
  const unsigned nb = (unsigned)c->nb;
  launch_hvp<T>(c, (const T*)c->np.p, (T*)c->nq.p, 1);
  if (sizeof(T) == 4) {
    k_cg_a4<<<nb, 128, 0, c->s>>>((const float*)c->ndinv.p, (const float*)c->np.p, (const float*)c->nq.p,
                                  (float*)c->nx.p, (float*)c->nr.p, dscal(c), part_a(c), 0);
    k_cg_b4<<<nb, 128, 0, c->s>>>((const float*)c->ndinv.p, (const float*)c->nmass.p, (const float*)c->nr.p,
                                  (float*)c->np.p, (float*)c->nq.p, dscal(c), part_b(c));
  } else {
    k_cg_a<T><<<nb, BV, 0, c->s>>>((const T*)c->ndinv.p, (const T*)c->np.p, (const T*)c->nq.p, (T*)c->nx.p,
                                  (T*)c->nr.p, dscal(c), part_a(c));
    k_cg_b<T><<<nb, BV, 0, c->s>>>((const T*)c->ndinv.p, (const T*)c->nmass.p, (const T*)c->nr.p, (T*)c->np.p,
                                  (T*)c->nq.p, dscal(c), part_b(c));
  }
  c->launches += 2;
}

// Condition of the graph-driven CG loop: continue while not converged, under
// the iteration cap, and under a hard cap on loop bodies (always terminates).
__global__ void k_cg_cond(DevScalars* sc, cudaGraphConditionalHandle h, int max_bodies) {
  const int b = sc->bodies + 1;
  sc->bodies = b;
  const int go = !(*(volatile int*)&sc->done) && sc->iters < sc->cg_max && b < max_bodies;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

constexpr int CG_UNROLL = 4;

template <typename T>
static int ensure_cg_graph(mpml_ctx_s* c, int cg_max) {
  const uintptr_t key[17] = {(uintptr_t)c->nb, (uintptr_t)c->ncb, (uintptr_t)c->np.p, (uintptr_t)c->nq.p,
                             (uintptr_t)c->nx.p, (uintptr_t)c->nr.p, (uintptr_t)c->ndinv.p, (uintptr_t)c->nmass.p,
                             (uintptr_t)c->cK.p, (uintptr_t)c->scal.p, (uintptr_t)c->profiling,
                             (uintptr_t)c->cblist.p, (uintptr_t)c->nbr.p, (uintptr_t)c->cflag.p,
                             (uintptr_t)cg_max, (uintptr_t)c->prof.p, (uintptr_t)(c->hvp_tile + 1)};
  if (c->cg_exec && memcmp(key, c->cg_key, sizeof key) == 0) return MPML_OK;
  if (c->cg_exec) {
    cudaGraphExecDestroy(c->cg_exec);
    c->cg_exec = nullptr;
  }
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return MPML_ERR_CUDA;
  cudaGraph_t g = nullptr;
  int rc = MPML_OK;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return MPML_ERR_CUDA;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) rc = MPML_ERR_CUDA;
  if (!rc) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) rc = MPML_ERR_CUDA;
  }
  if (!rc) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t user = c->s;
    c->s = c->cap_stream;  // the kernels below are recorded into the loop body
    if (cudaStreamBeginCaptureToGraph(c->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      rc = MPML_ERR_CUDA;
    } else {
      const int64_t before = c->launches;
      for (int u = 0; u < CG_UNROLL; ++u) cg_iteration<T>(c);
      k_cg_cond<<<1, 1, 0, c->s>>>(dscal(c), h, cg_max / CG_UNROLL + 2);
      c->launches = before;  // recorded, not launched
      cudaGraph_t out = nullptr;
      if (cudaStreamEndCapture(c->s, &out) != cudaSuccess) rc = MPML_ERR_CUDA;
    }
    c->s = user;
  }
  if (!rc && cudaGraphInstantiate(&c->cg_exec, g, 0) != cudaSuccess) {
    c->cg_exec = nullptr;
    rc = MPML_ERR_CUDA;
  }
  cudaGraphDestroy(g);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  memcpy(c->cg_key, key, sizeof key);
  return MPML_OK;
}

// [persistent-solver source: begin]
// ---------------------------------------------------------------------------
// Persistent Jacobi-PCG (FP32; NQC-number compressed or 45-number packed
// tangent): the whole CG solve in one cooperative launch.  Each iteration has
// two phases separated by grid barriers:
//   H: for every cell brick of this CTA, stage p_new = D^-1 r + beta p_old on
//      the 9^3 node block (the update of p fused into the halo staging; the
//      owner writes p_new to the other p buffer), apply K (the brick's tangent
//      block by one TMA bulk copy) in the column walk of phase_h_col and add
//      q; bricks holding only DOF nodes get p_new and the mass term.
//      Partials: p^T M p, p^T K p.
//   A: x += alpha p_new, r -= alpha q, q = 0, partials r^T D^-1 r, r^T r.
// Every CTA sums the per-CTA partials in the same order, so all take the same
// decisions (alpha, beta, convergence) without another barrier.  Barrier
// waits are bounded; a timeout sets ST_TIMEOUT and ends the solve.
// ---------------------------------------------------------------------------
struct PcgArgs {
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
  double* acc;    // [4][2] rotating accumulators of the phase sums
  unsigned* gbar; // grid-barrier counter (zero at launch)
  int ncb, nnob, nb, cg_max;
  unsigned spins;  // bound on the polls of one grid-barrier wait
  int* status;
  DevProf* pf;
};

// Warp sum of FP32 values in float-float arithmetic (error-free two-sum at
// every level, the rounding errors carried in a second float), returned as
// a double on lane 0: FP64-grade accuracy without a chain of FP64 additions.
__device__ __forceinline__ void warp_sum_ff(float v, float& hi_out, float& lo_out) {
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

// block sums of 2 FP32 per-thread partials (float-float within warps, FP64
// across warps) added atomically to acc[0..1] (thread 0)
__device__ __forceinline__ void block_atomic2(float a, float b, double* acc) {
  __shared__ double red2[2][32];
  float ah, al, bh, bl;
  warp_sum_ff(a, ah, al);
  warp_sum_ff(b, bh, bl);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {  // FP64 only on lane 0 (FP64 instructions are slow on this part)
    red2[0][wid] = (double)ah + (double)al;
    red2[1][wid] = (double)bh + (double)bl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red2[0][w];
      sb += red2[1][w];
    }
    atomicAdd(acc, sa);
    atomicAdd(acc + 1, sb);
  }
}

// every CTA: sums of the 2 partials of all CTAs (fixed order) -> s_out[2]
__device__ __forceinline__ void sum_partials2(const double* part, double* s_out) {
  __shared__ double red[2][32];
  double a = 0, b = 0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(&part[2 * k]);
    b += __ldcg(&part[2 * k + 1]);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    s_out[0] = sa;
    s_out[1] = sb;
  }
  __syncthreads();
}

// p_new at one node slot of brick t (0 where not a free DOF)
__device__ __forceinline__ float pnew_at(const PcgArgs& A, int64_t o, float beta, const float* pold) {
  const float di = A.dinv[o];
  return di > 0.f ? di * A.r[o] + beta * pold[o] : 0.f;
}


template <bool K45, bool GLOBAL = false>
__global__ void __launch_bounds__(256, 2) k_pcg_persistent(PcgArgs A) {
  constexpr unsigned KB = GLOBAL ? 0u : (K45 ? HVP_K_BYTES45 : HVP_C_BYTES);
  constexpr int NQ = K45 ? 45 : NQC;
  extern __shared__ __align__(128) unsigned char psm[];
  float* Cs = reinterpret_cast<float*>(psm);
  float (*sv)[729] = reinterpret_cast<float (*)[729]>(psm + KB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(psm + KB + sizeof(float) * 3 * 729 + 8 - (sizeof(float) * 3 * 729) % 8);
  // the CTA's cell bricks (jc = blockIdx.x + k G) and their neighbour rows are
  // the same in every iteration: kept in shared memory when there are at most
  // PCG_LOCAL of them, else read per brick
  constexpr int PCG_LOCAL = 8;
  __shared__ int s_nbr[NBR];
  __shared__ int s_ids[PCG_LOCAL];
  __shared__ int s_nbrs[PCG_LOCAL][NBR];
  __shared__ int s_flag;
  __shared__ float s_coef;  // alpha or beta, formed in FP64 by thread 0
  __shared__ int s_stop;    // breakdown / convergence decided by thread 0
  DevScalars* sc = A.sc;
  const int nloc = (int)blockIdx.x < A.ncb ? (A.ncb - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const bool cached = nloc <= PCG_LOCAL;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (cached) {
    for (int k = 0; k < nloc; ++k) {
      const int id = A.cblist[(int)blockIdx.x + k * (int)gridDim.x];
      if (threadIdx.x == 0) s_ids[k] = id;
      if (threadIdx.x < NBR) s_nbrs[k][threadIdx.x] = A.nbr[id * NBR + threadIdx.x];
    }
  }
  __syncthreads();
  unsigned tma_phase = 0;
  // compressed tangent staged by TMA: which local brick's tangent is in Cs (or on
  // its way), and whether a copy is in flight; the tangent does not change during
  // the solve, so a CTA with one brick copies it once, and a CTA with more starts
  // the copy of its first brick at the end of phase H for the next iteration
  constexpr bool KEEP = !K45 && !GLOBAL;
  int cs_k = -1;
  bool inflight = false;
  // FP64 scalar state of the recurrences: thread 0 only, in shared memory
  __shared__ double s_rz, s_rr_last, s_tol2;
  if (threadIdx.x == 0) {
    s_rz = sc->rz;
    s_tol2 = sc->tol2;
    s_rr_last = sc->rr_last;
  }
  int done = sc->done;
  int it = 0;
  float beta = 0.f;
  float* pold = A.pa;
  float* pnext = A.pb;
  const int G = gridDim.x;
  bool alive = true;
  while (!done && alive) {
    const unsigned long long t_h0 = (A.pf && blockIdx.x == 0 && threadIdx.x == 0) ? gtimer() : 0ull;
    // ---------------- phase H ----------------
    float pmp = 0.f, pkp = 0.f;  // per-thread FP32 partials, summed in FP64 below
    for (int kl = 0, jc = blockIdx.x; jc < A.ncb; ++kl, jc += G) {
      int id;
      const int* nb_row;
      if (cached) {
        id = s_ids[kl];
        nb_row = s_nbrs[kl];
      } else {
        id = A.cblist[jc];
        if (threadIdx.x < NBR) s_nbr[threadIdx.x] = A.nbr[id * NBR + threadIdx.x];
        __syncthreads();
        nb_row = s_nbr;
      }
      if (!GLOBAL && !(KEEP && cached && cs_k == kl)) {
        if (threadIdx.x == 0) {
          // order the previous brick's generic accesses to Cs before the async copy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_expect_tx(bar, KB);
          tma_load_1d(Cs, A.C + (int64_t)id * NQ * BV, KB, bar);
        }
        inflight = true;
        cs_k = kl;
      }
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
            const int t = (nx < 8 && ny < 8 && nz < 8) ? id : nb_row[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
            const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
            tt[k] = t;
            ll[k] = l;
            if (t >= 0) {
              const int64_t o = (int64_t)t * 3 * BV + l;
  #pragma unroll
              for (int a = 0; a < 3; ++a) {
                dv[k][a] = __ldcg(A.dinv + o + a * BV);
                rv[k][a] = __ldcg(A.r + o + a * BV);
                pv[k][a] = __ldcg(pold + o + a * BV);
              }
              if (t == id) mv[k] = __ldcg(A.m + (int64_t)id * BV + l);
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
      bool ok = true;
      if (!GLOBAL && inflight) {
        ok = mbar_wait_bounded(bar, tma_phase);
        tma_phase ^= 1u;
        inflight = false;
        if (!ok) {
          cs_k = -1;
          if (threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
        }
      }
      {
        // GLOBAL: the tangent is streamed from global memory; the exchange buffers
        // follow the halo (no shared-memory tangent block)
        float* Xs = GLOBAL ? reinterpret_cast<float*>(psm + sizeof(float) * 3 * 729 + 16 + 16)
                           : (K45 ? Cs : reinterpret_cast<float*>(psm + HVP_C_SMEM));
        const float* Ksrc = GLOBAL ? A.C + (int64_t)id * NQ * BV : Cs;
        pkp += phase_h_col<K45, GLOBAL>(id, nb_row, sv, Ksrc, A.cflag, A.m, A.q, Xs, Xs + HVP_X_FLOATS, ok);
        __syncthreads();  // Cs / sv / s_nbr / exchange buffers are reused by the next brick
      }
    }
    if (KEEP && cached && nloc > 1) {
      // the first brick's tangent for the next iteration (Cs is free: the last
      // brick's walk ended at the barrier above)
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, KB);
        tma_load_1d(Cs, A.C + (int64_t)s_ids[0] * NQ * BV, KB, bar);
      }
      inflight = true;
      cs_k = 0;
    }
    // bricks with DOF nodes but no cells: p_new and the mass term, dealt from the
    // last CTA down (the CTAs with the fewest cell bricks)
    for (int jn = G - 1 - (int)blockIdx.x; jn < A.nnob; jn += G) {
      const int id = A.nolist[jn];
      for (int l = threadIdx.x; l < BV; l += blockDim.x) {
        const int64_t o = (int64_t)id * 3 * BV + l;
        const float v0 = pnew_at(A, o, beta, pold), v1 = pnew_at(A, o + BV, beta, pold),
                    v2 = pnew_at(A, o + 2 * BV, beta, pold);
        pnext[o] = v0;
        pnext[o + BV] = v1;
        pnext[o + 2 * BV] = v2;
        const float mi = A.m[(int64_t)id * BV + l];
        pmp += mi * (v0 * v0 + v1 * v1 + v2 * v2);
        if (v0 != 0.f) atomicAdd(A.q + o, mi * v0);
        if (v1 != 0.f) atomicAdd(A.q + o + BV, mi * v1);
        if (v2 != 0.f) atomicAdd(A.q + o + 2 * BV, mi * v2);
      }
    }
    // phase sums go to slot k = (2 it) % 4; CTA 0 clears slot k + 2, last read
    // two barriers ago and next written two barriers later
    double* accH = A.acc + 2 * ((2 * it) & 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double* z = A.acc + 2 * ((2 * it + 2) & 3);
      z[0] = 0.0;
      z[1] = 0.0;
    }
    block_atomic2(pmp, pkp, accH);
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    // the scalar recurrences in FP64 on thread 0 only (FP64 is slow on this part)
    if (threadIdx.x == 0) {
      const double pq = __ldcg(accH) + __ldcg(accH + 1);
      s_stop = !(pq > 0.0);  // breakdown
      s_coef = s_stop ? 0.f : (float)(s_rz / pq);
      if (A.pf && blockIdx.x == 0) {
        A.pf->ns += gtimer() - t_h0;
        A.pf->count += 1;
      }
    }
    __syncthreads();
    if (s_stop) {
      done = 1;
      break;
    }
    const float alpha = s_coef;
    // ---------------- phase A ----------------
    float rzl = 0.f, rrl = 0.f;
    // two node bricks per pass, all loads issued before the updates
    for (int jb0 = blockIdx.x; jb0 < A.nb; jb0 += 2 * G) {
      float2 d2[2][3], p2[2][3], q2[2][3], x2[2][3], r2[2][3];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int jb = jb0 + u * G;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (jb < A.nb) {
            const int64_t o = ((int64_t)jb * 3 + a) * BV + 2 * threadIdx.x;
            d2[u][a] = __ldcg(reinterpret_cast<const float2*>(A.dinv + o));
            p2[u][a] = __ldcg(reinterpret_cast<const float2*>(pnext + o));
            q2[u][a] = __ldcg(reinterpret_cast<const float2*>(A.q + o));
            x2[u][a] = __ldcg(reinterpret_cast<const float2*>(A.x + o));
            r2[u][a] = __ldcg(reinterpret_cast<const float2*>(A.r + o));
          } else {
            d2[u][a] = p2[u][a] = q2[u][a] = x2[u][a] = r2[u][a] = make_float2(0.f, 0.f);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int jb = jb0 + u * G;
        if (jb >= A.nb) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int64_t o = ((int64_t)jb * 3 + a) * BV + 2 * threadIdx.x;
          const float2 d = d2[u][a], pp = p2[u][a], qq = q2[u][a];
          float2 xx = x2[u][a], rr = r2[u][a];
          if (d.x > 0.f) {
            xx.x += alpha * pp.x;
            rr.x -= alpha * qq.x;
          }
          if (d.y > 0.f) {
            xx.y += alpha * pp.y;
            rr.y -= alpha * qq.y;
          }
          *reinterpret_cast<float2*>(A.x + o) = xx;
          *reinterpret_cast<float2*>(A.r + o) = rr;
          *reinterpret_cast<float2*>(A.q + o) = make_float2(0.f, 0.f);
          const float srz = (d.x > 0.f ? rr.x * d.x * rr.x : 0.f) + (d.y > 0.f ? rr.y * d.y * rr.y : 0.f);
          const float srr = (d.x > 0.f ? rr.x * rr.x : 0.f) + (d.y > 0.f ? rr.y * rr.y : 0.f);
          rzl += srz;
          rrl += srr;
        }
      }
    }
    double* accA = A.acc + 2 * ((2 * it + 1) & 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double* z = A.acc + 2 * ((2 * it + 3) & 3);
      z[0] = 0.0;
      z[1] = 0.0;
    }
    block_atomic2(rzl, rrl, accA);
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    ++it;
    if (threadIdx.x == 0) {
      const double rzn = __ldcg(accA), rrn = __ldcg(accA + 1);
      s_rr_last = rrn;
      s_stop = (rrn <= s_tol2 || it >= A.cg_max || !(rrn == rrn)) ? 1 : 0;
      s_coef = (float)(rzn / s_rz);
      s_rz = rzn;
    }
    __syncthreads();
    done = s_stop;
    beta = s_coef;
    float* tmp = pold;
    pold = pnext;
    pnext = tmp;
  }
  if (!alive && threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
  // a prefetched tangent copy still in flight completes before the CTA exits
  if (!GLOBAL && inflight && !mbar_wait_bounded(bar, tma_phase) && threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->iters = it;
    sc->rr_last = s_rr_last;
    sc->rz = s_rz;
    sc->done = 1;
  }
}

// ---------------------------------------------------------------------------
// Persistent Jacobi-PCG, column-group form: the same iteration and phases as
// k_pcg_persistent, but in phase H each 64-thread group of a CTA owns a work
// unit of its own -- half a cell brick, four z-layers of cells (group g of CTA
// b takes the units b * 4 + g + k * 4 G, unit u = half u & 1 of cell brick
// u >> 1; halves balance the groups' work to within one unit) -- stages p_new on
// the unit's 9 x 9 x 5 node block (fused p update, as above) and the unit's cell
// flags and node masses in its own shared memory, and walks the 64 z-columns of
// cells with the tangent rows streamed from global memory (thread (x, y) walks
// column (x, y): lower and upper node layers in registers, node sums along x by
// shuffles, along y by shuffles and one row exchange per layer, a 64-thread
// named barrier per layer).  Four independent units per CTA and two to four
// CTAs per SM keep up to 45 outstanding tangent loads per thread in flight
// without any block-wide barrier inside phase H.
// ---------------------------------------------------------------------------
struct ColGroup {
  float sv[3][405];          // p_new on the unit's 9 x 9 x 5 node block
  float sxr[2][2][3][8];     // [z parity][E, E8 of row 3][a][x]
  float m[256];              // the masses of the unit's owned nodes
  int nbr[NBR];
  uint8_t cf[256];           // the unit's active-cell flags
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 64;" ::"r"(g + 1) : "memory");
}

// Half-brick work units: unit (brick, hz) holds the brick's cell layers 4hz .. 4hz+3
// and its node layers 4hz .. 4hz+4 (local layers 0 .. 4); it owns (writes p_new and
// adds the mass term for) the node layers 4hz .. 4hz+3 of the brick.  Node (nx, ny,
// local nzl) receives y[3]: plain store where only this unit contributes (owned,
// nx, ny >= 1 and 1 <= nzl <= 3), atomic add elsewhere.
__device__ __forceinline__ void col_emit_h(int id, const ColGroup& S, float* q, int nx, int ny, int nzl, int hz,
                                          const float y[3]) {
  const int nz = 4 * hz + nzl;
  if (nx < 8 && ny < 8 && nz < 8) {
    const int l = (nz * 8 + ny) * 8 + nx;
    float* dst = q + (int64_t)id * 3 * BV + l;
    const bool owned = nzl < 4;
    const float mi = owned ? S.m[l - 256 * hz] : 0.f;
    const int i = hidx(nx, ny, nzl);
    if (owned && nx >= 1 && ny >= 1 && nzl >= 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) dst[a * BV] = y[a] + mi * S.sv[a][i];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float val = y[a] + mi * S.sv[a][i];
        if (val != 0.f) atomicAdd(dst + a * BV, val);
      }
    }
  } else {
    const int t = S.nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
    if (t < 0) return;
    const int l = ((nz & 7) * 8 + (ny & 7)) * 8 + (nx & 7);
    float* dst = q + (int64_t)t * 3 * BV + l;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (y[a] != 0.f) atomicAdd(dst + a * BV, y[a]);
  }
}

template <bool K45, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pcg_groups(PcgArgs A) {
  constexpr int NQ = K45 ? 45 : NQC;
  constexpr bool PF = MINB <= 2;
  constexpr int SB = 3;  // halo nodes per thread and load batch
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ ColGroup gs[4];
  __shared__ int s_flag;
  __shared__ float s_coef;
  __shared__ int s_stop;
  __shared__ double s_rz, s_rr_last, s_tol2;
  DevScalars* sc = A.sc;
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63, x = t & 7, y = t >> 3, row = y & 3;
  ColGroup& S = gs[g];
  const int G = gridDim.x, NG = 4 * G, gid = 4 * (int)blockIdx.x + g;
  if (threadIdx.x == 0) {
    s_rz = sc->rz;
    s_tol2 = sc->tol2;
    s_rr_last = sc->rr_last;
  }

  int done = sc->done;
  int it = 0;
  float beta = 0.f;
  float* pold = A.pa;
  float* pnext = A.pb;
  bool alive = true;
  __syncthreads();
  while (!done && alive) {
    const unsigned long long t_h0 = (A.pf && blockIdx.x == 0 && threadIdx.x == 0) ? gtimer() : 0ull;
    // ---------------- phase H ----------------
    float pmp = 0.f, pkp = 0.f;
    for (int u = gid; u < 2 * A.ncb; u += NG) {
      const int id = A.cblist[u >> 1], hz = u & 1;
      if (t < NBR) S.nbr[t] = A.nbr[id * NBR + t];
      // the unit's active-cell flags (read by the walk from shared memory)
#pragma unroll
      for (int k = 0; k < 4; ++k) S.cf[t + 64 * k] = A.cflag[(int64_t)id * BV + 256 * hz + t + 64 * k];
      group_sync(g);
      // p_new on the unit's 9 x 9 x 5 node block, three nodes per thread and batch, all
      // loads first; the owned nodes' p_new and masses are written
      for (int i0 = t; i0 < 405; i0 += SB * 64) {
        int tb[SB], ll[SB];
        float dv[SB][3], rv[SB][3], pv[SB][3], mv[SB];
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          const int i = i0 + 64 * k;
          tb[k] = -1;
          ll[k] = 0;
          mv[k] = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a) dv[k][a] = rv[k][a] = pv[k][a] = 0.f;
          if (i < 405) {
            const int nx = i % 9, ny = (i / 9) % 9, nz = 4 * hz + i / 81;
            const int tt = (nx < 8 && ny < 8 && nz < 8) ? id : S.nbr[nbr_index(nx >> 3, ny >> 3, nz >> 3)];
            const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
            tb[k] = tt;
            ll[k] = l;
            if (tt >= 0) {
              const int64_t o = (int64_t)tt * 3 * BV + l;
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                dv[k][a] = __ldcg(A.dinv + o + a * BV);
                rv[k][a] = __ldcg(A.r + o + a * BV);
                pv[k][a] = __ldcg(pold + o + a * BV);
              }
              if (tt == id && i < 324) mv[k] = __ldcg(A.m + (int64_t)id * BV + l);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          const int i = i0 + 64 * k;
          if (i >= 405) continue;
          float v[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) v[a] = dv[k][a] > 0.f ? dv[k][a] * rv[k][a] + beta * pv[k][a] : 0.f;
          if (tb[k] == id && i < 324) {  // owned: own brick, local layers 0 .. 3
            const int64_t o = (int64_t)id * 3 * BV + ll[k];
            pnext[o] = v[0];
            pnext[o + BV] = v[1];
            pnext[o + 2 * BV] = v[2];
            pmp += mv[k] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            S.m[ll[k] - 256 * hz] = mv[k];
          }
          S.sv[0][i] = v[0];
          S.sv[1][i] = v[1];
          S.sv[2][i] = v[2];
        }
      }
      group_sync(g);
      // the z-column walk of this thread's column (x, y) over the unit's four cell layers
      const float* Kb = A.C + (int64_t)id * NQ * BV;
      float P0[2][2][3], Cz[2][2][3];
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            P0[ox][oy][a] = S.sv[a][hidx(x + ox, y + oy, 0)];
            Cz[ox][oy][a] = 0.f;
          }
      // prefetched tangent rows of the next layer's cell (PF builds)
      float kn[PF ? NQ : 1];
      int fn = 0;
      if (PF) {
        fn = S.cf[y * 8 + x];
        if (fn) {
#pragma unroll
          for (int qq = 0; qq < NQ; ++qq) kn[qq] = ld_stream(Kb + qq * BV + 256 * hz + y * 8 + x);
        }
      }
#pragma unroll
      for (int z = 0; z <= 4; ++z) {
        float N[2][2][3];
        if (z < 4) {
          float P1[2][2][3];
#pragma unroll
          for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int oy = 0; oy < 2; ++oy)
#pragma unroll
              for (int a = 0; a < 3; ++a) P1[ox][oy][a] = S.sv[a][hidx(x + ox, y + oy, z + 1)];
          const int lu = (z * 8 + y) * 8 + x, l = 256 * hz + lu;  // cell in the unit and in the brick
          float KD[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) KD[r] = 0.f;
          int fc;
          float kc[PF ? NQ : 1];
          if (PF) {
            fc = fn;
#pragma unroll
            for (int qq = 0; qq < (PF ? NQ : 1); ++qq) kc[qq] = kn[qq];
            fn = z < 3 ? S.cf[lu + 64] : 0;
            if (fn) {
#pragma unroll
              for (int qq = 0; qq < (PF ? NQ : 1); ++qq) kn[qq] = ld_stream(Kb + qq * BV + l + 64);
            }
          } else {
            fc = S.cf[lu];
          }
          if (fc) {
            float D[9];
            col_D(P0, P1, D);
            if (K45) {
              float k[45];
#pragma unroll
              for (int qq = 0; qq < 45; ++qq)
                k[qq] = PF ? kc[qq < (PF ? NQ : 1) ? qq : 0] : ld_stream(Kb + qq * BV + l);
#pragma unroll
              for (int r = 0; r < 9; ++r) {
                KD[r] += k[k45(r, r)] * D[r];
#pragma unroll
                for (int cc = r + 1; cc < 9; ++cc) {
                  KD[r] += k[k45(r, cc)] * D[cc];
                  KD[cc] += k[k45(r, cc)] * D[r];
                }
              }
            } else {
              float c[NQC];
#pragma unroll
              for (int qq = 0; qq < NQC; ++qq)
                c[qq] = PF ? kc[qq < (PF ? NQ : 1) ? qq : 0] : ld_stream(Kb + qq * BV + l);
              apply_cmp(c, D, KD);
            }
#pragma unroll
            for (int r = 0; r < 9; ++r) pkp += D[r] * KD[r];
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float X = KD[3 * a], Yv = KD[3 * a + 1], Z = KD[3 * a + 2];
            const float Ap = X + Yv, B = X - Yv;
            N[1][1][a] = Cz[1][1][a] + (Ap - Z);
            N[0][0][a] = Cz[0][0][a] - (Ap + Z);
            N[1][0][a] = Cz[1][0][a] + (B - Z);
            N[0][1][a] = Cz[0][1][a] - (B + Z);
            Cz[1][1][a] = Ap + Z;
            Cz[0][0][a] = Z - Ap;
            Cz[1][0][a] = B + Z;
            Cz[0][1][a] = Z - B;
          }
#pragma unroll
          for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int oy = 0; oy < 2; ++oy)
#pragma unroll
              for (int a = 0; a < 3; ++a) P0[ox][oy][a] = P1[ox][oy][a];
        } else {
#pragma unroll
          for (int ox = 0; ox < 2; ++ox)
#pragma unroll
            for (int oy = 0; oy < 2; ++oy)
#pragma unroll
              for (int a = 0; a < 3; ++a) N[ox][oy][a] = Cz[ox][oy][a];
        }
        // along x by shuffles; along y by shuffles of eight lanes and the row 3 -> 4
        // exchange (double-buffered by z parity: one barrier per layer)
        float E[2][3], E8[2][3];
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float left = __shfl_up_sync(FULL, N[1][oy][a], 1);
            E[oy][a] = N[0][oy][a] + (x > 0 ? left : 0.f);
            E8[oy][a] = N[1][oy][a];
          }
        const int buf = z & 1;
        if (y == 3) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            S.sxr[buf][0][a][x] = E[1][a];
            S.sxr[buf][1][a][x] = E8[1][a];
          }
        }
        group_sync(g);
        float T[3], T8[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float up = __shfl_up_sync(FULL, E[1][a], 8), up8 = __shfl_up_sync(FULL, E8[1][a], 8);
          float prev = 0.f, prev8 = 0.f;
          if (row > 0) {
            prev = up;
            prev8 = up8;
          } else if (y == 4) {
            prev = S.sxr[buf][0][a][x];
            prev8 = S.sxr[buf][1][a][x];
          }
          T[a] = E[0][a] + prev;
          T8[a] = E8[0][a] + prev8;
        }
        col_emit_h(id, S, A.q, x, y, z, hz, T);
        if (x == 7) col_emit_h(id, S, A.q, 8, y, z, hz, T8);
        if (y == 7) {
          col_emit_h(id, S, A.q, x, 8, z, hz, E[1]);
          if (x == 7) col_emit_h(id, S, A.q, 8, 8, z, hz, E8[1]);
        }
      }
      group_sync(g);  // S.sv, S.m, S.cf and S.nbr are reused by the group's next unit
    }
    // bricks with DOF nodes but no cells: p_new and the mass term
    for (int jn = G - 1 - (int)blockIdx.x; jn < A.nnob; jn += G) {
      const int id = A.nolist[jn];
      for (int l = threadIdx.x; l < BV; l += blockDim.x) {
        const int64_t o = (int64_t)id * 3 * BV + l;
        const float v0 = pnew_at(A, o, beta, pold), v1 = pnew_at(A, o + BV, beta, pold),
                    v2 = pnew_at(A, o + 2 * BV, beta, pold);
        pnext[o] = v0;
        pnext[o + BV] = v1;
        pnext[o + 2 * BV] = v2;
        const float mi = A.m[(int64_t)id * BV + l];
        pmp += mi * (v0 * v0 + v1 * v1 + v2 * v2);
        if (v0 != 0.f) atomicAdd(A.q + o, mi * v0);
        if (v1 != 0.f) atomicAdd(A.q + o + BV, mi * v1);
        if (v2 != 0.f) atomicAdd(A.q + o + 2 * BV, mi * v2);
      }
    }
    double* accH = A.acc + 2 * ((2 * it) & 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double* zz = A.acc + 2 * ((2 * it + 2) & 3);
      zz[0] = 0.0;
      zz[1] = 0.0;
    }
    block_atomic2(pmp, pkp, accH);
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    if (threadIdx.x == 0) {
      const double pq = __ldcg(accH) + __ldcg(accH + 1);
      s_stop = !(pq > 0.0);
      s_coef = s_stop ? 0.f : (float)(s_rz / pq);
      if (A.pf && blockIdx.x == 0) {
        A.pf->ns += gtimer() - t_h0;
        A.pf->count += 1;
      }
    }
    __syncthreads();
    if (s_stop) {
      done = 1;
      break;
    }
    const float alpha = s_coef;
    // ---------------- phase A ----------------
    float rzl = 0.f, rrl = 0.f;
    constexpr int PA = 1;  // node bricks per phase-A pass
    for (int jb0 = blockIdx.x; jb0 < A.nb; jb0 += PA * G) {
      // PA node bricks per pass, all loads issued first
      float2 d2[PA * 3], p2[PA * 3], q2[PA * 3], x2[PA * 3], r2[PA * 3];
#pragma unroll
      for (int e = 0; e < PA * 3; ++e) {
        const int jb = jb0 + (e / 3) * G, a = e % 3;
        if (jb < A.nb) {
          const int64_t o = ((int64_t)jb * 3 + a) * BV + 2 * threadIdx.x;
          d2[e] = __ldcg(reinterpret_cast<const float2*>(A.dinv + o));
          p2[e] = __ldcg(reinterpret_cast<const float2*>(pnext + o));
          q2[e] = __ldcg(reinterpret_cast<const float2*>(A.q + o));
          x2[e] = __ldcg(reinterpret_cast<const float2*>(A.x + o));
          r2[e] = __ldcg(reinterpret_cast<const float2*>(A.r + o));
        } else {
          d2[e] = p2[e] = q2[e] = x2[e] = r2[e] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int e = 0; e < PA * 3; ++e) {
        const int jb = jb0 + (e / 3) * G, a = e % 3;
        if (jb >= A.nb) continue;
        const int64_t o = ((int64_t)jb * 3 + a) * BV + 2 * threadIdx.x;
        const float2 d = d2[e], pp = p2[e], qq = q2[e];
        float2 xx = x2[e], rr = r2[e];
        if (d.x > 0.f) {
          xx.x += alpha * pp.x;
          rr.x -= alpha * qq.x;
        }
        if (d.y > 0.f) {
          xx.y += alpha * pp.y;
          rr.y -= alpha * qq.y;
        }
        *reinterpret_cast<float2*>(A.x + o) = xx;
        *reinterpret_cast<float2*>(A.r + o) = rr;
        *reinterpret_cast<float2*>(A.q + o) = make_float2(0.f, 0.f);
        rzl += (d.x > 0.f ? rr.x * d.x * rr.x : 0.f) + (d.y > 0.f ? rr.y * d.y * rr.y : 0.f);
        rrl += (d.x > 0.f ? rr.x * rr.x : 0.f) + (d.y > 0.f ? rr.y * rr.y : 0.f);
      }
    }
    double* accA = A.acc + 2 * ((2 * it + 1) & 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double* zz = A.acc + 2 * ((2 * it + 3) & 3);
      zz[0] = 0.0;
      zz[1] = 0.0;
    }
    block_atomic2(rzl, rrl, accA);
    if (!grid_barrier(A.gbar, &s_flag, A.spins)) {
      alive = false;
      break;
    }
    ++it;
    if (threadIdx.x == 0) {
      const double rzn = __ldcg(accA), rrn = __ldcg(accA + 1);
      s_rr_last = rrn;
      s_stop = (rrn <= s_tol2 || it >= A.cg_max || !(rrn == rrn)) ? 1 : 0;
      s_coef = (float)(rzn / s_rz);
      s_rz = rzn;
    }
    __syncthreads();
    done = s_stop;
    beta = s_coef;
    float* tmp = pold;
    pold = pnext;
    pnext = tmp;
  }
  if (!alive && threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->iters = it;
    sc->rr_last = s_rr_last;
    sc->rz = s_rz;
    sc->done = 1;
  }
}

// The kernels of the persistent solver: tangent format x staging (1 shared-memory
// block, 2 streamed rows, 3 column groups).
static const void* pcg_kernel(int k45, int staging, int ctas) {
  if (staging == MPML_PCG_COLUMNS) {
    if (ctas <= 2) return k45 ? (const void*)k_pcg_groups<true, 2> : (const void*)k_pcg_groups<false, 2>;
    if (ctas == 3) return k45 ? (const void*)k_pcg_groups<true, 3> : (const void*)k_pcg_groups<false, 3>;
    return k45 ? (const void*)k_pcg_groups<true, 4> : (const void*)k_pcg_groups<false, 4>;
  }
  const bool streamed = staging == MPML_PCG_STREAMED;
  return k45 ? (streamed ? (const void*)k_pcg_persistent<true, true> : (const void*)k_pcg_persistent<true>)
             : (streamed ? (const void*)k_pcg_persistent<false, true> : (const void*)k_pcg_persistent<false>);
}

static size_t pcg_smem(int k45, int staging, int ctas) {
  if (staging == MPML_PCG_COLUMNS) return 0;  // static shared memory only
  return staging == MPML_PCG_STREAMED ? sizeof(float) * (3 * 729 + HVP_X_FLOATS + HVP_R_FLOATS) + 32
                                      : (k45 ? HVP_K_SMEM45 : HVP_C_SMEM_COL);
}

// launch_fit slots: CTA-per-brick forms k45 + 2 (staging - 1); column groups by their build
static int pcg_slot(int k45, int staging, int ctas) {
  if (staging == MPML_PCG_COLUMNS) return LS_PCG + 4 + 3 * k45 + (ctas <= 2 ? 0 : ctas - 2);
  return LS_PCG + k45 + 2 * (staging - 1);
}

// the autotuner's shapes: (staging, CTAs per SM)
static const int PCG_SHAPE_TABLE[MPML_PCG_SHAPES][2] = {
    {MPML_PCG_STAGED, 1},  {MPML_PCG_STAGED, 2},  {MPML_PCG_STREAMED, 1}, {MPML_PCG_STREAMED, 2},
    {MPML_PCG_COLUMNS, 2}, {MPML_PCG_COLUMNS, 3}, {MPML_PCG_COLUMNS, 4}};

// tile-cache format keys of the persistent solver's shapes (the standalone HVP uses 25 and 45)
static int pcg_cache_format(int k45) { return k45 ? 145 : 125; }

// The shape (staging, CTAs per SM) of the next persistent launch: the context's
// explicit configuration, else the autotuned shape cached for this format and
// size class, else the fixed rule -- beyond eight cell bricks per SM the
// column-group solver at three CTAs per SM (256^3 slab on sand at impact, 45
// numbers: 186 us per CG iteration against 204 us at four CTAs per SM and 248 us
// for the shared-memory block; 3-8M pressed block, compressed: 73 us against
// 82 us streamed), below it the CTA-per-brick solver with the shared-memory
// block (two CTAs per SM).
static int pcg_shape(mpml_ctx_s* c, int* staging, int* ctas, int* nsm) {
  const int k45 = c->compressed ? 0 : 1;
  int st = c->pcg_cfg.tangent_staging, cp = c->pcg_cfg.ctas_per_sm;
  if (st == MPML_PCG_AUTO || cp == 0) {
    const int cached = tile_cache_lookup_fmt(pcg_cache_format(k45), c->ncb);
    if (cached >= 0 && cached < MPML_PCG_SHAPES) {
      if (st == MPML_PCG_AUTO) st = PCG_SHAPE_TABLE[cached][0];
      if (cp == 0 && st == PCG_SHAPE_TABLE[cached][0]) cp = PCG_SHAPE_TABLE[cached][1];
    }
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return MPML_ERR_CUDA;
  }
  if (st == MPML_PCG_AUTO) st = c->ncb > 4 * 2 * (int64_t)n ? MPML_PCG_COLUMNS : MPML_PCG_STAGED;
  // the column-group form has a build per CTA count (2, 3, 4); without a choice, three
  const int want = cp > 0 ? cp : (st == MPML_PCG_COLUMNS ? 3 : 2);
  const int fit = launch_fit(pcg_kernel(k45, st, want), 256, pcg_smem(k45, st, want), pcg_slot(k45, st, want), nullptr);
  if (fit <= 0) return MPML_ERR_CUDA;
  if (cp == 0) cp = fit < want ? fit : want;
  if (cp > fit) return MPML_ERR_ARG;
  *staging = st;
  *ctas = cp;
  *nsm = n;
  return MPML_OK;
}

// One cooperative launch of the persistent solver with the given shape;
// ev0 / ev1 (optional) are recorded around it on the context stream.
static int pcg_launch(mpml_ctx_s* c, int cg_max, int staging, int ctas, int nsm, cudaEvent_t ev0, cudaEvent_t ev1) {
  const int k45 = c->compressed ? 0 : 1;
  const void* kfn = pcg_kernel(k45, staging, ctas);
  const size_t smem = pcg_smem(k45, staging, ctas);
  const int G = ctas * nsm;
  int rc;
  // barrier words (2 unsigned) followed by the 4 x 2 rotating accumulators
  if ((rc = ensure(c->gbar, 16 + 8 * sizeof(double))) || (rc = ensure(c->np2, sizeof(float) * 3 * c->nb * BV)))
    return rc;
  cudaMemsetAsync(c->gbar.p, 0, 16 + 8 * sizeof(double), c->s);
  PcgArgs a;
  a.cblist = (const int*)c->cblist.p;
  a.nolist = (const int*)c->nolist.p;
  a.nbr = (const int*)c->nbr.p;
  a.cflag = (const uint8_t*)c->cflag.p;
  a.C = (const float*)c->cK.p;
  a.m = (const float*)c->nmass.p;
  a.dinv = (const float*)c->ndinv.p;
  a.x = (float*)c->nx.p;
  a.r = (float*)c->nr.p;
  a.pa = (float*)c->np.p;
  a.pb = (float*)c->np2.p;
  a.q = (float*)c->nq.p;
  a.sc = dscal(c);
  a.acc = (double*)((char*)c->gbar.p + 16);
  a.gbar = (unsigned*)c->gbar.p;
  a.ncb = (int)c->ncb;
  a.nnob = (int)c->nnob;
  a.nb = (int)c->nb;
  a.cg_max = cg_max;
  a.spins = c->pcg_cfg.barrier_spins ? c->pcg_cfg.barrier_spins : BARRIER_SPINS_DEFAULT;
  a.status = (int*)c->status.p;
  a.pf = c->profiling ? (DevProf*)c->prof.p : nullptr;
  // q starts at zero (the phase-A kernel zeroes it after each use)
  cudaMemsetAsync(c->nq.p, 0, sizeof(float) * 3 * c->nb * BV, c->s);
  void* args[] = {&a};
  if (ev0) cudaEventRecord(ev0, c->s);
  rc = cuda_status(cudaLaunchCooperativeKernel(kfn, dim3(G), dim3(256), args, smem, c->s));
  if (ev1) cudaEventRecord(ev1, c->s);
  c->launches++;
  c->pcg_last_staging = staging;
  c->pcg_last_ctas = ctas;
  return rc;
}

static int pcg_persistent(mpml_ctx_s* c, const mpml_solver_opts* o) {
  int staging = 0, ctas = 0, nsm = 0, rc;
  if ((rc = pcg_shape(c, &staging, &ctas, &nsm))) return rc;
  const bool timed = c->profiling && c->pcg_ev[0] && c->pcg_ev[1];
  return pcg_launch(c, o->cg_max, staging, ctas, nsm, timed ? c->pcg_ev[0] : nullptr, timed ? c->pcg_ev[1] : nullptr);
}

// Persistent-solver autotuner (mpml_autotune_pcg): linearises at the current
// iterate, then every shape runs `iters` CG iterations of that system from the
// same start (x, r, p and the
// scalars are saved before and restored after each run, with the stopping
// tolerance cleared so that every shape runs all iterations); best of reps.
int pcg_autotune(mpml_ctx_s* c, int iters, int reps, int* choice, float* ms) {
  if (c->fp64 || !c->have_lin) return MPML_ERR_ARG;
  if (iters < 1) iters = 1;
  if (reps < 1) reps = 1;
  for (int k = 0; k < MPML_PCG_SHAPES; ++k)
    if (ms) ms[k] = -1.f;
  if (c->ncb == 0) {
    if (choice) *choice = 0;
    return MPML_OK;
  }
  const int k45 = c->compressed ? 0 : 1;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || nsm <= 0) {
    cudaGetLastError();
    return MPML_ERR_CUDA;
  }
  const size_t vb = sizeof(float) * 3 * c->nb * BV;
  int rc;
  // the Newton system at the current iterate, with a fresh CG start (x = 0, r = -g)
  if ((rc = prep_t<float>(c, 1, 1, 1e-6, iters))) return rc;
  if ((rc = ensure(c->tuneq, 3 * vb + sizeof(DevScalars)))) return rc;
  char* save = (char*)c->tuneq.p;
  DevScalars* sv = (DevScalars*)(save + 3 * vb);
  cudaMemcpyAsync(save, c->nx.p, vb, cudaMemcpyDeviceToDevice, c->s);
  cudaMemcpyAsync(save + vb, c->nr.p, vb, cudaMemcpyDeviceToDevice, c->s);
  cudaMemcpyAsync(save + 2 * vb, c->np.p, vb, cudaMemcpyDeviceToDevice, c->s);
  cudaMemcpyAsync(sv, c->scal.p, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c->s);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return MPML_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return MPML_ERR_CUDA;
  }
  auto restore = [&]() {
    cudaMemcpyAsync(c->nx.p, save, vb, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(c->nr.p, save + vb, vb, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(c->np.p, save + 2 * vb, vb, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(c->scal.p, sv, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c->s);
  };
  float best = 0.f;
  int arg = -1;
  for (int shape = 0; shape < MPML_PCG_SHAPES && !rc; ++shape) {
    const int staging = PCG_SHAPE_TABLE[shape][0], ctas = PCG_SHAPE_TABLE[shape][1];
    const int fit = launch_fit(pcg_kernel(k45, staging, ctas), 256, pcg_smem(k45, staging, ctas),
                               pcg_slot(k45, staging, ctas), nullptr);
    if (fit < ctas) continue;
    float tbest = -1.f;
    for (int i = 0; i <= reps && !rc; ++i) {
      restore();
      cudaMemsetAsync(&((DevScalars*)c->scal.p)->tol2, 0, sizeof(double), c->s);
      cudaMemsetAsync(&((DevScalars*)c->scal.p)->done, 0, sizeof(int), c->s);
      if ((rc = pcg_launch(c, iters, staging, ctas, nsm, a, b))) break;
      if ((rc = cuda_status(cudaEventSynchronize(b)))) break;
      float e = 0.f;
      cudaEventElapsedTime(&e, a, b);
      if (i > 0 && (tbest < 0.f || e < tbest)) tbest = e;  // the first run is a warm-up
    }
    if (rc) break;
    if (ms) ms[shape] = tbest;
    if (arg < 0 || tbest < best) {
      best = tbest;
      arg = shape;
    }
  }
  restore();
  const int rc2 = cuda_status(cudaStreamSynchronize(c->s));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (rc2) return rc2;
  if (arg < 0) return MPML_ERR_CUDA;
  if (choice) *choice = arg;
  tile_cache_store_fmt(pcg_cache_format(k45), c->ncb, arg, best);
  return MPML_OK;
}

// after the solve has been read back: add the launch's event time and iterations
static void pcg_persistent_account(mpml_ctx_s* c) {
  if (!(c->profiling && c->pcg_ev[0] && c->pcg_ev[1])) return;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->pcg_ev[0], c->pcg_ev[1]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c->pcg_ms += ms;
  c->pcg_launches += 1;
  c->pcg_iters += c->hscal->iters;
}
// [persistent-solver source: end]

// ---------------------------------------------------------------------------
// Flexible CG with the learned preconditioner (FP32 contexts).  Notay's FCG
// with one stored direction: alpha = r^T z / p^T H p, beta = -z^T H p / p^T H p
// (equal to the Polak-Ribiere form).  Stall rule: z^T r <= 0, or no decrease
// of r^T r in 20 iterations -> the solve continues with Jacobi-PCG.
// ---------------------------------------------------------------------------
// sums of the per-brick (z^T q, z^T r) partials (one block, fixed order)
__global__ void __launch_bounds__(512) k_fcg_beta(const double* __restrict__ part, int nb, DevScalars* sc,
                                                  int init) {
  __shared__ double red[2][16];
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double zq = 0, zr = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    zq += red[0][w];
    zr += red[1][w];
  }
  if (sc->done) return;
  if (!(zr > 0.0)) {  // not a descent direction: fall back to Jacobi
    sc->fallback = 1;
    sc->done = 1;
    return;
  }
  sc->beta = init ? 0.0 : -zq / sc->pq;
  sc->rz = zr;
}

// p = z + beta p, q(face) = m p, sum m |p|^2
__global__ void __launch_bounds__(512) k_fcg_p(const float* __restrict__ z, const float* __restrict__ m, float* p,
                                               float* q, DevScalars* sc, double* part) {
  __shared__ int s_done;
  __shared__ float s_beta;
  if (threadIdx.x == 0) {
    s_done = sc->done;
    s_beta = (float)sc->beta;
  }
  __syncthreads();
  if (s_done) return;
  const int id = blockIdx.x, l = threadIdx.x;
  const bool face = (l & 7) == 0 || ((l >> 3) & 7) == 0 || (l >> 6) == 0;
  const float mi = m[(int64_t)id * BV + l];
  float pmp = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = ((int64_t)id * 3 + a) * BV + l;
    const float pv = z[o] + s_beta * p[o];
    p[o] = pv;
    if (face) q[o] = mi * pv;
    pmp += mi * pv * pv;
  }
  double vals[1] = {(double)pmp};
  block_store<1>(vals, part);
  if (arrive_last(&sc->counter[CNT_B])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    sc->pMp = tot[0];
    sc->counter[CNT_B] = 0;
  }
}

// r^T D^-1 r of the current residual; restart values for Jacobi-PCG
__global__ void __launch_bounds__(512) k_rz_jacobi(const float* __restrict__ r, const float* __restrict__ dinv,
                                                   DevScalars* sc, double* part, int restart) {
  const int id = blockIdx.x, l = threadIdx.x;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = ((int64_t)id * 3 + a) * BV + l;
    const float di = dinv[o];
    if (di > 0.f) s += r[o] * di * r[o];
  }
  double vals[1] = {(double)s};
  block_store<1>(vals, part);
  if (arrive_last(&sc->counter[CNT_MISC])) {
    double tot[1];
    block_sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    sc->rzj = tot[0];
    sc->nn_s = sc->nfree > 0 ? sqrt(tot[0] / sc->nfree) : 0.0;
    if (restart) {
      sc->rz = tot[0];
      sc->done = 0;
      sc->fallback = 0;
      sc->iters = 0;
    }
    sc->counter[CNT_MISC] = 0;
  }
}

static void fcg_iteration(mpml_ctx_s* c) {
  const unsigned nb = (unsigned)c->nb;
  DevScalars* d = dscal(c);
  launch_hvp<float>(c, (const float*)c->np.p, (float*)c->nq.p, 1);
  k_cg_a4<<<nb, 128, 0, c->s>>>((const float*)c->ndinv.p, (const float*)c->np.p, (const float*)c->nq.p,
                                (float*)c->nx.p, (float*)c->nr.p, d, part_a(c), 1);
  nn_apply(c, &d->nn_s, (const float*)c->nq.p, part_fin(c));
  k_fcg_beta<<<1, 512, 0, c->s>>>(part_fin(c), (int)c->nb, d, 0);
  k_fcg_p<<<nb, BV, 0, c->s>>>((const float*)c->nz.p, (const float*)c->nmass.p, (float*)c->np.p, (float*)c->nq.p, d,
                               part_b(c));
  c->launches += 4;
}

// flexible CG from the state left by prep (x = 0, r = -g, Jacobi scalars);
// returns iterations and whether it fell back
static int fcg_solve(mpml_ctx_s* c, const mpml_solver_opts* o, int* iters, int* fell_back) {
  int rc;
  DevScalars* d = dscal(c);
  if ((rc = nn_ensure(c))) return rc;
  const unsigned nb = (unsigned)c->nb;
  // z0 = B(r0), rz = z0^T r0, p0 = z0
  k_rz_jacobi<<<nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, d, part_b(c), 0);
  nn_apply(c, &d->nn_s, nullptr, part_fin(c));
  k_fcg_beta<<<1, 512, 0, c->s>>>(part_fin(c), (int)c->nb, d, 1);
  k_fcg_p<<<nb, BV, 0, c->s>>>((const float*)c->nz.p, (const float*)c->nmass.p, (float*)c->np.p, (float*)c->nq.p, d,
                               part_b(c));
  c->launches += 3;
  if ((rc = read_scalars(c))) return rc;
  const int every = o->check_every > 0 ? o->check_every : 8;
  int launched = 0;
  while (!c->hscal->done && launched < o->cg_max) {
    for (int j = 0; j < every && launched < o->cg_max; ++j, ++launched) fcg_iteration(c);
    if ((rc = cuda_status(cudaGetLastError()))) return rc;
    if ((rc = read_scalars(c))) return rc;
  }
  *iters = c->hscal->iters;
  *fell_back = c->hscal->fallback;
  return MPML_OK;
}

// ---------------------------------------------------------------------------
// training data and training (learned preconditioner)
// ---------------------------------------------------------------------------
// FP64 sum of a . b over free slots (atomic; training path only)
__global__ void __launch_bounds__(512) k_dot_ff(const float* __restrict__ a, const float* __restrict__ b,
                                                const float* __restrict__ dinv, double* out) {
  const int id = blockIdx.x, l = threadIdx.x;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t o = ((int64_t)id * 3 + c) * BV + l;
    if (dinv[o] > 0.f) s += a[o] * b[o];
  }
  double vals[1] = {(double)s};
  double* const dst[1] = {out};
  block_add<1>(vals, dst);
}

// y = a - b (free slots)
__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b, const float* __restrict__ dinv,
                      float* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = dinv[i] > 0.f ? a[i] - b[i] : 0.f;
}

// loss gradient w.r.t. the network output, L = 1 - a / sqrt(b c) with
// a = z^T r, b = z^T H z, c = e^T H e:
//   dL/dz = -r / sqrt(b c) + a H z / (sqrt(c) b^(3/2)),  gy = s sqrt(D^-1) dL/dz
__global__ void k_nn_gy(const float* __restrict__ hz, const float* __restrict__ r, const float* __restrict__ dinv,
                        const DevScalars* sc, double cden, float* gy, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float di = dinv[i];
  if (!(di > 0.f)) {
    gy[i] = 0.f;
    return;
  }
  const double a = sc->nn_a, b = sc->nn_b, s = sc->nn_s;
  const double sb = sqrt(b > 0.0 ? b : 1e-300), sc_ = sqrt(cden);
  const float cr = (float)(-s / (sb * sc_));
  const float ch = (float)(s * a / (sc_ * sb * sb * sb));
  gy[i] = sqrtf(di) * (cr * r[i] + ch * hz[i]);
}

// FP32 HVP y = H p on the current linearisation (q faces initialised to m p)
static void hvp_f32(mpml_ctx_s* c, const float* p, float* y) {
  const int64_t ns = c->nb * BV;
  cudaMemsetAsync(y, 0, sizeof(float) * 3 * ns, c->s);
  k_init_faces<float><<<(unsigned)c->nb, BV, 0, c->s>>>(p, (const float*)c->nmass.p, y);
  if (c->ncb > 0) launch_hvp<float>(c, p, y, 0);
  c->launches++;
}

// one training pair (r in c->nr; den = e^T H e): loss 1 - cos_H(z(r), e), and
// the weight gradient accumulated (scaled) on the device
static int nn_pair(mpml_ctx_s* c, double den, float scale, double* loss_out, bool backward) {
  DevScalars* d = dscal(c);
  const int64_t ns = c->nb * BV, n3 = 3 * ns;
  const unsigned nb = (unsigned)c->nb;
  k_rz_jacobi<<<nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, d, part_b(c), 0);
  nn_apply(c, &d->nn_s, nullptr, nullptr);
  float* z = (float*)c->nz.p;
  float* hz = (float*)c->nnhd.p;
  hvp_f32(c, z, hz);
  cudaMemsetAsync(&d->nn_a, 0, 2 * sizeof(double), c->s);
  k_dot_ff<<<nb, BV, 0, c->s>>>(z, (const float*)c->nr.p, (const float*)c->ndinv.p, &d->nn_a);
  k_dot_ff<<<nb, BV, 0, c->s>>>(z, hz, (const float*)c->ndinv.p, &d->nn_b);
  c->launches += 4;
  if (backward) {
    // gy overwrites z (no longer needed)
    k_nn_gy<<<div_up(n3, 256), 256, 0, c->s>>>(hz, (const float*)c->nr.p, (const float*)c->ndinv.p, d, den, z, n3);
    nn_backward(c, z, scale);
    c->launches++;
  }
  if (loss_out) {
    int rc = read_scalars(c);
    if (rc) return rc;
    const double a = c->hscal->nn_a, b = c->hscal->nn_b;
    *loss_out = b > 0.0 ? 1.0 - a / sqrt(b * den) : 1.0;
  }
  return cuda_status(cudaGetLastError());
}

int nn_collect(mpml_ctx_s* c, int nsamples, double rtol, int cg_max) {
  // the current Newton system: stretch + prep at vhat (Dirichlet values set)
  int rc;
  if (c->fp64 || !c->compressed) return MPML_ERR_ARG;
  if ((rc = stretch_all(c)) || (rc = alloc_solver<float>(c)) || (rc = nn_ensure(c))) return rc;
  const int64_t ns = c->nb * BV, n3 = 3 * ns;
  if (nsamples < 1) nsamples = 1;
  if ((rc = ensure(c->nns_r, sizeof(float) * n3 * nsamples)) || (rc = ensure(c->nns_e, sizeof(float) * n3 * nsamples)) ||
      (rc = ensure(c->nnhd, sizeof(float) * n3)))
    return rc;
  // first pass: iteration count of the solve
  if ((rc = prep_t<float>(c, 1, 1, rtol, cg_max)) || (rc = read_scalars(c))) return rc;
  int total = 0;
  while (!c->hscal->done && total < cg_max) {
    for (int j = 0; j < 16 && total < cg_max; ++j, ++total) cg_iteration<float>(c);
    if ((rc = read_scalars(c))) return rc;
  }
  total = c->hscal->iters;
  // second pass with snapshots of (r_k, x_k) at k_j = j total / nsamples
  if ((rc = prep_t<float>(c, 1, 1, rtol, cg_max)) || (rc = read_scalars(c))) return rc;
  float* R = (float*)c->nns_r.p;
  float* E = (float*)c->nns_e.p;
  int it = 0;
  for (int j = 0; j < nsamples; ++j) {
    const int target = (int)((int64_t)j * total / nsamples);
    while (it < target) {
      cg_iteration<float>(c);
      ++it;
    }
    cudaMemcpyAsync(R + (int64_t)j * n3, c->nr.p, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(E + (int64_t)j * n3, c->nx.p, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
  }
  if ((rc = read_scalars(c))) return rc;
  while (!c->hscal->done && it < cg_max) {
    for (int j = 0; j < 16 && it < cg_max; ++j, ++it) cg_iteration<float>(c);
    if ((rc = read_scalars(c))) return rc;
  }
  // e_j = x* - x_{k_j}
  for (int j = 0; j < nsamples; ++j)
    k_sub<<<div_up(n3, 256), 256, 0, c->s>>>((const float*)c->nx.p, E + (int64_t)j * n3, (const float*)c->ndinv.p,
                                             E + (int64_t)j * n3, n3);
  c->nn_nsamples = nsamples;
  return cuda_status(cudaStreamSynchronize(c->s));
}

int nn_train(mpml_ctx_s* c, int epochs, int batch, float lr, double* loss_first, double* loss_last) {
  int rc;
  if (!c->nn_ready || c->nn_nsamples < 1) return MPML_ERR_ARG;
  const int ns_ = c->nn_nsamples;
  const int64_t n3 = 3 * c->nb * BV;
  float* R = (float*)c->nns_r.p;
  float* E = (float*)c->nns_e.p;
  // e^T H e of every pair; pairs whose error is at rounding level (a late
  // sample of a stiff system, where x* - x_k keeps only FP32 noise) are not
  // used: their direction carries no information
  std::vector<double> den(ns_);
  std::vector<int> use;
  for (int j = 0; j < ns_; ++j) {
    float* e = E + (int64_t)j * n3;
    hvp_f32(c, e, (float*)c->nnhd.p);
    DevScalars* d = dscal(c);
    cudaMemsetAsync(&d->slope, 0, sizeof(double), c->s);
    k_dot_ff<<<(unsigned)c->nb, BV, 0, c->s>>>(e, (const float*)c->nnhd.p, (const float*)c->ndinv.p, &d->slope);
    if ((rc = read_scalars(c))) return rc;
    den[j] = c->hscal->slope;
    if (den[j] > 1e-10 * den[0] && std::isfinite(den[j])) use.push_back(j);
  }
  if (use.empty()) return MPML_ERR_NONFINITE;
  if (batch < 1) batch = 1;
  uint64_t rng = 0x9e3779b97f4a7c15ull;
  const int nu = (int)use.size();
  std::vector<int> order(nu);
  for (int ep = 0; ep < epochs; ++ep) {
    for (int j = 0; j < nu; ++j) order[j] = use[j];
    for (int j = nu - 1; j > 0; --j) {  // Fisher-Yates with a fixed LCG
      rng = rng * 6364136223846793005ull + 1442695040888963407ull;
      const int k = (int)((rng >> 33) % (uint64_t)(j + 1));
      std::swap(order[j], order[k]);
    }
    double lsum = 0;
    int inb = 0;
    for (int jj = 0; jj < nu; ++jj) {
      const int j = order[jj];
      cudaMemcpyAsync(c->nr.p, R + (int64_t)j * n3, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
      double l = 0;
      // lr = 0: evaluation only (no gradient, no update)
      if ((rc = nn_pair(c, den[j], 1.0f / (float)batch, &l, lr != 0.f))) return rc;
      lsum += l;
      if (++inb == batch || jj == nu - 1) {
        if (lr != 0.f) {
          nn_adam(c, lr, ++c->nn_adam_step);
          if ((rc = nn_refresh_weights(c))) return rc;
        }
        inb = 0;
      }
    }
    if (ep == 0 && loss_first) *loss_first = lsum / nu;
    if (loss_last) *loss_last = lsum / nu;
  }
  return cuda_status(cudaStreamSynchronize(c->s));
}

// z = B(r) for a given node vector (tests); needs a linearisation
int nn_apply_host(mpml_ctx_s* c, const void* r_nodes, void* z_nodes) {
  int rc;
  if (!c->nn_ready) return MPML_ERR_ARG;
  if ((rc = nn_ensure(c))) return rc;
  const int64_t n3 = 3 * c->nb * BV;
  cudaMemcpyAsync(c->nr.p, r_nodes, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
  DevScalars* d = dscal(c);
  k_rz_jacobi<<<(unsigned)c->nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, d, part_b(c), 0);
  nn_apply(c, &d->nn_s, nullptr, nullptr);
  cudaMemcpyAsync(z_nodes, c->nz.p, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
  return cuda_status(cudaStreamSynchronize(c->s));
}

// loss of one pair and its weight gradient (device grad buffer zeroed first)
int nn_loss_grad_host(mpml_ctx_s* c, const void* r_nodes, const void* e_nodes, double* loss) {
  int rc;
  if (!c->nn_ready) return MPML_ERR_ARG;
  const int64_t n3 = 3 * c->nb * BV;
  if ((rc = ensure(c->nnhd, sizeof(float) * n3)) || (rc = ensure(c->nns_e, sizeof(float) * n3))) return rc;
  cudaMemcpyAsync(c->nr.p, r_nodes, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
  float* e = (float*)c->nns_e.p;
  cudaMemcpyAsync(e, e_nodes, sizeof(float) * n3, cudaMemcpyDeviceToDevice, c->s);
  // den = e^T H e
  hvp_f32(c, e, (float*)c->nnhd.p);
  DevScalars* d = dscal(c);
  cudaMemsetAsync(&d->slope, 0, sizeof(double), c->s);
  k_dot_ff<<<(unsigned)c->nb, BV, 0, c->s>>>(e, (const float*)c->nnhd.p, (const float*)c->ndinv.p, &d->slope);
  if ((rc = read_scalars(c))) return rc;
  const double den = c->hscal->slope > 0 ? c->hscal->slope : 1.0;
  // zero the gradient accumulator, then one pair with scale 1
  std::vector<float> zeros((size_t)nn_weight_count(), 0.f);
  (void)zeros;
  return nn_pair(c, den, 1.0f, loss, true);
}

static int ensure_hvp_tile(mpml_ctx_s* c);

template <typename T>
static int pcg_t(mpml_ctx_s* c, const mpml_solver_opts* o, int* iters, double* rel) {
  int rc;
  if (sizeof(T) == 4 && o->precond == MPML_PRECOND_LEARNED && c->nn_ready && c->compressed) {
    int fit = 0, fb = 0;
    if ((rc = fcg_solve(c, o, &fit, &fb))) return rc;
    c->last_fcg_fallback = fb;
    if (!fb) {
      *iters = fit;
      const double rr0 = c->hscal->rr0;
      *rel = rr0 > 0 ? sqrt(c->hscal->rr_last / rr0) : 0.0;
      return MPML_OK;
    }
    // flexible CG stalled: continue from the current x, r with Jacobi-PCG
    k_rz_jacobi<<<(unsigned)c->nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, dscal(c),
                                                   part_b(c), 1);
    c->launches++;
    mpml_solver_opts j = *o;
    j.precond = MPML_PRECOND_JACOBI;
    j.cg_max = o->cg_max > fit ? o->cg_max - fit : 1;
    int jit = 0;
    if ((rc = pcg_t<T>(c, &j, &jit, rel))) return rc;
    *iters = fit + jit;
    return MPML_OK;
  }
  if (sizeof(T) == 4 && o->use_graph == 2) {
    if ((rc = pcg_persistent(c, o))) return rc;
    if ((rc = read_scalars(c))) return rc;
    pcg_persistent_account(c);
    *iters = c->hscal->iters;
    const double rr0p = c->hscal->rr0;
    *rel = rr0p > 0 ? sqrt(c->hscal->rr_last / rr0p) : 0.0;
    return MPML_OK;
  }
  if (sizeof(T) == 4 && (rc = ensure_hvp_tile(c))) return rc;
  if (o->use_graph && c->ncb > 0 && ensure_cg_graph<T>(c, o->cg_max) == MPML_OK) {
    if ((rc = cuda_status(cudaGraphLaunch(c->cg_exec, c->s)))) return rc;
    if ((rc = read_scalars(c))) return rc;
    c->launches += (int64_t)c->hscal->bodies * (3 * CG_UNROLL + 1);
  } else {
    const int every = o->check_every > 0 ? o->check_every : 16;
    int launched = 0;
    if ((rc = read_scalars(c))) return rc;
    while (!c->hscal->done && launched < o->cg_max) {
      for (int j = 0; j < every && launched < o->cg_max; ++j, ++launched) cg_iteration<T>(c);
      if ((rc = cuda_status(cudaGetLastError()))) return rc;
      if ((rc = read_scalars(c))) return rc;
    }
  }
  *iters = c->hscal->iters;
  const double rr0 = c->hscal->rr0;
  *rel = rr0 > 0 ? sqrt(c->hscal->rr_last / rr0) : 0.0;
  return MPML_OK;
}

template <typename T>
static int energy_t(mpml_ctx_s* c, double alpha, double* phi, int* infeasible) {
  SolveInfo si = solve_info(c);
  DevScalars* d = dscal(c);
  cudaMemsetAsync(&d->phi_in, 0, sizeof(double), c->s);
  cudaMemsetAsync(&d->phi_el, 0, sizeof(double), c->s);
  cudaMemsetAsync(&d->infeasible, 0, sizeof(int), c->s);
  k_energy_nodes<T><<<node_blocks(c->nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p,
                                                     (const double*)c->nvnew.p, (const T*)c->nx.p,
                                                     (const double*)c->nvhat.p, alpha, d, (int)c->nb);
  if (c->ncb > 0)
    k_energy_cells<T><<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                         (const uint8_t*)c->cflag.p, (const T*)c->cacc.p,
                                                         (const double*)(c->fp_active ? c->cB.p : c->cs.p), (const double*)c->nvnew.p,
                                                         (const T*)c->nx.p, alpha, si, d);
  c->launches += 2;
  int rc = read_scalars(c);
  if (rc) return rc;
  *infeasible = c->hscal->infeasible;
  *phi = c->hscal->phi_in + c->hscal->phi_el;
  return MPML_OK;
}

// ---- fixed-point plasticity (Sec. "Fixed-Point Plasticity") -------------------
// the general bases start as the stretch step's symmetric S - I
__global__ void __launch_bounds__(256) k_base_init(const int* __restrict__ cblist, const double* __restrict__ cs,
                                                   int nm, double* cb) {
  const int64_t id = cblist[blockIdx.x];
  for (int l = threadIdx.x; l < BV; l += blockDim.x)
    for (int k = 0; k < nm; ++k) {
      double bm[9];
      load_base(cs, 0, id, nm, k, l, bm);
#pragma unroll
      for (int q = 0; q < 9; ++q) cb[((id * nm + k) * 9 + q) * BV + l] = bm[q];
    }
}

// At the iterate v: each slot of a plastic material takes its trial F = (I + dt G_c(v)) B
// to the yield surface by the material's return map (FP64); where that changes F the
// base becomes B = (I + dt G_c(v))^{-1} F^E, so that F_c(v) = F^E.  The linear solves
// then see elasticity only.
__global__ void __launch_bounds__(256) k_plastic_fp(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                    const uint8_t* __restrict__ cflag, const void* __restrict__ accv,
                                                    int fp64, const double* __restrict__ v, SolveInfo si,
                                                    double* cb, int* changed) {
  __shared__ double sv[3][729];
  const int id = cblist[blockIdx.x];
  stage_nodes<double, double, double>(id, nbr, v, nullptr, 0.0, sv);
  __syncthreads();
  const double sgd = si.dt * 0.25 / si.dx;
  int nch = 0;
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    if (!cflag[(int64_t)id * BV + l]) continue;
    double D[9];
    gather_D<double>(l, sv, D);
    double A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = sgd * D[q] + ((q % 4 == 0) ? 1.0 : 0.0);
    const double cof[9] = {A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
                           A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
                           A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
    const double det = A[0] * cof[0] + A[1] * cof[3] + A[2] * cof[6];
    if (!(det > 0.0)) continue;
    for (int k = 0; k < si.nm; ++k) {
      if (si.plastic[k] == MPML_ELASTIC) continue;
      const double V = fp64 ? ((const double*)accv)[((int64_t)id * si.nf + acc_V(k)) * BV + l]
                             : (double)((const float*)accv)[((int64_t)id * si.nf + acc_V(k)) * BV + l];
      if (V == 0.0) continue;
      double bm[9], F[9];
      load_base(cb, 1, id, si.nm, k, l, bm);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          double acc = A[3 * a + b];
#pragma unroll
          for (int q = 0; q < 3; ++q) acc += A[3 * a + q] * bm[3 * q + b];
          F[3 * a + b] = acc;
        }
      if (!return_map<double>(si.plastic[k], si.mat[k].mu, si.mat[k].lam, si.ys[k], si.alpha[k], F)) continue;
      // B = A^{-1} F^E, stored as B - I
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double bv = (cof[3 * a] * F[b] + cof[3 * a + 1] * F[3 + b] + cof[3 * a + 2] * F[6 + b]) / det;
          cb[(((int64_t)id * si.nm + k) * 9 + 3 * a + b) * BV + l] = bv - ((a == b) ? 1.0 : 0.0);
        }
      ++nch;
    }
  }
  if (nch) atomicAdd(changed, nch);
}

// the general bases are used only inside one fixed-point solve
struct FixedPointScope {
  mpml_ctx_s* c;
  ~FixedPointScope() { c->fp_active = 0; }
};

// projection of every plastic slot at the current iterate; *changed += slots changed
template <typename T>
static int plastic_project(mpml_ctx_s* c, int* changed) {
  if (c->ncb == 0) return MPML_OK;
  DevScalars* d = dscal(c);
  cudaMemsetAsync(&d->nproj, 0, sizeof(int), c->s);
  k_plastic_fp<<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                  (const uint8_t*)c->cflag.p, c->cacc.p, sizeof(T) == 8,
                                                  (const double*)c->nvnew.p, solve_info(c), (double*)c->cB.p,
                                                  &d->nproj);
  c->launches++;
  int rc = read_scalars(c);
  if (rc) return rc;
  *changed += c->hscal->nproj;
  return MPML_OK;
}

// the CG stopping threshold |r|^2 <= tol2 of the next solve (inexact Newton)
__global__ void k_set_tol2(DevScalars* sc, double tol2) { sc->tol2 = tol2; }

int set_cg_tol2(mpml_ctx_s* c, cudaStream_t s, double tol2) {
  k_set_tol2<<<1, 1, 0, s>>>(dscal(c), tol2);
  c->launches++;
  return cuda_status(cudaGetLastError());
}

// Forcing term of Newton iteration k (opts.cg_forcing > 0): Eisenstat and Walker's
// second choice eta_k = 0.9 (|g_k| / |g_{k-1}|)^2 with their safeguard, capped at
// cg_forcing, floored at cg_rtol and at half of the reduction the Newton target still
// needs, and at most 0.5.
double newton_forcing(const mpml_solver_opts* o, int k, double gn, double gprev, double eta_prev, double target) {
  double eta = o->cg_forcing;
  if (k > 0 && gprev > 0.0) {
    const double q = gn / gprev;
    eta = 0.9 * q * q;
    const double sg = 0.9 * eta_prev * eta_prev;
    if (sg > 0.1 && sg > eta) eta = sg;
    if (eta > o->cg_forcing) eta = o->cg_forcing;
  }
  if (eta < o->cg_rtol) eta = o->cg_rtol;
  if (gn > 0.0 && eta < 0.5 * target / gn) eta = 0.5 * target / gn;
  return eta < 0.5 ? eta : 0.5;
}

template <typename T>
static int newton_t(mpml_ctx_s* c, const mpml_solver_opts* o, mpml_solve_stats* st) {
  int rc = alloc_solver<T>(c);
  if (rc) return rc;
  if (c->nb == 0) {
    st->status = MPML_OK;
    return MPML_OK;
  }
  bool fp = false;
  if (o->plastic_fixed_point)
    for (int k = 0; k < c->nm; ++k) fp = fp || c->mats[k].plastic != MPML_ELASTIC;
  FixedPointScope scope{c};
  if (fp) {
    if (c->compressed) return MPML_ERR_ARG;
    if ((rc = ensure(c->cB, sizeof(double) * 9 * c->nm * c->nb * BV))) return rc;
    if (c->ncb > 0) {
      k_base_init<<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const double*)c->cs.p, c->nm,
                                                      (double*)c->cB.p);
      c->launches++;
    }
    c->fp_active = 1;
  }
  if ((rc = prep_t<T>(c, 1, 1, o->cg_rtol, o->cg_max)) || (rc = read_scalars(c))) return rc;
  if (fp) {
    // project at v0 (prep has set it), then the gradient with the projected bases
    if ((rc = plastic_project<T>(c, &st->plastic_projections))) return rc;
    if ((rc = prep_t<T>(c, 1, 1, o->cg_rtol, o->cg_max)) || (rc = read_scalars(c))) return rc;
  }
  if (*c->hstatus & ST_NONFINITE) return MPML_ERR_NONFINITE;
  double g0 = sqrt(c->hscal->gg), gn = g0;
  const double gfloor = 1e-12 * sqrt(c->hscal->mv2);  // rounding level of the gradient
  double phi = c->hscal->phi_in + c->hscal->phi_el;
  double phi_el = c->hscal->phi_el;  // elastic energy at the current iterate
  st->g0_norm = g0;
  st->phi0 = phi;
  int status = MPML_OK, it = 0;
  double gprev = 0.0, eta = 0.0;
  const double target = fmax(o->newton_rtol * g0, o->newton_atol);
  while (true) {
    if (gn <= o->newton_rtol * g0 || gn <= o->newton_atol || gn <= gfloor) break;
    if (it >= o->newton_max) {
      status = MPML_WARN_NOT_CONVERGED;
      break;
    }
    if (o->cg_forcing > 0.0) {
      // inexact Newton: this solve stops at eta |g_k| (the prep set cg_rtol |g_k|)
      eta = newton_forcing(o, it, gn, gprev, eta, target);
      if ((rc = set_cg_tol2(c, c->s, eta * eta * gn * gn))) return rc;
    }
    gprev = gn;
    int cgit = 0;
    double rel = 0;
    c->last_fcg_fallback = 0;
    if ((rc = pcg_t<T>(c, o, &cgit, &rel))) return rc;
    st->fcg_fallbacks += c->last_fcg_fallback;
    if (it < 64) {
      st->cg_iters[it] = cgit;
      st->cg_rel_resid[it] = rel;
    }
    st->cg_iters_total += cgit;
    // slope g^T dx and the exact inertia change along dx
    DevScalars* d = dscal(c);
    cudaMemsetAsync(&d->slope, 0, 3 * sizeof(double), c->s);
    k_ls_setup<T><<<node_blocks(c->nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p,
                                                   (const double*)c->ng.p, (const double*)c->nvnew.p,
                                                   (const double*)c->nvhat.p, (const T*)c->nx.p, d, (int)c->nb);
    c->launches++;
    if ((rc = read_scalars(c))) return rc;
    const double slope = c->hscal->slope, lsA = c->hscal->ls_a, lsB = c->hscal->ls_b;
    double alpha = 1.0, phit = 0, phit_el = 0;
    bool accepted = false, linearised = false;
    int ls0 = 0;
    if (!fp) {
      // the full step first, by the prep at the trial iterate v + dx (without the CG start,
      // so that dx survives a rejection): its energy decides the Armijo test and, accepted,
      // it is the next iteration's linearisation (no separate line-search energy)
      k_axpy_out<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const T*)c->ndinv.p, (const T*)c->nx.p, 1.0,
                                                     (const double*)c->nvnew.p, (double*)c->nvtry.p);
      c->launches++;
      std::swap(c->nvnew, c->nvtry);
      if ((rc = prep_t<T>(c, 1, 0, o->cg_rtol, o->cg_max, 1, 1)) || (rc = read_scalars(c))) return rc;
      const double pel = c->hscal->phi_el, pin = c->hscal->phi_in, gg = c->hscal->gg;
      const double dphi = lsA + 0.5 * lsB + (pel - phi_el);
      if (c->hscal->infeasible == 0 && dphi <= o->ls_c1 * slope && gg == gg) {
        if ((rc = cg_start_t<T>(c, o->cg_rtol, o->cg_max))) return rc;
        accepted = linearised = true;
        phit = pin + pel;
        phit_el = pel;
        gn = sqrt(gg);
      } else {
        std::swap(c->nvnew, c->nvtry);  // back to v; dx is intact
        alpha = 0.5;
        ls0 = 1;
      }
    }
    for (int ls = ls0; !accepted && ls <= o->ls_max; ++ls) {
      int inf = 0;
      if ((rc = energy_t<T>(c, alpha, &phit, &inf))) return rc;
      phit_el = c->hscal->phi_el;
      // Armijo on the energy change: inertia part in closed form, elastic part as a
      // difference of the (accurately evaluated) elastic sums
      const double dphi = alpha * lsA + 0.5 * alpha * alpha * lsB + (phit_el - phi_el);
      if (inf == 0 && dphi <= o->ls_c1 * alpha * slope) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
    }
    if (it < 64) st->alpha[it] = accepted ? alpha : 0.0;
    ++it;
    if (!accepted) {
      status = MPML_WARN_NOT_CONVERGED;
      break;
    }
    if (linearised) {
      phi = phit;
      phi_el = phit_el;
      continue;
    }
    k_axpy<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const T*)c->ndinv.p, (const T*)c->nx.p, alpha, (double*)c->nvnew.p);
    c->launches++;
    if (fp) {
      // plastic projection at the new iterate; the energy changes with the bases
      if ((rc = plastic_project<T>(c, &st->plastic_projections))) return rc;
      if ((rc = prep_t<T>(c, 1, 1, o->cg_rtol, o->cg_max)) || (rc = read_scalars(c))) return rc;
      gn = sqrt(c->hscal->gg);
      phi = c->hscal->phi_in + c->hscal->phi_el;
      phi_el = c->hscal->phi_el;
      continue;
    }
    // the energy at the new iterate is the accepted line-search value (same formula
    // at v + alpha dx); prep skips it where its closed forms apply
    if ((rc = prep_t<T>(c, 1, 1, o->cg_rtol, o->cg_max, 0)) || (rc = read_scalars(c))) return rc;
    gn = sqrt(c->hscal->gg);
    phi = phit;
    phi_el = phit_el;
  }
  st->newton_iters = it;
  st->g_norm = gn;
  st->phi = phi;
  st->status = status;
  return status;
}

// ---- explicit integrator (Algorithm 3, explicit branch) ---------------------
// f_i = -sum_c sum_k V_ck tau_ck grad w_ic with grad w_ic = +-1/(4 dx) per
// component; the P2Q accumulators already hold the extensive V_ck tau_ck.
template <typename T>
__global__ void __launch_bounds__(256) k_explicit_cells(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                                        const uint8_t* __restrict__ cflag, const T* __restrict__ acc,
                                                        SolveInfo si, double* f) {
  const int id = cblist[blockIdx.x];
  const double gw = 0.25 / si.dx;
  for (int l = threadIdx.x; l < BV; l += blockDim.x) {
    if (!cflag[(int64_t)id * BV + l]) continue;
    double t6[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < si.nm; ++k)
#pragma unroll
      for (int q = 0; q < 6; ++q) t6[q] += (double)acc[((int64_t)id * si.nf + acc_tau(k) + q) * BV + l];
    const double Tm[9] = {t6[0], t6[3], t6[4], t6[3], t6[1], t6[5], t6[4], t6[5], t6[2]};
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const double g0 = (o & 1) ? gw : -gw, g1 = (o & 2) ? gw : -gw, g2 = (o & 4) ? gw : -gw;
      const int nx = lx + (o & 1), ny = ly + ((o >> 1) & 1), nz = lz + ((o >> 2) & 1);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double* fp = node_ptr(f, id, nbr, nx, ny, nz, a);
        if (fp) atomicAdd(fp, -(Tm[3 * a] * g0 + Tm[3 * a + 1] * g1 + Tm[3 * a + 2] * g2));
      }
    }
  }
}

// v^{n+1} = vhat + dt f / m on free DOFs, prescribed values on Dirichlet nodes
template <typename T>
__global__ void __launch_bounds__(512) k_explicit_nodes(const uint8_t* __restrict__ nflag, const T* __restrict__ m,
                                                        const double* __restrict__ vhat,
                                                        const double* __restrict__ vfix, const double* __restrict__ f,
                                                        double dt, double* vnew) {
  const int id = blockIdx.x, l = threadIdx.x;
  const int64_t slot = (int64_t)id * BV + l;
  const uint8_t fl = nflag[slot];
  const double mi = (double)m[slot];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t o = (int64_t)id * 3 * BV + a * BV + l;
    double v = 0.0;
    if (fl & NF_FIXED)
      v = vfix[o];
    else if ((fl & NF_DOF) && mi > 0.0)
      v = vhat[o] + dt * f[o] / mi;
    vnew[o] = v;
  }
}

template <typename T>
static int explicit_t(mpml_ctx_s* c) {
  int rc = alloc_solver<T>(c);
  if (rc) return rc;
  if (c->nb == 0) return MPML_OK;
  SolveInfo si = solve_info(c);
  double* f = (double*)c->ng.p;
  cudaMemsetAsync(f, 0, sizeof(double) * 3 * c->nb * BV, c->s);
  if (c->ncb > 0) {
    k_explicit_cells<T><<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                           (const uint8_t*)c->cflag.p, (const T*)c->cacc.p, si, f);
    c->launches++;
  }
  k_explicit_nodes<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const T*)c->nmass.p,
                                                       (const double*)c->nvhat.p, (const double*)c->nvfix.p, f,
                                                       c->d.dt, (double*)c->nvnew.p);
  c->launches++;
  return cuda_status(cudaGetLastError());
}

int explicit_solve(mpml_ctx_s* c) { return c->fp64 ? explicit_t<double>(c) : explicit_t<float>(c); }

int newton_solve(mpml_ctx_s* c, const mpml_solver_opts* o, mpml_solve_stats* st) {
  return c->fp64 ? newton_t<double>(c, o, st) : newton_t<float>(c, o, st);
}

// ---- operator-level helpers (introspection API) -----------------------------
template <typename T>
static int eval_t(mpml_ctx_s* c, const void* v, double* phi, void* grad) {
  int rc = alloc_solver<T>(c);
  if (rc) return rc;
  cudaMemcpyAsync(c->nvnew.p, v, sizeof(double) * 3 * c->nb * BV, cudaMemcpyDeviceToDevice, c->s);
  if ((rc = prep_t<T>(c, 1, 0, 1e-6, 1)) || (rc = read_scalars(c))) return rc;
  *phi = c->hscal->phi_in + c->hscal->phi_el;
  if (grad) cudaMemcpyAsync(grad, c->ng.p, sizeof(double) * 3 * c->nb * BV, cudaMemcpyDeviceToDevice, c->s);
  return cuda_status(cudaStreamSynchronize(c->s));
}

int eval_device(mpml_ctx_s* c, const void* v, double* phi, void* grad) {
  return c->fp64 ? eval_t<double>(c, v, phi, grad) : eval_t<float>(c, v, phi, grad);
}

int linearize_device(mpml_ctx_s* c, const void* v) {
  double phi;
  return eval_device(c, v, &phi, nullptr);
}

// q = m p on brick-face node slots (the HVP adds the elastic part there)
template <typename T>
__global__ void k_init_faces(const T* __restrict__ p, const T* __restrict__ m, T* q) {
  const int id = blockIdx.x, l = threadIdx.x;
  const bool face = (l & 7) == 0 || ((l >> 3) & 7) == 0 || (l >> 6) == 0;
  if (face) {
    const T mi = m[(int64_t)id * BV + l];
    for (int a = 0; a < 3; ++a) q[(int64_t)id * 3 * BV + a * BV + l] = mi * p[(int64_t)id * 3 * BV + a * BV + l];
  }
}

template <typename T>
static int hvp_t(mpml_ctx_s* c, const void* p, void* y) {
  cudaMemcpyAsync(c->np.p, p, sizeof(T) * 3 * c->nb * BV, cudaMemcpyDeviceToDevice, c->s);
  cudaMemsetAsync(c->nq.p, 0, sizeof(T) * 3 * c->nb * BV, c->s);
  if (c->nb > 0)
    k_init_faces<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const T*)c->np.p, (const T*)c->nmass.p, (T*)c->nq.p);
  if (c->ncb > 0) launch_hvp<T>(c, (const T*)c->np.p, (T*)c->nq.p, 0);
  cudaMemcpyAsync(y, c->nq.p, sizeof(T) * 3 * c->nb * BV, cudaMemcpyDeviceToDevice, c->s);
  return cuda_status(cudaStreamSynchronize(c->s));
}

int hvp_device(mpml_ctx_s* c, const void* p, void* y) {
  return c->fp64 ? hvp_t<double>(c, p, y) : hvp_t<float>(c, p, y);
}

template <typename T>
static int hvp_bench_t(mpml_ctx_s* c, int iters, double* mean_ms) {
  if (c->ncb == 0 || iters <= 0) {
    *mean_ms = 0;
    return MPML_OK;
  }
  // direction: the current p (left by the last solve) is fine; q faces zeroed per launch
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double tot = 0;
  for (int i = 0; i < iters; ++i) {
    k_init_faces<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const T*)c->np.p, (const T*)c->nmass.p, (T*)c->nq.p);
    cudaEventRecord(a, c->s);
    launch_hvp<T>(c, (const T*)c->np.p, (T*)c->nq.p, 0);
    cudaEventRecord(b, c->s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    tot += ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *mean_ms = tot / iters;
  return cuda_status(cudaGetLastError());
}

int hvp_bench(mpml_ctx_s* c, int iters, double* mean_ms) {
  return c->fp64 ? hvp_bench_t<double>(c, iters, mean_ms) : hvp_bench_t<float>(c, iters, mean_ms);
}

// Times every tile of the context's tangent format on the current linearisation
// (p = the solver's current direction, output into scratch, so the solver state
// is untouched): one untimed launch, then reps launches between CUDA events on
// the context stream; the mean per tile goes to ms[], the fastest becomes the
// context's tile and is recorded in the process-wide cache.
int hvp_autotune(mpml_ctx_s* c, int reps, int* choice, float* ms) {
  if (c->fp64) return MPML_ERR_ARG;
  if (reps < 1) reps = 1;
  if (c->ncb == 0) {
    if (choice) *choice = 0;
    return MPML_OK;
  }
  int rc;
  const int64_t n3 = 3 * c->nb * BV;
  if ((rc = ensure(c->tuneq, sizeof(float) * n3))) return rc;
  float* y = (float*)c->tuneq.p;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return MPML_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return MPML_ERR_CUDA;
  }
  float best = 0.f;
  int arg = 0;
  for (int t = 0; t < HVP_TILES && !rc; ++t) {
    float tot = 0.f;
    for (int i = 0; i <= reps; ++i) {
      k_init_faces<float><<<(unsigned)c->nb, BV, 0, c->s>>>((const float*)c->np.p, (const float*)c->nmass.p, y);
      cudaEventRecord(a, c->s);
      launch_hvp_f32(c, t, (const float*)c->np.p, y, 0);
      cudaEventRecord(b, c->s);
      if ((rc = cuda_status(cudaEventSynchronize(b)))) break;
      float e = 0.f;
      cudaEventElapsedTime(&e, a, b);
      if (i > 0) tot += e;
    }
    const float mean = tot / reps;
    if (ms) ms[t] = mean;
    if (t == 0 || mean < best) {
      best = mean;
      arg = t;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->launches += (int64_t)HVP_TILES * (reps + 1) * 2;
  if (rc) return rc;
  c->hvp_tile = arg;
  if (choice) *choice = arg;
  tile_cache_store(c->compressed, c->ncb, arg, best);
  return MPML_OK;
}

// tile for a standalone-HVP solve: the cached choice for this format and size,
// else a short autotuning run on the current system
static int ensure_hvp_tile(mpml_ctx_s* c) {
  if (c->fp64 || c->hvp_tile_fixed) return MPML_OK;
  const int cached = tile_cache_lookup(c->compressed, c->ncb);
  if (cached >= 0) {
    c->hvp_tile = cached;
    return MPML_OK;
  }
  return hvp_autotune(c, 3, nullptr, nullptr);
}

// ---- pieces of the solver used by the batched driver (k_batch.cu) ----------
int batch_alloc_solver(mpml_ctx_s* c) {
  int rc = alloc_solver<float>(c);
  if (rc) return rc;
  return ensure(c->np2, sizeof(float) * 3 * (c->nb ? c->nb : 1) * BV);
}

int batch_prep(mpml_ctx_s* c, double cg_rtol, int cg_max) { return prep_t<float>(c, 1, 1, cg_rtol, cg_max); }

void batch_slope_launch(mpml_ctx_s* c) {
  DevScalars* d = dscal(c);
  cudaMemsetAsync(&d->slope, 0, 3 * sizeof(double), c->s);
  k_ls_setup<float><<<node_blocks(c->nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const float*)c->nmass.p,
                                                     (const double*)c->ng.p, (const double*)c->nvnew.p,
                                                     (const double*)c->nvhat.p, (const float*)c->nx.p, d, (int)c->nb);
  c->launches++;
}

void batch_energy_launch(mpml_ctx_s* c, double alpha) {
  SolveInfo si = solve_info(c);
  DevScalars* d = dscal(c);
  cudaMemsetAsync(&d->phi_in, 0, sizeof(double), c->s);
  cudaMemsetAsync(&d->phi_el, 0, sizeof(double), c->s);
  cudaMemsetAsync(&d->infeasible, 0, sizeof(int), c->s);
  k_energy_nodes<float><<<node_blocks(c->nb), BV, 0, c->s>>>((const uint8_t*)c->nflag.p, (const float*)c->nmass.p,
                                                         (const double*)c->nvnew.p, (const float*)c->nx.p,
                                                         (const double*)c->nvhat.p, alpha, d, (int)c->nb);
  if (c->ncb > 0)
    k_energy_cells<float><<<(unsigned)c->ncb, 256, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                             (const uint8_t*)c->cflag.p, (const float*)c->cacc.p,
                                                             (const double*)(c->fp_active ? c->cB.p : c->cs.p), (const double*)c->nvnew.p,
                                                             (const float*)c->nx.p, alpha, si, d);
  c->launches += 2;
}

// the line search's full step (see newton_t): v + dx into the trial buffer, made current, and
// the prep there without the CG start; batch_trial_revert makes v current again
int batch_trial_launch(mpml_ctx_s* c, double cg_rtol, int cg_max) {
  k_axpy_out<float><<<(unsigned)c->nb, BV, 0, c->s>>>((const float*)c->ndinv.p, (const float*)c->nx.p, 1.0,
                                                     (const double*)c->nvnew.p, (double*)c->nvtry.p);
  c->launches++;
  std::swap(c->nvnew, c->nvtry);
  return prep_t<float>(c, 1, 0, cg_rtol, cg_max, 1, 1);
}
void batch_trial_revert(mpml_ctx_s* c) { std::swap(c->nvnew, c->nvtry); }
int batch_cg_start(mpml_ctx_s* c, double cg_rtol, int cg_max) { return cg_start_t<float>(c, cg_rtol, cg_max); }

void batch_axpy_launch(mpml_ctx_s* c, double alpha) {
  k_axpy<float><<<(unsigned)c->nb, BV, 0, c->s>>>((const float*)c->ndinv.p, (const float*)c->nx.p, alpha,
                                                 (double*)c->nvnew.p);
  c->launches++;
}

}  // namespace mpml
