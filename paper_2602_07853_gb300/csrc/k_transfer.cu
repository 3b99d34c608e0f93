// Algorithm 2 (Unload) transfers and Algorithm 4 (Load).
//
// P2Q (Sec. 3.1, 3.2): per particle, trilinear weights w_cp over the 8
//   centres around the base centre; accumulate m, m (v + G (x_c - x_p)),
//   m G, V_k and V_k tau_k.  One CTA per brick with cells, over the brick's
//   contiguous sorted particle range; a 9x9x9 block of centres (the brick
//   plus its upper halo) accumulates in shared memory and is written once:
//   centres owned only by this brick with plain stores, shared faces with
//   global atomics.
// Q2N (Sec. 3.3): nodal gather from the <= 8 surrounding centres with the
//   constant weight 1/8, (mv)_i = sum 1/8 (m_c v_c + m_c G_c (x_i - x_c));
//   no race (gather).
// N2Q (Sec. 3.3): v_c = sum_i 1/8 v_i, G_c = sum_i v_i (x) grad w_ic with
//   grad w_ic = (x_i - x_c) / (2 dx^2) = +-1/(4 dx) per component.
// G2P (Sec. 3.1, Algorithm 4): v_p = sum_c w_cp v_c, G_p = sum_c w_cp G_c,
//   x += dt v_p, F <- (I + dt G_p) F.
#include "mpml_internal.cuh"

namespace mpml {

struct XferInfo {
  int n[3];
  double inv_dx, dx, dt;
  double grav[3];
  int nm;
  int nf;  // accumulator fields
  MatParams<double> mat[MPML_MAX_MATS];
  // plasticity per material: kind, yield stress, Drucker-Prager alpha
  int plastic[MPML_MAX_MATS];
  double ys[MPML_MAX_MATS], alpha[MPML_MAX_MATS];
};

__device__ __forceinline__ void base_of(const double xa[3], double inv_dx, int b[3], double f[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double sa = __dsub_rn(__dmul_rn(xa[a], inv_dx), 0.5);
    double fl = floor(sa);
    b[a] = (int)fl;
    f[a] = __dsub_rn(sa, fl);
  }
}

// Kirchhoff stress tau = P(F) F^T of one particle (6 symmetric entries).
template <typename T>
__device__ void kirchhoff(const MatParams<T>& M, const T F[9], T tau[6]) {
  T H[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) H[i] = F[i] - ((i % 4 == 0) ? T(1) : T(0));
  if (M.model == MPML_WATER) {
    // Sec. "Water": tau = pi I, pi = kappa J (J - 1), J - 1 from the invariants of H
    T trH = H[0] + H[4] + H[8];
    T trH2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) trH2 += H[3 * a + b] * H[3 * b + a];
    T detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
             H[2] * (H[3] * H[7] - H[4] * H[6]);
    T Jm1 = trH + T(0.5) * (trH * trH - trH2) + detH;
    T pi = (M.lam + T(2) / T(3) * M.mu) * Jm1 * (T(1) + Jm1);
    tau[0] = tau[1] = tau[2] = pi;
    tau[3] = tau[4] = tau[5] = T(0);
    return;
  }
  if (M.model == MPML_NEO_HOOKEAN) {
    // split form of Sec. 4.3.2: mu J^{-2/3} dev(b) + kappa/2 (J^2 - 1) I,
    // with b - I = H + H^T + H H^T and J - 1 from the invariants of H.
    T B[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T acc = H[3 * a + b] + H[3 * b + a];
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += H[3 * a + k] * H[3 * b + k];
        B[3 * a + b] = acc;
      }
    T trH = H[0] + H[4] + H[8];
    T trH2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) trH2 += H[3 * a + b] * H[3 * b + a];
    T detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
             H[2] * (H[3] * H[7] - H[4] * H[6]);
    T Jm1 = trH + T(0.5) * (trH * trH - trH2) + detH;
    T kap = T(2) / T(3) * M.mu + M.lam;
    T c = exp_t(T(-2) / T(3) * log1p_t(Jm1));
    T trB = (B[0] + B[4] + B[8]) / T(3);
    T iso = T(0.5) * kap * Jm1 * (T(2) + Jm1);
    T mc = M.mu * c;
    tau[0] = mc * (B[0] - trB) + iso;
    tau[1] = mc * (B[4] - trB) + iso;
    tau[2] = mc * (B[8] - trB) + iso;
    tau[3] = mc * B[1];
    tau[4] = mc * B[2];
    tau[5] = mc * B[5];
    return;
  }
  if (M.model == MPML_HENCKY) {
    // small strain: tau = mu log(b) + lam/2 tr(log b) I with b - I = H + H^T + H H^T and
    // log(b) by its series (no eigen-decomposition); J > 0 from the invariants of H
    T e6[6];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      T acc = H[3 * ia[q] + ib[q]] + H[3 * ib[q] + ia[q]];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += H[3 * ia[q] + k] * H[3 * ib[q] + k];
      e6[q] = acc;
    }
    T trH = H[0] + H[4] + H[8], trH2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) trH2 += H[3 * a + b] * H[3 * b + a];
    const T detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                   H[2] * (H[3] * H[7] - H[4] * H[6]);
    const T Jm1h = trH + T(0.5) * (trH * trH - trH2) + detH;
    Sym3<T> L;
    if (Jm1h > T(-1) && log_spd_series(Sym3<T>{e6[0], e6[1], e6[2], e6[3], e6[4], e6[5]}, L)) {
      const T hl = T(0.5) * M.lam * (L.xx + L.yy + L.zz);
      tau[0] = M.mu * L.xx + hl;
      tau[1] = M.mu * L.yy + hl;
      tau[2] = M.mu * L.zz + hl;
      tau[3] = M.mu * L.xy;
      tau[4] = M.mu * L.xz;
      tau[5] = M.mu * L.yz;
      return;
    }
  }
  // fixed-corotated and Hencky: tau = U diag(s_i dpsi/ds_i) U^T (Sec. 4.3)
  T U[9], s[3], e[3], V[9], Jm1;
  svd_from_h(H, U, s, e, V, Jm1);
  Spec<T> sp;
  spectral<T, 1>(M, s, e, Jm1, sp);  // the principal stresses only
  T t[3] = {s[0] * sp.d1[0], s[1] * sp.d1[1], s[2] * sp.d1[2]};
  const int ra[6] = {0, 1, 2, 0, 0, 1}, rb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    T acc = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc += U[3 * ra[q] + k] * t[k] * U[3 * rb[q] + k];
    tau[q] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void sh_add(T* p, T v) {
  atomicAdd(p, v);
}

// dynamic smem: nf * 729 T
template <typename T>
__global__ void __launch_bounds__(384) k_p2q(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                             const int* __restrict__ start, const T* __restrict__ x,
                                             const T* __restrict__ v, const T* __restrict__ F,
                                             const T* __restrict__ G, const T* __restrict__ m,
                                             const T* __restrict__ Vp, const int32_t* __restrict__ mat,
                                             XferInfo xi, T* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  const int nf = xi.nf;
  const int id = cblist[blockIdx.x];
  for (int i = threadIdx.x; i < nf * 729; i += blockDim.x) sh[i] = T(0);
  __syncthreads();
  const int p0 = start[(int64_t)id * BV], p1 = start[(int64_t)id * BV + BV];
  MatParams<T> mats[MPML_MAX_MATS];
#pragma unroll
  for (int k = 0; k < MPML_MAX_MATS; ++k) {
    mats[k].model = xi.mat[k].model;
    mats[k].mu = (T)xi.mat[k].mu;
    mats[k].lam = (T)xi.mat[k].lam;
  }
  const T dx = (T)xi.dx;
  // the brick's particles are sorted by cell: lane l of a warp takes particle
  // l * ceil(n / 32) + j of the brick, so the lanes of one warp add into cells
  // far apart instead of contending for the same shared-memory words
  const int n = p1 - p0, qn = (n + 31) >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x >> 5; j < qn; j += blockDim.x >> 5) {
    const int pl = lane * qn + j;
    if (pl >= n) continue;
    const int p = p0 + pl;
    double xa[3] = {(double)x[3 * p], (double)x[3 * p + 1], (double)x[3 * p + 2]};
    int b[3];
    double f[3];
    base_of(xa, xi.inv_dx, b, f);
    T Fp[9], Gp[9], vp[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Fp[i] = F[9 * (int64_t)p + i];
      Gp[i] = G[9 * (int64_t)p + i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) vp[i] = v[3 * (int64_t)p + i];
    const T mp = m[p], Vq = Vp[p];
    const int k = mat[p];
    if (k < 0 || k >= xi.nm) continue;  // flagged by the sort (ST_BADMAT)
    T tau[6];
    kirchhoff(mats[k], Fp, tau);
    const int lb[3] = {b[0] & 7, b[1] & 7, b[2] & 7};
    // the base index and the 1-D factors f, 1 - f are formed in FP64, the weights
    // from them in the context precision: a factor rounds to zero only when it is
    // zero (a nonzero factor of a stored FP32 position is far above the FP32
    // underflow), so the zero pattern of the weights is the FP64 one
    T w1[3], w0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      w1[a] = (T)f[a];
      w0[a] = (T)(1.0 - f[a]);
    }
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      const T w = (oa[0] ? w1[0] : w0[0]) * (oa[1] ? w1[1] : w0[1]) * (oa[2] ? w1[2] : w0[2]);
      if (w == T(0)) continue;
      T d[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = (oa[a] ? w0[a] : -w1[a]) * dx;
      const int cell = ((lb[2] + oa[2]) * 9 + (lb[1] + oa[1])) * 9 + (lb[0] + oa[0]);
      const T wm = w * mp;
      sh_add(&sh[0 * 729 + cell], wm);
#pragma unroll
      for (int r = 0; r < 3; ++r)
        sh_add(&sh[(1 + r) * 729 + cell], wm * (vp[r] + Gp[3 * r] * d[0] + Gp[3 * r + 1] * d[1] + Gp[3 * r + 2] * d[2]));
#pragma unroll
      for (int r = 0; r < 9; ++r) sh_add(&sh[(4 + r) * 729 + cell], wm * Gp[r]);
      const T wV = w * Vq;
      sh_add(&sh[acc_V(k) * 729 + cell], wV);
#pragma unroll
      for (int q = 0; q < 6; ++q) sh_add(&sh[(acc_tau(k) + q) * 729 + cell], wV * tau[q]);
    }
  }
  __syncthreads();
  // write out the 9x9x9 block
  for (int cell = threadIdx.x; cell < 729; cell += blockDim.x) {
    if (sh[cell] == T(0)) continue;  // no particle weight here
    const int cx = cell % 9, cy = (cell / 9) % 9, cz = cell / 81;
    const int t = (cx < 8 && cy < 8 && cz < 8) ? id : nbr[id * NBR + nbr_index(cx >> 3, cy >> 3, cz >> 3)];
    if (t < 0) continue;
    const int l = (cz & 7) * 64 + (cy & 7) * 8 + (cx & 7);
    T* dst = acc + (int64_t)t * nf * BV + l;
    const bool excl = cx >= 1 && cx <= 7 && cy >= 1 && cy <= 7 && cz >= 1 && cz <= 7;
    if (excl) {
      for (int q = 0; q < nf; ++q) dst[q * BV] = sh[q * 729 + cell];
    } else {
      for (int q = 0; q < nf; ++q) {
        T val = sh[q * 729 + cell];
        if (val != T(0)) atomicAdd(&dst[q * BV], val);
      }
    }
  }
}

// Q2N gather, one CTA per brick (all bricks), one thread per node slot.
template <typename T>
__global__ void __launch_bounds__(512) k_q2n(const int* __restrict__ nbr, const uint8_t* __restrict__ nflag,
                                             const uint8_t* __restrict__ cflag, const T* __restrict__ acc,
                                             const double* __restrict__ vfix, XferInfo xi, T* __restrict__ nmass,
                                             double* __restrict__ nv, double* __restrict__ nvhat,
                                             double* __restrict__ vcur) {
  const int id = blockIdx.x, l = threadIdx.x;
  const int64_t slot = (int64_t)id * BV + l;
  const uint8_t fl = nflag[slot];
  double* vo = nv + (int64_t)id * 3 * BV + l;
  double* vh = nvhat + (int64_t)id * 3 * BV + l;
  double* vc = vcur + (int64_t)id * 3 * BV + l;
  if (!(fl & NF_DOF)) {
    nmass[slot] = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r) vo[r * BV] = vh[r * BV] = vc[r * BV] = 0.0;
    return;
  }
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const int nf = xi.nf;
  const T hdx = (T)(0.5 * xi.dx);
  T mi = 0, mv[3] = {0, 0, 0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    // the cell whose corner o is this node
    const int cx = lx - oa[0], cy = ly - oa[1], cz = lz - oa[2];
    const int t = (cx >= 0 && cy >= 0 && cz >= 0) ? id
                                                   : nbr[id * NBR + nbr_index(cx < 0 ? -1 : 0, cy < 0 ? -1 : 0,
                                                                              cz < 0 ? -1 : 0)];
    if (t < 0) continue;
    const int cl = ((cz & 7) * 8 + (cy & 7)) * 8 + (cx & 7);
    if (!cflag[(int64_t)t * BV + cl]) continue;
    const T* a = acc + (int64_t)t * nf * BV + cl;
    const T mc = a[0];
    // x_i - x_c = (o - 1/2) dx per axis
    const T d[3] = {oa[0] ? hdx : -hdx, oa[1] ? hdx : -hdx, oa[2] ? hdx : -hdx};
    mi += T(0.125) * mc;
#pragma unroll
    for (int r = 0; r < 3; ++r)
      mv[r] += T(0.125) * (a[(1 + r) * BV] + a[(4 + 3 * r) * BV] * d[0] + a[(5 + 3 * r) * BV] * d[1] +
                           a[(6 + 3 * r) * BV] * d[2]);
  }
  nmass[slot] = mi;
  const bool fixed = fl & NF_FIXED;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double vi = mi != T(0) ? (double)mv[r] / (double)mi : 0.0;
    double vhat = vi + xi.dt * xi.grav[r];
    vo[r * BV] = vi;
    vh[r * BV] = vhat;
    vc[r * BV] = fixed ? vfix[(int64_t)id * 3 * BV + r * BV + l] : vhat;
  }
}

// N2Q: v_c and G_c at active centres (cell-brick CTAs, 512 threads).
template <typename T>
__global__ void __launch_bounds__(512) k_n2q(const int* __restrict__ cblist, const int* __restrict__ nbr,
                                             const uint8_t* __restrict__ cflag, const double* __restrict__ vn,
                                             XferInfo xi, T* __restrict__ cnew) {
  __shared__ T sv[3][729];
  const int id = cblist[blockIdx.x];
  for (int i = threadIdx.x; i < 729; i += blockDim.x) {
    const int nx = i % 9, ny = (i / 9) % 9, nz = i / 81;
    const int t = (nx < 8 && ny < 8 && nz < 8) ? id : nbr[id * NBR + nbr_index(nx >> 3, ny >> 3, nz >> 3)];
    const int l = (nz & 7) * 64 + (ny & 7) * 8 + (nx & 7);
#pragma unroll
    for (int r = 0; r < 3; ++r) sv[r][i] = t >= 0 ? (T)vn[(int64_t)t * 3 * BV + r * BV + l] : T(0);
  }
  __syncthreads();
  const int l = threadIdx.x;
  if (!cflag[(int64_t)id * BV + l]) return;
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const T gw = (T)(0.25 / xi.dx);
  T vc[3] = {0, 0, 0}, Gc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    const int i = ((lz + oa[2]) * 9 + (ly + oa[1])) * 9 + (lx + oa[0]);
    const T g[3] = {oa[0] ? gw : -gw, oa[1] ? gw : -gw, oa[2] ? gw : -gw};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T va = sv[a][i];
      vc[a] += T(0.125) * va;
#pragma unroll
      for (int b = 0; b < 3; ++b) Gc[3 * a + b] += va * g[b];
    }
  }
  T* dst = cnew + (int64_t)id * 12 * BV + l;
#pragma unroll
  for (int a = 0; a < 3; ++a) dst[a * BV] = vc[a];
#pragma unroll
  for (int q = 0; q < 9; ++q) dst[(3 + q) * BV] = Gc[q];
}

// G2P: particles in sorted order; writes the caller's arrays.
template <typename T>
__global__ void __launch_bounds__(256) k_g2p(int64_t np, const T* __restrict__ xs, const T* __restrict__ Fs,
                                             const T* __restrict__ ms, const T* __restrict__ Vs,
                                             const int32_t* __restrict__ mats, const int* __restrict__ bmap,
                                             const T* __restrict__ cnew, int NB0, int NB1, XferInfo xi, T* xo,
                                             T* vo, T* Fo, T* Go, T* mo, T* Vo, int32_t* mato) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double xa[3] = {(double)xs[3 * p], (double)xs[3 * p + 1], (double)xs[3 * p + 2]};
  int b[3];
  double f[3];
  base_of(xa, xi.inv_dx, b, f);
  T vp[3] = {0, 0, 0}, Gp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  // weights from FP64 factors in the context precision (zero pattern as in P2Q)
  T w1[3], w0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w1[a] = (T)f[a];
    w0[a] = (T)(1.0 - f[a]);
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    const T w = (oa[0] ? w1[0] : w0[0]) * (oa[1] ? w1[1] : w0[1]) * (oa[2] ? w1[2] : w0[2]);
    if (w == T(0)) continue;
    const int c[3] = {b[0] + oa[0], b[1] + oa[1], b[2] + oa[2]};
    const int t = bmap[((int64_t)(c[2] >> 3) * NB1 + (c[1] >> 3)) * NB0 + (c[0] >> 3)];
    const T* src = cnew + (int64_t)t * 12 * BV + ((c[2] & 7) * 64 + (c[1] & 7) * 8 + (c[0] & 7));
#pragma unroll
    for (int a = 0; a < 3; ++a) vp[a] += w * src[a * BV];
#pragma unroll
    for (int q = 0; q < 9; ++q) Gp[q] += w * src[(3 + q) * BV];
  }
  const T dt = (T)xi.dt;
  T Fp[9], Fn[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Fp[i] = Fs[9 * p + i];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      T acc = Fp[3 * r + cc];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += dt * Gp[3 * r + k] * Fp[3 * k + cc];
      Fn[3 * r + cc] = acc;
    }
  const int km = mats[p];
  if (km >= 0 && km < xi.nm && xi.plastic[km] != MPML_ELASTIC)
    return_map<T>(xi.plastic[km], xi.mat[km].mu, xi.mat[km].lam, xi.ys[km], xi.alpha[km], Fn);
  if (km >= 0 && km < xi.nm && xi.mat[km].model == MPML_WATER) {
    // Sec. "Water": J <- (1 + dt tr G_p) J, F kept isotropic; J <= 0 gives NaN
    const T J0 = Fp[0] * (Fp[4] * Fp[8] - Fp[5] * Fp[7]) - Fp[1] * (Fp[3] * Fp[8] - Fp[5] * Fp[6]) +
                 Fp[2] * (Fp[3] * Fp[7] - Fp[4] * Fp[6]);
    const T Jn = (T(1) + dt * (Gp[0] + Gp[4] + Gp[8])) * J0;
    const T c = Jn > T(0) ? cbrt(Jn) : T(NAN);
#pragma unroll
    for (int i = 0; i < 9; ++i) Fn[i] = (i % 4 == 0) ? c : T(0);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) Fo[9 * p + i] = Fn[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xo[3 * p + a] = xs[3 * p + a] + dt * vp[a];
    vo[3 * p + a] = vp[a];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) Go[9 * p + q] = Gp[q];
  mo[p] = ms[p];
  Vo[p] = Vs[p];
  mato[p] = mats[p];
}

static XferInfo xfer_info(mpml_ctx_s* c) {
  XferInfo xi;
  for (int a = 0; a < 3; ++a) {
    xi.n[a] = c->d.n[a];
    xi.grav[a] = c->d.gravity[a];
  }
  xi.inv_dx = c->d.inv_dx;
  xi.dx = c->d.dx;
  xi.dt = c->d.dt;
  xi.nm = c->nm;
  xi.nf = acc_fields(c->nm);
  for (int k = 0; k < MPML_MAX_MATS; ++k) {
    const mpml_material& m = c->mats[k < c->nm ? k : 0];
    xi.mat[k].model = m.model;
    xi.mat[k].mu = m.mu;
    xi.mat[k].lam = m.lambda;
    xi.plastic[k] = k < c->nm ? m.plastic : MPML_ELASTIC;
    xi.ys[k] = m.yield_stress;
    const double sp = sin(m.friction_angle);
    xi.alpha[k] = sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp);
  }
  return xi;
}

template <typename T>
static int p2q_q2n_t(mpml_ctx_s* c) {
  const int64_t nslots = c->nb * BV;
  XferInfo xi = xfer_info(c);
  const size_t es = sizeof(T);
  int rc;
  const size_t ds = sizeof(double);
  if ((rc = ensure(c->cacc, es * xi.nf * nslots)) || (rc = ensure(c->nmass, es * nslots)) ||
      (rc = ensure(c->nv, ds * 3 * nslots)) || (rc = ensure(c->nvhat, ds * 3 * nslots)) ||
      (rc = ensure(c->nvnew, ds * 3 * nslots)))
    return rc;
  if (nslots > 0) cudaMemsetAsync(c->cacc.p, 0, es * xi.nf * nslots, c->s);
  if (c->ncb > 0) {
    size_t smem = es * xi.nf * 729;
    cudaFuncSetAttribute(k_p2q<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_p2q<T><<<(unsigned)c->ncb, 384, smem, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                  (const int*)c->start.p, (const T*)c->px.p, (const T*)c->pv.p,
                                                  (const T*)c->pF.p, (const T*)c->pG.p, (const T*)c->pm.p,
                                                  (const T*)c->pV.p, (const int32_t*)c->pmat.p, xi, (T*)c->cacc.p);
    c->launches++;
  }
  if (c->nb > 0) {
    k_q2n<T><<<(unsigned)c->nb, BV, 0, c->s>>>((const int*)c->nbr.p, (const uint8_t*)c->nflag.p,
                                               (const uint8_t*)c->cflag.p, (const T*)c->cacc.p,
                                               (const double*)c->nvfix.p, xi, (T*)c->nmass.p, (double*)c->nv.p,
                                               (double*)c->nvhat.p, (double*)c->nvnew.p);
    c->launches++;
  }
  return cuda_status(cudaGetLastError());
}

int p2q_q2n(mpml_ctx_s* c) { return c->fp64 ? p2q_q2n_t<double>(c) : p2q_q2n_t<float>(c); }

template <typename T>
static int n2q_t(mpml_ctx_s* c) {
  int rc;
  if ((rc = ensure(c->cnew, sizeof(T) * 12 * c->nb * BV))) return rc;
  XferInfo xi = xfer_info(c);
  if (c->ncb > 0) {
    k_n2q<T><<<(unsigned)c->ncb, BV, 0, c->s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                (const uint8_t*)c->cflag.p, (const double*)c->nvnew.p, xi,
                                                (T*)c->cnew.p);
    c->launches++;
  }
  return cuda_status(cudaGetLastError());
}

int n2q_device(mpml_ctx_s* c) { return c->fp64 ? n2q_t<double>(c) : n2q_t<float>(c); }

template <typename T>
static int g2p_t(mpml_ctx_s* c, void* x, void* v, void* F, void* G, void* m, void* V, int32_t* mat) {
  int rc = n2q_t<T>(c);
  if (rc) return rc;
  XferInfo xi = xfer_info(c);
  const int64_t np = c->np_count;
  if (np > 0) {
    k_g2p<T><<<div_up(np, 256), 256, 0, c->s>>>(np, (const T*)c->px.p, (const T*)c->pF.p, (const T*)c->pm.p,
                                                (const T*)c->pV.p, (const int32_t*)c->pmat.p,
                                                (const int*)c->bmap.p, (const T*)c->cnew.p, c->NB[0], c->NB[1], xi,
                                                (T*)x, (T*)v, (T*)F, (T*)G, (T*)m, (T*)V, mat);
    c->launches++;
  }
  return cuda_status(cudaGetLastError());
}

int g2p_device(mpml_ctx_s* c, void* x, void* v, void* F, void* G, void* m, void* V, int32_t* mat) {
  return c->fp64 ? g2p_t<double>(c, x, v, F, G, m, V, mat) : g2p_t<float>(c, x, v, F, G, m, V, mat);
}

}  // namespace mpml
