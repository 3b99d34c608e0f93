/*
 * FP64 CPU oracle for the MPM Lite implicit time step (arXiv 2602.07853).
 * TEST INFRASTRUCTURE ONLY (see mpml_oracle.h).  Plain loops, double
 * precision, no blocking or fusion.  Compiled with -ffp-contract=off so that
 * the integer decisions (base cell, active set, Dirichlet set) are taken on
 * exactly the rounded products and sums written here.
 */
#include "mpml_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ========================================================================
 * Small dense linear algebra (row-major 3x3: M[3*r+c])
 * ====================================================================== */
static void m3_mul(const double* A, const double* B, double* C) {
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      T[3 * r + c] = s;
    }
  memcpy(C, T, sizeof T);
}
static void m3_mul_bt(const double* A, const double* B, double* C) { /* A B^T */
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * c + k];
      T[3 * r + c] = s;
    }
  memcpy(C, T, sizeof T);
}
static void m3_mul_at(const double* A, const double* B, double* C) { /* A^T B */
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * k + r] * B[3 * k + c];
      T[3 * r + c] = s;
    }
  memcpy(C, T, sizeof T);
}
static double m3_det(const double* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 9).
 * evecs is row-major with eigenvector j in column j. */
void orc_sym_eigen(int n, const double* Ain, double* evals, double* evecs) {
  double A[81], V[81];
  memcpy(A, Ain, sizeof(double) * n * n);
  for (int i = 0; i < n * n; ++i) V[i] = 0;
  for (int i = 0; i < n; ++i) V[i * n + i] = 1;
  double fro = 0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off == 0.0 || off <= 1e-34 * fro) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
        double c = 1 / sqrt(t * t + 1), s = t * c;
        /* A <- J^T A J with J the (p,q) rotation */
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
  memcpy(evecs, V, sizeof(double) * n * n);
}

/* Signed SVD F = U diag(s) V^T with U, V rotations, s0 >= s1 >= |s2|.
 * From the eigen-decomposition of F^T F; the sign of s2 carries det F. */
void orc_svd3(const double F[9], double U[9], double s[3], double V[9]) {
  double C[9], lam[3], W[9];
  m3_mul_at(F, F, C);
  orc_sym_eigen(3, C, lam, W);
  int idx[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[idx[j]] > lam[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) V[3 * r + c] = W[3 * r + idx[c]];
  if (m3_det(V) < 0)
    for (int r = 0; r < 3; ++r) V[3 * r + 2] = -V[3 * r + 2];
  double B[9];
  m3_mul(F, V, B); /* column j = s_j u_j */
  double b[3][3];
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < 3; ++r) b[j][r] = B[3 * r + j];
  double u0[3], u1[3], u2[3];
  double n0 = sqrt(b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2]);
  if (n0 > 1e-300) {
    for (int r = 0; r < 3; ++r) u0[r] = b[0][r] / n0;
  } else {
    u0[0] = 1; u0[1] = 0; u0[2] = 0;
  }
  double d = u0[0] * b[1][0] + u0[1] * b[1][1] + u0[2] * b[1][2];
  for (int r = 0; r < 3; ++r) u1[r] = b[1][r] - d * u0[r];
  double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
  if (n1 > 1e-300) {
    for (int r = 0; r < 3; ++r) u1[r] /= n1;
  } else { /* any unit vector orthogonal to u0 */
    double a[3] = {1, 0, 0};
    if (fabs(u0[0]) > 0.9) { a[0] = 0; a[1] = 1; }
    double e = a[0] * u0[0] + a[1] * u0[1] + a[2] * u0[2];
    for (int r = 0; r < 3; ++r) u1[r] = a[r] - e * u0[r];
    double nn = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    for (int r = 0; r < 3; ++r) u1[r] /= nn;
  }
  u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
  u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
  u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
  s[0] = n0;
  s[1] = u1[0] * b[1][0] + u1[1] * b[1][1] + u1[2] * b[1][2];
  s[2] = u2[0] * b[2][0] + u2[1] * b[2][1] + u2[2] * b[2][2];
  for (int r = 0; r < 3; ++r) {
    U[3 * r + 0] = u0[r];
    U[3 * r + 1] = u1[r];
    U[3 * r + 2] = u2[r];
  }
}

/* ========================================================================
 * Isotropic energies in principal stretches (Sec. 4.3)
 *   psi_hat(s), d1[i] = dpsi/ds_i, d2 = 3x3 Hessian in s,
 *   pairs (0,1),(0,2),(1,2): pp = (d1_i - d1_j)/(s_i - s_j),
 *                            pm = (d1_i + d1_j)/(s_i + s_j),
 * each written in a closed form that stays finite when s_i == s_j.
 * ====================================================================== */
typedef struct {
  double psi, d1[3], d2[9], pp[3], pm[3];
} spec_t;

static const int PAIR_I[3] = {0, 0, 1}, PAIR_J[3] = {1, 2, 2}, PAIR_K[3] = {2, 1, 0};

/* returns 0, or 1 when the energy is undefined at s (J <= 0 where the model
 * needs J > 0) */
static int spectral(int model, double mu, double lam, const double s[3], spec_t* o) {
  double J = s[0] * s[1] * s[2];
  if (model == ORC_FIXED_COROTATED) {
    /* psi = mu sum (s_i - 1)^2 + lam/2 (J - 1)^2  (fixed-corotated; the
     * model named by the workloads, not written in the paper) */
    o->psi = 0;
    for (int i = 0; i < 3; ++i) o->psi += mu * (s[i] - 1) * (s[i] - 1);
    o->psi += 0.5 * lam * (J - 1) * (J - 1);
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      o->d1[i] = 2 * mu * (s[i] - 1) + lam * (J - 1) * s[j] * s[k];
      o->d2[3 * i + i] = 2 * mu + lam * (s[j] * s[k]) * (s[j] * s[k]);
    }
    for (int p = 0; p < 3; ++p) {
      int i = PAIR_I[p], j = PAIR_J[p], k = PAIR_K[p];
      o->d2[3 * i + j] = o->d2[3 * j + i] = lam * s[k] * (2 * J - 1);
      o->pp[p] = 2 * mu - lam * (J - 1) * s[k];
      o->pm[p] = 2 * mu * (1 - 2 / (s[i] + s[j])) + lam * (J - 1) * s[k];
    }
    return 0;
  }
  if (model == ORC_NEO_HOOKEAN) {
    /* Split Neo-Hookean, Sec. 4.3.2:
     *   psi = mu/2 (J^{-2/3} I1 - 3) + kappa/4 (J^2 - 1 - 2 log J),
     *   kappa = 2/3 mu + lam, I1 = sum s_i^2 */
    if (!(J > 0)) return 1;
    double kap = 2.0 / 3.0 * mu + lam;
    double I1 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    double c = pow(J, -2.0 / 3.0);
    o->psi = 0.5 * mu * (c * I1 - 3) + 0.25 * kap * (J * J - 1 - 2 * log(J));
    for (int i = 0; i < 3; ++i) {
      o->d1[i] = mu * c * (s[i] - I1 / (3 * s[i])) + 0.5 * kap * (J * J - 1) / s[i];
      o->d2[3 * i + i] = mu * c * (-1.0 / 3.0 + 5 * I1 / (9 * s[i] * s[i])) +
                         0.5 * kap * (J * J + 1) / (s[i] * s[i]);
    }
    for (int p = 0; p < 3; ++p) {
      int i = PAIR_I[p], j = PAIR_J[p];
      double sij = s[i] * s[j];
      o->d2[3 * i + j] = o->d2[3 * j + i] =
          mu * c / sij * (-2.0 / 3.0 * s[i] * s[i] - 2.0 / 3.0 * s[j] * s[j] + 2.0 / 9.0 * I1) +
          kap * J * J / sij;
      o->pp[p] = mu * c * (1 + I1 / (3 * sij)) - 0.5 * kap * (J * J - 1) / sij;
      o->pm[p] = mu * c * (1 - I1 / (3 * sij)) + 0.5 * kap * (J * J - 1) / sij;
    }
    return 0;
  }
  if (model == ORC_WATER) {
    /* Sec. "Water": psi = kappa/2 (J - 1)^2, kappa = lam + 2/3 mu (bulk modulus);
     * undefined for J <= 0 (no inverted fluid) */
    if (!(J > 0)) return 1;
    double kap = lam + 2.0 / 3.0 * mu;
    o->psi = 0.5 * kap * (J - 1) * (J - 1);
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      o->d1[i] = kap * (J - 1) * s[j] * s[k];
      o->d2[3 * i + i] = kap * (s[j] * s[k]) * (s[j] * s[k]);
    }
    for (int p = 0; p < 3; ++p) {
      int i = PAIR_I[p], j = PAIR_J[p], k = PAIR_K[p];
      o->d2[3 * i + j] = o->d2[3 * j + i] = kap * s[k] * (2 * J - 1);
      o->pp[p] = -kap * (J - 1) * s[k];
      o->pm[p] = kap * (J - 1) * s[k];
    }
    return 0;
  }
  if (model == ORC_HENCKY) {
    /* StVK with Hencky strain, Sec. 4.3.1:
     *   psi = mu sum (log s_i)^2 + lam/2 (sum log s_i)^2 */
    if (!(s[0] > 0 && s[1] > 0 && s[2] > 0)) return 1;
    double e[3] = {log(s[0]), log(s[1]), log(s[2])};
    double tr = e[0] + e[1] + e[2];
    o->psi = mu * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) + 0.5 * lam * tr * tr;
    for (int i = 0; i < 3; ++i) {
      o->d1[i] = (2 * mu * e[i] + lam * tr) / s[i];
      o->d2[3 * i + i] = (2 * mu + lam - 2 * mu * e[i] - lam * tr) / (s[i] * s[i]);
    }
    for (int p = 0; p < 3; ++p) {
      int i = PAIR_I[p], j = PAIR_J[p];
      o->d2[3 * i + j] = o->d2[3 * j + i] = lam / (s[i] * s[j]);
      /* (log s_i - log s_j)/(s_i - s_j) * s_j = log1p(z)/z, z = s_i/s_j - 1 */
      double z = (s[i] - s[j]) / s[j];
      double L = fabs(z) < 1e-8 ? 1 - 0.5 * z : log1p(z) / z;
      o->pp[p] = (2 * mu * (L - e[j]) - lam * tr) / (s[i] * s[j]);
      double ti = 2 * mu * e[i] + lam * tr, tj = 2 * mu * e[j] + lam * tr;
      o->pm[p] = (ti * s[j] + tj * s[i]) / (s[i] * s[j] * (s[i] + s[j]));
    }
    return 0;
  }
  return 1;
}

/* Split Neo-Hookean energy of Sec. 4.3.2, mu/2 (J^(-2/3) I1 - 3) + kappa/4 (J^2 - 1
 * - 2 log J), evaluated from H = F - I so that small strains keep their relative
 * accuracy: the energy is second order in H but both brackets are differences of
 * first-order terms.  With c = J^(-2/3) - 1 (binomial series in x = J - 1 for
 * |x| < 0.05, coefficients C(-2/3, k) by their product recurrence),
 *   J^(-2/3) I1 - 3 = [3 c + 2 x] + [(I1 - 3) - 2 x] + c (I1 - 3),
 * where 3 c + 2 x drops the series' linear term, (I1 - 3) - 2 x = |H|^2 + tr(H^2)
 * - (tr H)^2 - 2 det H, and J^2 - 1 - 2 log J = x^2 + 2 (x - log(1 + x)) with
 * x - log(1 + x) from its Taylor series for |x| < 0.05. */
static double nh_energy(double mu, double lam, const double F[9]) {
  double H[9];
  for (int i = 0; i < 9; ++i) H[i] = F[i] - ((i % 4 == 0) ? 1.0 : 0.0);
  double trH = H[0] + H[4] + H[8], hF2 = 0, trH2 = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      hF2 += H[3 * a + b] * H[3 * a + b];
      trH2 += H[3 * a + b] * H[3 * b + a];
    }
  double detH = m3_det(H);
  double x = trH + 0.5 * (trH * trH - trH2) + detH; /* J - 1 */
  if (!(x > -1)) return INFINITY;
  double I1m3 = 2 * trH + hF2, b2 = hF2 + trH2 - trH * trH - 2 * detH;
  double kap = 2.0 / 3.0 * mu + lam;
  double c, a2, xml;
  if (fabs(x) < 0.05) {
    double coef = 1, pw = 1;
    c = 0;
    a2 = 0;
    for (int k = 1; k <= 16; ++k) {
      coef *= (-2.0 / 3.0 - (k - 1)) / k;
      pw *= x;
      c += coef * pw;
      if (k >= 2) a2 += 3 * coef * pw;
    }
    xml = 0;
    pw = x;
    for (int k = 2; k <= 18; ++k) {
      pw *= x;
      xml += ((k % 2) ? -pw : pw) / k;
    }
  } else {
    c = pow(1 + x, -2.0 / 3.0) - 1;
    a2 = 3 * c + 2 * x;
    xml = x - log1p(x);
  }
  return 0.5 * mu * (a2 + b2 + c * I1m3) + 0.25 * kap * (x * x + 2 * xml);
}

int orc_psi(int model, double mu, double lam, const double F[9], double* psi) {
  double U[9], s[3], V[9];
  spec_t sp;
  if (model == ORC_NEO_HOOKEAN) {
    *psi = nh_energy(mu, lam, F);
    return isfinite(*psi) ? 0 : 1;
  }
  orc_svd3(F, U, s, V);
  if (spectral(model, mu, lam, s, &sp)) { *psi = INFINITY; return 1; }
  *psi = sp.psi;
  return 0;
}

/* P = U diag(dpsi/ds_i) V^T */
int orc_piola(int model, double mu, double lam, const double F[9], double P[9]) {
  double U[9], s[3], V[9], D[9] = {0};
  spec_t sp;
  orc_svd3(F, U, s, V);
  if (spectral(model, mu, lam, s, &sp)) return 1;
  for (int i = 0; i < 3; ++i) D[3 * i + i] = sp.d1[i];
  m3_mul(U, D, D);
  m3_mul_bt(D, V, P);
  return 0;
}

/* Kirchhoff stress tau = P F^T (Algorithm 2, Stress(F_p)). */
int orc_kirchhoff(int model, double mu, double lam, const double F[9], double tau[9]) {
  double P[9];
  if (orc_piola(model, mu, lam, F, P)) return 1;
  m3_mul_bt(P, F, tau);
  for (int r = 0; r < 3; ++r)
    for (int c = r + 1; c < 3; ++c) {
      double a = 0.5 * (tau[3 * r + c] + tau[3 * c + r]);
      tau[3 * r + c] = tau[3 * c + r] = a;
    }
  return 0;
}

/* dP/dF in the standard basis.  In the frame of the signed SVD the tangent of
 * an isotropic energy acts on dFh = U^T dF V as: the diagonal of dFh through
 * the 3x3 Hessian d2, and each off-diagonal pair (dFh_ij, dFh_ji) through a
 * 2x2 block with eigenvalues pp (vector (1,1)) and pm (vector (1,-1)).
 * With project != 0 the resulting 9x9 matrix is projected onto the PSD cone
 * by a full 9x9 eigen-decomposition with negative eigenvalues set to zero. */
int orc_tangent(int model, double mu, double lam, const double F[9], int project,
                double A[81]) {
  double U[9], s[3], V[9];
  spec_t sp;
  orc_svd3(F, U, s, V);
  if (spectral(model, mu, lam, s, &sp)) return 1;
  for (int col = 0; col < 9; ++col) {
    double dF[9] = {0}, dFh[9], dPh[9] = {0}, dP[9];
    dF[col] = 1;
    m3_mul_at(U, dF, dFh);
    m3_mul(dFh, V, dFh);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dPh[3 * i + i] += sp.d2[3 * i + j] * dFh[3 * j + j];
    for (int p = 0; p < 3; ++p) {
      int i = PAIR_I[p], j = PAIR_J[p];
      double a = 0.5 * (sp.pp[p] + sp.pm[p]), b = 0.5 * (sp.pp[p] - sp.pm[p]);
      dPh[3 * i + j] = a * dFh[3 * i + j] + b * dFh[3 * j + i];
      dPh[3 * j + i] = b * dFh[3 * i + j] + a * dFh[3 * j + i];
    }
    m3_mul(U, dPh, dP);
    m3_mul_bt(dP, V, dP);
    for (int r = 0; r < 9; ++r) A[9 * r + col] = dP[r];
  }
  for (int r = 0; r < 9; ++r)
    for (int c = r + 1; c < 9; ++c) {
      double a = 0.5 * (A[9 * r + c] + A[9 * c + r]);
      A[9 * r + c] = A[9 * c + r] = a;
    }
  if (project) {
    double ev[9], Q[81];
    orc_sym_eigen(9, A, ev, Q);
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c < 9; ++c) {
        double acc = 0;
        for (int k = 0; k < 9; ++k)
          if (ev[k] > 0) acc += Q[9 * r + k] * ev[k] * Q[9 * c + k];
        A[9 * r + c] = acc;
      }
  }
  return 0;
}

/* ========================================================================
 * Stretch reconstruction, Sec. 4.3: tau = U diag(tau_i) U^T, solve the
 * principal relation tau_i = s_i dpsi/ds_i for s_i, S = U diag(s_i) U^T.
 * ====================================================================== */
static double cbrt_signed(double z) { return z >= 0 ? cbrt(z) : -cbrt(-z); }

/* fixed-corotated principal stretch at a given J on the s >= 1/2 branch:
 * tau_i = 2 mu s_i (s_i - 1) + lam J (J - 1) */
static int fc_sigma(double mu, double lam, const double t[3], double J, double s[3]) {
  double c = lam * J * (J - 1);
  for (int i = 0; i < 3; ++i) {
    double disc = 0.25 + (t[i] - c) / (2 * mu);
    if (disc < -1e-12) return 1;
    s[i] = 0.5 + sqrt(disc > 0 ? disc : 0);
  }
  return 0;
}
static double fc_h(double mu, double lam, const double t[3], double J) {
  double s[3];
  fc_sigma(mu, lam, t, J, s);
  return s[0] * s[1] * s[2] - J;
}

int orc_stretch_from_tau(int model, double mu, double lam, const double tau[9], double S[9]) {
  double T[9], t[3], Q[9], s[3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) T[3 * r + c] = 0.5 * (tau[3 * r + c] + tau[3 * c + r]);
  orc_sym_eigen(3, T, t, Q);
  if (model == ORC_HENCKY) {
    /* Sec. 4.3.1: s = tr tau / (2 mu + d lam), e_i = (tau_i - lam s)/(2 mu) */
    if (!(mu > 0 && lam > -2 * mu / 3)) return ORC_ERR_STRETCH;
    double tr = t[0] + t[1] + t[2];
    double ls = tr / (2 * mu + 3 * lam);
    for (int i = 0; i < 3; ++i) s[i] = exp((t[i] - lam * ls) / (2 * mu));
  } else if (model == ORC_NEO_HOOKEAN) {
    /* Sec. 4.3.2 and App. C: J from the spherical part, deviatoric offsets,
     * depressed cubic m^3 + S2 m + S3 - J^2 = 0 solved by Cardano; the
     * largest real root is the one with all m + delta_i > 0. */
    double kap = 2.0 / 3.0 * mu + lam;
    double alpha = (t[0] + t[1] + t[2]) / 3;
    double arg = 1 + 2 * alpha / kap;
    if (!(arg > 0)) return ORC_ERR_STRETCH;
    double J = sqrt(arg);
    double sc = mu * pow(J, -2.0 / 3.0);
    double dl[3];
    for (int i = 0; i < 3; ++i) dl[i] = (t[i] - alpha) / sc;
    double p = dl[0] * dl[1] + dl[1] * dl[2] + dl[2] * dl[0];
    double q = dl[0] * dl[1] * dl[2] - J * J;
    double disc = (q / 2) * (q / 2) + (p / 3) * (p / 3) * (p / 3);
    double m;
    if (disc >= 0) {
      /* Cardano's one-real-root formula, u + v with u v = -p/3.  The cube
       * root of the smaller-magnitude radicand cancels catastrophically when
       * the deviator is small, so v is taken from u v = -p/3 (same root). */
      double sd = sqrt(disc);
      double u = cbrt_signed(-q / 2 + (q <= 0 ? sd : -sd));
      double v = (u != 0) ? -p / (3 * u) : 0;
      m = u + v;
    } else {
      double r = 2 * sqrt(-p / 3);
      double a = 3 * q / (2 * p) * sqrt(-3 / p);
      if (a > 1) a = 1;
      if (a < -1) a = -1;
      m = r * cos(acos(a) / 3);
    }
    for (int i = 0; i < 3; ++i) {
      double beta = m + dl[i];
      if (!(beta > 0)) return ORC_ERR_STRETCH;
      s[i] = sqrt(beta);
    }
  } else if (model == ORC_FIXED_COROTATED) {
    /* Not in the paper (it gives the general recipe of Sec. 4.3 and notes new
     * inverses may be needed).  tau_i = 2 mu s_i (s_i - 1) + lam J (J - 1);
     * for fixed J each s_i is the root >= 1/2 of that quadratic, which is
     * real for J <= Jb (lam J (J - 1) <= tau_min + mu/2).  h(J) =
     * prod_i s_i(J) - J is strictly decreasing for J >= 1/2, so a root in
     * [1/2, Jb] is unique and plain bisection finds it.  Below J = 1/2 h is
     * not monotone (several roots can exist): such states (more than half
     * the volume lost) are rejected with ORC_ERR_STRETCH. */
    if (!(mu > 0) || lam < 0) return ORC_ERR_STRETCH;
    if (lam == 0) {
      if (fc_sigma(mu, lam, t, 1.0, s)) return ORC_ERR_STRETCH;
    } else {
      double tmin = fmin(t[0], fmin(t[1], t[2]));
      double d = 0.25 + (tmin + 0.5 * mu) / lam;
      if (d < 0) return ORC_ERR_STRETCH;
      double lo = 0.5, hi = 0.5 + sqrt(d);
      if (fc_h(mu, lam, t, lo) < 0 || fc_h(mu, lam, t, hi) > 0) return ORC_ERR_STRETCH;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (fc_h(mu, lam, t, mid) > 0) lo = mid; else hi = mid;
      }
      if (fc_sigma(mu, lam, t, 0.5 * (lo + hi), s)) return ORC_ERR_STRETCH;
    }
  } else if (model == ORC_WATER) {
    /* Sec. "Water": the pressure pi = tr(tau)/3 = kappa J (J - 1) inverted on the
     * root J >= 1/2, J = (1 + sqrt(1 + 4 pi / kappa)) / 2; S = J^(1/3) I */
    double kap = lam + 2.0 / 3.0 * mu;
    if (!(kap > 0)) return ORC_ERR_STRETCH;
    double pi = (t[0] + t[1] + t[2]) / 3;
    double d = 1 + 4 * pi / kap;
    if (!(d >= 0)) return ORC_ERR_STRETCH;
    double J = 0.5 * (1 + sqrt(d));
    s[0] = s[1] = s[2] = cbrt(J);
  } else {
    return ORC_ERR_ARG;
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double a = 0;
      for (int k = 0; k < 3; ++k) a += Q[3 * r + k] * s[k] * Q[3 * c + k];
      S[3 * r + c] = a;
    }
  return ORC_OK;
}

/* ========================================================================
 * Grid bookkeeping
 * ====================================================================== */
struct orc_state {
  orc_scene sc;
  long np;
  double *x, *v, *F, *G, *mp, *Vp;
  int* mat;
  long* perm;
  long long* pkey;
  int* base;     /* np*3 */
  double* frac;  /* np*3 */
  /* active cells */
  long nc;
  long long* ckey;
  int* cijk;       /* nc*3 */
  int* cell_index; /* dense cells -> compact or -1 */
  int* corner;     /* nc*8 compact node index of corner (o0,o1,o2), o = bit */
  double *m_c, *v_c, *G_c, *V_ck, *tau_ck, *S_ck;
  double *v_c_new, *G_c_new;
  /* DOF nodes */
  long nn;
  long long* nkey;
  int* nijk;
  int* node_index; /* dense nodes -> compact or -1 */
  double *m_i, *v_i, *vhat, *vfix, *vnew;
  int* fixed;
  /* linearisation */
  double* K;  /* nc*81: per-cell Hessian acting on D = sum_i p_i (x) grad w_ic */
  int have_lin;
};

static long cells_total(const orc_scene* s) { return (long)s->n[0] * s->n[1] * s->n[2]; }
static long nodes_total(const orc_scene* s) {
  return (long)(s->n[0] + 1) * (s->n[1] + 1) * (s->n[2] + 1);
}
static long cell_dense(const orc_scene* s, int i, int j, int k) {
  return ((long)k * s->n[1] + j) * s->n[0] + i;
}
static long node_dense(const orc_scene* s, int i, int j, int k) {
  return ((long)k * (s->n[1] + 1) + j) * (s->n[0] + 1) + i;
}
/* Brick-major key with 8^3 bricks: bricks in (z,y,x) lexicographic order,
 * cells (or nodes) inside a brick in (z,y,x) order.  The brick grid is
 * (n_a >> 3) + 1 bricks per axis for both cells and nodes. */
static long long brick_key(const orc_scene* s, int i, int j, int k) {
  long long nbx = (s->n[0] >> 3) + 1, nby = (s->n[1] >> 3) + 1;
  long long b = ((long long)(k >> 3) * nby + (j >> 3)) * nbx + (i >> 3);
  return b * 512 + (k & 7) * 64 + (j & 7) * 8 + (i & 7);
}

orc_state* orc_create(const orc_scene* sc) {
  orc_state* st = (orc_state*)calloc(1, sizeof(orc_state));
  st->sc = *sc;
  return st;
}

static void free_all(orc_state* st) {
  void* ptrs[] = {st->x, st->v, st->F, st->G, st->mp, st->Vp, st->mat, st->perm, st->pkey,
                  st->base, st->frac, st->ckey, st->cijk, st->cell_index, st->corner,
                  st->m_c, st->v_c, st->G_c, st->V_ck, st->tau_ck, st->S_ck, st->v_c_new,
                  st->G_c_new, st->nkey, st->nijk, st->node_index, st->m_i, st->v_i,
                  st->vhat, st->vfix, st->vnew, st->fixed, st->K};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
  orc_scene sc = st->sc;
  memset(st, 0, sizeof *st);
  st->sc = sc;
}

void orc_destroy(orc_state* st) {
  if (!st) return;
  free_all(st);
  free(st);
}

void orc_set_time(orc_state* st, double t) { st->sc.time = t; }

typedef struct { long long key; long idx; } kv_t;
static int kv_cmp(const void* a, const void* b) {
  const kv_t *x = (const kv_t*)a, *y = (const kv_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}
static int ll_cmp(const void* a, const void* b) {
  long long x = *(const long long*)a, y = *(const long long*)b;
  return x < y ? -1 : (x > y);
}

/* Dirichlet rule (the paper only says boundaries become unambiguous):
 * sticky walls on the outer wall_layers node layers, then an optional
 * axis-aligned box moving with plate_vel. */
static int dirichlet(const orc_scene* s, int i, int j, int k, double vel[3]) {
  int id[3] = {i, j, k};
  for (int a = 0; a < 3; ++a)
    if (id[a] < s->wall_layers || id[a] > s->n[a] - s->wall_layers) {
      vel[0] = vel[1] = vel[2] = 0;
      return 1;
    }
  if (s->has_plate) {
    int in = 1;
    for (int a = 0; a < 3; ++a) {
      double xa = (double)id[a] * s->dx;
      double sh = s->plate_vel[a] * s->time;
      double lo = s->plate_lo[a] + sh, hi = s->plate_hi[a] + sh;
      if (!(xa >= lo && xa <= hi)) in = 0;
    }
    if (in) {
      for (int a = 0; a < 3; ++a) vel[a] = s->plate_vel[a];
      return 1;
    }
  }
  return 0;
}

/* ========================================================================
 * Algorithm 2: Unload
 * ====================================================================== */
int orc_unload(orc_state* st, long np, const double* x, const double* v, const double* F,
               const double* G, const double* mp, const double* Vp, const int* mat) {
  free_all(st);
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  st->np = np;
  st->base = (int*)malloc(sizeof(int) * 3 * (np ? np : 1));
  st->frac = (double*)malloc(sizeof(double) * 3 * (np ? np : 1));
  long long* key = (long long*)malloc(sizeof(long long) * (np ? np : 1));
  /* base centre b = floor(x/dx - 1/2) and fraction f, both from the stored x;
   * w_cp is the trilinear weight over the 8 surrounding centres (Sec. 3.1). */
  for (long p = 0; p < np; ++p) {
    int b[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double xa = x[3 * p + a];
      if (!isfinite(xa)) { free(key); return ORC_ERR_NONFINITE; }
      double sa = xa * s->inv_dx - 0.5;
      double fl = floor(sa);
      if (fl < 0 || fl + 1 > s->n[a] - 1) { free(key); return ORC_ERR_OUT_OF_DOMAIN; }
      b[a] = (int)fl;
      f[a] = sa - fl;
    }
    key[p] = brick_key(s, b[0], b[1], b[2]);
    for (int a = 0; a < 3; ++a) {
      st->base[3 * p + a] = b[a];
      st->frac[3 * p + a] = f[a];
    }
  }
  /* stable sort by key */
  kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * (np ? np : 1));
  for (long p = 0; p < np; ++p) { kv[p].key = key[p]; kv[p].idx = p; }
  qsort(kv, np, sizeof(kv_t), kv_cmp);
  st->perm = (long*)malloc(sizeof(long) * (np ? np : 1));
  st->pkey = (long long*)malloc(sizeof(long long) * (np ? np : 1));
  st->x = (double*)malloc(sizeof(double) * 3 * (np ? np : 1));
  st->v = (double*)malloc(sizeof(double) * 3 * (np ? np : 1));
  st->F = (double*)malloc(sizeof(double) * 9 * (np ? np : 1));
  st->G = (double*)malloc(sizeof(double) * 9 * (np ? np : 1));
  st->mp = (double*)malloc(sizeof(double) * (np ? np : 1));
  st->Vp = (double*)malloc(sizeof(double) * (np ? np : 1));
  st->mat = (int*)malloc(sizeof(int) * (np ? np : 1));
  int* nb = (int*)malloc(sizeof(int) * 3 * (np ? np : 1));
  double* nf = (double*)malloc(sizeof(double) * 3 * (np ? np : 1));
  for (long q = 0; q < np; ++q) {
    long p = kv[q].idx;
    st->perm[q] = p;
    st->pkey[q] = kv[q].key;
    memcpy(st->x + 3 * q, x + 3 * p, 3 * sizeof(double));
    memcpy(st->v + 3 * q, v + 3 * p, 3 * sizeof(double));
    memcpy(st->F + 9 * q, F + 9 * p, 9 * sizeof(double));
    memcpy(st->G + 9 * q, G + 9 * p, 9 * sizeof(double));
    st->mp[q] = mp[p];
    st->Vp[q] = Vp[p];
    st->mat[q] = mat[p];
    if (mat[p] < 0 || mat[p] >= K) { free(kv); free(key); free(nb); free(nf); return ORC_ERR_ARG; }
    memcpy(nb + 3 * q, st->base + 3 * p, 3 * sizeof(int));
    memcpy(nf + 3 * q, st->frac + 3 * p, 3 * sizeof(double));
  }
  free(st->base); free(st->frac);
  st->base = nb; st->frac = nf;
  free(kv); free(key);

  /* active cells: c is active iff some particle has w_cp > 0, i.e. on every
   * axis c_a = b_a, or c_a = b_a + 1 with f_a > 0 (Algorithm 2, m_c != 0) */
  long ncell = cells_total(s), nnode = nodes_total(s);
  unsigned char* cflag = (unsigned char*)calloc(ncell, 1);
  for (long p = 0; p < np; ++p) {
    const int* b = st->base + 3 * p;
    const double* f = st->frac + 3 * p;
    for (int o = 0; o < 8; ++o) {
      int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1}, ok = 1;
      for (int a = 0; a < 3; ++a) if (oa[a] == 1 && !(f[a] > 0)) ok = 0;
      if (ok) cflag[cell_dense(s, b[0] + oa[0], b[1] + oa[1], b[2] + oa[2])] = 1;
    }
  }
  long nc = 0;
  for (long c = 0; c < ncell; ++c) nc += cflag[c];
  st->nc = nc;
  st->ckey = (long long*)malloc(sizeof(long long) * (nc ? nc : 1));
  {
    long q = 0;
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i)
          if (cflag[cell_dense(s, i, j, k)]) st->ckey[q++] = brick_key(s, i, j, k);
  }
  qsort(st->ckey, nc, sizeof(long long), ll_cmp);
  /* decode keys back to (i,j,k) */
  st->cijk = (int*)malloc(sizeof(int) * 3 * (nc ? nc : 1));
  st->cell_index = (int*)malloc(sizeof(int) * ncell);
  for (long c = 0; c < ncell; ++c) st->cell_index[c] = -1;
  long long nbx = (s->n[0] >> 3) + 1, nby = (s->n[1] >> 3) + 1;
  for (long c = 0; c < nc; ++c) {
    long long kk = st->ckey[c], b = kk / 512, l = kk % 512;
    int i = (int)((b % nbx) * 8 + (l % 8));
    int j = (int)(((b / nbx) % nby) * 8 + ((l / 8) % 8));
    int k = (int)((b / (nbx * nby)) * 8 + (l / 64));
    st->cijk[3 * c] = i; st->cijk[3 * c + 1] = j; st->cijk[3 * c + 2] = k;
    st->cell_index[cell_dense(s, i, j, k)] = (int)c;
  }
  free(cflag);
  /* DOF nodes: corners of active cells */
  unsigned char* nflag = (unsigned char*)calloc(nnode, 1);
  for (long c = 0; c < nc; ++c)
    for (int o = 0; o < 8; ++o)
      nflag[node_dense(s, st->cijk[3 * c] + (o & 1), st->cijk[3 * c + 1] + ((o >> 1) & 1),
                       st->cijk[3 * c + 2] + ((o >> 2) & 1))] = 1;
  long nn = 0;
  for (long i = 0; i < nnode; ++i) nn += nflag[i];
  st->nn = nn;
  st->nkey = (long long*)malloc(sizeof(long long) * (nn ? nn : 1));
  {
    long q = 0;
    for (int k = 0; k <= s->n[2]; ++k)
      for (int j = 0; j <= s->n[1]; ++j)
        for (int i = 0; i <= s->n[0]; ++i)
          if (nflag[node_dense(s, i, j, k)]) st->nkey[q++] = brick_key(s, i, j, k);
  }
  qsort(st->nkey, nn, sizeof(long long), ll_cmp);
  free(nflag);
  st->nijk = (int*)malloc(sizeof(int) * 3 * (nn ? nn : 1));
  st->node_index = (int*)malloc(sizeof(int) * nnode);
  for (long i = 0; i < nnode; ++i) st->node_index[i] = -1;
  for (long q = 0; q < nn; ++q) {
    long long kk = st->nkey[q], b = kk / 512, l = kk % 512;
    int i = (int)((b % nbx) * 8 + (l % 8));
    int j = (int)(((b / nbx) % nby) * 8 + ((l / 8) % 8));
    int k = (int)((b / (nbx * nby)) * 8 + (l / 64));
    st->nijk[3 * q] = i; st->nijk[3 * q + 1] = j; st->nijk[3 * q + 2] = k;
    st->node_index[node_dense(s, i, j, k)] = (int)q;
  }
  st->corner = (int*)malloc(sizeof(int) * 8 * (nc ? nc : 1));
  for (long c = 0; c < nc; ++c)
    for (int o = 0; o < 8; ++o)
      st->corner[8 * c + o] =
          st->node_index[node_dense(s, st->cijk[3 * c] + (o & 1), st->cijk[3 * c + 1] + ((o >> 1) & 1),
                                    st->cijk[3 * c + 2] + ((o >> 2) & 1))];

  /* P2Q (Algorithm 2 loop over p; Sec. 3.1 and 3.2) */
  long C1 = nc ? nc : 1;
  st->m_c = (double*)calloc(C1, sizeof(double));
  st->v_c = (double*)calloc(3 * C1, sizeof(double));
  st->G_c = (double*)calloc(9 * C1, sizeof(double));
  st->V_ck = (double*)calloc(K * C1, sizeof(double));
  st->tau_ck = (double*)calloc(9 * K * C1, sizeof(double));
  st->S_ck = (double*)calloc(9 * K * C1, sizeof(double));
  st->v_c_new = (double*)calloc(3 * C1, sizeof(double));
  st->G_c_new = (double*)calloc(9 * C1, sizeof(double));
  const double dx = s->dx;
  for (long p = 0; p < np; ++p) {
    double tau[9];
    int k = st->mat[p];
    if (orc_kirchhoff(s->model[k], s->mu[k], s->lam[k], st->F + 9 * p, tau))
      return ORC_ERR_NONFINITE;
    const int* b = st->base + 3 * p;
    const double* f = st->frac + 3 * p;
    const double* xp = st->x + 3 * p;
    const double* vp = st->v + 3 * p;
    const double* Gp = st->G + 9 * p;
    for (int o = 0; o < 8; ++o) {
      int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      double w = 1;
      for (int a = 0; a < 3; ++a) w *= oa[a] ? f[a] : 1 - f[a];
      if (w == 0) continue;
      int ci = b[0] + oa[0], cj = b[1] + oa[1], ck = b[2] + oa[2];
      long c = st->cell_index[cell_dense(s, ci, cj, ck)];
      double xc[3] = {(ci + 0.5) * dx, (cj + 0.5) * dx, (ck + 0.5) * dx};
      double d[3] = {xc[0] - xp[0], xc[1] - xp[1], xc[2] - xp[2]};
      double wm = w * st->mp[p];
      st->m_c[c] += wm;
      for (int r = 0; r < 3; ++r) {
        double aff = Gp[3 * r] * d[0] + Gp[3 * r + 1] * d[1] + Gp[3 * r + 2] * d[2];
        st->v_c[3 * c + r] += wm * (vp[r] + aff);
      }
      for (int r = 0; r < 9; ++r) st->G_c[9 * c + r] += wm * Gp[r];
      double wV = w * st->Vp[p];
      st->V_ck[K * c + k] += wV;
      for (int r = 0; r < 9; ++r) st->tau_ck[9 * (K * c + k) + r] += wV * tau[r];
    }
  }
  /* normalise (Algorithm 2, cells with m_c != 0 and V_ck != 0) */
  for (long c = 0; c < nc; ++c) {
    if (st->m_c[c] != 0) {
      for (int r = 0; r < 3; ++r) st->v_c[3 * c + r] /= st->m_c[c];
      for (int r = 0; r < 9; ++r) st->G_c[9 * c + r] /= st->m_c[c];
    }
    for (int k = 0; k < K; ++k)
      if (st->V_ck[K * c + k] != 0)
        for (int r = 0; r < 9; ++r) st->tau_ck[9 * (K * c + k) + r] /= st->V_ck[K * c + k];
  }
  /* Q2N (Sec. 3.3): w_ic = 1/8, (mv)_i += w m_c (v_c + G_c (x_i - x_c)) */
  long N1 = nn ? nn : 1;
  st->m_i = (double*)calloc(N1, sizeof(double));
  st->v_i = (double*)calloc(3 * N1, sizeof(double));
  st->vhat = (double*)calloc(3 * N1, sizeof(double));
  st->vfix = (double*)calloc(3 * N1, sizeof(double));
  st->vnew = (double*)calloc(3 * N1, sizeof(double));
  st->fixed = (int*)calloc(N1, sizeof(int));
  for (long c = 0; c < nc; ++c) {
    if (st->m_c[c] == 0) continue;
    for (int o = 0; o < 8; ++o) {
      int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      long i = st->corner[8 * c + o];
      double d[3];
      for (int a = 0; a < 3; ++a)
        d[a] = (st->cijk[3 * c + a] + oa[a]) * dx - (st->cijk[3 * c + a] + 0.5) * dx;
      double wm = 0.125 * st->m_c[c];
      st->m_i[i] += wm;
      for (int r = 0; r < 3; ++r) {
        const double* Gc = st->G_c + 9 * c;
        st->v_i[3 * i + r] +=
            wm * (st->v_c[3 * c + r] + Gc[3 * r] * d[0] + Gc[3 * r + 1] * d[1] + Gc[3 * r + 2] * d[2]);
      }
    }
  }
  for (long i = 0; i < nn; ++i) {
    if (st->m_i[i] != 0)
      for (int r = 0; r < 3; ++r) st->v_i[3 * i + r] /= st->m_i[i];
    /* external force folded into the inertia target: vhat = v^n + dt g */
    for (int r = 0; r < 3; ++r) st->vhat[3 * i + r] = st->v_i[3 * i + r] + s->dt * s->gravity[r];
    st->fixed[i] = dirichlet(s, st->nijk[3 * i], st->nijk[3 * i + 1], st->nijk[3 * i + 2],
                             st->vfix + 3 * i);
  }
  st->K = (double*)calloc(81 * C1, sizeof(double));
  st->have_lin = 0;
  return ORC_OK;
}

/* ========================================================================
 * Algorithm 3, implicit branch
 * ====================================================================== */
int orc_stretch(orc_state* st) {
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  for (long c = 0; c < st->nc; ++c)
    for (int k = 0; k < K; ++k) {
      double* S = st->S_ck + 9 * (K * c + k);
      if (st->V_ck[K * c + k] == 0) {
        memset(S, 0, 9 * sizeof(double));
        continue;
      }
      int rc = orc_stretch_from_tau(s->model[k], s->mu[k], s->lam[k],
                                    st->tau_ck + 9 * (K * c + k), S);
      if (rc) return rc;
    }
  return ORC_OK;
}

/* grad w_ic at x_c = (x_i - x_c) / (2^{d-2} dx^2), d = 3 (Sec. 3.3) */
static void grad_w(const orc_scene* s, int o, double g[3]) {
  for (int a = 0; a < 3; ++a) {
    int oa = (o >> a) & 1;
    double d = (oa ? 0.5 : -0.5) * s->dx;
    g[a] = d / (2 * s->dx * s->dx);
  }
}

/* G_c(v) = sum_i v_i (x) grad w_ic */
static void cell_vgrad(const orc_state* st, long c, const double* v, double Gc[9]) {
  for (int r = 0; r < 9; ++r) Gc[r] = 0;
  for (int o = 0; o < 8; ++o) {
    double g[3];
    grad_w(&st->sc, o, g);
    const double* vi = v + 3 * st->corner[8 * c + o];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Gc[3 * a + b] += vi[a] * g[b];
  }
}

/* F_c(v) = (I + dt G_c(v)) S_c  (Sec. 4.2) */
static void trial_F(const orc_scene* s, const double Gc[9], const double S[9], double Fc[9]) {
  double A[9];
  for (int r = 0; r < 9; ++r) A[r] = s->dt * Gc[r];
  A[0] += 1; A[4] += 1; A[8] += 1;
  m3_mul(A, S, Fc);
}

/* the incremental potential's two parts: inertia (returned in *e_in) and the
 * elastic sum (*e_el); the gradient when grad != NULL */
static int eval_parts(orc_state* st, const double* v, double* e_in, double* e_el, double* grad) {
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  double Ein = 0, E = 0;
  if (grad) memset(grad, 0, sizeof(double) * 3 * st->nn);
  for (long i = 0; i < st->nn; ++i)
    for (int r = 0; r < 3; ++r) {
      double d = v[3 * i + r] - st->vhat[3 * i + r];
      Ein += 0.5 * st->m_i[i] * d * d;
      if (grad) grad[3 * i + r] += st->m_i[i] * d;
    }
  int bad = 0;
  for (long c = 0; c < st->nc; ++c) {
    double Gc[9];
    cell_vgrad(st, c, v, Gc);
    for (int k = 0; k < K; ++k) {
      double Vck = st->V_ck[K * c + k];
      if (Vck == 0) continue;
      const double* S = st->S_ck + 9 * (K * c + k);
      double Fc[9], psi;
      trial_F(s, Gc, S, Fc);
      if (orc_psi(s->model[k], s->mu[k], s->lam[k], Fc, &psi)) { bad = 1; continue; }
      E += Vck * psi;
      if (grad) {
        /* g_i += dt V P S^T grad w_ic */
        double P[9], PS[9];
        orc_piola(s->model[k], s->mu[k], s->lam[k], Fc, P);
        m3_mul_bt(P, S, PS);
        for (int o = 0; o < 8; ++o) {
          double g[3];
          grad_w(s, o, g);
          long i = st->corner[8 * c + o];
          for (int a = 0; a < 3; ++a)
            grad[3 * i + a] += s->dt * Vck * (PS[3 * a] * g[0] + PS[3 * a + 1] * g[1] + PS[3 * a + 2] * g[2]);
        }
      }
    }
  }
  if (grad)
    for (long i = 0; i < st->nn; ++i)
      if (st->fixed[i]) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = 0;
  *e_in = Ein;
  *e_el = bad ? INFINITY : E;
  return bad;
}

int orc_eval(orc_state* st, const double* v, double* phi, double* grad) {
  double ein, eel;
  int bad = eval_parts(st, v, &ein, &eel, grad);
  *phi = bad ? INFINITY : ein + eel;
  return bad;
}

/* K_c acting on D (9-vector, D_ab = sum_i p_i[a] grad w_ic[b]):
 * K_c = dt^2 sum_k V_ck L_S^T A_k L_S with (L_S D) = D S. */
int orc_linearize(orc_state* st, const double* v, int project) {
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  for (long c = 0; c < st->nc; ++c) {
    double* Kc = st->K + 81 * c;
    memset(Kc, 0, 81 * sizeof(double));
    double Gc[9];
    cell_vgrad(st, c, v, Gc);
    for (int k = 0; k < K; ++k) {
      double Vck = st->V_ck[K * c + k];
      if (Vck == 0) continue;
      const double* S = st->S_ck + 9 * (K * c + k);
      double Fc[9], A[81];
      trial_F(s, Gc, S, Fc);
      if (orc_tangent(s->model[k], s->mu[k], s->lam[k], Fc, project, A)) return ORC_ERR_NONFINITE;
      for (int col = 0; col < 9; ++col) {
        double D[9] = {0}, dF[9], dP[9], Y[9];
        D[col] = 1;
        m3_mul(D, S, dF);
        for (int r = 0; r < 9; ++r) {
          double acc = 0;
          for (int q = 0; q < 9; ++q) acc += A[9 * r + q] * dF[q];
          dP[r] = acc;
        }
        m3_mul_bt(dP, S, Y);
        for (int r = 0; r < 9; ++r) Kc[9 * r + col] += s->dt * s->dt * Vck * Y[r];
      }
    }
  }
  st->have_lin = 1;
  return ORC_OK;
}

void orc_hvp(const orc_state* st, const double* p, double* y) {
  const orc_scene* s = &st->sc;
  for (long i = 0; i < st->nn; ++i)
    for (int r = 0; r < 3; ++r) y[3 * i + r] = st->m_i[i] * p[3 * i + r];
  for (long c = 0; c < st->nc; ++c) {
    double D[9], KD[9];
    cell_vgrad(st, c, p, D);
    const double* Kc = st->K + 81 * c;
    for (int r = 0; r < 9; ++r) {
      double acc = 0;
      for (int q = 0; q < 9; ++q) acc += Kc[9 * r + q] * D[q];
      KD[r] = acc;
    }
    for (int o = 0; o < 8; ++o) {
      double g[3];
      grad_w(s, o, g);
      long i = st->corner[8 * c + o];
      for (int a = 0; a < 3; ++a)
        y[3 * i + a] += KD[3 * a] * g[0] + KD[3 * a + 1] * g[1] + KD[3 * a + 2] * g[2];
    }
  }
  for (long i = 0; i < st->nn; ++i)
    if (st->fixed[i]) y[3 * i] = y[3 * i + 1] = y[3 * i + 2] = 0;
}

void orc_diag(const orc_state* st, double* d) {
  const orc_scene* s = &st->sc;
  for (long i = 0; i < st->nn; ++i)
    for (int r = 0; r < 3; ++r) d[3 * i + r] = st->m_i[i];
  for (long c = 0; c < st->nc; ++c) {
    const double* Kc = st->K + 81 * c;
    for (int o = 0; o < 8; ++o) {
      double g[3];
      grad_w(s, o, g);
      long i = st->corner[8 * c + o];
      for (int a = 0; a < 3; ++a) {
        double acc = 0;
        for (int b = 0; b < 3; ++b)
          for (int bb = 0; bb < 3; ++bb) acc += Kc[9 * (3 * a + b) + (3 * a + bb)] * g[b] * g[bb];
        d[3 * i + a] += acc;
      }
    }
  }
  for (long i = 0; i < st->nn; ++i)
    if (st->fixed[i]) d[3 * i] = d[3 * i + 1] = d[3 * i + 2] = 0;
}

/* f_i = - sum_c sum_k V_ck tau_ck grad w_ic (Algorithm 3, explicit branch) */
void orc_explicit_force(const orc_state* st, double* f) {
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  memset(f, 0, sizeof(double) * 3 * st->nn);
  for (long c = 0; c < st->nc; ++c)
    for (int k = 0; k < K; ++k) {
      double Vck = st->V_ck[K * c + k];
      const double* T = st->tau_ck + 9 * (K * c + k);
      for (int o = 0; o < 8; ++o) {
        double g[3];
        grad_w(s, o, g);
        long i = st->corner[8 * c + o];
        for (int a = 0; a < 3; ++a)
          f[3 * i + a] -= Vck * (T[3 * a] * g[0] + T[3 * a + 1] * g[1] + T[3 * a + 2] * g[2]);
      }
    }
}

/* Algorithm 3, explicit branch: f_i = -sum_c sum_k V_ck tau_ck grad w_ic
 * (the explicit internal force of Sec. 4), v_i^{n+1} = vhat_i + dt f_i / m_i
 * on free DOFs (gravity is in vhat as in the implicit branch), prescribed
 * values on Dirichlet nodes. */
int orc_explicit(orc_state* st) {
  double* f = (double*)malloc(sizeof(double) * 3 * (st->nn ? st->nn : 1));
  orc_explicit_force(st, f);
  for (long i = 0; i < st->nn; ++i)
    for (int r = 0; r < 3; ++r)
      st->vnew[3 * i + r] = st->fixed[i] ? st->vfix[3 * i + r]
                                         : st->vhat[3 * i + r] + st->sc.dt * f[3 * i + r] / st->m_i[i];
  free(f);
  return ORC_OK;
}

static double dot(long n, const double* a, const double* b) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Jacobi-PCG (diag of H, zero on fixed DOFs) on H x = b, x0 = 0. */
int orc_pcg(const orc_state* st, const double* b, double* x, double rtol, int maxit,
            double* rel_resid) {
  long n = 3 * st->nn;
  double *r = (double*)malloc(sizeof(double) * (n ? n : 1)), *z = (double*)malloc(sizeof(double) * (n ? n : 1));
  double *p = (double*)malloc(sizeof(double) * (n ? n : 1)), *q = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* d = (double*)malloc(sizeof(double) * (n ? n : 1));
  orc_diag(st, d);
  for (long i = 0; i < n; ++i) {
    x[i] = 0;
    r[i] = d[i] > 0 ? b[i] : 0;
    z[i] = d[i] > 0 ? r[i] / d[i] : 0;
    p[i] = z[i];
  }
  double rz = dot(n, r, z), r0 = sqrt(dot(n, r, r)), rn = r0;
  int it = 0;
  if (r0 > 0) {
    while (it < maxit) {
      orc_hvp(st, p, q);
      double pq = dot(n, p, q);
      ++it;
      if (!(pq > 0)) break;
      double al = rz / pq;
      for (long i = 0; i < n; ++i) { x[i] += al * p[i]; r[i] -= al * q[i]; }
      rn = sqrt(dot(n, r, r));
      if (rn <= rtol * r0) break;
      for (long i = 0; i < n; ++i) z[i] = d[i] > 0 ? r[i] / d[i] : 0;
      double rz2 = dot(n, r, z), be = rz2 / rz;
      rz = rz2;
      for (long i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
    }
  }
  if (rel_resid) *rel_resid = r0 > 0 ? rn / r0 : 0;
  free(r); free(z); free(p); free(q); free(d);
  return it;
}

/* Newton on Phi(v) (Algorithm 3), x0 = vhat with Dirichlet values.
 * Stop when ||g|| <= max(newton_rtol ||g(v0)||, newton_atol, 1e-12 ||M vhat||)
 * (the last term is the rounding level of the gradient: a body at rest or in
 * free fall starts at g(v0) = 0 up to rounding, which the relative test cannot
 * reduce further); Jacobi-PCG to cg_rtol; Armijo backtracking by halving. */
/* Sec. "Fixed-Point Plasticity" (plasticity updated inside each Newton
 * iteration, the linear solves see elasticity only): at iterate v, each slot of
 * a plastic material takes its trial F = (I + dt G_c(v)) B to the yield surface
 * by the material's return map; where that changes F, the slot's base becomes
 * B = (I + dt G_c(v))^{-1} F^E, so that F_c(v) = F^E.  Returns the number of
 * slots changed. */
static long plastic_project(orc_state* st, const double* v) {
  const orc_scene* s = &st->sc;
  const int K = s->n_mats;
  long changed = 0;
  for (long c = 0; c < st->nc; ++c) {
    double Gc[9], A[9], Ai[9];
    cell_vgrad(st, c, v, Gc);
    for (int r = 0; r < 9; ++r) A[r] = s->dt * Gc[r];
    A[0] += 1; A[4] += 1; A[8] += 1;
    double det = m3_det(A);
    if (!(det > 0)) continue;
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det; Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det; Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det; Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det; Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    for (int k = 0; k < K; ++k) {
      if (st->V_ck[K * c + k] == 0 || s->plastic[k] == ORC_ELASTIC) continue;
      double* B = st->S_ck + 9 * (K * c + k);
      double F[9];
      m3_mul(A, B, F);
      if (orc_return_map(s->plastic[k], s->mu[k], s->lam[k], s->yield_stress[k], s->friction_angle[k], F) == 0)
        continue;
      m3_mul(Ai, F, B);
      ++changed;
    }
  }
  return changed;
}

int orc_newton(orc_state* st, const orc_solver* opt, orc_stats* stats) {
  long n = 3 * st->nn;
  double* v = st->vnew;
  double* g = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* dv = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* vt = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* rhs = (double*)malloc(sizeof(double) * (n ? n : 1));
  memset(stats, 0, sizeof *stats);
  for (long i = 0; i < st->nn; ++i)
    for (int r = 0; r < 3; ++r)
      v[3 * i + r] = st->fixed[i] ? st->vfix[3 * i + r] : st->vhat[3 * i + r];
  if (opt->fixed_point) plastic_project(st, v);
  double phi;
  orc_eval(st, v, &phi, g);
  double g0 = sqrt(dot(n, g, g)), gn = g0;
  double mv2 = 0;
  for (long i = 0; i < st->nn; ++i)
    if (!st->fixed[i])
      for (int r = 0; r < 3; ++r) mv2 += (st->m_i[i] * st->vhat[3 * i + r]) * (st->m_i[i] * st->vhat[3 * i + r]);
  const double gfloor = 1e-12 * sqrt(mv2);
  stats->g0_norm = g0;
  stats->phi0 = phi;
  int status = ORC_OK, it = 0;
  while (1) {
    if (gn <= opt->newton_rtol * g0 || gn <= opt->newton_atol || gn <= gfloor) break;
    if (it >= opt->newton_max) { status = ORC_WARN_NOT_CONVERGED; break; }
    if (orc_linearize(st, v, 1)) { status = ORC_ERR_NONFINITE; break; }
    for (long i = 0; i < n; ++i) rhs[i] = -g[i];
    double rr;
    int cgit = orc_pcg(st, rhs, dv, opt->cg_rtol, opt->cg_max, &rr);
    if (it < 64) stats->cg_iters[it] = cgit;
    stats->cg_iters_total += cgit;
    /* Armijo test of App. B on the energy change Phi(v + a dv) - Phi(v): the
     * inertia part is a A + a^2 B / 2 in closed form (A = sum m (v - vhat).dv,
     * B = sum m |dv|^2), the elastic part a difference of elastic sums, so that
     * no two nearly equal inertia sums are subtracted */
    double slope = dot(n, g, dv), alpha = 1, A = 0, B = 0;
    for (long i = 0; i < st->nn; ++i)
      for (int r = 0; r < 3; ++r) {
        const long q = 3 * i + r;
        A += st->m_i[i] * (v[q] - st->vhat[q]) * dv[q];
        B += st->m_i[i] * dv[q] * dv[q];
      }
    double ein0, eel0, eint, eelt = INFINITY;
    eval_parts(st, v, &ein0, &eel0, NULL);
    int accepted = 0;
    for (int ls = 0; ls <= opt->ls_max; ++ls) {
      for (long i = 0; i < n; ++i) vt[i] = v[i] + alpha * dv[i];
      int bad = eval_parts(st, vt, &eint, &eelt, NULL);
      double dphi = alpha * A + 0.5 * alpha * alpha * B + (eelt - eel0);
      if (!bad && dphi <= opt->ls_c1 * alpha * slope) { accepted = 1; break; }
      alpha *= 0.5;
    }
    if (it < 64) stats->alpha[it] = accepted ? alpha : 0;
    ++it;
    if (!accepted) { status = ORC_WARN_NOT_CONVERGED; break; }
    memcpy(v, vt, sizeof(double) * n);
    if (opt->fixed_point) plastic_project(st, v);
    orc_eval(st, v, &phi, g);
    gn = sqrt(dot(n, g, g));
  }
  stats->newton_iters = it;
  stats->g_norm = gn;
  stats->phi = phi;
  stats->status = status;
  free(g); free(dv); free(vt); free(rhs);
  return status;
}

void orc_set_node_velocity(orc_state* st, const double* v_new) {
  memcpy(st->vnew, v_new, sizeof(double) * 3 * st->nn);
}

/* ========================================================================
 * Algorithm 4: Load
 * ====================================================================== */
/* ------------------------------------------------------------------------
 * Plasticity (config-5 materials).  The paper lists von Mises (li2022) and
 * Drucker-Prager sand (klar2016) among the materials MPM Lite runs and, in
 * its plasticity discussion, applies the return map to the particle's
 * elastic F after the update of Load (the semi-implicit treatment).  Both
 * maps act on the Hencky strain eps_i = log s_i of F = U diag(s) V^T with the
 * StVK-Hencky Kirchhoff stress tau = 2 mu eps + lam tr(eps) I:
 *   von Mises: |dev tau| <= sqrt(2/3) sigma_y; outside, the deviatoric strain
 *     is scaled back to the surface (radial return), tr(eps) kept.
 *   Drucker-Prager (cohesionless, friction angle phi):
 *     |dev tau| + alpha tr(tau) <= 0, alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi));
 *     tr(eps) > 0 (tension): projected to the apex, eps = 0; otherwise the
 *     excess dgamma = |dev eps| + (3 lam + 2 mu) / (2 mu) alpha tr(eps), when
 *     positive, is removed from |dev eps| along dev eps, tr(eps) kept.
 * ---------------------------------------------------------------------- */
int orc_return_map(int plastic, double mu, double lam, double yield_stress, double friction_angle,
                   double F[9]) {
  if (plastic == ORC_ELASTIC) return 0;
  double U[9], sg[3], V[9];
  orc_svd3(F, U, sg, V);
  if (!(sg[0] > 0 && sg[1] > 0 && sg[2] > 0)) return -1;
  double e[3] = {log(sg[0]), log(sg[1]), log(sg[2])};
  const double tr = e[0] + e[1] + e[2];
  double d[3] = {e[0] - tr / 3, e[1] - tr / 3, e[2] - tr / 3};
  const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  int kind = 0;
  if (plastic == ORC_VON_MISES) {
    const double lim = sqrt(2.0 / 3.0) * yield_stress / (2 * mu); /* |dev eps| on the surface */
    if (dn <= lim) return 0;
    for (int i = 0; i < 3; ++i) e[i] = tr / 3 + d[i] * (lim / dn);
    kind = 1;
  } else if (plastic == ORC_DRUCKER_PRAGER) {
    const double sp = sin(friction_angle);
    const double alpha = sqrt(2.0 / 3.0) * 2 * sp / (3 - sp);
    if (tr > 0) {
      e[0] = e[1] = e[2] = 0;
      kind = 2;
    } else {
      const double dg = dn + (3 * lam + 2 * mu) / (2 * mu) * tr * alpha;
      if (dg <= 0) return 0;
      for (int i = 0; i < 3; ++i) e[i] -= dg * d[i] / dn;
      kind = 3;
    }
  } else {
    return -1;
  }
  /* F = U diag(exp(eps)) V^T */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += U[3 * r + k] * exp(e[k]) * V[3 * c + k];
      F[3 * r + c] = acc;
    }
  return kind;
}

int orc_load(orc_state* st, double* x, double* v, double* F, double* G, double* mp,
             double* Vp, int* mat) {
  const orc_scene* s = &st->sc;
  int bad_j = 0;
  for (long c = 0; c < st->nc; ++c) {
    double* vc = st->v_c_new + 3 * c;
    vc[0] = vc[1] = vc[2] = 0;
    if (st->m_c[c] == 0) continue;
    for (int o = 0; o < 8; ++o) {
      const double* vi = st->vnew + 3 * st->corner[8 * c + o];
      for (int a = 0; a < 3; ++a) vc[a] += 0.125 * vi[a];
    }
    cell_vgrad(st, c, st->vnew, st->G_c_new + 9 * c);
  }
  for (long p = 0; p < st->np; ++p) {
    const int* b = st->base + 3 * p;
    const double* f = st->frac + 3 * p;
    double vp[3] = {0, 0, 0}, Gp[9] = {0};
    for (int o = 0; o < 8; ++o) {
      int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      double w = 1;
      for (int a = 0; a < 3; ++a) w *= oa[a] ? f[a] : 1 - f[a];
      if (w == 0) continue;
      long c = st->cell_index[cell_dense(s, b[0] + oa[0], b[1] + oa[1], b[2] + oa[2])];
      for (int a = 0; a < 3; ++a) vp[a] += w * st->v_c_new[3 * c + a];
      for (int r = 0; r < 9; ++r) Gp[r] += w * st->G_c_new[9 * c + r];
    }
    double A[9], Fn[9];
    for (int r = 0; r < 9; ++r) A[r] = s->dt * Gp[r];
    A[0] += 1; A[4] += 1; A[8] += 1;
    m3_mul(A, st->F + 9 * p, Fn);
    {
      const int k = st->mat[p];
      if (s->plastic[k] != ORC_ELASTIC)
        orc_return_map(s->plastic[k], s->mu[k], s->lam[k], s->yield_stress[k], s->friction_angle[k], Fn);
      if (s->model[k] == ORC_WATER) {
        /* Sec. "Water": J_p^{n+1} = (1 + dt tr(G_p^{n+1})) J_p^n, F kept isotropic;
         * a non-positive J is an error (F set to NaN) */
        double Jn = (1 + s->dt * (Gp[0] + Gp[4] + Gp[8])) * m3_det(st->F + 9 * p);
        double c = Jn > 0 ? cbrt(Jn) : NAN;
        for (int r = 0; r < 9; ++r) Fn[r] = (r % 4 == 0) ? c : 0.0;
        if (!(Jn > 0)) bad_j = 1;
      }
    }
    for (int a = 0; a < 3; ++a) {
      x[3 * p + a] = st->x[3 * p + a] + s->dt * vp[a];
      v[3 * p + a] = vp[a];
    }
    memcpy(F + 9 * p, Fn, sizeof Fn);
    memcpy(G + 9 * p, Gp, sizeof Gp);
    if (mp) mp[p] = st->mp[p];
    if (Vp) Vp[p] = st->Vp[p];
    if (mat) mat[p] = st->mat[p];
  }
  return bad_j ? ORC_ERR_NONFINITE : ORC_OK;
}

/* ========================================================================
 * Introspection
 * ====================================================================== */
long orc_count(const orc_state* st, int what) {
  if (what == ORC_N_PARTICLES) return st->np;
  if (what == ORC_N_CELLS) return st->nc;
  if (what == ORC_N_NODES) return st->nn;
  return -1;
}
void orc_get_perm(const orc_state* st, long* perm) { memcpy(perm, st->perm, sizeof(long) * st->np); }
void orc_get_particle_keys(const orc_state* st, long long* k) { memcpy(k, st->pkey, sizeof(long long) * st->np); }
void orc_get_cell_keys(const orc_state* st, long long* k) { memcpy(k, st->ckey, sizeof(long long) * st->nc); }
void orc_get_node_keys(const orc_state* st, long long* k) { memcpy(k, st->nkey, sizeof(long long) * st->nn); }

void orc_get_field(const orc_state* st, int field, double* out) {
  const int K = st->sc.n_mats;
  switch (field) {
    case ORC_C_MASS: memcpy(out, st->m_c, sizeof(double) * st->nc); break;
    case ORC_C_VEL: memcpy(out, st->v_c, sizeof(double) * 3 * st->nc); break;
    case ORC_C_VGRAD: memcpy(out, st->G_c, sizeof(double) * 9 * st->nc); break;
    case ORC_C_VOL: memcpy(out, st->V_ck, sizeof(double) * K * st->nc); break;
    case ORC_C_TAU: memcpy(out, st->tau_ck, sizeof(double) * 9 * K * st->nc); break;
    case ORC_C_STRETCH: memcpy(out, st->S_ck, sizeof(double) * 9 * K * st->nc); break;
    case ORC_C_VEL_NEW: memcpy(out, st->v_c_new, sizeof(double) * 3 * st->nc); break;
    case ORC_C_VGRAD_NEW: memcpy(out, st->G_c_new, sizeof(double) * 9 * st->nc); break;
    case ORC_N_MASS: memcpy(out, st->m_i, sizeof(double) * st->nn); break;
    case ORC_N_VEL: memcpy(out, st->v_i, sizeof(double) * 3 * st->nn); break;
    case ORC_N_VHAT: memcpy(out, st->vhat, sizeof(double) * 3 * st->nn); break;
    case ORC_N_FIXED:
      for (long i = 0; i < st->nn; ++i) out[i] = st->fixed[i];
      break;
    case ORC_N_VNEW: memcpy(out, st->vnew, sizeof(double) * 3 * st->nn); break;
    default: break;
  }
}
