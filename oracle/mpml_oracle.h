/*
 * FP64 CPU oracle for the MPM Lite implicit time step (arXiv 2602.07853).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  The
 * product path (the CUDA library) never calls it and shares no code with it.
 *
 * Everything here is plain double-precision loops over dense grids and
 * compact active-cell / DOF-node lists, written to be checked by eye
 * against the paper:
 *   - Algorithm 1 (one time step): Unload -> Integrate -> Load
 *   - Algorithm 2 (Unload): Sec. 3.1 kinematic unload, Sec. 3.2 stress
 *     unload, Sec. 3.3 centre-to-node gather
 *   - Algorithm 3 (Integrate, implicit branch): Sec. 4.2 rotation-free
 *     stretch reference, Sec. 4.3 stretch reconstruction, the incremental
 *     potential of Sec. 4.2 minimised by Newton with Jacobi-PCG and a
 *     backtracking line search (App. B mentions "standard damping/line-search")
 *   - Algorithm 4 (Load): Sec. 3.3 node-to-centre sampling, Sec. 3.1
 *     centre-to-particle interpolation, advection and F update.
 *
 * Where the paper leaves a passage open, the reading taken is stated at the
 * function that uses it.
 */
#ifndef MPML_ORACLE_H
#define MPML_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_MATS 4

/* ORC_WATER: the inviscid fluid of Sec. "Water": psi(J) = kappa/2 (J - 1)^2 of
 * J = det F only, kappa = lam + 2/3 mu; pressure pi = kappa J (J - 1);
 * base Jacobian by the closed-form root J >= 1/2, S = J^(1/3) I; particles
 * carry F = J^(1/3) I and update J by the grid divergence. */
enum { ORC_FIXED_COROTATED = 0, ORC_NEO_HOOKEAN = 1, ORC_HENCKY = 2, ORC_WATER = 3 };
enum { ORC_ELASTIC = 0, ORC_VON_MISES = 1, ORC_DRUCKER_PRAGER = 2 };

enum {
  ORC_OK = 0,
  ORC_WARN_NOT_CONVERGED = 1,
  ORC_ERR_ARG = -1,
  ORC_ERR_OUT_OF_DOMAIN = -2,
  ORC_ERR_NONFINITE = -3,
  ORC_ERR_STRETCH = -4
};

typedef struct {
  int n[3];            /* cells per axis; nodes are 0..n[a] */
  double dx;           /* cell size */
  double inv_dx;       /* exactly 1/dx as the caller defines it */
  double dt;
  double gravity[3];
  int n_mats;
  int model[ORC_MAX_MATS];
  double mu[ORC_MAX_MATS], lam[ORC_MAX_MATS];
  int wall_layers;     /* node index < wall_layers or > n - wall_layers: sticky */
  int has_plate;       /* moving Dirichlet box */
  double plate_lo[3], plate_hi[3], plate_vel[3];
  double time;         /* time at the start of the step (moves the plate) */
  /* plasticity per material (0 none): return map on the particle's elastic
   * F after its update in Load; yield stress (von Mises), friction angle in
   * radians (Drucker-Prager) */
  int plastic[ORC_MAX_MATS];
  double yield_stress[ORC_MAX_MATS];
  double friction_angle[ORC_MAX_MATS];
} orc_scene;

typedef struct {
  double cg_rtol;      /* ||r|| <= cg_rtol * ||r0|| */
  int cg_max;
  double newton_rtol;  /* ||g|| <= newton_rtol * ||g(v0)|| */
  double newton_atol;  /* or ||g|| <= newton_atol */
  int newton_max;
  double ls_c1;        /* Armijo constant */
  int ls_max;          /* halvings */
  int fixed_point;     /* Sec. "Fixed-Point Plasticity": project the plastic slots'
                          trial F onto the yield surface at every Newton iterate */
} orc_solver;

typedef struct {
  int status;
  int newton_iters;
  int cg_iters_total;
  int cg_iters[64];    /* per Newton iteration (first 64) */
  double alpha[64];
  double g0_norm, g_norm;
  double phi0, phi;
} orc_stats;

typedef struct orc_state orc_state;

/* ---- whole-step API ---------------------------------------------------- */
orc_state* orc_create(const orc_scene* sc);
void orc_destroy(orc_state* st);
void orc_set_time(orc_state* st, double t);

/* Algorithm 2.  Particles are given in any order; the oracle stably sorts
 * them by the brick-major key of their base cell and keeps the sorted copy.
 * x,v: np*3; F,G: np*9 row-major; mp, Vp: np; mat: np.               */
int orc_unload(orc_state* st, long np, const double* x, const double* v,
               const double* F, const double* G, const double* mp,
               const double* Vp, const int* mat);
/* Algorithm 3 (implicit): stretch reconstruction then the Newton solve. */
int orc_stretch(orc_state* st);
int orc_newton(orc_state* st, const orc_solver* opt, orc_stats* stats);
/* Algorithm 3, explicit branch (after orc_unload): v^{n+1} = vhat + dt f / m
 * with the explicit internal force, Dirichlet values on fixed nodes. */
int orc_explicit(orc_state* st);
/* Algorithm 4.  Writes the updated particles in the sorted order. */
int orc_load(orc_state* st, double* x, double* v, double* F, double* G,
             double* mp, double* Vp, int* mat);

/* ---- introspection ------------------------------------------------------ */
enum {
  ORC_N_PARTICLES = 0, ORC_N_CELLS = 1, ORC_N_NODES = 2
};
long orc_count(const orc_state* st, int what);
/* perm[s] = index (in the orc_unload input) of the s-th sorted particle */
void orc_get_perm(const orc_state* st, long* perm);
void orc_get_particle_keys(const orc_state* st, long long* keys); /* sorted */
void orc_get_cell_keys(const orc_state* st, long long* keys);
void orc_get_node_keys(const orc_state* st, long long* keys);
enum {
  ORC_C_MASS = 0,   /* 1  */
  ORC_C_VEL = 1,    /* 3  */
  ORC_C_VGRAD = 2,  /* 9  */
  ORC_C_VOL = 3,    /* n_mats */
  ORC_C_TAU = 4,    /* n_mats*9 */
  ORC_C_STRETCH = 5,/* n_mats*9 */
  ORC_C_VEL_NEW = 6,   /* 3, after Load */
  ORC_C_VGRAD_NEW = 7, /* 9, after Load */
  ORC_N_MASS = 10,  /* 1 */
  ORC_N_VEL = 11,   /* 3 (v_i^n) */
  ORC_N_VHAT = 12,  /* 3 */
  ORC_N_FIXED = 13, /* 1 (1.0 for Dirichlet) */
  ORC_N_VNEW = 14   /* 3 (v_i^{n+1}) */
};
void orc_get_field(const orc_state* st, int field, double* out);
void orc_set_node_velocity(orc_state* st, const double* v_new); /* for Load tests */

/* ---- operator-level access (tests) -------------------------------------- */
/* Phi and its gradient (masked to free DOFs) at node velocities v (nn*3). */
int orc_eval(orc_state* st, const double* v, double* phi, double* grad);
/* Linearise at v: per-cell tangent, projected to PSD if project != 0. */
int orc_linearize(orc_state* st, const double* v, int project);
/* y = H p with the last linearisation (masked). */
void orc_hvp(const orc_state* st, const double* p, double* y);
/* Jacobi diagonal of H (free DOFs; 0 on fixed DOFs). */
void orc_diag(const orc_state* st, double* d);
/* Explicit internal force of Algorithm 3 (explicit branch): f_i. */
void orc_explicit_force(const orc_state* st, double* f);
/* Jacobi-PCG on H x = b (masked), returns iterations. */
int orc_pcg(const orc_state* st, const double* b, double* x, double rtol,
            int maxit, double* rel_resid);

/* ---- constitutive pieces (tests) ---------------------------------------- */
int orc_psi(int model, double mu, double lam, const double F[9], double* psi);
int orc_piola(int model, double mu, double lam, const double F[9], double P[9]);
/* dP/dF as 81 doubles, A[9*(3a+b) + 3c+d] = dP_ab/dF_cd */
int orc_tangent(int model, double mu, double lam, const double F[9],
                int project, double A[81]);
int orc_kirchhoff(int model, double mu, double lam, const double F[9],
                  double tau[9]);
int orc_stretch_from_tau(int model, double mu, double lam,
                         const double tau[9], double S[9]);
void orc_svd3(const double F[9], double U[9], double s[3], double V[9]);
/* Plastic return map of one elastic deformation gradient (in place), in the
 * Hencky strain eps = log(s) of F = U diag(s) V^T; U, V kept.  Returns
 * 0 (admissible, unchanged), 1 (von Mises radial return), 2 (Drucker-Prager
 * apex: s = 1), 3 (Drucker-Prager cone), -1 (det F <= 0: unchanged). */
int orc_return_map(int plastic, double mu, double lam, double yield_stress, double friction_angle,
                   double F[9]);
void orc_sym_eigen(int n, const double* A, double* evals, double* evecs);

#ifdef __cplusplus
}
#endif
#endif
