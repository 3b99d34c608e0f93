/*
 * mpml.h - C ABI of the GB300 (sm_103a) MPM Lite hot path.
 *
 * MPM Lite (arXiv 2602.07853) advances particles by one implicit time step
 * in three calls that follow Algorithm 1 of the paper:
 *
 *   mpml_resample     Algorithm 2 (Unload): particle binning and sort, the
 *                     trilinear particle-to-centre transfer of mass, APIC
 *                     momentum, velocity gradient, volume and extensive
 *                     Kirchhoff stress (Sec. 3.1, 3.2), and the constant
 *                     weight centre-to-node gather (Sec. 3.3).
 *   mpml_newton_step  Algorithm 3 (Integrate, implicit): rotation-free stretch
 *                     reconstruction at every active centre (Sec. 4.2, 4.3)
 *                     and Newton on the incremental potential of Sec. 4.2,
 *                     matrix-free Jacobi-PCG (or learned-preconditioner
 *                     flexible CG) with a backtracking line search.
 *   mpml_g2p          Algorithm 4 (Load): node-to-centre sampling of v and
 *                     its gradient (Sec. 3.3), trilinear interpolation to the
 *                     particles (Sec. 3.1), advection, F update.
 *
 * Conventions
 *   - Plain C types only.  Pointers are either device pointers (MPML_MEM_DEVICE)
 *     or host pointers (MPML_MEM_HOST, pinned or pageable); the caller owns
 *     them and the library never frees them.
 *   - Particle arrays are array-of-structures: x, v are n*3, F, G are n*9
 *     row-major (F[9p + 3r + c]), mass, volume are n, mat is n int32.  Their
 *     element type is float in an MPML_FP32 context and double in MPML_FP64.
 *   - Every call is asynchronous on the context's CUDA stream except where
 *     it says it synchronises.  A status returned by a call is the status of
 *     what that call could check; errors detected on the device (particle
 *     outside the grid, non-finite input, failed stretch inversion) are
 *     latched and returned by the next synchronising call.
 *   - The library owns one context's scratch (grid, cell, node and solver
 *     buffers), allocated with cudaMalloc and grown only inside
 *     mpml_resample; mpml_destroy frees it.
 *   - Grid: n[a] cells per axis of size dx, nodes 0..n[a], origin 0.  Cells
 *     and nodes are grouped in 8x8x8 bricks; "key" below means the
 *     brick-major index ((bz*NBy + by)*NBx + bx)*512 + (lz*64 + ly*8 + lx)
 *     with NB_a = (n[a] >> 3) + 1.
 */
#ifndef MPML_H
#define MPML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPML_MAX_MATS 4

typedef struct mpml_ctx_s* mpml_ctx;

typedef enum {
  MPML_OK = 0,
  MPML_WARN_NOT_CONVERGED = 1, /* Newton hit its cap or the line search failed */
  MPML_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, call order) */
  MPML_ERR_OUT_OF_DOMAIN = -2, /* a particle's 2x2x2 centre stencil leaves the grid */
  MPML_ERR_NONFINITE = -3,     /* NaN/Inf in particle input or in the solve */
  MPML_ERR_STRETCH = -4,       /* stress-to-stretch inversion has no admissible root */
  MPML_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  MPML_ERR_CUDA = -6,          /* a CUDA runtime call failed */
  MPML_ERR_NOMEM = -7,         /* device allocation failed */
  MPML_ERR_TOO_LARGE = -8      /* size above a fixed capacity (mpml_sort_particles_noalloc) */
} mpml_status;

enum { MPML_FIXED_COROTATED = 0, MPML_NEO_HOOKEAN = 1, MPML_HENCKY = 2, MPML_WATER = 3 };
enum { MPML_FP32 = 0, MPML_FP64 = 1 };
enum { MPML_MEM_DEVICE = 0, MPML_MEM_HOST = 1 };
enum { MPML_PRECOND_JACOBI = 0, MPML_PRECOND_LEARNED = 1 };

/* Isotropic hyperelastic material with Lame parameters (mu, lambda).
 * MPML_HENCKY: StVK with Hencky strain (Sec. 4.3.1); MPML_NEO_HOOKEAN: split
 * Neo-Hookean, kappa = 2/3 mu + lambda (Sec. 4.3.2); MPML_FIXED_COROTATED:
 * psi = mu sum(s_i - 1)^2 + lambda/2 (J - 1)^2 (its stretch inverse is the
 * library's, the paper gives the general recipe of Sec. 4.3); MPML_WATER: the
 * inviscid fluid of Sec. "Water", psi = kappa/2 (J - 1)^2 with the bulk modulus
 * kappa = lambda + 2/3 mu > 0 (mu >= 0 may be 0), undefined for J <= 0: the base
 * Jacobian is the root J >= 1/2 of kappa J (J - 1) = tr(tau)/3, S = J^(1/3) I;
 * G2P sets such a particle's F to J^(1/3) I with J <- (1 + dt tr G_p) J (a
 * non-positive J makes F NaN, reported by the next resample); elastic only. */
typedef struct {
  int model;
  double mu, lambda;
  /* Plasticity (0 = elastic): MPML_VON_MISES (yield_stress sigma_y) or
   * MPML_DRUCKER_PRAGER (cohesionless, friction_angle in radians).  The return
   * map acts on each particle's elastic F after its update in mpml_g2p, in
   * the Hencky strain eps = log(s) of F = U diag(s) V^T (U, V kept):
   *   von Mises: |dev tau| <= sqrt(2/3) sigma_y with tau = 2 mu eps +
   *     lambda tr(eps) I; outside, dev eps is scaled back to the surface.
   *   Drucker-Prager: |dev tau| + alpha tr(tau) <= 0,
   *     alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi)); tr(eps) > 0 maps to
   *     eps = 0, otherwise the excess of |dev eps| is removed.
   * The paper lists both materials and treats plasticity on the particle F
   * after Load's update (the semi-implicit form). */
  int plastic;
  double yield_stress, friction_angle;
} mpml_material;
enum { MPML_ELASTIC = 0, MPML_VON_MISES = 1, MPML_DRUCKER_PRAGER = 2 };

/* Scene: grid, time step, gravity (folded into the inertia target
 * vhat = v^n + dt g), precision, Dirichlet boundary.  Nodes with an index
 * below wall_layers or above n - wall_layers on any axis are sticky (v = 0);
 * when has_plate, nodes whose position lies in [plate_lo + t plate_vel,
 * plate_hi + t plate_vel] (t from mpml_set_time) move with plate_vel. */
typedef struct {
  int n[3];
  double dx;
  double inv_dx; /* exactly 1/dx as the caller defines it; used for binning */
  double dt;
  double gravity[3];
  int precision; /* MPML_FP32 or MPML_FP64 */
  int wall_layers;
  int has_plate;
  double plate_lo[3], plate_hi[3], plate_vel[3];
} mpml_scene_desc;

typedef struct {
  int64_t n;
  int mem;          /* MPML_MEM_DEVICE or MPML_MEM_HOST */
  void* x;          /* n*3 */
  void* v;          /* n*3 */
  void* F;          /* n*9 */
  void* G;          /* n*9 */
  void* mass;       /* n */
  void* volume;     /* n */
  int32_t* mat;     /* n, material index < n_mats */
  int32_t* perm;    /* optional (may be NULL), written by mpml_resample:
                       perm[s] = index before the call of the s-th sorted particle */
} mpml_particles;

typedef struct {
  double cg_rtol;      /* stop CG when ||r|| <= cg_rtol ||r0|| (default 1e-6) */
  int cg_max;          /* CG iteration cap per Newton iteration */
  double newton_rtol;  /* stop Newton when ||g|| <= newton_rtol ||g(v0)|| */
  double newton_atol;  /* ... or when ||g|| <= newton_atol (and always when ||g|| <= 1e-12 ||M vhat||,
                          the rounding level of the gradient: a body at rest or in free fall
                          starts from g(v0) = 0 up to rounding) */
  int newton_max;      /* Newton iteration cap */
  double ls_c1;        /* Armijo constant */
  int ls_max;          /* maximal number of step halvings */
  int precond;         /* MPML_PRECOND_JACOBI or MPML_PRECOND_LEARNED */
  int check_every;     /* CG iterations between convergence polls (host-driven loop) */
  int use_graph;       /* how the CG loop runs: 0 host-driven launches; 1 one CUDA graph launch
                          with a device-side conditional WHILE loop; 2 (default when opts is
                          NULL) one persistent cooperative kernel with bounded grid barriers
                          (FP32 contexts; FP64 contexts use 1) */
  int plastic_fixed_point; /* 0 (default): plasticity by the particles' return map after G2P
                          (semi-implicit); 1: Sec. "Fixed-Point Plasticity": at v0 and after
                          every accepted Newton step each plastic slot's trial F =
                          (I + dt G_c(v)) B is return-mapped and its base replaced by
                          B = (I + dt G_c(v))^-1 F^E (a general 3x3 base for the rest of the
                          solve), so the converged grid state satisfies the yield condition;
                          the linear solves see elasticity only.  Single-scene solver only
                          (mpml_newton_step_batch rejects it with MPML_ERR_ARG). */
  double cg_forcing;   /* Not in the paper (which leaves the CG tolerance open).  0 (default):
                          every CG solve stops at cg_rtol ||g_k||.  In (0, 0.5]: inexact
                          Newton -- the CG of Newton iteration k stops at eta_k ||g_k|| with
                          eta_0 = cg_forcing and eta_k = min(cg_forcing, 0.9 (||g_k|| /
                          ||g_{k-1}||)^2) (Eisenstat and Walker's second forcing choice, with
                          their safeguard max(eta_k, 0.9 eta_{k-1}^2) when the latter exceeds
                          0.1), never below cg_rtol nor below half of what the Newton target
                          still needs (0.5 max(newton_rtol ||g_0||, newton_atol) / ||g_k||),
                          capped at 0.5.  Newton's own test (newton_rtol on the FP64 gradient)
                          is unchanged.  The batched solver applies it per scene.  Other
                          values are MPML_ERR_ARG. */
} mpml_solver_opts;

typedef struct {
  int status;
  int newton_iters;
  int cg_iters_total;
  int cg_iters[64];          /* per Newton iteration (first 64) */
  double alpha[64];          /* accepted line-search step per Newton iteration */
  double cg_rel_resid[64];   /* CG recurrence residual ||r||/||r0|| at exit */
  double g0_norm, g_norm;    /* ||g(v0)||, ||g|| at exit (FP64 sums) */
  double phi0, phi;          /* incremental potential at v0 and at exit */
  int64_t n_particles, n_cells, n_nodes, n_bricks;
  int fcg_fallbacks;         /* learned solves that continued with Jacobi-PCG */
  int plastic_projections;   /* fixed-point plasticity: slot projections that changed a base */
} mpml_solve_stats;

/* Lifecycle ----------------------------------------------------------- */
/* stream: a cudaStream_t (NULL = legacy default stream).  n_mats <= MPML_MAX_MATS.
 * Returns MPML_ERR_ARG for invalid sizes (n[a] < 2, dx <= 0, dt <= 0, ...). */
int mpml_create(const mpml_scene_desc* desc, const mpml_material* mats, int n_mats,
                void* stream, mpml_ctx* out);
int mpml_destroy(mpml_ctx ctx);
const char* mpml_status_str(int status);
/* Sets the time used by the moving Dirichlet box for the next step. */
int mpml_set_time(mpml_ctx ctx, double t);
/* Blocks until the context's stream is idle; returns the latched device status. */
int mpml_sync(mpml_ctx ctx);

/* Algorithm 1 ---------------------------------------------------------- */
/* Algorithm 2.  Reads the particles, sorts a library-owned copy by the key
 * of the base centre floor(x/dx - 1/2) (stable), builds the active cells
 * (centres with a nonzero trilinear weight) and DOF nodes (their corners),
 * and runs P2Q and Q2N.  Synchronises once (to size the grid).  Returns
 * MPML_ERR_OUT_OF_DOMAIN / MPML_ERR_NONFINITE for bad particles. */
int mpml_resample(mpml_ctx ctx, const mpml_particles* p);
/* Algorithm 3, implicit.  Synchronises (convergence tests); fills stats if
 * non-NULL.  opts may be NULL (defaults). */
int mpml_newton_step(mpml_ctx ctx, const mpml_solver_opts* opts, mpml_solve_stats* stats);
/* Algorithm 3, explicit branch (after mpml_resample; instead of
 * mpml_newton_step): node velocities v^{n+1} = vhat + dt f / m with the
 * explicit internal force f_i = -sum_c sum_k V_ck tau_ck grad w_ic (Sec. 4),
 * Dirichlet values on fixed nodes; no stretch reconstruction or solve.  The
 * step is stable only below the elastic CFL limit (dt < dx / sqrt(E / rho)
 * roughly).  Asynchronous; follow with mpml_g2p. */
int mpml_explicit_step(mpml_ctx ctx);
/* Batches of independent scenes (one context each, on one device; each context
 * on its own stream or a shared one; at most MPML_BATCH_MAX, all distinct).
 * Not in the paper: the workload statement asks for many scenes of uneven
 * size solved in one persistent launch.
 * mpml_resample_batch: Algorithm 2 for every scene with one host wait for the
 *   whole batch (device particle arrays only; parts is an array of n).
 * mpml_newton_step_batch: Algorithm 3 for every scene (FP32 single-material
 *   contexts, already resampled).  Each scene follows exactly the Newton /
 *   Jacobi-PCG / line-search logic of mpml_newton_step with its own
 *   tolerances and iteration counts, but the scenes advance in lockstep and
 *   every round of their CG solves is one persistent cooperative launch over
 *   all active scenes' bricks (per-scene scalars and FP64 sums), issued on
 *   ctxs[0]'s stream after every scene's stream and followed by all of them
 *   (events).  stats: array of n (may be NULL).  The batch's scratch lives in
 *   ctxs[0].  Synchronises; returns the first error, else
 *   MPML_WARN_NOT_CONVERGED if any scene did not converge. */
#define MPML_BATCH_MAX 128
int mpml_resample_batch(mpml_ctx* ctxs, const mpml_particles* parts, int n);
int mpml_newton_step_batch(mpml_ctx* ctxs, int n, const mpml_solver_opts* opts, mpml_solve_stats* stats);
/* Algorithm 4.  Writes x, v, F, G, mass, volume, mat of p (the same arrays
 * or others of the same size) in the sorted order of the last resample.
 * Asynchronous for device memory; for MPML_MEM_HOST it synchronises after
 * the device-to-host copies. */
int mpml_g2p(mpml_ctx ctx, const mpml_particles* p);

/* Introspection and operator access (host buffers; synchronising) ------ */
/* out[0..3] = particles, active cells, DOF nodes, bricks of the last resample */
int mpml_counts(mpml_ctx ctx, int64_t out[4]);
enum { MPML_KEYS_PARTICLES = 0, MPML_KEYS_CELLS = 1, MPML_KEYS_NODES = 2 };
/* Sorted particle keys, active-cell keys or DOF-node keys (ascending). */
int mpml_get_keys(mpml_ctx ctx, int what, int64_t* out);
enum {
  MPML_F_CELL_MASS = 0,      /* m_c                       1 per active cell  */
  MPML_F_CELL_VEL = 1,       /* v_c                       3                  */
  MPML_F_CELL_VGRAD = 2,     /* G_c                       9 row-major        */
  MPML_F_CELL_VOL = 3,       /* V_ck                      n_mats             */
  MPML_F_CELL_TAU = 4,       /* tau_ck                    n_mats*9           */
  MPML_F_CELL_STRETCH = 5,   /* S_ck (after newton_step)  n_mats*9           */
  MPML_F_CELL_VEL_NEW = 6,   /* v_c^{n+1} (after g2p)     3                  */
  MPML_F_CELL_VGRAD_NEW = 7, /* G_c^{n+1} (after g2p)     9                  */
  MPML_F_NODE_MASS = 10,     /* m_i                       1 per DOF node     */
  MPML_F_NODE_VEL = 11,      /* v_i^n                     3                  */
  MPML_F_NODE_VHAT = 12,     /* vhat_i                    3                  */
  MPML_F_NODE_FIXED = 13,    /* 1.0 on Dirichlet nodes    1                  */
  MPML_F_NODE_VNEW = 14      /* v_i^{n+1}                 3                  */
};
/* Copies a field, in key order of active cells / DOF nodes, as double. */
int mpml_get_field(mpml_ctx ctx, int field, double* out);
/* Overrides v^{n+1} at the DOF nodes (n_nodes*3 doubles in key order). */
int mpml_set_node_velocity(mpml_ctx ctx, const double* v);
/* Reconstructs the stretches (Algorithm 3 line 9) without solving. */
int mpml_stretch(mpml_ctx ctx);
/* Incremental potential and its gradient (masked to free DOFs) at node
 * velocities v (n_nodes*3, key order).  grad may be NULL. */
int mpml_eval(mpml_ctx ctx, const double* v, double* phi, double* grad);
/* Builds the per-cell projected tangent at v (n_nodes*3). */
int mpml_linearize(mpml_ctx ctx, const double* v);
/* y = H p with the last linearisation (masked), n_nodes*3 each. */
int mpml_hvp(mpml_ctx ctx, const double* p, double* y);

/* Profiling: when enabled, every HVP kernel launch (also inside the
 * graph-driven CG loop) is timed on the device from the earliest block start
 * to the last block end with the GPU global timer; mpml_hvp_timing returns
 * the number of timed launches, their total milliseconds and the bytes one
 * launch moves by the library's count (K_c, p, q, m per active brick).
 * Enabling (or re-enabling) resets the counters.  Synchronising. */
int mpml_set_profiling(mpml_ctx ctx, int enable);
int mpml_hvp_timing(mpml_ctx ctx, int64_t* launches, double* total_ms, double* bytes_per_launch);
/* Runs `iters` back-to-back HVPs on the current linearisation with a
 * device-resident direction and returns the mean kernel milliseconds
 * (CUDA events on the context stream).  Synchronising. */
int mpml_hvp_bench(mpml_ctx ctx, int iters, double* mean_ms);
/* With profiling enabled: the persistent cooperative PCG kernel (use_graph = 2)
 * is bracketed by CUDA events on the context stream; returns its launches
 * since profiling was enabled, the CG iterations they ran and their total
 * milliseconds.  With profiling enabled on the first context of a batch, the
 * batched solver's launches are counted there (CG iterations: the largest
 * count among the launch's scenes).  Host-side only (no synchronisation). */
int mpml_pcg_timing(mpml_ctx ctx, int64_t* launches, int64_t* cg_iters, double* total_ms);
/* Number of kernel launches issued on the context stream since creation. */
int64_t mpml_kernel_launches(mpml_ctx ctx);

/* HVP launch-shape autotuner --------------------------------------------
 * Not in the paper (the workload asks for brick tile shapes chosen by an
 * autotuner).  The standalone FP32 HVP of the graph-driven and host-driven CG
 * loops (and of flexible CG) has MPML_HVP_TILES launch shapes per tangent
 * format: the brick kernel (one 8^3 cell brick per 256-thread CTA, two cells
 * per thread, node sums gathered through shared memory) and the z-column
 * kernel (one brick per 64-thread CTA, thread (x, y) walks the 8 cells of its
 * column, node sums by register carries and warp shuffles) at different
 * CTAs per SM.  The persistent solver (use_graph = 2) has a single shape.
 *
 * mpml_autotune_hvp times every shape on the current linearisation (one
 * untimed launch, then `reps` launches between CUDA events on the context
 * stream; the solver's vectors are left untouched), keeps the fastest for the
 * context, records it in a process-wide cache keyed by tangent format and
 * log2 of the active brick count, and returns the shape index and (if `ms` is
 * not NULL) the mean milliseconds of each of the MPML_HVP_TILES shapes.
 * FP32 contexts after a linearisation (MPML_ERR_ARG otherwise).  Synchronising.
 *
 * Without a call, the first standalone-HVP solve of a context takes the
 * cached shape for its format and size, else autotunes with reps = 3.
 * mpml_set_hvp_tile fixes the shape (0 .. MPML_HVP_TILES-1; -1 returns to
 * automatic choice); mpml_get_hvp_tile returns the shape in use (-1: not yet
 * chosen) and a one-line description (static storage).
 * mpml_tile_cache_save / _load write and read the cache as text, one line
 * "format log2_bricks tile mean_ms" per entry (format 25: compressed tangent,
 * 45: packed); loading merges into the cache (malformed lines: MPML_ERR_ARG, nothing merged; unreadable or
 * unwritable file: MPML_ERR_ARG).  Host-only, thread-safe. */
#define MPML_HVP_TILES 3
int mpml_autotune_hvp(mpml_ctx ctx, int reps, int* tile, float* ms);
int mpml_set_hvp_tile(mpml_ctx ctx, int tile);
int mpml_get_hvp_tile(mpml_ctx ctx, int* tile, const char** description);
int mpml_tile_cache_save(const char* path);
int mpml_tile_cache_load(const char* path);
void mpml_tile_cache_clear(void);

/* Persistent-solver launch controls -------------------------------------
 * Not in the paper.  The persistent Jacobi-PCG kernel (use_graph = 2) applies
 * the tangent of each cell brick in one of three ways:
 *   MPML_PCG_STAGED    the CTA's 256 threads work on one brick at a time; its
 *                      whole tangent block comes in by one bulk copy into
 *                      shared memory (kept there for the solve when a CTA owns
 *                      one brick)
 *   MPML_PCG_STREAMED  the same, with the rows read from global memory as the
 *                      column walk needs them (no shared-memory block)
 *   MPML_PCG_COLUMNS   each 64-thread group of a CTA works on half a brick
 *                      (four z-layers of cells) of its own, rows streamed from
 *                      global memory (four half-bricks in flight per CTA; builds
 *                      for 2, 3 and 4 CTAs per SM, the 2-CTA one loading each
 *                      layer's rows one layer ahead)
 *   MPML_PCG_AUTO      the shape mpml_autotune_pcg chose for this tangent format
 *                      and size class, else a fixed rule: above 8 cell bricks
 *                      per SM column groups at 3 CTAs per SM, staged at 2
 *                      otherwise
 * ctas_per_sm: CTAs per SM of the cooperative launch (0 = the autotuned or
 *   fixed-rule count, capped at what fits; at most 2 for the first two forms
 *   and 4 for the third; a value above what fits is MPML_ERR_ARG at the next
 *   solve).
 * barrier_spins: bound on the polls of one grid-barrier wait (0 = the default
 *   2^25 polls of 32 ns, about a second).  A wait that runs out ends the solve:
 *   mpml_newton_step returns MPML_ERR_TIMEOUT; the next mpml_resample clears the
 *   latched status and the context is usable again.  A bound of a few polls
 *   makes the waits run out on purpose (how the tests exercise that path).
 * The configuration applies to every later solve of the context (also the
 * learned solver's Jacobi fallback; the batched solver uses ctas_per_sm and
 * barrier_spins of its first context).  mpml_get_pcg_config returns it, and in
 * last_staging / last_ctas_per_sm (either may be NULL) the shape the last
 * persistent launch used (0 before the first). */
enum { MPML_PCG_AUTO = 0, MPML_PCG_STAGED = 1, MPML_PCG_STREAMED = 2, MPML_PCG_COLUMNS = 3 };
typedef struct {
  int tangent_staging;
  int ctas_per_sm;
  unsigned barrier_spins;
} mpml_pcg_config;
int mpml_set_pcg_config(mpml_ctx ctx, const mpml_pcg_config* cfg);
int mpml_get_pcg_config(mpml_ctx ctx, mpml_pcg_config* cfg, int* last_staging, int* last_ctas_per_sm);

/* Persistent-solver autotuner: times the MPML_PCG_SHAPES shapes of the
 * persistent solve (index: 0 staged x 1 CTA/SM, 1 staged x 2, 2 streamed x 1,
 * 3 streamed x 2, 4 column groups x 2, 5 column groups x 3, 6 column groups
 * x 4; shapes that do not fit are skipped, their time reported as -1) on the
 * Newton system at the current iterate: each runs `iters` Jacobi-PCG
 * iterations from the same start (the solver's state is restored afterwards),
 * CUDA events on the context stream, best of `reps`.  The fastest becomes the
 * context's shape under MPML_PCG_AUTO and is recorded in the process-wide tile
 * cache under format 125 (compressed) or 145 (45 numbers) and log2 of the cell
 * bricks.  FP32 contexts after a linearisation (mpml_linearize or
 * mpml_newton_step), MPML_ERR_ARG otherwise.  Synchronising. */
#define MPML_PCG_SHAPES 7
int mpml_autotune_pcg(mpml_ctx ctx, int iters, int reps, int* shape, float* ms);

/* Lame parameters of an isotropic material from Young's modulus E > 0 and
 * Poisson's ratio -1 < nu < 1/2: mu = E / (2 (1 + nu)),
 * lambda = E nu / ((1 + nu)(1 - 2 nu)) (the standard relations; the paper
 * quotes E and nu).  MPML_ERR_ARG outside that range. */
int mpml_lame_parameters(double E, double nu, double* mu, double* lambda);

/* Learned preconditioner ------------------------------------------------
 * Not in the paper: the workload asks for a small 3D convolutional network
 * on the node grid used inside flexible CG.  Network: three bias-free
 * 3x3x3 convolutions 3 -> 16 -> 16 -> 3 channels, ReLU after the first two,
 * outputs kept on DOF nodes (free DOFs for the last layer); BF16 weights and
 * activations with FP32 accumulation on the tensor cores.  Preconditioner:
 *   z = D^-1 r + s D^-1/2 NN(D^-1/2 r / s),  s = RMS of D^-1/2 r,
 * D the Jacobi diagonal.  With opts->precond = MPML_PRECOND_LEARNED (FP32,
 * single-material contexts, weights set) mpml_newton_step runs flexible CG;
 * when it stalls (z^T r <= 0, or no decrease of ||r|| in 20 iterations) the
 * solve continues with Jacobi-PCG from the current iterate.
 * Weights use the layout per layer (27 taps, C_out, C_in), tap
 * (dz+1)*9 + (dy+1)*3 + (dx+1), layers concatenated (9504 floats). */
typedef struct {
  int samples;   /* (residual, error) pairs taken from one Jacobi-PCG solve */
  double rtol;   /* tolerance of that solve (the pairs' reference solution) */
  int cg_max;
  int epochs;
  int batch;     /* pairs per Adam step */
  float lr;
} mpml_train_opts;
typedef struct {
  int samples;
  double loss_first;  /* mean loss of the first epoch */
  double loss_last;   /* ... of the last epoch */
} mpml_train_stats;
int mpml_nn_weight_count(void);
int mpml_nn_set_weights(mpml_ctx ctx, const float* w);
int mpml_nn_get_weights(mpml_ctx ctx, float* w);
/* Accumulated weight gradient (same layout), as left by mpml_nn_loss_grad. */
int mpml_nn_get_grad(mpml_ctx ctx, float* g);
/* z = preconditioner(r) on the current linearisation (DOF order, n*3). */
int mpml_nn_apply(mpml_ctx ctx, const double* r, double* z);
/* Loss L = 1 - z^T H e / sqrt(z^T H z * e^T H e) (one minus the H-cosine of
 * z(r) and the error e; only the direction of z counts, as in CG) of one pair
 * and its weight gradient (written to the gradient accumulator, which is
 * zeroed first). */
int mpml_nn_loss_grad(mpml_ctx ctx, const double* r, const double* e, double* loss);
/* One Adam step (learning rate lr > 0) with the weight gradient left by
 * mpml_nn_loss_grad, which it then zeroes: training on caller-chosen pairs. */
int mpml_nn_adam_step(mpml_ctx ctx, float lr);
/* Trains on the current Newton system (after mpml_resample): reconstructs the
 * stretches, solves the first Newton system with Jacobi-PCG, takes
 * `samples` pairs (r_k, x* - x_k) along the way and runs Adam on the loss
 * of mpml_nn_loss_grad.  Weights must be set (e.g. a seeded initialisation).
 * Pairs whose error is at rounding level are skipped.  lr = 0 evaluates the
 * current weights instead (mean loss in loss_first, weights unchanged). */
int mpml_nn_train(mpml_ctx ctx, const mpml_train_opts* opts, mpml_train_stats* stats);

/* Allocation-free particle sort ----------------------------------------
 * No counterpart in the paper: a service for callers that must not allocate
 * device memory when they sort, e.g. an application whose own arena owns all
 * device memory, or a time-critical loop that cannot take cudaMalloc's
 * implicit device-wide synchronisation.  It needs no context and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Computes the order mpml_resample gives the particles: ascending brick-major
 * key of the base centre floor(x/dx - 1/2), ties by input index.
 *   n, inv_dx   the grid of an mpml_scene_desc (n[a] >= 2, inv_dx > 0)
 *   precision   MPML_FP32 (x is float) or MPML_FP64 (double)
 *   x           device pointer, n_particles*3 positions (read only)
 *   perm        device pointer, n_particles int32: perm[s] = input index of
 *               the s-th particle in sorted order (written)
 *   keys        device pointer, n_particles int64 keys of the sorted
 *               particles (written), or NULL
 *   stream      a cudaStream_t (NULL = legacy default stream)
 * Its scratch is one fixed array in device memory (about 16 MiB, which every
 * GPU that loads this library holds until the process exits): a grid with
 * NB_x*NB_y*NB_z*512 > MPML_NOALLOC_MAX_SLOTS (e.g. more than 127 cells per
 * axis of a cube) is rejected with MPML_ERR_TOO_LARGE, n_particles above
 * INT32_MAX with MPML_ERR_ARG.  The CUDA runtime loads the library's device
 * code, and with it places the array, on a device at the first use of the
 * library there -- possibly this call: make that first call (the device
 * current) before an arena claims the device's memory and before any stream
 * capture.  Every call looks up the array's address on the current device.
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other threads) race.  Cost: linear in the particles, plus a
 * quadratic term per centre in the particles of that centre (cheap up to a
 * few thousand per centre; typical scenes hold 8-24).  Synchronises the
 * stream; returns MPML_ERR_OUT_OF_DOMAIN / MPML_ERR_NONFINITE for bad
 * particles (perm is then incomplete). */
#define MPML_NOALLOC_MAX_SLOTS (1 << 21)
int mpml_sort_particles_noalloc(const int n[3], double inv_dx, int precision, const void* x,
                                int64_t n_particles, int32_t* perm, int64_t* keys, void* stream);

#ifdef __cplusplus
}
#endif
#endif
