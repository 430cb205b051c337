/*
 * ofdft.h - C ABI of the GB300 (sm_103a) library for the Augmented Lagrangian
 * formulation of orbital-free DFT (Suryanarayana & Phanish, arXiv:1405.6456).
 *
 * The library finds the electronic ground state u* = sqrt(rho*) of an isolated
 * cluster of M nuclei (Sec. 2, Eq. GroundStateElectronic) on a uniform
 * finite-difference grid with zero Dirichlet values for u and phi (Sec. 4), using
 * the Augmented Lagrangian outer loop of Algorithm 1 around Polak-Ribiere nonlinear
 * CG (Sec. 4), one conjugate-gradient Poisson solve per gradient evaluation
 * (Sec. 4, Eq. Poisson:Discretized), and returns the energy and the forces of
 * Eq. Force:Nuclei.
 *
 * Conventions shared by every call:
 *   - atomic units (bohr, hartree); R is M x 3 row-major, Z has M entries;
 *   - a grid has n[0] x n[1] x n[2] nodes of spacing h; node (i,j,k) sits at
 *     origin + (i+1/2, j+1/2, k+1/2) h; field arrays are x-fastest:
 *     idx = i + n[0]*(j + n[1]*k), no padding;
 *   - fd_order = 2n, n = 1..6 (Eq. FD:Laplacian, radius-n star stencil);
 *   - `prec` (OFDFT_PREC_FP64 or OFDFT_PREC_MIXED) fixes the element type of every
 *     device field buffer a call takes: double for FP64, float for MIXED.  In
 *     MIXED mode stencils, CG vectors and the functional run in FP32 while every
 *     dot product, the constraint, the multipliers, energies and forces are
 *     accumulated in FP64, and Poisson solves end with an FP64 residual
 *     correction;
 *   - device pointers are CUDA device addresses on the context's device, owned
 *     by the caller, at least 256-byte aligned for best speed (any element
 *     alignment is accepted); host pointers are ordinary host memory owned by
 *     the caller;
 *   - calls that return host scalars synchronise the context's stream; others
 *     are asynchronous on it;
 *   - every call returns an ofdft_status; on failure ofdft_last_error(ctx)
 *     describes it.  No C++ exception crosses this interface.  A context is not
 *     safe for concurrent use from several host threads.
 */
#ifndef OFDFT_H
#define OFDFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OFDFT_OK = 0,
  OFDFT_EINVAL = 1,     /* bad argument (sizes, order, null pointer, ...) */
  OFDFT_ENOMEM = 2,     /* device workspace does not fit */
  OFDFT_ENOTCONV = 3,   /* an iteration hit its cap before its tolerance */
  OFDFT_ENONFINITE = 4, /* NaN or Inf in an input or an intermediate scalar */
  OFDFT_ETIMEOUT = 5,   /* a bounded device wait ran out */
  OFDFT_ECUDA = 6       /* a CUDA runtime error */
} ofdft_status;

enum { OFDFT_PREC_FP64 = 0, OFDFT_PREC_MIXED = 1 };

/* energy terms of Eq. F (Sec. 2) */
enum { OFDFT_TERM_TF = 1, OFDFT_TERM_VW = 2, OFDFT_TERM_XC = 4, OFDFT_TERM_ES = 8,
       OFDFT_TERM_ALL = 15 };

/* constraint treatment (Sec. 5.3.2): Algorithm 1 (augmented Lagrangian), the
 * penalty method (Algorithm 1 with eta_q = 0), or the Lagrange-multiplier method
 * (PR nonlinear CG on the sphere h^3 sum u^2 = N with the gradient projected
 * orthogonal to u, eta = G_E.u / (2 u.u), Brent's line search on the angle of
 * the norm-preserving rotation; single solves only: the batch engine rejects it) */
enum { OFDFT_METHOD_AL = 0, OFDFT_METHOD_PENALTY = 1, OFDFT_METHOD_LM = 2 };

/* force expression: Eq. Force:Nuclei with the FD gradient of Sec. 4 (paper), or
 * the exact derivative of the discrete energy at fixed grid (exact). */
enum { OFDFT_FORCE_PAPER = 0, OFDFT_FORCE_EXACT = 1 };

typedef struct ofdft_ctx ofdft_ctx;

typedef struct {
  int n[3];
  double h;
  double origin[3];
} ofdft_grid;

typedef struct {
  int fd_order;       /* 2n: 2, 4, ..., 12 (Sec. 4) */
  int terms;          /* OFDFT_TERM_* mask */
  int method;         /* OFDFT_METHOD_* */
  int precision;      /* OFDFT_PREC_* */
  double lambda;      /* vW weight, 0.2 (Sec. 5) */
  double eta0, mu0, kappa; /* Algorithm 1 inputs: -0.2, 1, 0.1 (Sec. 5.3.1) */
  double sigma, rc;   /* Gaussian nuclei V_J = -Z erf(r/sigma)/r, b_J cut at r_c */
  double guess_sigma, guess_cut; /* Gaussian atomic densities of the starting guess */
  double tol_E;       /* Algorithm 1 stops when |E_{q+1} - E_q| < tol_E * M (Ha/atom) */
  double tol_inner;   /* NLCG stops when h^3 r.s < tol_inner * M (Ha/atom) */
  double tol_poisson; /* CG stops when ||r||_2 <= tol_poisson ||4 pi rho||_2 */
  int max_outer, max_nlcg, max_cg, max_secant;
  double sigma0;      /* secant trial step along the preconditioned direction */
  double eps_secant;  /* secant loop stops when alpha^2 h^3 d.d <= eps_secant^2 N */
  int restart_every;  /* Polak-Ribiere restart period */
  int force_variant;  /* OFDFT_FORCE_* */
  int ezz_correction; /* 1: add the Gaussian-overlap repulsion correction (App. A) */
  double vacuum;      /* box rule of ofdft_grid_for_atoms: vacuum on every side */
  int round_to;       /* box rule: node counts rounded up to a multiple of this */
  int refine_every;   /* MIXED: FP64 residual correction after at most this many FP32 CG steps
                         (sooner once the FP32 residual fell by 1e-4 or to half the tolerance);
                         default 200: much longer FP32 runs let the q = A p recurrence drift */
  double trial_max_rel; /* cap of the trial step: h^3 |sig d|^2 <= trial_max_rel^2 N (0: no cap) */
  int max_backtrack;  /* halvings of the secant step while L does not decrease (0: none) */
  int precond_rank1;  /* 1: the preconditioner also inverts the rank-one term (4h^3/mu) u u^T
                         of the augmented Lagrangian's Hessian exactly (Sherman-Morrison) */
  double poisson_adapt; /* c > 0: inside a solve's NLCG, Poisson solves stop at
                           min(1e-4, max(tol_poisson, c tol_poisson sqrt(rs / (tol_inner M)))),
                           rs = h^3 r.s at the current point: loose while the gradient is
                           large, tol_poisson as the NLCG converges; 0: always tol_poisson */
  double trial_poisson_loosen; /* >= 1: the Poisson solve at a secant trial point (whose gradient only
                                  sets the secant step) stops at this multiple of the current
                                  tolerance, at most 1e-4; 1: the same tolerance as every other solve */
} ofdft_params;

typedef struct {
  int iterations;      /* CG iterations (stencil applications inside the CG) */
  double rel_residual; /* final ||r|| / ||4 pi rho|| */
} ofdft_cg_stats;

typedef struct {
  double L;       /* augmented Lagrangian, Eq. AugLag */
  double E;       /* discrete energy (Eq. F at the computed phi, Sec. 4 quadrature) */
  double E_tf, E_vw, E_xc, E_es, E_self, E_zz_corr;
  double C;       /* C_h(u) = h^3 sum u^2 - N (Sec. 4) */
  double gd;      /* h^3 G.d when d was given */
  double gs_old;  /* h^3 G.s_old when s_old was given */
  double gnorm2;  /* h^3 G.G */
  double rs;      /* h^3 r.s, r = -G, s = r / Jacobi diagonal (NLCG stopping measure) */
  double rs_pc;   /* h^3 r.s with the preconditioner the solver applies (Polak-Ribiere beta) */
  ofdft_cg_stats poisson;
} ofdft_energy;

typedef struct {
  double E, eta, C;   /* E*, eta* (Algorithm 1 output), C_h(u*) */
  ofdft_energy parts; /* terms at u* */
  int outer_iters, nlcg_iters, grad_evals, cg_iters;
  int energy_evals;       /* energy-only evaluations (line searches of OFDFT_METHOD_LM) */
  long long stencil_apps; /* "matrix-vector products" counted as in Sec. 5.3 */
  int converged;
  ofdft_grid grid;    /* grid the solve used */
} ofdft_solve_stats;

/* Fills p with the paper's defaults (Sec. 5) and this library's readings of the
 * knobs the paper leaves open (NLCG constants, Gaussian nuclei, box rule). */
void ofdft_default_params(ofdft_params* p);

/* Creates a context on CUDA device `device` whose work goes to `cuda_stream`
 * (a cudaStream_t; NULL means the legacy default stream).  The context owns its
 * device workspaces; they grow on demand and are freed by ofdft_destroy.
 * The first Poisson solve on a new grid times a few launch shapes of the CG
 * stencil pass and keeps the fastest for the context's lifetime (the shape sets
 * the order of the reductions' partial sums, so two contexts may differ in the
 * last bits); environment variable OFDFT_AUTOTUNE=0 at creation turns this off
 * and keeps the fixed one-wave shape.  Other variables read at creation:
 * OFDFT_PRECOND=0 (plain Poisson CG, as ofdft_set_poisson_precond), OFDFT_MG_OMEGA
 * (multigrid Jacobi weight in (0, 1), default 0.9), OFDFT_MG_SWEEPS (bottom-level
 * sweeps, default 20), OFDFT_COOP=1 (plain CG iterations in one persistent
 * cooperative launch per eight iterations where the grid's blocks fit on the
 * device at once), OFDFT_CG_FOLD_BYTES (bytes of the five CG vectors above which
 * a CG folds its iterate update into the next stencil pass; default 96 MiB),
 * multigrid variants (each gives the same preconditioner up to rounding):
 * OFDFT_MG_ZSTREAM=1 (level smoothing passes as radius-1 z-streaming stencils
 * instead of row-per-warp kernels), OFDFT_MG_FUSE_NODES / OFDFT_MG_FUSE_BELOW
 * (levels of at least / coarser levels of at most this many nodes run smoothing,
 * residual and restriction as one fused pass and prolongation and smoothing as
 * another), OFDFT_MG_CLUSTER=1 (the coarse levels whose z-plane slabs fit and
 * the coarse end in one launch of an 8-block thread-block cluster, in its
 * distributed shared memory), OFDFT_MG_FINEST_SMOOTH=0 (no sweeps on the finest
 * level: r_c = R r, z = s r + P e_c; a different, cheaper preconditioner);
 * OFDFT_FF_RESIDUAL=0 (MIXED: FP64 stencil in the residual pass of each Poisson
 * round instead of the float-float one), OFDFT_COND_GRAPHS=0 (CG chunks of eight
 * iterations polled by the host instead of a device-side loop in a CUDA graph
 * with a conditional node), OFDFT_TMA=1 (FP32 z-streaming passes stage their
 * planes with tiled TMA copies where the tile allows it; results are identical),
 * OFDFT_PDL=1 (CG-loop kernels with programmatic dependent launch; results are
 * identical), OFDFT_FUNC_SPLIT_DOTS=1 (G.d and G.s_old of an evaluation by a pass
 * after the functional instead of inside it), OFDFT_MG_ZSTREAM_NODES (z-streaming
 * smoothing on the levels of at least this many nodes), OFDFT_TRACE=1 (one stderr
 * line per evaluation). */
int ofdft_create(ofdft_ctx** ctx, int device, void* cuda_stream);
int ofdft_destroy(ofdft_ctx* ctx);

/* Preconditioner of the Poisson CG (S3) for every later solve on ctx
 * (ofdft_poisson, ofdft_energy_grad, ofdft_solve and the calls built on them;
 * not the batch engine, which keeps plain CG).  The paper's Krylov solve has
 * none; the choice changes the iteration count, not the solution (phi to the
 * same relative residual).
 *   OFDFT_PRECOND_NONE: plain CG (the oracle's iteration, iteration for
 *     iteration up to rounding).
 *   OFDFT_PRECOND_MG (default): z = M r with M one symmetric V(1,1)-cycle of the
 *     second-order 7-point Laplacian (damped Jacobi, full weighting, trilinear
 *     prolongation, coarse node I on fine node 2I+1, zero Dirichlet values);
 *     grids whose coarsest level would keep more than 4096 nodes (an extent
 *     below 4 with the others large) fall back to plain CG.
 * Returns OFDFT_EINVAL for an unknown kind. */
enum { OFDFT_PRECOND_NONE = 0, OFDFT_PRECOND_MG = 1 };
int ofdft_set_poisson_precond(ofdft_ctx* ctx, int kind);
/* Message describing the last failure on ctx (never NULL; "" after success). */
const char* ofdft_last_error(const ofdft_ctx* ctx);

/* Box rule (host only, Sec. 4): bounding box of R grown by `vacuum` on each side,
 * n_d = ceil(L_d/h) rounded up to a multiple of round_to, nodes cell-centred with
 * the spare length split evenly.  Output grid g. */
int ofdft_grid_for_atoms(const double* R, int M, double h, double vacuum, int round_to,
                         ofdft_grid* g);

/* S2 - out = L_h f, the radius-n star stencil of Sec. 4 Eq. FD:Laplacian with
 * weights w_0 = -(1/h^2) sum 1/q^2 (centre counted six times) and
 * w_p = 2(-1)^{p+1}(n!)^2/(h^2 p^2 (n-p)!(n+p)!), zero at every index outside the
 * grid.  f and out: device arrays of n[0]n[1]n[2] elements of the `prec` type;
 * they must not overlap. */
int ofdft_stencil(ofdft_ctx* ctx, const ofdft_grid* g, int fd_order, int prec, const void* f,
                  void* out);

/* S1 - nuclear pseudocharge b = sum_J b_J with b_J = -(1/4 pi) L_h V_J on nodes
 * within r_c of R_J (Sec. 4, Eq. b:Pseudopotential), V_J = -Z_J erf(r/sigma)/r
 * evaluated analytically at every stencil neighbour, and the self energy
 * E_self = (1/2) sum_J h^3 sum b_J V_J (Eq. ElectroststaticReformulation).
 * R (M x 3) and Z (M) are host arrays; b is a device array of the `prec` type
 * (overwritten); *E_self (host) is computed in FP64. */
int ofdft_pseudocharge(ofdft_ctx* ctx, const ofdft_grid* g, int fd_order, const double* R,
                       const double* Z, int M, double sigma, double rc, int prec, void* b,
                       double* E_self);

/* S1 - starting guess of Sec. 4: sqrt of the superposed Gaussian atomic densities
 * Z_J (2 pi s^2)^{-3/2} exp(-r^2/(2 s^2)) (r < cut), scaled so h^3 sum u^2 = N.
 * u: device array of the `prec` type (overwritten). */
int ofdft_initial_guess(ofdft_ctx* ctx, const ofdft_grid* g, const double* R, const double* Z,
                        int M, double guess_sigma, double guess_cut, double N, int prec,
                        void* u);

/* S3 - Poisson problem of Sec. 4 (Eq. Poisson:Discretized):
 * -(1/4 pi) L_h phi = rho with zero Dirichlet values, written as the SPD system
 * (-L_h) phi = 4 pi rho and solved by conjugate gradients (the paper uses GMRES;
 * both reach the same solution of this SPD system) from the incoming phi (the
 * previous solution, Sec. 4).  rho is the device array `rho` if it is not NULL,
 * otherwise u^2 + b from the device arrays u and b.  Stops when
 * ||r||_2 <= tol ||4 pi rho||_2 or after max_it iterations (then OFDFT_ENOTCONV,
 * phi holds the last iterate).  phi: device array, in: guess, out: solution. */
int ofdft_poisson(ofdft_ctx* ctx, const ofdft_grid* g, int fd_order, int prec, const void* rho,
                  const void* u, const void* b, void* phi, double tol, int max_it,
                  ofdft_cg_stats* st);

/* S3+S4+S5+S6 - one evaluation of the augmented Lagrangian (Eq. AugLag) and its
 * gradient at u (the unit of work of the method):
 *   if solve_poisson, phi is first updated by ofdft_poisson from its incoming
 *   value (tolerance p->tol_poisson); then at that phi
 *   E = h^3 sum [C_F u^{10/3} + eps_xc(u) u^2] - (lambda/2) h^3 u.L_h u
 *       + h^3 sum [phi L_h phi/(8 pi) + (u^2 + b) phi] - E_self   (Eq. F)
 *   C = h^3 sum u^2 - N,  L = E - eta C + C^2/(2 mu)
 *   G = -lambda L_h u + 2 (V_K + V_xc + phi) u + 2 (-eta + C/mu) u
 * G is (1/h^3) dL/du, twice the discrete Euler-Lagrange expression of Sec. 4
 * (Eq. EulerLagrangeDiscretized).  Optional device outputs: grad (G) and s (the
 * preconditioned residual: -G/diag, and with p->precond_rank1 the exact inverse of
 * diag + (4h^3/mu) u u^T applied to -G); optional device inputs d and s_old
 * give out->gd = h^3 G.d and out->gs_old = h^3 G.s_old.  mu = +inf drops the
 * penalty term.  u, b, phi, grad, s, d, s_old: device arrays of the `prec` type
 * (p->precision).  Synchronises; results in *out. */
int ofdft_energy_grad(ofdft_ctx* ctx, const ofdft_grid* g, const ofdft_params* p, const void* u,
                      const void* b, void* phi, double E_self, double eta, double mu, double N,
                      int solve_poisson, void* grad, void* s, const void* d, const void* s_old,
                      ofdft_energy* out);

/* S9 - forces on the nuclei (Eq. Force:Nuclei) at phi:
 *   OFDFT_FORCE_PAPER: f_J = h^3 sum_{|x-R_J|<r_c} grad_h b_J (phi - V_J), grad_h the
 *                      FD gradient of Sec. 4 with weights w~_p;
 *   OFDFT_FORCE_EXACT: f_J = -h^3 sum (db_J/dR_J)(phi - V_J) with
 *                      db_J/dR_J = (1/4 pi) L_h grad V_J (exact derivative of the
 *                      discrete energy at fixed grid).
 * phi: device array of the `prec` type; F: host array M x 3 (output, FP64). */
int ofdft_forces(ofdft_ctx* ctx, const ofdft_grid* g, int fd_order, const double* R,
                 const double* Z, int M, double sigma, double rc, int variant, int prec,
                 const void* phi, double* F);

/* App. A - correction of the repulsive energy and the forces for overlapping
 * pseudocharges, in the paper's general form (Eq. RepulsiveCorrection2 and the
 * force expression after it): reference charges b~_J, Gaussian nuclei of width
 * sigma_ref cut at rc_ref (each of charge Z_J on the grid; their balls must not
 * overlap: every pair of atoms more than 2 rc_ref apart, else OFDFT_EINVAL), beside
 * the method's b_J (sigma, rc); V and V~ from (-1/4 pi) L_h V = b and
 * (-1/4 pi) L_h V~ = b~ (two FP64 Poisson solves to relative residual tol, so
 * V_c = V~ - V), and
 *   E_c = 1/2 h^3 sum (b~ + b) V_c + E_self(b) - E_self(b~),
 *   f_J = h^3 sum grad_h b~_J (V~ - V~_J) - h^3 sum grad_h b_J (V - V_J)
 * (the paper-form force of ofdft_forces at each potential).  Add E_c to the
 * energy and f to the forces of a ground state computed with b.  For Gaussian
 * nuclei E_c tends to sum_{I<J} Z_I Z_J erfc(R_IJ/(sqrt2 sigma))/R_IJ as h -> 0 (the
 * closed form ofdft_params.ezz_correction adds).  E_c: host scalar; F_c: host
 * array M x 3.  Synchronises. */
int ofdft_overlap_correction(ofdft_ctx* ctx, const ofdft_grid* g, int fd_order, const double* R,
                             const double* Z, int M, double sigma, double rc, double sigma_ref,
                             double rc_ref, double tol, double* E_c, double* F_c);

/* S1..S9 - ground state at fixed nuclei (Eq. GroundStateElectronic) by
 * Algorithm 1 (or the penalty method) around PR nonlinear CG with a secant line
 * search, the Jacobi preconditioner and u <- |u| (Sec. 4), then the forces.
 *   grid: the grid to use, or NULL for ofdft_grid_for_atoms(R, M, h, p->vacuum,
 *         p->round_to) (the grid used is returned in st->grid);
 *   u_out, phi_out: optional device arrays (p->precision type) receiving u*, phi*
 *         (they must hold the grid's node count; query it with
 *         ofdft_grid_for_atoms first when grid is NULL);
 *   energy: host scalar E* (Ha); forces: host M x 3 array or NULL; st: stats.
 * Returns OFDFT_ENOTCONV when Algorithm 1 hits p->max_outer (results are still
 * written), OFDFT_ENOMEM when the workspace does not fit on the device. */
int ofdft_solve(ofdft_ctx* ctx, const ofdft_grid* grid, const double* R, const double* Z, int M,
                double h, const ofdft_params* p, void* u_out, void* phi_out, double* energy,
                double* forces, ofdft_solve_stats* st);

/* Warm-started ground state: as ofdft_solve, with the NLCG starting from u_in
 * (device array of p->precision type on `grid`, rescaled to h^3 sum u^2 = N)
 * instead of the Gaussian guess, and the Poisson solves from phi_in instead of
 * zero.  Either may be NULL; grid must be given when either is.  u_in and
 * phi_in may be the same arrays as u_out and phi_out.  Algorithm 1 starts from
 * p->eta0 and p->mu0: to resume from a previous ground state pass its eta* and
 * the last penalty weight (mu0 kappa^(outer_iters - 1)), as ofdft_relax does. */
int ofdft_solve_from(ofdft_ctx* ctx, const ofdft_grid* grid, const double* R, const double* Z, int M, double h,
                     const ofdft_params* p, const void* u_in, const void* phi_in, void* u_out, void* phi_out,
                     double* energy, double* forces, ofdft_solve_stats* st);

typedef struct {
  int steps;          /* geometry steps taken */
  int solves;         /* ground states computed (two or three per step) */
  long long cg_iters; /* Poisson CG iterations over all of them */
  double max_force;   /* largest atomic force norm at the final geometry (Ha/bohr) */
  double energy;      /* E* at the final geometry */
  int converged;      /* 1 once max_force < f_tol */
} ofdft_relax_stats;

/* Geometry relaxation (Sec. 3, the nuclei at the minimum of E over R with the
 * forces of Eq. Force:Nuclei): Polak-Ribiere CG over the 3M coordinates with a
 * secant step on F.d between the current geometry and a trial geometry whose
 * largest atomic move is max_move (bohr), each ground state warm-started from
 * the previous one (ofdft_solve_from) on one fixed grid (the caller's, or the
 * box rule at the starting geometry).  R (host, M x 3) is updated in place;
 * energy and forces (host, M x 3) are those of the final geometry.  Stops when
 * the largest atomic force norm is below f_tol or after max_steps steps
 * (OFDFT_ENOTCONV). */
int ofdft_relax(ofdft_ctx* ctx, const ofdft_grid* grid, double* R, const double* Z, int M, double h,
                const ofdft_params* p, int max_steps, double f_tol, double max_move, double* energy,
                double* forces, ofdft_relax_stats* st);

/* Kernel kinds counted by the context (trace counters). */
enum {
  OFDFT_K_STENCIL = 0,          /* S2 plain stencil */
  OFDFT_K_CG_DIR_STENCIL = 1,   /* S3 CG: p = r + beta p, Ap = -L_h p, p.Ap */
  OFDFT_K_CG_UPDATE = 2,        /* S3 CG: x += alpha p, r -= alpha Ap, r.r */
  OFDFT_K_RESIDUAL = 3,         /* S3/S5/S10 residual 4 pi rho + L_h phi (FP64 in MIXED) */
  OFDFT_K_FUNCTIONAL = 4,       /* S4 fused energy + gradient */
  OFDFT_K_VECTOR = 5,           /* S6/S7 dots, NLCG updates, conversions */
  OFDFT_K_ATOMS = 6,            /* S1/S9 pseudocharge, guess, forces */
  OFDFT_K_CG_PERSISTENT = 7,    /* S3 CG: whole iterations (both halves) in one cooperative launch */
  OFDFT_K_MG = 8,               /* S3 multigrid preconditioner passes */
  OFDFT_K_COUNT = 9
};

typedef struct {
  long long launches;                      /* kernels launched by this context */
  long long kind_launches[OFDFT_K_COUNT];  /* per OFDFT_K_* kind */
  long long timed_launches[OFDFT_K_COUNT]; /* launches bracketed by CUDA events */
  double timed_ms[OFDFT_K_COUNT];          /* summed event durations (ms) */
  long long persistent_cg_iters;           /* CG iterations run by OFDFT_K_CG_PERSISTENT launches */
  long long tma_launches;                  /* z-streaming passes whose planes were staged by TMA */
} ofdft_counters;

/* Tracing (no counterpart in the paper, which reports wall time and counts of
 * matrix-vector products): every launch is counted per kind; launches of the
 * kinds whose bit (1 << OFDFT_K_*) is set in kind_mask are also bracketed by a
 * pair of CUDA events on the context's stream and their durations summed
 * (kind_mask = -1: all kinds, 0: counting only).  Costs two event records per
 * timed launch. */
int ofdft_profile(ofdft_ctx* ctx, int kind_mask);
/* Copies the counters (synchronises the stream first). */
int ofdft_get_counters(ofdft_ctx* ctx, ofdft_counters* out);
int ofdft_reset_counters(ofdft_ctx* ctx);

/* S11/S12 - batched and continuously served ground states.  A batch holds
 * solve requests (the same inputs as ofdft_solve) and advances every admitted
 * solve by one evaluation round per ofdft_batch_step: the rounds of all active
 * solves are packed into shared launches over work lists of tiles of their
 * (uneven) grids, and a solve whose CG has converged leaves the list.  Requests
 * are admitted in submission order between rounds while their workspace
 * (ofdft_batch_bytes) fits in hbm_budget_bytes (a request larger than the budget
 * is admitted alone).  Every solve keeps u, phi, its CG and NLCG vectors and
 * (eta, mu) resident on the device between rounds.  All requests of a batch use
 * `precision`.  Results are identical in method to ofdft_solve: the same
 * Algorithm 1 and nonlinear CG, only the launches are shared. */
typedef struct ofdft_batch ofdft_batch;
int ofdft_batch_create(ofdft_ctx* ctx, int precision, long long hbm_budget_bytes, ofdft_batch** out);
int ofdft_batch_destroy(ofdft_batch* b);
/* Queues a solve; R, Z host arrays (copied), grid as in ofdft_solve (may be NULL).
 * *request_id identifies it in ofdft_batch_poll. */
int ofdft_batch_submit(ofdft_batch* b, const double* R, const double* Z, int M, double h,
                       const ofdft_params* p, const ofdft_grid* grid, int* request_id);
/* One round: admit, advance every active solve to its next evaluation, run the
 * packed work, retire finished solves (forces computed at retirement).
 * Outputs the numbers of active and queued solves. */
int ofdft_batch_step(ofdft_batch* b, int* n_active, int* n_queued);
/* *done = 1 once request_id finished; then energy, forces (M x 3, may be NULL)
 * and stats are written and the request is forgotten.  Returns the solve's
 * status (OFDFT_OK, OFDFT_ENOTCONV, ...). */
int ofdft_batch_poll(ofdft_batch* b, int request_id, int* done, double* energy, double* forces,
                     ofdft_solve_stats* st);
/* Steps until no solve is active or queued. */
int ofdft_batch_run(ofdft_batch* b);
/* Device bytes one batched solve of grid g holds while admitted. */
long long ofdft_batch_bytes(const ofdft_grid* g, int prec);

/* Launch statistics of a batch (no counterpart in the paper).  The CG loop of
 * each Poisson round runs as one CUDA graph launch: a device-side WHILE loop
 * over one iteration of every solve in the round (V-cycles, stencil pass,
 * update, all solves packed into shared launches), captured the first time a
 * set of solves meets and replayed while the set stays the same (it changes on
 * admission and retirement).  The first time a grid shape meets the batch
 * engine of a context, the autotuner times that grid's batched CG stencil pass
 * at 8, 16, 32 and 64 planes per CTA (z-tile depth) and keeps the fastest for
 * that shape (the depth sets the order of the grid's partial sums, so one
 * choice per shape keeps every request's result independent of the mix); the CTA shape
 * itself (32 x 8 threads, 2 rows x 2 columns per thread in FP32, 2 x 1 in FP64)
 * is fixed by the register-blocked kernel. */
typedef struct {
  long long rounds;            /* ofdft_batch_step calls that ran a round */
  long long graph_captures;    /* CG loop graphs captured */
  long long graph_replays;     /* CG loops run as one graph launch */
  long long graph_iterations;  /* CG iterations run inside those graphs (largest per loop, summed) */
  long long eager_iterations;  /* CG iterations launched one by one (one ahead of each graph launch) */
  int z_depth;                 /* planes per CTA of the most recently tuned grid's tiles (each grid shape
                                  is tuned once per context; the depth fixes the order of its sums) */
  int z_tuned;                 /* 1 once the autotuner has chosen a depth */
  int tune_candidates;         /* entries of tune_depth / tune_us from the last tuning */
  int tune_depth[8];
  double tune_us[8];           /* mean duration of the batched CG stencil pass at that depth */
} ofdft_batch_stats;
int ofdft_batch_info(const ofdft_batch* b, ofdft_batch_stats* out);

/* Allocation-free variant of ofdft_poisson (FP64), for callers that cannot
 * allocate device memory: an application whose framework owns every device
 * allocation, or code that must not call cudaMalloc on a latency-critical path.
 * The paper has no counterpart; this is an interface of this library only.
 * It needs no context.  Its CG vectors, reduction scratch and CG scalars live
 * in one file-scope device array of about 6.1 MB that every GPU which loads the
 * library holds until the process exits, so it accepts grids of at most
 * 262144 nodes (64^3) and returns OFDFT_EINVAL beyond that.  The first call on
 * a device sets that device up (the array's device address through
 * cudaGetSymbolAddress, the SM count, the kernels' shared-memory limits), so make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (the reduction counter is cleared at the
 * start of each call): calls that overlap on the GPU, on any stream or from any
 * thread, race and must be serialised by the caller.  rho, phi: device arrays
 * (double) of the grid's node count; phi in: guess, out: solution of
 * (-L_h) phi = 4 pi rho with zero Dirichlet values, as ofdft_poisson.  Work is
 * enqueued on cuda_stream and the call synchronises it. */
int ofdft_poisson_noalloc(const ofdft_grid* g, int fd_order, const double* rho, double* phi,
                          double tol, int max_it, void* cuda_stream, ofdft_cg_stats* st);

/* Device bytes a solve of this grid needs in the context workspace (for
 * admission control by callers that pack several solves on one device). */
long long ofdft_workspace_bytes(const ofdft_grid* g, int fd_order, int prec);

/* Host only (no device work): the multigrid levels the Poisson preconditioner
 * (OFDFT_PRECOND_MG) builds for grid g in precision prec.  *levels = number of
 * levels from g itself down to the bottom (each level halves every extent,
 * n_c = floor(n / 2); coarsening stops once an extent is below 4);
 * dims (nullable, 3 * 24 ints) receives the extents of each level.
 * *coarse_level = first level handled by the one-block coarse kernel (the first
 * with at most 4096 nodes), or -1 when even the bottom level is larger: the CG
 * then runs without preconditioner.  *bytes (nullable) = device bytes of the
 * preconditioner's vectors (0 when it does not apply).  OFDFT_EINVAL for a NULL
 * or empty grid. */
int ofdft_mg_plan(const ofdft_grid* g, int prec, int* levels, int* coarse_level, int* dims, long long* bytes);

/* sizeof of the named ABI struct ("ofdft_grid", "ofdft_params", "ofdft_cg_stats",
 * "ofdft_energy", "ofdft_solve_stats", "ofdft_counters", "ofdft_relax_stats",
 * "ofdft_batch_stats"), or -1 for any other
 * name: lets a binding check its struct layouts against the library's.  Host
 * only, no context needed. */
long long ofdft_struct_bytes(const char* name);

#ifdef __cplusplus
}
#endif
#endif /* OFDFT_H */
