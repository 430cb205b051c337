/*
 * FP64 CPU oracle for the Augmented Lagrangian formulation of orbital-free DFT
 * (Suryanarayana & Phanish, arXiv:1405.6456).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct reference that the
 * GPU library is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Conventions (all atomic units: bohr, hartree):
 *   - uniform grid of n1 x n2 x n3 nodes, spacing h (Sec. 4); node (i,j,k),
 *     0-based, sits at origin + (i+1/2, j+1/2, k+1/2) h, so the cube of side h
 *     around each node tiles the box exactly (the quadrature of Sec. 4);
 *   - arrays are x-fastest: idx = i + n1*(j + n2*k);
 *   - every index outside the grid holds 0 for u and for phi (zero Dirichlet,
 *     Sec. 4);
 *   - fd_n is the stencil radius n; the FD order is 2n.
 */
#ifndef OFDFT_ORACLE_H
#define OFDFT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_N 8

typedef struct {
  int n1, n2, n3;
  double h;
  double origin[3];
} orc_grid;

/* Energy terms switched on in the functional (the TFW family of Sec. 2). */
enum { ORC_TF = 1, ORC_VW = 2, ORC_XC = 4, ORC_ES = 8, ORC_ALL = 15 };
/* Constraint treatment (Sec. 5.3.2): Augmented Lagrangian, penalty, Lagrange multiplier. */
enum { ORC_AL = 0, ORC_PENALTY = 1, ORC_LM = 2 };

typedef struct {
  int fd_n;            /* stencil radius n (order 2n) */
  int terms;           /* ORC_TF|ORC_VW|ORC_XC|ORC_ES */
  double lambda;       /* von Weizsaecker weight, 0.2 in Sec. 5 */
  double eta0, mu0, kappa; /* Algorithm 1 inputs */
  int method;          /* ORC_AL, ORC_PENALTY, ORC_LM */
  double tol_E;        /* stop when |E_{q+1}-E_q| < tol_E (Ha, whole system) */
  double tol_inner;    /* NLCG stops when h^3 r.s < tol_inner (Ha) */
  double tol_poisson;  /* CG stops when ||r|| <= tol_poisson ||rhs|| */
  int max_outer, max_nlcg, max_cg, max_secant;
  double sigma0;       /* secant trial step along the preconditioned direction */
  double eps_secant;   /* secant loop stops when alpha^2 d.d <= eps_secant^2 */
  int restart_every;   /* PR restart period */
  /* pseudocharge model: Gaussian nuclei V_J = -Z erf(r/sigma)/r, cut at r_c */
  double sigma, rc;
  double guess_sigma, guess_cut; /* initial guess: Gaussian atoms, width, cutoff */
  int ezz_correction;  /* add the Gaussian-overlap repulsion correction (App. A) */
  double trial_max_rel; /* trial step capped to h^3 |sig d|^2 <= trial_max_rel^2 N (0: no cap) */
  int max_backtrack;   /* halvings of the secant step while L does not decrease */
  int precond_rank1;   /* also invert the rank-one term (4 h^3/mu) u u^T of the Hessian exactly */
} orc_params;

typedef struct {
  double L;        /* augmented Lagrangian value, Eq. AugLag */
  double E;        /* discrete energy E_h (Eq. F at the computed phi) */
  double E_tf, E_vw, E_xc, E_es, E_self, E_zz_corr;
  double C;        /* C_h(u) = h^3 sum u^2 - N */
  double gnorm2;   /* h^3 sum G^2 */
  double rs;       /* h^3 r.s with r = -G, s = r/M (Jacobi diagonal alone): stopping measure */
  double rs_pc;    /* h^3 r.s with s the preconditioned residual actually used (PR beta) */
  int cg_iters;
  double cg_relres;
} orc_energy;

typedef struct {
  double E, eta, C;
  orc_energy parts;
  int outer_iters, nlcg_iters, grad_evals, energy_evals, cg_iters;
  long long stencil_apps;
  int converged;
} orc_result;

/* OpenMP threads used by the grid-sized loops (no effect without OpenMP). */
void orc_set_threads(int n);
int orc_get_threads(void);
void orc_default_params(orc_params* p);
int orc_lap_weights(int n, double h, double* w);
int orc_grad_weights(int n, double h, double* wt);
void orc_laplacian(const orc_grid* g, int n, const double* f, double* out);
void orc_xc(double u, double* eps_xc, double* v_xc);
int orc_grid_for_atoms(const double* R, int M, double h, double vacuum, int round_to, orc_grid* g);
double orc_gauss_potential(double Z, double sigma, double r);
void orc_pseudocharge(const orc_grid* g, int n, const double* R, const double* Z, int M,
                      double sigma, double rc, double* b, double* E_self);
void orc_initial_guess(const orc_grid* g, const double* R, const double* Z, int M,
                       double gsigma, double gcut, double N, double* u);
int orc_poisson(const orc_grid* g, int n, const double* rho, double* phi, double tol,
                int max_it, double* relres);
void orc_functional(const orc_grid* g, const orc_params* p, const double* u, const double* b,
                    const double* phi, double E_self, double eta, double mu, double N,
                    double* G, double* s, orc_energy* out);
int orc_energy_grad(const orc_grid* g, const orc_params* p, const double* u, const double* b,
                    double* phi, double E_self, double eta, double mu, double N, double* G,
                    double* s, orc_energy* out);
int orc_solve(const orc_grid* g, const orc_params* p, const double* R, const double* Z, int M,
              double* u, double* phi, double* b, orc_result* res);
void orc_forces(const orc_grid* g, int n, const double* R, const double* Z, int M, double sigma,
                double rc, const double* phi, int exact_variant, double* F);
double orc_ezz_correction(const double* R, const double* Z, int M, double sigma, double* F);

#ifdef __cplusplus
}
#endif
#endif
