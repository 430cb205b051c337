/*
 * FP64 CPU oracle for the Augmented Lagrangian formulation of orbital-free DFT
 * (Suryanarayana & Phanish, arXiv:1405.6456).  TEST INFRASTRUCTURE ONLY: see
 * ofdft_oracle.h.  Plain loops, FP64 throughout, no blocking or fusion beyond
 * what the paper's definitions state.  Shares nothing with the CUDA library.
 *
 * Readings of points the paper leaves open (each is stated where used):
 *   R1 node placement: cell-centred nodes, zeros at every index outside the grid;
 *   R2 discrete energy: Eq. F of Sec. 2 with integrals replaced by the h^3 sum of
 *      Sec. 4, |grad u|^2 by -u.L_h u and -|grad phi|^2 by phi.L_h phi
 *      (summation by parts under zero Dirichlet values);
 *   R3 gradient: G = (1/h^3) dL_h/du, which is twice the discrete Euler-Lagrange
 *      expression of Sec. 4 (Eq. EulerLagrangeDiscretized); same zero set;
 *   R4 Jacobi preconditioner: the diagonal of dG/du with the nonlocal Hartree and
 *      the rank-one constraint parts left out, floored to stay positive (optionally
 *      with the rank-one part inverted exactly, Sherman-Morrison);
 *   R5 secant line search and Polak-Ribiere update as in the reference the paper
 *      names for them (Shewchuk 1994), with |u| taken after every update (Sec. 4);
 *      the trial step is sigma0 along d, capped so that its RMS size is at most
 *      trial_max_rel times that of u, and a secant step that does not lower L is
 *      halved up to max_backtrack times;
 *   R6 pseudocharge: Gaussian nuclei V_J = -Z erf(r/sigma)/r (the paper's GNH
 *      parameters are not given), b_J from Eq. b_J of Sec. 4 inside r < r_c;
 *   R7 initial guess: superposed Gaussian atomic densities (isolated-atom
 *      densities are not given), rescaled to h^3 sum u^2 = N;
 *   R8 XC density floor: eps_xc = V_xc = 0 where u^2 < 1e-30.
 */
#include "ofdft_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Threads: the grid-sized loops below are split over OpenMP threads when the
 * library is built with OpenMP.  Every sum over the grid is taken in ORC_NCH
 * fixed contiguous chunks whose partial sums are added in chunk order, so
 * results do not depend on the number of threads. */
#define ORC_NCH 256

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static long chunk_lo(long G, int c) { return G * c / ORC_NCH; }

static double fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}

void orc_default_params(orc_params* p) {
  memset(p, 0, sizeof(*p));
  p->fd_n = 6;
  p->terms = ORC_ALL;
  p->lambda = 0.2;     /* Sec. 5 */
  p->eta0 = -0.2;      /* Sec. 5.3.1 */
  p->mu0 = 1.0;
  p->kappa = 0.1;
  p->method = ORC_AL;
  p->tol_E = 1e-6;
  p->tol_inner = 1e-9;
  p->tol_poisson = 1e-11;
  p->max_outer = 30;
  p->max_nlcg = 2000;
  p->max_cg = 20000;
  p->max_secant = 1;
  p->sigma0 = 0.5;
  p->eps_secant = 1e-7;
  p->restart_every = 20;
  p->sigma = 1.0;
  p->rc = 7.0;
  p->guess_sigma = 2.0;
  p->guess_cut = 8.0;
  p->ezz_correction = 0;
  p->trial_max_rel = 0.2;
  p->max_backtrack = 2;
  p->precond_rank1 = 1;
}

/* Laplacian weights of Sec. 4, Eq. FD:Laplacian: w_0 = -(1/h^2) sum_{q=1}^n 1/q^2,
 * w_p = 2(-1)^{p+1} (n!)^2 / (h^2 p^2 (n-p)! (n+p)!).  The p = 0 term of the
 * stencil sums f at the centre six times, so the centre coefficient is 6 w_0. */
int orc_lap_weights(int n, double h, double* w) {
  if (n < 1 || n > ORC_MAX_N || !(h > 0)) return -1;
  double s = 0.0;
  for (int q = 1; q <= n; ++q) s += 1.0 / ((double)q * q);
  w[0] = -s / (h * h);
  double nf2 = fact(n) * fact(n);
  for (int p = 1; p <= n; ++p) {
    double sign = (p % 2 == 1) ? 1.0 : -1.0;
    w[p] = 2.0 * sign * nf2 / (h * h * (double)p * p * fact(n - p) * fact(n + p));
  }
  return 0;
}

/* Gradient weights of Sec. 4: w~_p = (-1)^{p+1} (n!)^2 / (h p (n-p)! (n+p)!). */
int orc_grad_weights(int n, double h, double* wt) {
  if (n < 1 || n > ORC_MAX_N || !(h > 0)) return -1;
  wt[0] = 0.0;
  double nf2 = fact(n) * fact(n);
  for (int p = 1; p <= n; ++p) {
    double sign = (p % 2 == 1) ? 1.0 : -1.0;
    wt[p] = sign * nf2 / (h * (double)p * fact(n - p) * fact(n + p));
  }
  return 0;
}

/* Radius-n star stencil of Eq. FD:Laplacian with zero Dirichlet values (Sec. 4):
 * the field is copied into a zero-padded box so every out-of-grid index reads 0. */
void orc_laplacian(const orc_grid* g, int n, const double* f, double* out) {
  double w[ORC_MAX_N + 1];
  orc_lap_weights(n, g->h, w);
  const int n1 = g->n1, n2 = g->n2, n3 = g->n3;
  const long P1 = n1 + 2 * n, P2 = n2 + 2 * n, P3 = n3 + 2 * n;
  double* fp = (double*)calloc((size_t)(P1 * P2 * P3), sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 0; k < n3; ++k)
    for (int j = 0; j < n2; ++j)
      for (int i = 0; i < n1; ++i)
        fp[(i + n) + P1 * ((j + n) + P2 * (long)(k + n))] = f[i + (long)n1 * (j + (long)n2 * k)];
  const long sy = P1, sz = P1 * P2;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < n3; ++k)
    for (int j = 0; j < n2; ++j)
      for (int i = 0; i < n1; ++i) {
        const long c = (i + n) + P1 * ((j + n) + P2 * (long)(k + n));
        double acc = 6.0 * w[0] * fp[c];
        for (int p = 1; p <= n; ++p)
          acc += w[p] * (fp[c + p] + fp[c - p] + fp[c + p * sy] + fp[c - p * sy] +
                         fp[c + p * sz] + fp[c - p * sz]);
        out[i + (long)n1 * (j + (long)n2 * k)] = acc;
      }
  free(fp);
}

/* LDA exchange-correlation per particle and potential, Ceperley-Alder form with
 * the constants of Sec. 2 (eps_x, eps_c) and Sec. 3 (V_x, V_c); r_s = (3/(4 pi u^2))^{1/3}. */
void orc_xc(double u, double* eps_xc, double* v_xc) {
  const double rho = u * u;
  if (rho < 1e-30) { /* R8 */
    *eps_xc = 0.0;
    *v_xc = 0.0;
    return;
  }
  const double g1 = -0.1423, b1 = 1.0529, b2 = 0.3334;
  const double A1 = 0.0311, B1 = -0.048, C1 = 0.002, D1 = -0.0116;
  const double u23 = cbrt(rho); /* u^{2/3} */
  const double c3pi = cbrt(3.0 / M_PI);
  const double ex = -0.75 * c3pi * u23;
  const double vx = -c3pi * u23;
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  double ec, vc;
  if (rs >= 1.0) {
    const double srs = sqrt(rs);
    const double den = 1.0 + b1 * srs + b2 * rs;
    ec = g1 / den;
    vc = (g1 + (7.0 / 6.0) * g1 * b1 * srs + (4.0 / 3.0) * g1 * b2 * rs) / (den * den);
  } else {
    const double lr = log(rs);
    ec = A1 * lr + B1 + C1 * rs * lr + D1 * rs;
    vc = (A1 + (2.0 / 3.0) * C1 * rs) * lr + (B1 - A1 / 3.0) + (1.0 / 3.0) * (2.0 * D1 - C1) * rs;
  }
  *eps_xc = ex + ec;
  *v_xc = vx + vc;
}

/* Box rule: bounding box of the atoms plus `vacuum` on every side, n_d = ceil(L_d/h)
 * rounded up to a multiple of round_to, extra length split evenly (R1). */
int orc_grid_for_atoms(const double* R, int M, double h, double vacuum, int round_to, orc_grid* g) {
  if (M < 1 || !(h > 0) || round_to < 1) return -1;
  int nd[3];
  for (int d = 0; d < 3; ++d) {
    double lo = R[d], hi = R[d];
    for (int J = 1; J < M; ++J) {
      if (R[3 * J + d] < lo) lo = R[3 * J + d];
      if (R[3 * J + d] > hi) hi = R[3 * J + d];
    }
    lo -= vacuum;
    hi += vacuum;
    const double L = hi - lo;
    int n = (int)ceil(L / h - 1e-9);
    if (n < 1) n = 1;
    n = ((n + round_to - 1) / round_to) * round_to;
    nd[d] = n;
    g->origin[d] = lo - 0.5 * (n * h - L);
  }
  g->n1 = nd[0];
  g->n2 = nd[1];
  g->n3 = nd[2];
  g->h = h;
  return 0;
}

/* Gaussian-nucleus potential V(r) = -Z erf(r/sigma)/r, with its r -> 0 limit (R6). */
double orc_gauss_potential(double Z, double sigma, double r) {
  if (r < 1e-12 * sigma) return -2.0 * Z / (sigma * sqrt(M_PI));
  return -Z * erf(r / sigma) / r;
}

static double node_coord(const orc_grid* g, int d, long i) { return g->origin[d] + ((double)i + 0.5) * g->h; }

/* Integer box of lattice nodes that can lie within radius r of point x (per axis). */
static void ball_range(const orc_grid* g, const double* x, double r, long lo[3], long hi[3]) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = (long)floor((x[d] - r - g->origin[d]) / g->h - 0.5) - 1;
    hi[d] = (long)ceil((x[d] + r - g->origin[d]) / g->h - 0.5) + 1;
  }
}

/* Tabulated b_J on the lattice box [lo-pad, hi+pad] (nodes inside or outside the
 * grid): b_J = -(1/4 pi) L_h V_J at nodes with |x - R_J| < r_c, 0 elsewhere (Sec. 4,
 * Eq. b_J; V_J analytic at every stencil neighbour). */
typedef struct {
  long lo[3], dim[3];
  double* v; /* V_J on the box extended by n more nodes */
  double* b; /* b_J on the box */
  long vlo[3], vdim[3];
} atom_box;

static void atom_box_build(const orc_grid* g, int n, const double* RJ, double ZJ, double sigma,
                           double rc, long pad, atom_box* ab) {
  long lo[3], hi[3];
  ball_range(g, RJ, rc, lo, hi);
  for (int d = 0; d < 3; ++d) {
    ab->lo[d] = lo[d] - pad;
    ab->dim[d] = hi[d] - lo[d] + 1 + 2 * pad;
    ab->vlo[d] = ab->lo[d] - n;
    ab->vdim[d] = ab->dim[d] + 2 * n;
  }
  const long VV = ab->vdim[0] * ab->vdim[1] * ab->vdim[2];
  ab->v = (double*)malloc(sizeof(double) * VV);
  for (long c = 0; c < ab->vdim[2]; ++c)
    for (long b = 0; b < ab->vdim[1]; ++b)
      for (long a = 0; a < ab->vdim[0]; ++a) {
        const double dx = node_coord(g, 0, ab->vlo[0] + a) - RJ[0];
        const double dy = node_coord(g, 1, ab->vlo[1] + b) - RJ[1];
        const double dz = node_coord(g, 2, ab->vlo[2] + c) - RJ[2];
        ab->v[a + ab->vdim[0] * (b + ab->vdim[1] * c)] =
            orc_gauss_potential(ZJ, sigma, sqrt(dx * dx + dy * dy + dz * dz));
      }
  double w[ORC_MAX_N + 1];
  orc_lap_weights(n, g->h, w);
  const long BB = ab->dim[0] * ab->dim[1] * ab->dim[2];
  ab->b = (double*)malloc(sizeof(double) * BB);
  const long sy = ab->vdim[0], sz = ab->vdim[0] * ab->vdim[1];
  for (long c = 0; c < ab->dim[2]; ++c)
    for (long b = 0; b < ab->dim[1]; ++b)
      for (long a = 0; a < ab->dim[0]; ++a) {
        const double dx = node_coord(g, 0, ab->lo[0] + a) - RJ[0];
        const double dy = node_coord(g, 1, ab->lo[1] + b) - RJ[1];
        const double dz = node_coord(g, 2, ab->lo[2] + c) - RJ[2];
        double val = 0.0;
        if (sqrt(dx * dx + dy * dy + dz * dz) < rc) {
          const long vc = (a + n) + sy * (b + n) + sz * (c + n);
          double acc = 6.0 * w[0] * ab->v[vc];
          for (int p = 1; p <= n; ++p)
            acc += w[p] * (ab->v[vc + p] + ab->v[vc - p] + ab->v[vc + p * sy] + ab->v[vc - p * sy] +
                           ab->v[vc + p * sz] + ab->v[vc - p * sz]);
          val = -acc / (4.0 * M_PI);
        }
        ab->b[a + ab->dim[0] * (b + ab->dim[1] * c)] = val;
      }
}

static void atom_box_free(atom_box* ab) {
  free(ab->v);
  free(ab->b);
}

static double ab_v(const atom_box* ab, long i, long j, long k) {
  return ab->v[(i - ab->vlo[0]) + ab->vdim[0] * ((j - ab->vlo[1]) + ab->vdim[1] * (k - ab->vlo[2]))];
}
static double ab_b(const atom_box* ab, long i, long j, long k) {
  if (i < ab->lo[0] || j < ab->lo[1] || k < ab->lo[2] || i >= ab->lo[0] + ab->dim[0] ||
      j >= ab->lo[1] + ab->dim[1] || k >= ab->lo[2] + ab->dim[2])
    return 0.0;
  return ab->b[(i - ab->lo[0]) + ab->dim[0] * ((j - ab->lo[1]) + ab->dim[1] * (k - ab->lo[2]))];
}

/* b = sum_J b_J on the grid (Sec. 4) and the self energy E_self = (1/2) sum_J h^3
 * sum b_J V_J (last term of Eq. ElectroststaticReformulation). */
void orc_pseudocharge(const orc_grid* g, int n, const double* R, const double* Z, int M,
                      double sigma, double rc, double* b, double* E_self) {
  const long G = (long)g->n1 * g->n2 * g->n3;
  const double h3 = g->h * g->h * g->h;
  memset(b, 0, sizeof(double) * G);
  double es = 0.0;
  /* the atoms' tables are built in parallel in groups; their contributions are
     added to b in atom order */
  enum { GROUP = 32 };
  atom_box boxes[GROUP];
  for (int J0 = 0; J0 < M; J0 += GROUP) {
    const int nj = (M - J0 < GROUP) ? M - J0 : GROUP;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nj; ++t) atom_box_build(g, n, R + 3 * (J0 + t), Z[J0 + t], sigma, rc, 0, &boxes[t]);
    for (int t = 0; t < nj; ++t) {
      atom_box* ab = &boxes[t];
      for (long c = 0; c < ab->dim[2]; ++c)
        for (long bb = 0; bb < ab->dim[1]; ++bb)
          for (long a = 0; a < ab->dim[0]; ++a) {
            const long i = ab->lo[0] + a, j = ab->lo[1] + bb, k = ab->lo[2] + c;
            if (i < 0 || j < 0 || k < 0 || i >= g->n1 || j >= g->n2 || k >= g->n3) continue;
            const double bj = ab_b(ab, i, j, k);
            if (bj == 0.0) continue;
            b[i + (long)g->n1 * (j + (long)g->n2 * k)] += bj;
            es += 0.5 * h3 * bj * ab_v(ab, i, j, k);
          }
      atom_box_free(ab);
    }
  }
  *E_self = es;
}

/* Starting guess (Sec. 4): superposed atomic densities projected inside a ball;
 * R7: rho_J = Z_J (2 pi s^2)^{-3/2} exp(-r^2/(2 s^2)) for r < cut; u_0 = sqrt(rho_0)
 * rescaled so that h^3 sum u_0^2 = N. */
void orc_initial_guess(const orc_grid* g, const double* R, const double* Z, int M,
                       double gsigma, double gcut, double N, double* u) {
  const long G = (long)g->n1 * g->n2 * g->n3;
  const double h3 = g->h * g->h * g->h;
  double* rho = (double*)calloc(G, sizeof(double));
  const double norm = pow(2.0 * M_PI * gsigma * gsigma, -1.5);
  for (int J = 0; J < M; ++J) {
    long lo[3], hi[3];
    ball_range(g, R + 3 * J, gcut, lo, hi);
    for (long k = lo[2]; k <= hi[2]; ++k)
      for (long j = lo[1]; j <= hi[1]; ++j)
        for (long i = lo[0]; i <= hi[0]; ++i) {
          if (i < 0 || j < 0 || k < 0 || i >= g->n1 || j >= g->n2 || k >= g->n3) continue;
          const double dx = node_coord(g, 0, i) - R[3 * J];
          const double dy = node_coord(g, 1, j) - R[3 * J + 1];
          const double dz = node_coord(g, 2, k) - R[3 * J + 2];
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < gcut * gcut) rho[i + g->n1 * (j + (long)g->n2 * k)] += Z[J] * norm * exp(-r2 / (2.0 * gsigma * gsigma));
        }
  }
  double s = 0.0;
  for (long x = 0; x < G; ++x) s += rho[x];
  const double scale = (s > 0.0) ? sqrt(N / (h3 * s)) : 0.0;
  for (long x = 0; x < G; ++x) u[x] = scale * sqrt(rho[x]);
  free(rho);
}

static double dot(const double* a, const double* b, long G) {
  double part[ORC_NCH];
#pragma omp parallel for schedule(static)
  for (int c = 0; c < ORC_NCH; ++c) {
    double s = 0.0;
    for (long x = chunk_lo(G, c); x < chunk_lo(G, c + 1); ++x) s += a[x] * b[x];
    part[c] = s;
  }
  double s = 0.0;
  for (int c = 0; c < ORC_NCH; ++c) s += part[c];
  return s;
}

/* Discrete Poisson problem of Sec. 4 (Eq. Poisson:Discretized), written as the SPD
 * system (-L_h) phi = 4 pi rho, solved by plain conjugate gradients from the
 * incoming phi (the previous solution, Sec. 4).  The paper uses GMRES; on this SPD
 * system both reach the same solution.  Stops when ||r||_2 <= tol ||4 pi rho||_2.
 * Returns the iteration count; *relres gets the final recursive relative residual. */
int orc_poisson(const orc_grid* g, int n, const double* rho, double* phi, double tol,
                int max_it, double* relres) {
  const long G = (long)g->n1 * g->n2 * g->n3;
  double* r = (double*)malloc(sizeof(double) * G);
  double* p = (double*)malloc(sizeof(double) * G);
  double* Ap = (double*)malloc(sizeof(double) * G);
  orc_laplacian(g, n, phi, Ap);
  double part[ORC_NCH];
#pragma omp parallel for schedule(static)
  for (int c = 0; c < ORC_NCH; ++c) {
    double s = 0.0;
    for (long x = chunk_lo(G, c); x < chunk_lo(G, c + 1); ++x) {
      const double rhs = 4.0 * M_PI * rho[x];
      r[x] = rhs + Ap[x]; /* rhs - (-L phi) */
      p[x] = r[x];
      s += rhs * rhs;
    }
    part[c] = s;
  }
  double bb = 0.0;
  for (int c = 0; c < ORC_NCH; ++c) bb += part[c];
  const double bnorm = sqrt(bb) > 0.0 ? sqrt(bb) : 1.0;
  double rr = dot(r, r, G);
  int it = 0;
  while (it < max_it && sqrt(rr) > tol * bnorm) {
    orc_laplacian(g, n, p, Ap);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < G; ++x) Ap[x] = -Ap[x];
    const double pAp = dot(p, Ap, G);
    const double alpha = rr / pAp;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < G; ++x) {
      phi[x] += alpha * p[x];
      r[x] -= alpha * Ap[x];
    }
    const double rr_new = dot(r, r, G);
    const double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < G; ++x) p[x] = r[x] + beta * p[x];
    rr = rr_new;
    ++it;
  }
  if (relres) *relres = sqrt(rr) / bnorm;
  free(r);
  free(p);
  free(Ap);
  return it;
}

/* The discrete functional and its gradient at fixed phi (R2, R3, R4).
 *   E_tf = h^3 sum C_F u^{10/3}                       (Eq. KineticEnergy)
 *   E_vw = -(lambda/2) h^3 sum u L_h u                (Eq. KineticEnergy, by parts)
 *   E_xc = h^3 sum eps_xc(u) u^2                      (Eq. E_xc)
 *   E_es = h^3 sum [ phi L_h phi / (8 pi) + (u^2 + b) phi ] - E_self   (Eq. F)
 *   C    = h^3 sum u^2 - N                            (Sec. 4, C_h)
 *   L    = E - eta C + C^2 / (2 mu)                   (Eq. AugLag)
 *   G    = -lambda L_h u + 2 (V_K + V_xc + phi) u + 2 (-eta + C/mu) u
 * with V_K = (5/3) C_F u^{4/3} (Sec. 3).  mu = +inf drops the penalty term.
 * If s != NULL it receives s = -G / Mdiag (Jacobi-preconditioned residual). */
void orc_functional(const orc_grid* g, const orc_params* p, const double* u, const double* b,
                    const double* phi, double E_self, double eta, double mu, double N,
                    double* G, double* s, orc_energy* out) {
  const long NG = (long)g->n1 * g->n2 * g->n3;
  const double h3 = g->h * g->h * g->h;
  const double CF = 0.3 * pow(3.0 * M_PI * M_PI, 2.0 / 3.0);
  const int tf = p->terms & ORC_TF, vw = p->terms & ORC_VW, xc = p->terms & ORC_XC,
            es = p->terms & ORC_ES;
  double w[ORC_MAX_N + 1];
  orc_lap_weights(p->fd_n, g->h, w);
  double* Lu = (double*)malloc(sizeof(double) * NG);
  double* Lphi = (double*)malloc(sizeof(double) * NG);
  orc_laplacian(g, p->fd_n, u, Lu);
  if (es) orc_laplacian(g, p->fd_n, phi, Lphi);
  /* per-chunk partial sums, added in chunk order below:
     tf, vw, xc, es, G.G, G.G/diag, u.s, u.u/diag */
  enum { NS = 8 };
  double part[ORC_NCH][NS];
  const double s_uu = dot(u, u, NG);
  const double C = h3 * s_uu - N;
  const double inv_mu = 1.0 / mu;
  const double mult = -eta + C * inv_mu;
  double* winv = (p->precond_rank1 && s) ? (double*)malloc(sizeof(double) * NG) : NULL;
#pragma omp parallel for schedule(static)
  for (int c = 0; c < ORC_NCH; ++c) {
    double s_tf = 0, s_vw = 0, s_xc = 0, s_es = 0, g2 = 0.0, rs = 0.0, us = 0.0, uwu = 0.0;
    for (long x = chunk_lo(NG, c); x < chunk_lo(NG, c + 1); ++x) {
      const double ux = fabs(u[x]);
      double e_xc = 0.0, v_xc = 0.0;
      if (xc) orc_xc(ux, &e_xc, &v_xc);
      const double u43 = pow(ux, 4.0 / 3.0);
      const double vk = tf ? (5.0 / 3.0) * CF * u43 : 0.0;
      if (tf) s_tf += CF * u43 * ux * ux;
      if (vw) s_vw += u[x] * Lu[x];
      if (xc) s_xc += e_xc * ux * ux;
      double ph = 0.0;
      if (es) {
        ph = phi[x];
        s_es += ph * Lphi[x] / (8.0 * M_PI) + (u[x] * u[x] + b[x]) * ph;
      }
      const double gx = (vw ? -p->lambda * Lu[x] : 0.0) + 2.0 * (vk + v_xc + ph) * u[x] + 2.0 * mult * u[x];
      const double kin = (vw ? -6.0 * p->lambda * w[0] : 0.0) + (14.0 / 3.0) * vk;
      double md = kin + 2.0 * (v_xc + ph + mult);
      if (md < 0.25 * kin) md = 0.25 * kin;
      if (md < 1e-10) md = 1e-10;
      if (G) G[x] = gx;
      if (s) s[x] = -gx / md;
      if (winv) winv[x] = u[x] / md;
      g2 += gx * gx;
      rs += gx * gx / md;
      us += u[x] * (-gx / md);
      uwu += u[x] * u[x] / md;
    }
    part[c][0] = s_tf;
    part[c][1] = s_vw;
    part[c][2] = s_xc;
    part[c][3] = s_es;
    part[c][4] = g2;
    part[c][5] = rs;
    part[c][6] = us;
    part[c][7] = uwu;
  }
  double s_tf = 0, s_vw = 0, s_xc = 0, s_es = 0, g2 = 0.0, rs = 0.0, us = 0.0, uwu = 0.0;
  for (int c = 0; c < ORC_NCH; ++c) {
    s_tf += part[c][0];
    s_vw += part[c][1];
    s_xc += part[c][2];
    s_es += part[c][3];
    g2 += part[c][4];
    rs += part[c][5];
    us += part[c][6];
    uwu += part[c][7];
  }
  double rs_pc = rs;
  if (winv && s) {
    /* rank-one term (4 h^3/mu) u u^T of dG/du inverted exactly (Sherman-Morrison) */
    const double cpen = 4.0 * h3 * inv_mu;
    const double gamma = cpen * us / (1.0 + cpen * uwu);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < NG; ++x) s[x] -= gamma * winv[x];
    rs_pc -= gamma * us;
  }
  free(winv);
  out->E_tf = h3 * s_tf;
  out->E_vw = -0.5 * p->lambda * h3 * s_vw;
  out->E_xc = h3 * s_xc;
  out->E_self = es ? E_self : 0.0;
  out->E_es = es ? h3 * s_es - E_self : 0.0;
  out->E = out->E_tf + out->E_vw + out->E_xc + out->E_es + out->E_zz_corr;
  out->C = C;
  out->L = out->E - eta * C + 0.5 * C * C * inv_mu;
  out->gnorm2 = h3 * g2;
  out->rs = h3 * rs;
  out->rs_pc = h3 * rs_pc;
  free(Lu);
  free(Lphi);
}

/* One evaluation of the augmented Lagrangian and its gradient: a Poisson solve for
 * phi at the current u, warm-started from the incoming phi (Sec. 4), then the
 * functional.  Returns the CG iteration count (-1 if the CG did not converge). */
int orc_energy_grad(const orc_grid* g, const orc_params* p, const double* u, const double* b,
                    double* phi, double E_self, double eta, double mu, double N, double* G,
                    double* s, orc_energy* out) {
  const long NG = (long)g->n1 * g->n2 * g->n3;
  int it = 0;
  double rel = 0.0;
  double ezz = out->E_zz_corr;
  if (p->terms & ORC_ES) {
    double* rho = (double*)malloc(sizeof(double) * NG);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < NG; ++x) rho[x] = u[x] * u[x] + b[x];
    it = orc_poisson(g, p->fd_n, rho, phi, p->tol_poisson, p->max_cg, &rel);
    free(rho);
  }
  memset(out, 0, sizeof(*out));
  out->E_zz_corr = ezz;
  orc_functional(g, p, u, b, phi, E_self, eta, mu, N, G, s, out);
  out->cg_iters = it;
  out->cg_relres = rel;
  return (rel <= p->tol_poisson) ? it : -1;
}

/* ---------------------------------------------------------------------------
 * Solver state shared by the constrained minimisers.
 * ------------------------------------------------------------------------- */
typedef struct {
  const orc_grid* g;
  const orc_params* p;
  const double* b;
  double E_self, N, ezz;
  double *u, *phi, *G, *s;
  orc_energy e;
  orc_result* res;
  long NG;
  double h3;
} solver;

static void sv_eval(solver* S, const double* u, double eta, double mu) {
  S->e.E_zz_corr = S->ezz;
  orc_energy_grad(S->g, S->p, u, S->b, S->phi, S->E_self, eta, mu, S->N, S->G, S->s, &S->e);
  S->res->grad_evals++;
  S->res->cg_iters += S->e.cg_iters;
  S->res->stencil_apps += S->e.cg_iters + 1 + 2;
}

/* Polak-Ribiere nonlinear CG with a secant line search and the Jacobi
 * preconditioner (Sec. 4, R5), u <- |u| after every update, minimising
 * L(u, eta, mu) from the incoming u.  Returns 1 when h^3 r.s < tol_inner. */
static int nlcg(solver* S, double eta, double mu) {
  const orc_params* p = S->p;
  const long NG = S->NG;
  const double h3 = S->h3;
  double* d = (double*)malloc(sizeof(double) * NG);
  double* s_old = (double*)malloc(sizeof(double) * NG);
  double* ut = (double*)malloc(sizeof(double) * NG);
  double* Gt = (double*)malloc(sizeof(double) * NG);
  double* st = (double*)malloc(sizeof(double) * NG);
  int converged = 0;
  sv_eval(S, S->u, eta, mu);
  memcpy(d, S->s, sizeof(double) * NG);
  double delta_new = S->e.rs_pc;
  int k = 0;
  for (int it = 0; it < p->max_nlcg; ++it) {
    if (S->e.rs < p->tol_inner) {
      converged = 1;
      break;
    }
    if (!isfinite(S->e.L) || !isfinite(S->e.rs)) break; /* diverged: report non-convergence */
    S->res->nlcg_iters++;
    memcpy(s_old, S->s, sizeof(double) * NG);
    double g0 = h3 * dot(S->G, d, NG);
    if (!(g0 < 0.0)) { /* not a descent direction: restart along s */
      memcpy(d, S->s, sizeof(double) * NG);
      k = 0;
      g0 = h3 * dot(S->G, d, NG);
    }
    const double dd = h3 * dot(d, d, NG);
    /* trial point at sig along d: sigma0, capped so that its RMS size is at most
       trial_max_rel times that of u (R5) */
    double sig = p->sigma0;
    if (p->trial_max_rel > 0.0 && dd > 0.0 && p->trial_max_rel * sqrt(S->N / dd) < sig)
      sig = p->trial_max_rel * sqrt(S->N / dd);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < NG; ++x) ut[x] = fabs(S->u[x] + sig * d[x]);
    {
      double* Gs = S->G;
      double* ss = S->s;
      S->G = Gt;
      S->s = st;
      sv_eval(S, ut, eta, mu);
      S->G = Gs;
      S->s = ss;
    }
    double gt = h3 * dot(Gt, d, NG);
    double alpha = -sig, gprev = gt, gcur = g0;
    if (!((gcur - gprev) / alpha > 0.0)) {
      /* no positive curvature between 0 and sigma0: keep the trial point */
      memcpy(S->u, ut, sizeof(double) * NG);
      memcpy(S->G, Gt, sizeof(double) * NG);
      memcpy(S->s, st, sizeof(double) * NG);
    } else {
      const double L0 = S->e.L;
      for (int j = 1; j <= p->max_secant; ++j) {
        alpha = alpha * gcur / (gprev - gcur);
#pragma omp parallel for schedule(static)
        for (long x = 0; x < NG; ++x) ut[x] = fabs(S->u[x] + alpha * d[x]);
        sv_eval(S, ut, eta, mu);
        for (int bt = 0; bt < p->max_backtrack && !(S->e.L <= L0); ++bt) {
          alpha *= 0.5; /* the secant step did not lower L: halve it */
#pragma omp parallel for schedule(static)
          for (long x = 0; x < NG; ++x) ut[x] = fabs(S->u[x] + alpha * d[x]);
          sv_eval(S, ut, eta, mu);
        }
        memcpy(S->u, ut, sizeof(double) * NG);
        gprev = gcur;
        gcur = h3 * dot(S->G, d, NG);
        if (j == p->max_secant || alpha * alpha * dd <= p->eps_secant * p->eps_secant * S->N) break;
        if (!((gcur - gprev) / alpha > 0.0)) break;
      }
    }
    /* Polak-Ribiere direction update with restarts */
    const double delta_old = delta_new;
    const double delta_mid = -h3 * dot(S->G, s_old, NG);
    delta_new = S->e.rs_pc;
    const double beta = (delta_new - delta_mid) / delta_old;
    ++k;
    if (k >= p->restart_every || !(beta > 0.0)) {
      memcpy(d, S->s, sizeof(double) * NG);
      k = 0;
    } else {
#pragma omp parallel for schedule(static)
      for (long x = 0; x < NG; ++x) d[x] = S->s[x] + beta * d[x];
    }
  }
  if (!converged && S->e.rs < p->tol_inner) converged = 1;
  free(d);
  free(s_old);
  free(ut);
  free(Gt);
  free(st);
  return converged;
}

/* Brent's minimiser (parabolic interpolation with golden-section fallback, Brent
 * 1973) on a bracket a < x < c with f(x) < f(a), f(x) < f(c). */
typedef double (*scalar_fn)(void* ctx, double t);
static double brent_min(scalar_fn f, void* ctx, double a, double x, double c, double fx, double tol,
                        int max_it, double* fmin) {
  const double cg = 0.3819660112501051;
  double lo = a < c ? a : c, hi = a < c ? c : a;
  double w = x, v = x, fw = fx, fv = fx;
  double e = 0.0, step = 0.0;
  for (int it = 0; it < max_it; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double t1 = tol * fabs(x) + 1e-12, t2 = 2.0 * t1;
    if (fabs(x - mid) <= t2 - 0.5 * (hi - lo)) break;
    int golden = 1;
    if (fabs(e) > t1) {
      /* parabola through (x,fx), (w,fw), (v,fv) */
      double r = (x - w) * (fx - fv);
      double q = (x - v) * (fx - fw);
      double pn = (x - v) * q - (x - w) * r;
      q = 2.0 * (q - r);
      if (q > 0.0) pn = -pn;
      q = fabs(q);
      const double e_prev = e;
      e = step;
      if (fabs(pn) < fabs(0.5 * q * e_prev) && pn > q * (lo - x) && pn < q * (hi - x)) {
        step = pn / q;
        const double t = x + step;
        if (t - lo < t2 || hi - t < t2) step = (x < mid) ? t1 : -t1;
        golden = 0;
      }
    }
    if (golden) {
      e = (x >= mid) ? lo - x : hi - x;
      step = cg * e;
    }
    const double t = (fabs(step) >= t1) ? x + step : x + (step > 0 ? t1 : -t1);
    const double ft = f(ctx, t);
    if (ft <= fx) {
      if (t >= x) lo = x; else hi = x;
      v = w; fv = fw;
      w = x; fw = fx;
      x = t; fx = ft;
    } else {
      if (t < x) lo = t; else hi = t;
      if (ft <= fw || w == x) {
        v = w; fv = fw;
        w = t; fw = ft;
      } else if (ft <= fv || v == x || v == w) {
        v = t; fv = ft;
      }
    }
  }
  *fmin = fx;
  return x;
}

typedef struct {
  solver* S;
  const double* u0;
  const double* dh;
  double* ut;
} lm_line;

/* E_h(|cos t u + sin t dhat|): the norm-preserving rotation of the Lagrange
 * multiplier method (Sec. 5.3.2), one Poisson solve per call. */
static double lm_energy_at(void* ctx, double t) {
  lm_line* L = (lm_line*)ctx;
  solver* S = L->S;
  const double ct = cos(t), st = sin(t);
  for (long x = 0; x < S->NG; ++x) L->ut[x] = fabs(ct * L->u0[x] + st * L->dh[x]);
  orc_energy e;
  e.E_zz_corr = S->ezz;
  double* Gs = (double*)malloc(sizeof(double) * S->NG);
  orc_energy_grad(S->g, S->p, L->ut, S->b, S->phi, S->E_self, 0.0, INFINITY, S->N, Gs, NULL, &e);
  free(Gs);
  S->res->energy_evals++;
  S->res->cg_iters += e.cg_iters;
  S->res->stencil_apps += e.cg_iters + 1 + 2;
  return e.E;
}

/* Lagrange multiplier method (Sec. 5.3.2): PR nonlinear CG on the sphere
 * h^3 sum u^2 = N with the gradient projected orthogonal to u, eta = G_E.u/(2 u.u),
 * the Jacobi preconditioner, Brent's line search on the rotation angle, |u|. */
static int lm_solve(solver* S) {
  const orc_params* p = S->p;
  const long NG = S->NG;
  const double h3 = S->h3;
  double* d = (double*)calloc(NG, sizeof(double));
  double* sv = (double*)malloc(sizeof(double) * NG);
  double* s_old = (double*)calloc(NG, sizeof(double));
  double* g = (double*)malloc(sizeof(double) * NG);
  double* g_old = (double*)calloc(NG, sizeof(double));
  double* dh = (double*)malloc(sizeof(double) * NG);
  double* ut = (double*)malloc(sizeof(double) * NG);
  double* u0 = (double*)malloc(sizeof(double) * NG);
  double w[ORC_MAX_N + 1];
  orc_lap_weights(p->fd_n, S->g->h, w);
  const double CF = 0.3 * pow(3.0 * M_PI * M_PI, 2.0 / 3.0);
  int converged = 0, k = 0;
  double delta_new = 0.0, eta = 0.0;
  /* normalise */
  {
    const double nn = h3 * dot(S->u, S->u, NG);
    const double sc = sqrt(S->N / nn);
    for (long x = 0; x < NG; ++x) S->u[x] *= sc;
  }
  for (int it = 0; it <= p->max_nlcg; ++it) {
    sv_eval(S, S->u, 0.0, INFINITY); /* G = gradient of E_h alone */
    const double Ecur = S->e.E;
    eta = dot(S->G, S->u, NG) / (2.0 * dot(S->u, S->u, NG));
    double rs = 0.0, rs_mid = 0.0;
    for (long x = 0; x < NG; ++x) {
      g[x] = S->G[x] - 2.0 * eta * S->u[x];
      const double ux = fabs(S->u[x]);
      double e_xc = 0.0, v_xc = 0.0;
      if (p->terms & ORC_XC) orc_xc(ux, &e_xc, &v_xc);
      const double vk = (p->terms & ORC_TF) ? (5.0 / 3.0) * CF * pow(ux, 4.0 / 3.0) : 0.0;
      const double ph = (p->terms & ORC_ES) ? S->phi[x] : 0.0;
      const double kin = ((p->terms & ORC_VW) ? -6.0 * p->lambda * w[0] : 0.0) + (14.0 / 3.0) * vk;
      double md = kin + 2.0 * (v_xc + ph - eta);
      if (md < 0.25 * kin) md = 0.25 * kin;
      if (md < 1e-10) md = 1e-10;
      sv[x] = -g[x] / md;
    }
    /* project s onto the tangent space of the sphere */
    const double su = dot(sv, S->u, NG) / dot(S->u, S->u, NG);
    for (long x = 0; x < NG; ++x) sv[x] -= su * S->u[x];
    for (long x = 0; x < NG; ++x) {
      rs += -g[x] * sv[x];
      rs_mid += -g[x] * s_old[x];
    }
    rs *= h3;
    rs_mid *= h3;
    S->e.rs = rs;
    if (rs < p->tol_inner) {
      converged = 1;
      (void)Ecur;
      break;
    }
    if (it == p->max_nlcg) break;
    S->res->nlcg_iters++;
    double beta = (it == 0) ? 0.0 : (rs - rs_mid) / delta_new;
    delta_new = rs;
    ++k;
    if (it == 0 || k >= p->restart_every || !(beta > 0.0)) {
      memcpy(d, sv, sizeof(double) * NG);
      k = 0;
    } else {
      for (long x = 0; x < NG; ++x) d[x] = sv[x] + beta * d[x];
    }
    {
      const double du = dot(d, S->u, NG) / dot(S->u, S->u, NG);
      for (long x = 0; x < NG; ++x) d[x] -= du * S->u[x];
    }
    if (!(dot(g, d, NG) < 0.0)) {
      memcpy(d, sv, sizeof(double) * NG);
      k = 0;
    }
    memcpy(s_old, sv, sizeof(double) * NG);
    memcpy(g_old, g, sizeof(double) * NG);
    const double dnorm = sqrt(h3 * dot(d, d, NG));
    const double sc = sqrt(S->N) / dnorm;
    for (long x = 0; x < NG; ++x) dh[x] = d[x] * sc;
    /* bracket the minimum along the rotation angle, then Brent */
    memcpy(u0, S->u, sizeof(double) * NG);
    lm_line L = {S, u0, dh, ut};
    double t1 = dnorm / sqrt(S->N);
    if (t1 > 0.3) t1 = 0.3;
    double fa = Ecur, ta = 0.0;
    double tb = t1, fb = lm_energy_at(&L, tb);
    double tc, fc;
    int shrink = 0;
    while (fb >= fa && shrink < 30) {
      tb *= 0.25;
      fb = lm_energy_at(&L, tb);
      ++shrink;
    }
    if (fb >= fa) break; /* no decrease found along d */
    tc = tb * 2.0;
    fc = lm_energy_at(&L, tc);
    int grow = 0;
    while (fc < fb && grow < 40) {
      ta = tb;
      fa = fb;
      tb = tc;
      fb = fc;
      tc = tb * 1.618034 + 0.0;
      fc = lm_energy_at(&L, tc);
      ++grow;
    }
    double fmin;
    const double tmin = brent_min(lm_energy_at, &L, ta, tb, tc, fb, 1e-4, 60, &fmin);
    const double ct = cos(tmin), st = sin(tmin);
    for (long x = 0; x < NG; ++x) S->u[x] = fabs(ct * u0[x] + st * dh[x]);
  }
  S->res->eta = eta;
  free(d);
  free(sv);
  free(s_old);
  free(g);
  free(g_old);
  free(dh);
  free(ut);
  free(u0);
  return converged;
}

/* Repulsion correction for overlapping Gaussian nuclei (Appendix A, reduced to a
 * closed form): the electrostatic reformulation counts the Gaussian-Gaussian
 * repulsion Z_I Z_J erf(R_IJ/(sqrt2 sigma))/R_IJ instead of Z_I Z_J/R_IJ (Eq. EZZ),
 * so the correction is sum_{I<J} Z_I Z_J erfc(R_IJ/(sqrt2 sigma))/R_IJ; F (if not
 * NULL) receives its contribution -dE_c/dR to the forces. */
double orc_ezz_correction(const double* R, const double* Z, int M, double sigma, double* F) {
  double E = 0.0;
  if (F) memset(F, 0, sizeof(double) * 3 * M);
  const double a = 1.0 / (sqrt(2.0) * sigma);
  for (int I = 0; I < M; ++I)
    for (int J = I + 1; J < M; ++J) {
      double dx[3], r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        dx[d] = R[3 * I + d] - R[3 * J + d];
        r2 += dx[d] * dx[d];
      }
      const double r = sqrt(r2);
      const double zz = Z[I] * Z[J];
      E += zz * erfc(a * r) / r;
      if (F) {
        /* d/dr [erfc(a r)/r] = -erfc(a r)/r^2 - (2a/sqrt(pi)) exp(-a^2 r^2)/r */
        const double dEdr = zz * (-erfc(a * r) / r2 - 2.0 * a / sqrt(M_PI) * exp(-a * a * r2) / r);
        for (int d = 0; d < 3; ++d) {
          F[3 * I + d] -= dEdr * dx[d] / r;
          F[3 * J + d] += dEdr * dx[d] / r;
        }
      }
    }
  return E;
}

/* Ground state at fixed nuclei (Eq. GroundStateElectronic): Algorithm 1 (AL),
 * the penalty method (AL with eta_q = 0) or the Lagrange multiplier method.
 * On entry u may hold a starting guess (all zeros selects the R7 guess); on exit
 * u, phi, b hold u*, phi*, b.  Returns 0 on convergence, 1 otherwise. */
int orc_solve(const orc_grid* g, const orc_params* p, const double* R, const double* Z, int M,
              double* u, double* phi, double* b, orc_result* res) {
  memset(res, 0, sizeof(*res));
  solver S;
  memset(&S, 0, sizeof(S));
  S.g = g;
  S.p = p;
  S.NG = (long)g->n1 * g->n2 * g->n3;
  S.h3 = g->h * g->h * g->h;
  S.res = res;
  double N = 0.0;
  for (int J = 0; J < M; ++J) N += Z[J];
  S.N = N;
  orc_pseudocharge(g, p->fd_n, R, Z, M, p->sigma, p->rc, b, &S.E_self);
  S.ezz = p->ezz_correction ? orc_ezz_correction(R, Z, M, p->sigma, NULL) : 0.0;
  S.b = b;
  int all_zero = 1;
  for (long x = 0; x < S.NG; ++x)
    if (u[x] != 0.0) {
      all_zero = 0;
      break;
    }
  if (all_zero) orc_initial_guess(g, R, Z, M, p->guess_sigma, p->guess_cut, N, u);
  S.u = u;
  S.phi = phi;
  S.G = (double*)malloc(sizeof(double) * S.NG);
  S.s = (double*)malloc(sizeof(double) * S.NG);
  int converged = 0;
  if (p->method == ORC_LM) {
    converged = lm_solve(&S);
    sv_eval(&S, u, 0.0, INFINITY);
    res->E = S.e.E;
    res->C = S.e.C;
    res->outer_iters = 1;
  } else {
    double eta = (p->method == ORC_PENALTY) ? 0.0 : p->eta0;
    double mu = p->mu0;
    sv_eval(&S, u, eta, mu);
    double E_prev = S.e.E;
    for (int q = 0; q < p->max_outer; ++q) {
      nlcg(&S, eta, mu);
      res->outer_iters++;
      const double E = S.e.E, C = S.e.C;
      if (!isfinite(E) || !isfinite(C)) break;
      const double eta_eff = eta - C / mu; /* Algorithm 1 multiplier update */
      res->eta = eta_eff;
      if (p->method == ORC_AL) eta = eta_eff;
      mu = p->kappa * mu;
      if (fabs(E - E_prev) < p->tol_E) {
        converged = 1;
        break;
      }
      E_prev = E;
    }
    res->E = S.e.E;
    res->C = S.e.C;
  }
  res->parts = S.e;
  res->converged = converged;
  free(S.G);
  free(S.s);
  return converged ? 0 : 1;
}

/* Forces on the nuclei (Eq. Force:Nuclei) at the ground state phi*:
 *   paper form   : f_J = h^3 sum_{ball J} grad_h b_J (phi* - V_J), with the FD
 *                  gradient of Sec. 4 (weights w~_p) applied to b_J;
 *   exact variant: f_J = -h^3 sum_{ball J} (db_J/dR_J)(phi* - V_J) with
 *                  db_J/dR_J = (1/4 pi) L_h (grad V_J) from the analytic gradient,
 *                  the exact derivative of the discrete energy for fixed grid.
 * Sums run over grid nodes within r_c of R_J. */
void orc_forces(const orc_grid* g, int n, const double* R, const double* Z, int M, double sigma,
                double rc, const double* phi, int exact_variant, double* F) {
  const double h3 = g->h * g->h * g->h;
  double wt[ORC_MAX_N + 1], w[ORC_MAX_N + 1];
  orc_grad_weights(n, g->h, wt);
  orc_lap_weights(n, g->h, w);
#pragma omp parallel for schedule(dynamic, 1)
  for (int J = 0; J < M; ++J) {
    atom_box ab;
    atom_box_build(g, n, R + 3 * J, Z[J], sigma, rc, n, &ab);
    double f[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < ab.dim[2]; ++c)
      for (long bb = 0; bb < ab.dim[1]; ++bb)
        for (long a = 0; a < ab.dim[0]; ++a) {
          const long i = ab.lo[0] + a, j = ab.lo[1] + bb, k = ab.lo[2] + c;
          if (i < 0 || j < 0 || k < 0 || i >= g->n1 || j >= g->n2 || k >= g->n3) continue;
          const double dx = node_coord(g, 0, i) - R[3 * J];
          const double dy = node_coord(g, 1, j) - R[3 * J + 1];
          const double dz = node_coord(g, 2, k) - R[3 * J + 2];
          if (!(sqrt(dx * dx + dy * dy + dz * dz) < rc)) continue;
          const double pv = phi[i + (long)g->n1 * (j + (long)g->n2 * k)] - ab_v(&ab, i, j, k);
          double grad[3] = {0.0, 0.0, 0.0};
          if (!exact_variant) {
            for (int p = 1; p <= n; ++p) {
              grad[0] += wt[p] * (ab_b(&ab, i + p, j, k) - ab_b(&ab, i - p, j, k));
              grad[1] += wt[p] * (ab_b(&ab, i, j + p, k) - ab_b(&ab, i, j - p, k));
              grad[2] += wt[p] * (ab_b(&ab, i, j, k + p) - ab_b(&ab, i, j, k - p));
            }
          } else {
            /* -db_J/dR = -(1/4 pi) L_h grad V_J, analytic grad V_J at every stencil node */
            for (int d = 0; d < 3; ++d) {
              double acc = 0.0;
              for (int p = -n; p <= n; ++p)
                for (int ax = 0; ax < 3; ++ax) {
                  if (p == 0 && ax > 0) continue;
                  const long ii = i + (ax == 0 ? p : 0), jj = j + (ax == 1 ? p : 0), kk = k + (ax == 2 ? p : 0);
                  const double ex = node_coord(g, 0, ii) - R[3 * J];
                  const double ey = node_coord(g, 1, jj) - R[3 * J + 1];
                  const double ez = node_coord(g, 2, kk) - R[3 * J + 2];
                  const double r = sqrt(ex * ex + ey * ey + ez * ez);
                  /* dV/dr for V = -Z erf(r/s)/r */
                  double gv = 0.0;
                  if (r > 1e-12 * sigma) {
                    const double dVdr = Z[J] * erf(r / sigma) / (r * r) -
                                        Z[J] * 2.0 / (sigma * sqrt(M_PI)) * exp(-(r / sigma) * (r / sigma)) / r;
                    const double comp = (d == 0 ? ex : (d == 1 ? ey : ez)) / r;
                    gv = dVdr * comp;
                  }
                  const double wp = (p == 0) ? 6.0 * w[0] : w[p < 0 ? -p : p];
                  acc += wp * gv;
                }
              grad[d] = -acc / (4.0 * M_PI);
            }
          }
          f[0] += h3 * grad[0] * pv;
          f[1] += h3 * grad[1] * pv;
          f[2] += h3 * grad[2] * pv;
        }
    F[3 * J] = f[0];
    F[3 * J + 1] = f[1];
    F[3 * J + 2] = f[2];
    atom_box_free(&ab);
  }
}
