/* FP64 CPU oracle for the Wilson-Dirac operator and its solvers.
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU baseline load it; the library does not. Definitions and layout are in
 * wilson_oracle.h. Everything here is plain double-precision C with the
 * operator written out from its definition; OpenMP only splits site loops.
 */
#include "wilson_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* gamma matrices, chiral basis (textbook; the paper does not fix one) */
/* ------------------------------------------------------------------ */

static cplx GAMMA[4][4][4]; /* GAMMA[mu][row][col] */
static int gamma_ready = 0;

static void build_gammas(void) {
  if (gamma_ready) return;
  /* Pauli matrices sigma_1..3 */
  const cplx sig[3][2][2] = {
      {{0, 1}, {1, 0}},
      {{0, -I}, {I, 0}},
      {{1, 0}, {0, -1}},
  };
  memset(GAMMA, 0, sizeof(GAMMA));
  for (int k = 0; k < 3; ++k) {
    /* g_k = [[0, -i sigma_k], [i sigma_k, 0]] */
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        GAMMA[k][a][2 + b] = -I * sig[k][a][b];
        GAMMA[k][2 + a][b] = I * sig[k][a][b];
      }
  }
  /* g_4 = [[0, 1], [1, 0]] */
  for (int a = 0; a < 2; ++a) {
    GAMMA[3][a][2 + a] = 1;
    GAMMA[3][2 + a][a] = 1;
  }
  gamma_ready = 1;
}

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
  long long L[4];
  long long V;
} geom;

static int make_geom(const int dims[4], geom* g) {
  g->V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] <= 0) return ORACLE_BADARG;
    g->L[mu] = dims[mu];
    g->V *= dims[mu];
  }
  return ORACLE_OK;
}

static void coords(const geom* g, long long s, long long c[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = s % g->L[mu];
    s /= g->L[mu];
  }
}

static long long index_of(const geom* g, const long long c[4]) {
  return c[0] + g->L[0] * (c[1] + g->L[1] * (c[2] + g->L[2] * c[3]));
}

static int parity_of(const long long c[4]) { return (int)((c[0] + c[1] + c[2] + c[3]) & 1); }

/* ------------------------------------------------------------------ */
/* the hopping term at one site                                         */
/* ------------------------------------------------------------------ */

/* acc = sum_mu [ eta+ (1 - sgn g_mu) U_mu(x) psi(x+mu) + eta- (1 + sgn g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 * sgn = +1 for D, -1 for D^dag. */
static void hop_site(const geom* g, int t_bc, const cplx* U, const cplx* psi, long long s,
                     int dagger, cplx acc[4][3]) {
  const double sgn = dagger ? -1.0 : 1.0;
  long long c[4];
  coords(g, s, c);
  memset(acc, 0, sizeof(cplx) * 12);
  for (int mu = 0; mu < 4; ++mu) {
    for (int dir = 0; dir < 2; ++dir) { /* 0 forward, 1 backward */
      long long n[4] = {c[0], c[1], c[2], c[3]};
      double eta = 1.0;
      const cplx* link;
      if (dir == 0) {
        n[mu] = (c[mu] + 1) % g->L[mu];
        if (mu == 3 && c[3] == g->L[3] - 1) eta = (double)t_bc;
        link = U + (s * 4 + mu) * 9;
      } else {
        n[mu] = (c[mu] - 1 + g->L[mu]) % g->L[mu];
        if (mu == 3 && c[3] == 0) eta = (double)t_bc;
        link = U + (index_of(g, n) * 4 + mu) * 9;
      }
      const cplx* ps = psi + index_of(g, n) * 12;
      /* chi[spin][a] = (link or link^dag)[a][b] psi[spin][b] */
      cplx chi[4][3];
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
          cplx v = 0;
          for (int b = 0; b < 3; ++b) {
            cplx u = (dir == 0) ? link[a * 3 + b] : conj(link[b * 3 + a]);
            v += u * ps[sp * 3 + b];
          }
          chi[sp][a] = v;
        }
      /* projector P = 1 - sgn g_mu (forward) or 1 + sgn g_mu (backward) */
      const double sg = (dir == 0) ? -sgn : sgn;
      for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) {
          cplx v = chi[i][a];
          for (int j = 0; j < 4; ++j) v += sg * GAMMA[mu][i][j] * chi[j][a];
          acc[i][a] += eta * v;
        }
    }
  }
}

/* ------------------------------------------------------------------ */
/* operators                                                            */
/* ------------------------------------------------------------------ */

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int hop_impl(const int dims[4], int t_bc, const cplx* U, const cplx* psi, cplx* out,
                    int only_parity, int dagger) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return ORACLE_BADARG;
  build_gammas();
#pragma omp parallel for schedule(static)
  for (long long s = 0; s < g.V; ++s) {
    long long c[4];
    coords(&g, s, c);
    if (only_parity >= 0 && parity_of(c) != only_parity) {
      memset(out + s * 12, 0, sizeof(cplx) * 12);
      continue;
    }
    cplx acc[4][3];
    hop_site(&g, t_bc, U, psi, s, dagger, acc);
    memcpy(out + s * 12, acc, sizeof(cplx) * 12);
  }
  return ORACLE_OK;
}

int oracle_hop(const int dims[4], int t_bc, const double* U, const double* psi, double* out,
               int dagger) {
  return hop_impl(dims, t_bc, (const cplx*)U, (const cplx*)psi, (cplx*)out, -1, dagger);
}

int oracle_hop_eo(const int dims[4], int t_bc, const double* U, const double* psi, double* out,
                  int out_parity, int dagger) {
  if (out_parity != 0 && out_parity != 1) return ORACLE_BADARG;
  return hop_impl(dims, t_bc, (const cplx*)U, (const cplx*)psi, (cplx*)out, out_parity, dagger);
}

int oracle_hop_sites(const int dims[4], int t_bc, const double* U, const double* psi,
                     const long long* sites, long long nsites, double* out, int dagger) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return ORACLE_BADARG;
  build_gammas();
  for (long long i = 0; i < nsites; ++i)
    if (sites[i] < 0 || sites[i] >= g.V) return ORACLE_BADARG;
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < nsites; ++i) {
    cplx acc[4][3];
    hop_site(&g, t_bc, (const cplx*)U, (const cplx*)psi, sites[i], dagger, acc);
    memcpy((cplx*)out + i * 12, acc, sizeof(cplx) * 12);
  }
  return ORACLE_OK;
}

/* g5 = diag(1, 1, -1, -1) in the chiral basis: sign of spin component sp */
static double g5_sign(int sp) { return sp < 2 ? 1.0 : -1.0; }

/* out = c * (1 + i tau g5) psi at every site of parity `only` (all sites if only < 0) */
static void twist(const geom* g, cplx c, double tau, const cplx* psi, cplx* out, int only) {
#pragma omp parallel for schedule(static)
  for (long long s = 0; s < g->V; ++s) {
    long long cc[4];
    coords(g, s, cc);
    if (only >= 0 && parity_of(cc) != only) continue;
    for (int sp = 0; sp < 4; ++sp)
      for (int a = 0; a < 3; ++a) {
        const long long i = s * 12 + sp * 3 + a;
        out[i] = c * (1.0 + I * tau * g5_sign(sp)) * psi[i];
      }
  }
}

int oracle_apply_M(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                   const double* psi, double* out, int dagger) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return ORACLE_BADARG;
  int rc = oracle_hop(dims, t_bc, U, psi, out, dagger);
  if (rc) return rc;
  cplx* o = (cplx*)out;
  const cplx* p = (const cplx*)psi;
  /* M = 1 - kappa D + 2 i kappa mu g5 ;  M^dag = 1 - kappa D^dag - 2 i kappa mu g5 */
  const double tm = (dagger ? -2.0 : 2.0) * kappa * mu;
#pragma omp parallel for schedule(static)
  for (long long s = 0; s < g.V; ++s)
    for (int sp = 0; sp < 4; ++sp)
      for (int a = 0; a < 3; ++a) {
        const long long i = s * 12 + sp * 3 + a;
        o[i] = p[i] - kappa * o[i] + I * tm * g5_sign(sp) * p[i];
      }
  return ORACLE_OK;
}

/* Mhat = A - kappa^2 D_eo A^-1 D_oe on the even sites (Schur complement of M), with
 * A = 1 + i a g5, a = 2 kappa mu, A^-1 = (1 - i a g5) / (1 + a^2).
 * For dagger: Mhat^dag = A^dag - kappa^2 (D^dag)_eo (A^-1)^dag (D^dag)_oe. */
int oracle_apply_Mhat(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                      const double* psi, double* out, int dagger) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return ORACLE_BADARG;
  const double a = (dagger ? -2.0 : 2.0) * kappa * mu;
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * 12 * g.V);
  cplx* tmp2 = (cplx*)malloc(sizeof(cplx) * 12 * g.V);
  cplx* apsi = (cplx*)malloc(sizeof(cplx) * 12 * g.V);
  if (!tmp || !tmp2 || !apsi) return ORACLE_BADARG;
  hop_impl(dims, t_bc, (const cplx*)U, (const cplx*)psi, tmp, 1, dagger);
  twist(&g, 1.0 / (1.0 + a * a), -a, tmp, tmp2, 1);
  hop_impl(dims, t_bc, (const cplx*)U, tmp2, (cplx*)out, 0, dagger);
  twist(&g, 1.0, a, (const cplx*)psi, apsi, 0);
  free(tmp);
  free(tmp2);
  cplx* o = (cplx*)out;
#pragma omp parallel for schedule(static)
  for (long long s = 0; s < g.V; ++s) {
    long long c[4];
    coords(&g, s, c);
    for (int k = 0; k < 12; ++k)
      o[s * 12 + k] = (parity_of(c) == 0) ? apsi[s * 12 + k] - kappa * kappa * o[s * 12 + k] : 0;
  }
  free(apsi);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* vector helpers (n complex entries)                                   */
/* ------------------------------------------------------------------ */

static cplx vdot(const cplx* a, const cplx* b, long long n) { /* <a, b> = sum conj(a) b */
  double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
  for (long long i = 0; i < n; ++i) {
    cplx v = conj(a[i]) * b[i];
    re += creal(v);
    im += cimag(v);
  }
  return re + I * im;
}

static double vnorm2(const cplx* a, long long n) { return creal(vdot(a, a, n)); }

/* ------------------------------------------------------------------ */
/* solvers                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
  const int* dims;
  int t_bc;
  const double* U;
  double kappa;
  double mu;
  int eo;
  long long n; /* complex entries per vector (full lattice) */
  cplx* tmp;
} opctx;

/* y = A v with A = M (eo = 0) or Mhat (eo = 1) */
static void op_apply(const opctx* c, const cplx* v, cplx* y, int dagger) {
  if (c->eo)
    oracle_apply_Mhat(c->dims, c->t_bc, c->U, c->kappa, c->mu, (const double*)v, (double*)y, dagger);
  else
    oracle_apply_M(c->dims, c->t_bc, c->U, c->kappa, c->mu, (const double*)v, (double*)y, dagger);
}

/* Hestenes-Stiefel CG on A^dag A x = A^dag rhs, x0 = 0; stop on ||rhs - A x|| <= abs_tol. */
static int cg_normal(const opctx* c, const cplx* rhs, cplx* x, double abs_tol, int maxiter,
                     int* iters) {
  long long n = c->n;
  cplx* r = calloc(n, sizeof(cplx));
  cplx* p = calloc(n, sizeof(cplx));
  cplx* q = calloc(n, sizeof(cplx));
  cplx* w = calloc(n, sizeof(cplx));
  cplx* res = calloc(n, sizeof(cplx));
  memset(x, 0, sizeof(cplx) * n);
  op_apply(c, rhs, r, 1); /* r = A^dag rhs - A^dag A 0 */
  memcpy(p, r, sizeof(cplx) * n);
  double rr = vnorm2(r, n);
  int status = ORACLE_MAXITER, k = 0;
  if (sqrt(vnorm2(rhs, n)) <= abs_tol) status = ORACLE_OK;
  while (status != ORACLE_OK && k < maxiter) {
    op_apply(c, p, q, 0); /* q = A p */
    op_apply(c, q, w, 1); /* w = A^dag A p */
    double pap = vnorm2(q, n);
    if (pap == 0.0) { status = ORACLE_BREAKDOWN; break; }
    double alpha = rr / pap;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * w[i];
    }
    ++k;
    /* true residual of the (un-normalised) system */
    op_apply(c, x, res, 0);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) res[i] = rhs[i] - res[i];
    if (sqrt(vnorm2(res, n)) <= abs_tol) { status = ORACLE_OK; break; }
    double rr_new = vnorm2(r, n);
    double beta = rr_new / rr;
    rr = rr_new;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
  *iters = k;
  free(r); free(p); free(q); free(w); free(res);
  return status;
}

/* van der Vorst BiCGStab on A x = rhs, x0 = 0, shadow residual r0. */
static int bicgstab(const opctx* c, const cplx* rhs, cplx* x, double abs_tol, int maxiter,
                    int* iters) {
  long long n = c->n;
  cplx* r = calloc(n, sizeof(cplx));
  cplx* r0 = calloc(n, sizeof(cplx));
  cplx* p = calloc(n, sizeof(cplx));
  cplx* v = calloc(n, sizeof(cplx));
  cplx* s = calloc(n, sizeof(cplx));
  cplx* t = calloc(n, sizeof(cplx));
  cplx* res = calloc(n, sizeof(cplx));
  memset(x, 0, sizeof(cplx) * n);
  memcpy(r, rhs, sizeof(cplx) * n);
  memcpy(r0, rhs, sizeof(cplx) * n);
  cplx rho = 1, alpha = 1, omega = 1;
  int status = ORACLE_MAXITER, k = 0;
  if (sqrt(vnorm2(rhs, n)) <= abs_tol) status = ORACLE_OK;
  while (status != ORACLE_OK && k < maxiter) {
    cplx rho_new = vdot(r0, r, n);
    if (cabs(rho_new) == 0.0 || cabs(omega) == 0.0) { status = ORACLE_BREAKDOWN; break; }
    cplx beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    op_apply(c, p, v, 0);
    cplx r0v = vdot(r0, v, n);
    if (cabs(r0v) == 0.0) { status = ORACLE_BREAKDOWN; break; }
    alpha = rho / r0v;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    op_apply(c, s, t, 0);
    double tt = vnorm2(t, n);
    omega = (tt == 0.0) ? 0.0 : vdot(t, s, n) / tt;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) {
      x[i] += alpha * p[i] + omega * s[i];
      r[i] = s[i] - omega * t[i];
    }
    ++k;
    op_apply(c, x, res, 0);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) res[i] = rhs[i] - res[i];
    if (sqrt(vnorm2(res, n)) <= abs_tol) { status = ORACLE_OK; break; }
  }
  *iters = k;
  free(r); free(r0); free(p); free(v); free(s); free(t); free(res);
  return status;
}

double oracle_true_residual(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                            const double* b, const double* x) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return -1.0;
  long long n = 12 * g.V;
  cplx* y = malloc(sizeof(cplx) * n);
  oracle_apply_M(dims, t_bc, U, kappa, mu, x, (double*)y, 0);
  const cplx* bb = (const cplx*)b;
  for (long long i = 0; i < n; ++i) y[i] = bb[i] - y[i];
  double res = sqrt(vnorm2(y, n)) / sqrt(vnorm2(bb, n));
  free(y);
  return res;
}

int oracle_solve(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                 const double* b, double* x, double tol, int maxiter, int method, double* info) {
  geom g;
  if (make_geom(dims, &g) != ORACLE_OK) return ORACLE_BADARG;
  if (method < 0 || method > 2) return ORACLE_BADARG;
  build_gammas();
  long long n = 12 * g.V;
  const cplx* bb = (const cplx*)b;
  cplx* xx = (cplx*)x;
  double bnorm = sqrt(vnorm2(bb, n));
  double abs_tol = tol * bnorm;
  opctx c = {dims, t_bc, U, kappa, mu, method != 0, n, NULL};
  int iters = 0, status;
  if (method == 0) {
    status = cg_normal(&c, bb, xx, abs_tol, maxiter, &iters);
  } else {
    /* Schur complement with A = 1 + i a g5 (a = 2 kappa mu):
     *   bhat_e = b_e + kappa D_eo A^-1 b_o ;  x_o = A^-1 (b_o + kappa D_oe x_e).
     * The residual of Mhat on the even sites equals the full residual there,
     * and the odd residual vanishes by construction, so the same abs_tol applies. */
    const double a = 2.0 * kappa * mu;
    cplx* bhat = calloc(n, sizeof(cplx));
    cplx* xe = calloc(n, sizeof(cplx));
    cplx* tmp = calloc(n, sizeof(cplx));
    cplx* ainv_bo = calloc(n, sizeof(cplx));
    twist(&g, 1.0 / (1.0 + a * a), -a, bb, ainv_bo, 1);
    oracle_hop_eo(dims, t_bc, U, (const double*)ainv_bo, (double*)tmp, 0, 0);
    for (long long s = 0; s < g.V; ++s) {
      long long cc[4];
      coords(&g, s, cc);
      for (int k = 0; k < 12; ++k)
        bhat[s * 12 + k] = parity_of(cc) == 0 ? bb[s * 12 + k] + kappa * tmp[s * 12 + k] : 0;
    }
    if (method == 1)
      status = cg_normal(&c, bhat, xe, abs_tol, maxiter, &iters);
    else
      status = bicgstab(&c, bhat, xe, abs_tol, maxiter, &iters);
    oracle_hop_eo(dims, t_bc, U, (const double*)xe, (double*)tmp, 1, 0);
    for (long long s = 0; s < g.V; ++s) {
      long long cc[4];
      coords(&g, s, cc);
      for (int k = 0; k < 12; ++k)
        tmp[s * 12 + k] = parity_of(cc) == 1 ? bb[s * 12 + k] + kappa * tmp[s * 12 + k] : 0;
    }
    twist(&g, 1.0 / (1.0 + a * a), -a, tmp, tmp, 1);
    for (long long s = 0; s < g.V; ++s) {
      long long cc[4];
      coords(&g, s, cc);
      for (int k = 0; k < 12; ++k)
        xx[s * 12 + k] = parity_of(cc) == 0 ? xe[s * 12 + k] : tmp[s * 12 + k];
    }
    free(ainv_bo);
    free(bhat); free(xe); free(tmp);
  }
  if (info) {
    info[0] = iters;
    info[1] = oracle_true_residual(dims, t_bc, U, kappa, mu, b, x);
  }
  return status;
}
