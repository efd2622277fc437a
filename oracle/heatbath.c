/* FP64 CPU oracle of the SU(3) heatbath (test infrastructure only; see heatbath.h
 * for the algorithm, its reading of the paper and the pins). */
#include "heatbath.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define MAX_ATTEMPTS 1000
static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------ Philox4x64-10 */

/* Philox4x64 (SC'11): multipliers and Weyl key increments of the published definition */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL, PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL, PHILOX_W1 = 0xBB67AE8584CAA73BULL;

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  const unsigned __int128 p = (unsigned __int128)a * b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void oracle_philox4x64(const uint64_t counter[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = counter[0], c1 = counter[1], c2 = counter[2], c3 = counter[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo64(PHILOX_M1, c2, &hi1, &lo1);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* (0, 1]: 53 high bits, plus one unit */
static double unit_open0(uint64_t r) { return ((double)(r >> 11) + 1.0) * 0x1.0p-53; }

/* ------------------------------------------------------------ SU(2) draw (Creutz) */

/* b with density ~ exp(alpha b0) on the 3-sphere; counters (c0, c1, c2, attempt).
 * Returns 1 if accepted, 0 after MAX_ATTEMPTS (b = identity then). */
static int su2_draw(double alpha, uint64_t seed, uint64_t c0, uint64_t c1, uint64_t c2, double b[4]) {
  const uint64_t key[2] = {seed, 0};
  for (uint64_t attempt = 0; attempt < MAX_ATTEMPTS; ++attempt) {
    const uint64_t ctr[4] = {c0, c1, c2, attempt};
    uint64_t r[4];
    oracle_philox4x64(ctr, key, r);
    const double u0 = unit_open0(r[0]), u1 = unit_open0(r[1]);
    const double u2 = unit_open0(r[2]), u3 = unit_open0(r[3]);
    double b0;
    if (alpha < 1e-12) {
      b0 = 1.0 - 2.0 * u0;  /* uniform on [-1, 1): alpha -> 0 limit */
    } else {
      /* y = 1 - u0 (1 - exp(-2 alpha)) in [exp(-2 alpha), 1), b0 = 1 + ln(y) / alpha */
      b0 = 1.0 + log1p(-u0 * (-expm1(-2.0 * alpha))) / alpha;
    }
    const double s2 = 1.0 - b0 * b0;
    if (u1 * u1 <= s2) {
      const double rr = sqrt(s2 > 0.0 ? s2 : 0.0);
      const double ct = 2.0 * u2 - 1.0;
      const double st2 = 1.0 - ct * ct;
      const double st = sqrt(st2 > 0.0 ? st2 : 0.0);
      const double phi = TWO_PI * u3;
      b[0] = b0;
      b[1] = rr * st * cos(phi);
      b[2] = rr * st * sin(phi);
      b[3] = rr * ct;
      return 1;
    }
  }
  b[0] = 1.0;
  b[1] = b[2] = b[3] = 0.0;
  return 0;
}

long long oracle_su2_draws(double alpha, uint64_t seed, long long n, double* out) {
  long long fails = 0;
  for (long long i = 0; i < n; ++i) fails += !su2_draw(alpha, seed, (uint64_t)i, 0, 0, out + 4 * i);
  return fails;
}

/* ------------------------------------------------------------ lattice helpers */

typedef struct {
  int L[4];
  long long V;
} Lat;

static int lat_init(Lat* g, const int dims[4]) {
  g->V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || dims[m] % 2) return -1;
    g->L[m] = dims[m];
    g->V *= dims[m];
  }
  return 0;
}

static void coords(const Lat* g, long long s, int c[4]) {
  for (int m = 0; m < 4; ++m) {
    c[m] = (int)(s % g->L[m]);
    s /= g->L[m];
  }
}

static long long index_of(const Lat* g, const int c[4]) {
  return c[0] + (long long)g->L[0] * (c[1] + (long long)g->L[1] * (c[2] + (long long)g->L[2] * c[3]));
}

/* site s shifted by +d along mu (d = +-1) */
static long long shift(const Lat* g, long long s, int mu, int d) {
  int c[4];
  coords(g, s, c);
  c[mu] = (c[mu] + d + g->L[mu]) % g->L[mu];
  return index_of(g, c);
}

static const cplx* link(const double* U, long long s, int mu) { return (const cplx*)U + (s * 4 + mu) * 9; }
static cplx* link_w(double* U, long long s, int mu) { return (cplx*)U + (s * 4 + mu) * 9; }

/* C = A B, C = A B^dag, C = A^dag B for 3x3 complex matrices */
static void mul_nn(const cplx* A, const cplx* B, cplx* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
      C[i * 3 + j] = s;
    }
}
static void mul_nd(const cplx* A, const cplx* B, cplx* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * conj(B[j * 3 + k]);
      C[i * 3 + j] = s;
    }
}
static void mul_dn(const cplx* A, const cplx* B, cplx* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx s = 0;
      for (int k = 0; k < 3; ++k) s += conj(A[k * 3 + i]) * B[k * 3 + j];
      C[i * 3 + j] = s;
    }
}

static void staple(const Lat* g, const double* U, long long s, int mu, cplx* W) {
  for (int i = 0; i < 9; ++i) W[i] = 0;
  const long long sp = shift(g, s, mu, +1);
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    cplx T[9], T2[9];
    /* upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    const long long spn = shift(g, s, nu, +1);
    mul_nd(link(U, sp, nu), link(U, spn, mu), T);
    mul_nd(T, link(U, s, nu), T2);
    for (int i = 0; i < 9; ++i) W[i] += T2[i];
    /* lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) */
    const long long smn = shift(g, s, nu, -1);
    const long long spmn = shift(g, sp, nu, -1);
    cplx A[9];
    mul_nn(link(U, smn, mu), link(U, spmn, nu), A); /* U_mu(x-nu) U_nu(x+mu-nu) */
    mul_dn(A, link(U, smn, nu), T2);                /* (U_mu U_nu)^dag U_nu(x-nu) */
    for (int i = 0; i < 9; ++i) W[i] += T2[i];
  }
}

void oracle_staple(const int dims[4], const double* U, long long s, int mu, double* W) {
  Lat g;
  if (lat_init(&g, dims)) return;
  staple(&g, U, s, mu, (cplx*)W);
}

/* ------------------------------------------------------------ Cabibbo-Marinari */

static const int SUB[3][2] = {{0, 1}, {1, 2}, {0, 2}};

/* U <- R U for the three SU(2) subgroups in turn; returns subgroups left unchanged */
static int update_link(cplx* U, const cplx* W, double beta, uint64_t seed, uint64_t link_id,
                       uint64_t sweep) {
  int fails = 0;
  for (int k = 0; k < 3; ++k) {
    const int i = SUB[k][0], j = SUB[k][1];
    cplx V[9];
    mul_nn(U, W, V);
    /* subgroup block X of V and c with Re Tr(a X) = a . c, a = a0 + i a.sigma */
    const cplx x00 = V[i * 3 + i], x01 = V[i * 3 + j], x10 = V[j * 3 + i], x11 = V[j * 3 + j];
    double c[4];
    c[0] = creal(x00 + x11);
    c[1] = -cimag(x01 + x10);
    c[2] = creal(x10 - x01);
    c[3] = -cimag(x00 - x11);
    const double kk = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
    double v[4] = {1.0, 0.0, 0.0, 0.0};
    if (kk > 0.0)
      for (int m = 0; m < 4; ++m) v[m] = c[m] / kk;
    double b[4];
    if (!su2_draw(beta * kk / 3.0, seed, link_id, sweep, (uint64_t)k, b)) {
      ++fails;
      continue;
    }
    /* a = b v as 2x2 matrices: mat(q) = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]] */
    const cplx B[4] = {b[0] + I * b[3], b[2] + I * b[1], -b[2] + I * b[1], b[0] - I * b[3]};
    const cplx Vm[4] = {v[0] + I * v[3], v[2] + I * v[1], -v[2] + I * v[1], v[0] - I * v[3]};
    cplx A[4];
    for (int r = 0; r < 2; ++r)
      for (int q = 0; q < 2; ++q) A[r * 2 + q] = B[r * 2 + 0] * Vm[0 * 2 + q] + B[r * 2 + 1] * Vm[1 * 2 + q];
    /* U <- R U with R the embedding of A on rows / columns (i, j) */
    for (int col = 0; col < 3; ++col) {
      const cplx ui = U[i * 3 + col], uj = U[j * 3 + col];
      U[i * 3 + col] = A[0] * ui + A[1] * uj;
      U[j * 3 + col] = A[2] * ui + A[3] * uj;
    }
  }
  return fails;
}

static int parity_of(const Lat* g, long long s) {
  int c[4];
  coords(g, s, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

int oracle_heatbath_link(const int dims[4], double* U, double beta, uint64_t seed, uint64_t sweep,
                         long long s, int mu) {
  Lat g;
  if (lat_init(&g, dims) || s < 0 || s >= g.V || mu < 0 || mu > 3) return -1;
  cplx W[9];
  staple(&g, U, s, mu, W);
  return update_link(link_w(U, s, mu), W, beta, seed, (uint64_t)(4 * s + mu), sweep);
}

static void reunit_one(cplx* u) {
  double n0 = 0;
  for (int c = 0; c < 3; ++c) n0 += creal(u[c] * conj(u[c]));
  n0 = 1.0 / sqrt(n0);
  for (int c = 0; c < 3; ++c) u[c] *= n0;
  cplx p = 0; /* <row0, row1> */
  for (int c = 0; c < 3; ++c) p += conj(u[c]) * u[3 + c];
  for (int c = 0; c < 3; ++c) u[3 + c] -= p * u[c];
  double n1 = 0;
  for (int c = 0; c < 3; ++c) n1 += creal(u[3 + c] * conj(u[3 + c]));
  n1 = 1.0 / sqrt(n1);
  for (int c = 0; c < 3; ++c) u[3 + c] *= n1;
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

void oracle_reunitarise(const int dims[4], double* U) {
  Lat g;
  if (lat_init(&g, dims)) return;
#pragma omp parallel for schedule(static)
  for (long long s = 0; s < g.V; ++s)
    for (int mu = 0; mu < 4; ++mu) reunit_one(link_w(U, s, mu));
}

long long oracle_heatbath(const int dims[4], double* U, double beta, uint64_t seed, uint64_t sweep0,
                          int nsweeps, int reunit) {
  Lat g;
  if (lat_init(&g, dims) || nsweeps < 0 || !(beta >= 0.0)) return -1;
  long long fails = 0;
  for (int sw = 0; sw < nsweeps; ++sw) {
    const uint64_t sweep = sweep0 + (uint64_t)sw;
    for (int mu = 0; mu < 4; ++mu)
      for (int par = 0; par < 2; ++par) {
        /* links of one (mu, parity) class share no staple: any order gives the same result */
#pragma omp parallel for schedule(static) reduction(+ : fails)
        for (long long s = 0; s < g.V; ++s) {
          if (parity_of(&g, s) != par) continue;
          cplx W[9];
          staple(&g, U, s, mu, W);
          fails += update_link(link_w(U, s, mu), W, beta, seed, (uint64_t)(4 * s + mu), sweep);
        }
      }
    if (reunit) oracle_reunitarise(dims, U);
  }
  return fails;
}

double oracle_plaquette(const int dims[4], const double* U) {
  Lat g;
  if (lat_init(&g, dims)) return NAN;
  double sum = 0.0;
  for (long long s = 0; s < g.V; ++s)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        /* Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag = Re Tr A B^dag with
         * A = U_mu(x) U_nu(x+mu), B = U_nu(x) U_mu(x+nu) */
        cplx A[9], B[9];
        mul_nn(link(U, s, mu), link(U, shift(&g, s, mu, +1), nu), A);
        mul_nn(link(U, s, nu), link(U, shift(&g, s, nu, +1), mu), B);
        double tr = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) tr += creal(A[i * 3 + k] * conj(B[i * 3 + k]));
        sum += tr;
      }
  return sum / (18.0 * (double)g.V);
}
