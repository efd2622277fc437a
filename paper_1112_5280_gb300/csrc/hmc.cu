// Hybrid Monte Carlo for N_f = 2 (twisted-mass) Wilson fermions with even-odd
// preconditioning (paper Section 3: an HMC with even-odd preconditioning, the 2MN
// integrator and multiple integration timescales for N_f = 2 twisted-mass Wilson
// fermions).
//
//   S = S_g + S_f, S_g = beta sum_P (1 - Re Tr U_P / 3), S_f = phi^dag (Mhat^dag Mhat)^-1 phi
//   on the even sites, Mhat = A - kappa^2 D_eo A^-1 D_oe, A = 1 + i a g5, a = 2 kappa mu.
//   Momenta P traceless anti-Hermitian; H = -sum Tr(P^2) / 2 + S; dU/dt = P U, dP/dt = -G.
//   G is the su(3) gradient: dS/de = -sum Tr(H G) for U -> exp(e H) U, so a term
//   c Re Tr(U B) gives G = -c TA(U B), TA(M) = (M - M^dag)/2 - Tr(M - M^dag)/6.
//     gauge:   G_g = (beta/3) TA(U W), W the staple sum;
//     fermion: X = (Mhat^dag Mhat)^-1 phi, Y = Mhat X, Phi = X_e + A^-1 D_oe X_e,
//              Psi = Y_e + A^-dag (D^dag)_oe Y_e, and
//              G_f = -2 kappa^2 eta TA(U [ ((1 - g_mu) Phi(x+mu))^T conj(Psi(x))
//                                          + Psi(x+mu)^T conj((1 + g_mu) Phi(x)) ]),
//              spin summed, colour indices left as a 3 x 3 matrix, eta the t-boundary sign.
//   S_f = |Y|^2 comes free with each force.
// Integrators: leapfrog and the second-order minimum-norm scheme of Omelyan, Mryglod and
// Folk (lambda = 0.1931833275037836), the gauge force on a nested inner level. Kicks at
// the same links are merged (one solve where two fermion kicks meet).
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "gauge_field.cuh"
#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {
namespace {

using namespace gf;

constexpr int HMC_THREADS = 128;

__device__ __forceinline__ int eo_index(const Geom& g, const Site& s) {
  return (s.c[0] >> 1) + g.Lxh * (s.c[1] + g.L[1] * (s.c[2] + g.L[2] * s.c[3]));
}

// P_mu(x) += c TA(V) for a double-float V: TA(V)_ii = i (Im V_ii - Im tr V / 3),
// TA(V)_ij = (V_ij - conj V_ji) / 2, TA_ji = -conj TA_ij; only the accumulation into the FP64
// momenta runs in FP64
__device__ __forceinline__ void add_ta(double2* P, const Geom& g, const Site& x, int mu, const M3d& V, double c) {
  const size_t b = link_base(g, x, mu);
  const size_t vh = (size_t)g.Vh;
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = (double)V.e[k * 4].im;
  const double tr = (d[0] + d[1] + d[2]) / 3.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double2 q = P[b + (size_t)(k * 4) * vh];
    q.y += c * (d[k] - tr);
    P[b + (size_t)(k * 4) * vh] = q;
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int col = r + 1; col < 3; ++col) {
      const C2d x1 = V.e[r * 3 + col], y1 = V.e[col * 3 + r];
      const double re = 0.5 * (double)df_add_u(x1.re, -y1.re), im = 0.5 * (double)df_add_u(x1.im, y1.im);
      double2 q = P[b + (size_t)(r * 3 + col) * vh];
      q.x += c * re;
      q.y += c * im;
      P[b + (size_t)(r * 3 + col) * vh] = q;
      q = P[b + (size_t)(col * 3 + r) * vh];
      q.x -= c * re;
      q.y += c * im;
      P[b + (size_t)(col * 3 + r) * vh] = q;
    }
}

// P_mu(x) += c TA(U W), c = coeff beta / 3: the staple sum, U W and the anti-Hermitian
// part in double-float from the copy Ud (FP32 pipes), only the accumulation into the FP64
// momenta in FP64. All four directions in one launch (blockIdx.y = mu), one thread per
// link, mu a run-time value so that the four share one instruction stream.
// 2 CTAs per SM (254 registers, no spill): 3 (168 registers, a 68-byte spill) measured 3%
// slower over a 16^3x32 HMC trajectory on GB300.
#ifndef LQCD_GF_MIN_BLOCKS
#define LQCD_GF_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(HMC_THREADS, LQCD_GF_MIN_BLOCKS) k_gauge_force(const float4* Ud, Geom g, double c, double2* P) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2LL * g.Vh) return;
  const int mu = blockIdx.y;
  const Site x = site_of(g, (int)(i / g.Vh), (int)(i % g.Vh));
  add_ta(P, g, x, mu, mul_d<false, false>(load_link_df(Ud, g, x, mu), staple_df(Ud, g, x, mu)), c);
}

// gamma_mu v on one colour's four spins in double-float (chiral basis, as in the Dslash:
// g_k = [[0, -i s_k], [i s_k, 0]] for mu = 0, 1, 2, g_t = [[0, 1], [1, 0]])
__device__ __forceinline__ C2d ti_d(const C2d& a) { return {-a.im, a.re}; }
__device__ __forceinline__ C2d tmi_d(const C2d& a) { return {a.im, -a.re}; }
__device__ __forceinline__ C2d neg_d(const C2d& a) { return {-a.re, -a.im}; }
template <int MU>
__device__ __forceinline__ void gamma_mul_d(const C2d v[4], C2d o[4]) {
  if (MU == 0) {
    o[0] = tmi_d(v[3]); o[1] = tmi_d(v[2]); o[2] = ti_d(v[1]); o[3] = ti_d(v[0]);
  } else if (MU == 1) {
    o[0] = neg_d(v[3]); o[1] = v[2]; o[2] = v[1]; o[3] = neg_d(v[0]);
  } else if (MU == 2) {
    o[0] = tmi_d(v[2]); o[1] = ti_d(v[3]); o[2] = ti_d(v[0]); o[3] = tmi_d(v[1]);
  } else {
    o[0] = v[2]; o[1] = v[3]; o[2] = v[0]; o[3] = v[1];
  }
}

// acc += a conj(b), unnormalised double-float
__device__ __forceinline__ void cmacc_d(C2d& acc, const C2d& a, const C2d& b) {
  df_mac_u(acc.re, a.re, b.re);
  df_mac_u(acc.re, a.im, b.im);
  df_mac_u(acc.im, a.im, b.re);
  df_mac_u(acc.im, -a.re, b.im);
}

// P_mu(x) += c eta TA(U B), B = ((1 - g_mu) Phi(x+mu))^T conj(Psi(x)) + Psi(x+mu)^T conj((1 + g_mu) Phi(x)),
// all in double-float from the double-float fields Phi, Psi and links Ud; one thread per link
// of direction MU. B's entries accumulate unnormalised and are normalised once.
template <int MU>
__global__ void __launch_bounds__(HMC_THREADS) k_fermion_force(const float4* Ud, Geom g, const void* phi_e,
                                                              const void* phi_o, const void* psi_e,
                                                              const void* psi_o, double c, double2* P) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2LL * g.Vh) return;
  const int par = (int)(i / g.Vh), h = (int)(i % g.Vh);
  const Site x = site_of(g, par, h);
  const Site xp = shifted(g, x, MU, 1);
  const int hp = eo_index(g, xp);
  const void* phi_x = par ? phi_o : phi_e;
  const void* psi_x = par ? psi_o : psi_e;
  const void* phi_n = par ? phi_e : phi_o;
  const void* psi_n = par ? psi_e : psi_o;
  M3d Bm;
#pragma unroll
  for (int k = 0; k < 9; ++k) Bm.e[k] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
  {
    df64 s[24];  // Psi(x)
    SpinorIO<P_DF64>::load(psi_x, g.Vh, h, s);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      df64 f[8];  // colour b of Phi(x + mu)
      SpinorIO<P_DF64>::load_colour(phi_n, g.Vh, hp, b, f);
      C2d v[4], gv[4];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) v[sp] = {f[2 * sp], f[2 * sp + 1]};
      gamma_mul_d<MU>(v, gv);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) v[sp] = {df_add_u(v[sp].re, -gv[sp].re), df_add_u(v[sp].im, -gv[sp].im)};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
          cmacc_d(Bm.e[b * 3 + a], v[sp], C2d{s[sidx(sp, a)], s[sidx(sp, a) + 1]});
    }
  }
  {
    df64 f[24];  // Phi(x)
    SpinorIO<P_DF64>::load(phi_x, g.Vh, h, f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      df64 t[8];  // colour a of Psi(x + mu)
      SpinorIO<P_DF64>::load_colour(psi_n, g.Vh, hp, a, t);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        C2d v[4], gv[4];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) v[sp] = {f[sidx(sp, b)], f[sidx(sp, b) + 1]};
        gamma_mul_d<MU>(v, gv);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const C2d w{df_add_u(v[sp].re, gv[sp].re), df_add_u(v[sp].im, gv[sp].im)};  // (1 + g_mu) Phi(x)
          cmacc_d(Bm.e[a * 3 + b], C2d{t[2 * sp], t[2 * sp + 1]}, w);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) Bm.e[k] = {df_norm(Bm.e[k].re), df_norm(Bm.e[k].im)};
  const double eta = (MU == 3 && x.c[3] == g.L[3] - 1) ? (double)g.t_bc : 1.0;
  add_ta(P, g, x, MU, mul_d<false, false>(load_link_df(Ud, g, x, MU), Bm), c * eta);
}

// 1/k! for the Taylor coefficients as double-float constants (k! is exact in FP64 for
// k <= 22; the pair is the FP64 value split into two floats at compile time)
struct DFConst {
  float hi, lo;
};
constexpr DFConst dfc(double v) { return {(float)v, (float)(v - (double)(float)v)}; }
__constant__ DFConst kInvFact[18] = {
    dfc(1.0), dfc(1.0), dfc(1.0 / 2.0), dfc(1.0 / 6.0), dfc(1.0 / 24.0), dfc(1.0 / 120.0), dfc(1.0 / 720.0),
    dfc(1.0 / 5040.0), dfc(1.0 / 40320.0), dfc(1.0 / 362880.0), dfc(1.0 / 3628800.0), dfc(1.0 / 39916800.0),
    dfc(1.0 / 479001600.0), dfc(1.0 / 6227020800.0), dfc(1.0 / 87178291200.0), dfc(1.0 / 1307674368000.0),
    dfc(1.0 / 20922789888000.0), dfc(1.0 / 355687428096000.0)};

// U <- exp(eps P) U in double-float: the Taylor polynomial of degree n after scaling
// |eps P| below 1/2 (n from the norm, at most 16), then squaring; U read from the
// double-float copy Ud, the product written to Ud and, when write_master, to the FP64
// master U (else the caller rebuilds the master from Ud before reading it).
// The polynomial is reduced by Cayley-Hamilton: with c2 = tr X, c1 = (tr(X)^2 - tr X^2) / 2
// and c0 = det X, X^3 = c2 X^2 - c1 X + c0 I, so every power X^k = a_k I + b_k X + g_k X^2
// with the scalar recursion a_{k+1} = g_k c0, b_{k+1} = a_k - g_k c1, g_{k+1} = b_k + g_k c2,
// and sum_k X^k / k! = (sum a_k / k!) I + (sum b_k / k!) X + (sum g_k / k!) X^2: one matrix
// product (X^2) for any degree. Everything runs on the FP32 pipes: P is split into
// double-float pairs by integer operations, and the norm and the degree, which only need
// to bound the Taylor tail, are taken in FP32 with a margin.
__global__ void k_expm_update(double2* U, float4* Ud, Geom g, const double2* P, double eps, bool write_master) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (par, mu, h)
  if (i >= 8LL * g.Vh) return;
  const int h = (int)(i % g.Vh);
  const size_t base = (size_t)(i / g.Vh) * 9 * g.Vh + h;
  const df64 e_df = df_split_bits(eps);
  M3d A;
  float n2 = 0.0f;
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const double2 q = P[base + (size_t)w * g.Vh];
    A.e[w] = {e_df * df_split_bits(q.x), e_df * df_split_bits(q.y)};
    n2 = __fmaf_rn(A.e[w].re.hi, A.e[w].re.hi, __fmaf_rn(A.e[w].im.hi, A.e[w].im.hi, n2));
  }
  // Frobenius norm of eps P (submultiplicative, so it bounds the Taylor tail), rounded up
  float nrm = sqrtf(n2) * (1.0f + 0x1.0p-16f);
  int sq = 0;
  while (nrm > 0.5f && sq < 60) {
    nrm *= 0.5f;
    ++sq;
  }
  if (sq > 0) {
    const float sc = __uint_as_float((unsigned)(127 - sq) << 23);  // 2^-sq, exact scaling
#pragma unroll
    for (int w = 0; w < 9; ++w) {
      A.e[w].re = df64(A.e[w].re.hi * sc, A.e[w].re.lo * sc);
      A.e[w].im = df64(A.e[w].im.hi * sc, A.e[w].im.lo * sc);
    }
  }
  // degree: the smallest n with nrm^(n+1) / (n+1)! below 2^-50 (n <= 16 as nrm <= 1/2)
  int order = 1;
  for (float term = nrm; order < 16; ++order) {
    term *= __fdividef(nrm, (float)(order + 1));
    if (term < 0x1.0p-50f) break;
  }
  const M3d A2 = mul_d<false, false>(A, A);
  const C2d t1 = cadd_d(cadd_d(A.e[0], A.e[4]), A.e[8]);
  const C2d t2 = cadd_d(cadd_d(A2.e[0], A2.e[4]), A2.e[8]);
  const C2d c2 = t1;
  const C2d c1 = cscale_d(df64(0.5f, 0.0f), csub_d(cmul_d(t1, t1), t2));
  const C2d m0 = csub_d(cmul_d(A.e[4], A.e[8]), cmul_d(A.e[5], A.e[7]));
  const C2d m1 = csub_d(cmul_d(A.e[3], A.e[8]), cmul_d(A.e[5], A.e[6]));
  const C2d m2 = csub_d(cmul_d(A.e[3], A.e[7]), cmul_d(A.e[4], A.e[6]));
  const C2d c0 = cadd_d(csub_d(cmul_d(A.e[0], m0), cmul_d(A.e[1], m1)), cmul_d(A.e[2], m2));
  const C2d zero = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
  C2d a = {df64(1.0f, 0.0f), df64(0.0f, 0.0f)}, b = zero, gm = zero;  // X^0 = I
  C2d sa = a, sb = b, sg = gm;                                        // sums over k of X^k / k!
  for (int k = 1; k <= order; ++k) {
    const C2d na = cmul_d(gm, c0), nb = csub_d(a, cmul_d(gm, c1)), ng = cadd_d(b, cmul_d(gm, c2));
    a = na;
    b = nb;
    gm = ng;
    const df64 f(kInvFact[k].hi, kInvFact[k].lo);
    sa = cadd_d(sa, cscale_d(f, a));
    sb = cadd_d(sb, cscale_d(f, b));
    sg = cadd_d(sg, cscale_d(f, gm));
  }
  M3d E;
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    C2d e = cadd_d(cmul_d(sb, A.e[w]), cmul_d(sg, A2.e[w]));
    if (w % 4 == 0) e = cadd_d(e, sa);
    E.e[w] = e;
  }
  for (int k = 0; k < sq; ++k) E = mul_d<false, false>(E, E);
  M3d u;
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const float4 d = Ud[base + (size_t)w * g.Vh];
    u.e[w] = {df64(d.x, d.y), df64(d.z, d.w)};
  }
  const M3d un = mul_d<false, false>(E, u);
#pragma unroll
  for (int w = 0; w < 9; ++w)
    Ud[base + (size_t)w * g.Vh] = make_float4(un.e[w].re.hi, un.e[w].re.lo, un.e[w].im.hi, un.e[w].im.lo);
  if (write_master) {
#pragma unroll
    for (int w = 0; w < 9; ++w)
      U[base + (size_t)w * g.Vh] = make_double2((double)un.e[w].re, (double)un.e[w].im);
  }
}

constexpr int RED_THREADS = 256;
// per-CTA partial of sum |P_ij|^2 / 2
__global__ void __launch_bounds__(RED_THREADS) k_kinetic(const double2* P, long long n, double* partials) {
  __shared__ double red[RED_THREADS];
  double acc = 0.0;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 d = P[i];
    acc = 0.5 * (d.x * d.x + d.y * d.y);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* partials, int n, double* out) {
  __shared__ double red[RED_THREADS];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += RED_THREADS) acc += partials[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int check_mom(const lqcd_gauge* g, const lqcd_mom* m) {
  if (!g || !m) return set_error(LQCD_EINVAL, "NULL gauge or momentum field");
  if (g->ctx != m->ctx || memcmp(g->g.L, m->g.L, sizeof g->g.L))
    return set_error(LQCD_EINVAL, "gauge and momentum field differ in context or lattice");
  return LQCD_OK;
}

// the gauge field's double-float copy (made when missing; kept current by every update here)
int df_links(const lqcd_gauge* g, float4** out) {
  const void* base;
  int nr;
  LQCD_TRY(gauge_links(g, P_DF64, &base, &nr));
  *out = static_cast<float4*>(const_cast<void*>(base));
  return LQCD_OK;
}

int gauge_force_impl(const lqcd_gauge* g, double beta, double coeff, lqcd_mom* m) {
  const double c = coeff * beta / 3.0;
  float4* Ud = nullptr;
  LQCD_TRY(df_links(g, &Ud));
  const unsigned nb = blocks(2LL * g->g.Vh, HMC_THREADS);
  cudaStream_t st = g->ctx->stream;
  k_gauge_force<<<dim3(nb, 4), HMC_THREADS, 0, st>>>(Ud, g->g, c, m->d);
  g->ctx->launches++;
  LQCD_CK(cudaGetLastError());
  return LQCD_OK;
}

// |half|^2 (other == NULL) or Re <half, other> of FP64 half fields, synchronous
int half_norm2(lqcd_ctx* c, const void* half, const Geom& g, double* out, const void* other = nullptr) {
  LQCD_TRY(ctx_partials(c, 3 * (size_t)((g.Vh + TILE - 1) / TILE)));
  Work w = blank_work(g);
  w.sc = c->scratch_sc;
  w.in = half;
  w.y1 = other;
  w.red = 1;
  w.fin = FIN_STORE0;
  LQCD_CK(launch_blas(P_F64, other ? B_RDOT : B_NORM, single_launch(w, c->partials), 0, c->stream));
  c->launches++;
  LQCD_CK(cudaMemcpyAsync(c->host_sc, c->scratch_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  *out = c->host_sc->res[0];
  return LQCD_OK;
}

// From X (even half of x, FP64): Y = Mhat X, the odd halves of Phi and Psi, S_f and
// P += coeff G_f. x and y are FULL FP64 fields (y's even half receives Y); xd and yd are
// FULL double-float work fields that end up holding Phi = (X_e, A^-1 D_oe X_e) and
// Psi = (Y_e, A^-dag (D^dag)_oe Y_e). The Dslash applications and the force kernel run
// in double-float (FP64 runs at 1/64 of the FP32 rate here).
// S_f: with phi, the variational 2 Re <phi, X> - |Y|^2, whose error is quadratic in the
// solve's (X = X* - e gives S* - |Mhat e|^2); without, |Y|^2 = phi^dag X (linear error).
int fermion_force_from_x(const lqcd_gauge* g, double kappa, double mu, lqcd_field* x, lqcd_field* y,
                         lqcd_field* xd, lqcd_field* yd, double coeff, lqcd_mom* m, double* s_f,
                         const lqcd_field* phi = nullptr) {
  const double a = 2.0 * kappa * mu, s = 1.0 / (1.0 + a * a);
  const int Vh = g->g.Vh;
  cudaStream_t st = g->ctx->stream;
  float4* Ud = nullptr;
  LQCD_TRY(df_links(g, &Ud));
  LQCD_CK(spinor_convert(x->half[0], P_F64, xd->half[0], P_DF64, Vh, 1.0, st));
  LQCD_TRY(lqcd_apply_Mhat_tm(g, kappa, mu, xd, yd, 0));
  // Phi_o = A^-1 D_oe X_e, Psi_o = A^-dag (D^dag)_oe Y_e
  LQCD_TRY(dslash_tw(g, P_DF64, xd->half[0], xd->half[1], nullptr, nullptr, 1.0, 0.0, 0.0, 1, false, s, -a, 0.0));
  LQCD_TRY(dslash_tw(g, P_DF64, yd->half[0], yd->half[1], nullptr, nullptr, 1.0, 0.0, 0.0, 1, true, s, a, 0.0));
  LQCD_CK(spinor_convert(yd->half[0], P_DF64, y->half[0], P_F64, Vh, 1.0, st));
  g->ctx->launches += 2;
  double yy = 0.0;
  LQCD_TRY(half_norm2(g->ctx, y->half[0], g->g, &yy));
  if (phi) {
    double px = 0.0;
    LQCD_TRY(half_norm2(g->ctx, x->half[0], g->g, &px, phi->half[0]));
    yy = 2.0 * px - yy;
  }
  if (s_f) *s_f = yy;
  const double c = -2.0 * kappa * kappa * coeff;
  const unsigned nb = blocks(2LL * g->g.Vh, HMC_THREADS);
  const void *pe = xd->half[0], *po = xd->half[1], *se = yd->half[0], *so = yd->half[1];
  k_fermion_force<0><<<nb, HMC_THREADS, 0, st>>>(Ud, g->g, pe, po, se, so, c, m->d);
  k_fermion_force<1><<<nb, HMC_THREADS, 0, st>>>(Ud, g->g, pe, po, se, so, c, m->d);
  k_fermion_force<2><<<nb, HMC_THREADS, 0, st>>>(Ud, g->g, pe, po, se, so, c, m->d);
  k_fermion_force<3><<<nb, HMC_THREADS, 0, st>>>(Ud, g->g, pe, po, se, so, c, m->d);
  g->ctx->launches += 4;
  LQCD_CK(cudaGetLastError());
  return LQCD_OK;
}

// x0 (may be NULL): the starting even half of the solve (else x = 0)
int solve_normal_with(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* phi, double kappa, double mu,
                      double tol, lqcd_field* x, lqcd_solve_info* info, const lqcd_field* x0 = nullptr) {
  long long id = 0;
  if (x0)
    LQCD_TRY(engine_submit_normal_guess(e, g, phi, x0, kappa, mu, tol, &id));
  else
    LQCD_TRY(lqcd_engine_submit_normal(e, g, phi, kappa, mu, tol, &id));
  int active = 1;
  while (active > 0) LQCD_TRY(lqcd_engine_step(e, &active));
  return lqcd_engine_result(e, id, x, info);
}

// master: also write the FP64 master and rebuild the other link copies now; else only the
// double-float copy moves, and the caller runs links_from_df before anything else reads links
int update_links(lqcd_gauge* g, const lqcd_mom* m, double eps, bool master) {
  float4* Ud = nullptr;
  LQCD_TRY(df_links(g, &Ud));
  k_expm_update<<<blocks(8LL * g->g.Vh, 128), 128, 0, g->ctx->stream>>>(static_cast<double2*>(g->copy[P_F64][0]),
                                                                          Ud, g->g, m->d, eps, master);
  g->ctx->launches++;
  LQCD_CK(cudaGetLastError());
  return master ? refresh_gauge_copies(g, true) : LQCD_OK;
}

int kinetic_impl(const lqcd_mom* m, double* out) {
  lqcd_ctx* c = m->ctx;
  const long long n = 72LL * m->g.Vh;  // complex entries: 2 parities x 4 mu x 9 x V/2
  const int nb = (int)blocks(n, RED_THREADS);
  LQCD_TRY(ctx_partials(c, (size_t)nb + 1));
  k_kinetic<<<nb, RED_THREADS, 0, c->stream>>>(m->d, n, c->partials);
  k_sum_partials<<<1, RED_THREADS, 0, c->stream>>>(c->partials, nb, c->partials + nb);
  c->launches += 2;
  LQCD_CK(cudaGetLastError());
  LQCD_CK(cudaMemcpyAsync(out, c->partials + nb, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

}  // namespace
}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_mom_create(lqcd_ctx* c, const int dims[4], lqcd_mom** out) {
  clear_error();
  if (!c || !dims || !out) return set_error(LQCD_EINVAL, "NULL argument");
  *out = nullptr;
  Geom g;
  LQCD_TRY(make_geom(dims, -1, g));
  LQCD_CK(cudaSetDevice(c->device));
  lqcd_mom* m = new lqcd_mom();
  m->ctx = c;
  m->g = g;
  m->bytes = gauge_copy_bytes(P_F64, 18, g.Vh);
  if (cudaMalloc(&m->d, m->bytes) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return set_error(LQCD_ENOMEM, "momentum field (%zu bytes)", gauge_copy_bytes(P_F64, 18, g.Vh));
  }
  cudaError_t e = cudaMemsetAsync(m->d, 0, m->bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(m->d);
    delete m;
    return set_error(LQCD_ECUDA, "momentum field: %s", cudaGetErrorString(e));
  }
  ctx_retain(c);
  *out = m;
  return LQCD_OK;
}

void lqcd_mom_destroy(lqcd_mom* m) {
  if (!m) return;
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  cudaFree(m->d);
  lqcd_ctx* c = m->ctx;
  delete m;
  ctx_release(c);
}

int lqcd_mom_upload(lqcd_mom* m, const double* host) {
  clear_error();
  if (!m || !host) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = m->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  LQCD_TRY(ctx_staging(c, m->bytes));
  LQCD_CK(cudaMemcpyAsync(c->staging, host, m->bytes, cudaMemcpyHostToDevice, c->stream));
  LQCD_CK(gauge_from_aos(c->staging, m->g, P_F64, 18, m->d, c->stream));
  c->launches++;
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

int lqcd_mom_download(const lqcd_mom* m, double* host) {
  clear_error();
  if (!m || !host) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = m->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  LQCD_TRY(ctx_staging(c, m->bytes));
  LQCD_CK(links_to_aos(m->d, m->g, reinterpret_cast<double2*>(c->staging), c->stream));
  c->launches++;
  LQCD_CK(cudaMemcpyAsync(host, c->staging, m->bytes, cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

int lqcd_mom_zero(lqcd_mom* m) {
  clear_error();
  if (!m) return set_error(LQCD_EINVAL, "NULL argument");
  LQCD_CK(cudaSetDevice(m->ctx->device));
  LQCD_CK(cudaMemsetAsync(m->d, 0, m->bytes, m->ctx->stream));
  return LQCD_OK;
}

int lqcd_mom_kinetic(const lqcd_mom* m, double* energy) {
  LQCD_TRACE("lqcd_mom_kinetic");
  clear_error();
  if (!m || !energy) return set_error(LQCD_EINVAL, "NULL argument");
  LQCD_CK(cudaSetDevice(m->ctx->device));
  return kinetic_impl(m, energy);
}

int lqcd_gauge_force(const lqcd_gauge* g, double beta, double coeff, lqcd_mom* m) {
  LQCD_TRACE("lqcd_gauge_force");
  clear_error();
  LQCD_TRY(check_mom(g, m));
  if (!std::isfinite(beta) || !std::isfinite(coeff)) return set_error(LQCD_EINVAL, "beta and coeff must be finite");
  LQCD_CK(cudaSetDevice(g->ctx->device));
  return gauge_force_impl(g, beta, coeff, m);
}

int lqcd_fermion_force(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* x, double coeff,
                       lqcd_mom* m, double* s_f) {
  LQCD_TRACE("lqcd_fermion_force");
  PdlSolverScope pdl_scope(g && pdl_solver_off((g->g.Vh + TILE - 1) / TILE));  // large: no PDL
  clear_error();
  LQCD_TRY(check_mom(g, m));
  if (!x || x->prec != LQCD_F64 || x->subset != LQCD_FULL || memcmp(x->g.L, g->g.L, sizeof g->g.L))
    return set_error(LQCD_EINVAL, "x must be a FULL FP64 field of the gauge's lattice");
  if (!std::isfinite(kappa) || !std::isfinite(mu) || !std::isfinite(coeff))
    return set_error(LQCD_EINVAL, "kappa, mu and coeff must be finite");
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  int dims[4] = {g->g.L[0], g->g.L[1], g->g.L[2], g->g.L[3]};
  lqcd_field *xx = nullptr, *y = nullptr, *xd = nullptr, *yd = nullptr;
  int rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &xx);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &y);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_DF64, LQCD_FULL, &xd);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_DF64, LQCD_FULL, &yd);
  if (rc == LQCD_OK) rc = lqcd_field_copy(xx, x, 1.0);
  if (rc == LQCD_OK) rc = fermion_force_from_x(g, kappa, mu, xx, y, xd, yd, coeff, m, s_f);
  for (lqcd_field* f : {xx, y, xd, yd}) lqcd_field_destroy(f);
  return rc;
}

int lqcd_gauge_update(lqcd_gauge* g, const lqcd_mom* m, double eps) {
  LQCD_TRACE("lqcd_gauge_update");
  clear_error();
  LQCD_TRY(check_mom(g, m));
  if (!std::isfinite(eps)) return set_error(LQCD_EINVAL, "eps must be finite");
  LQCD_CK(cudaSetDevice(g->ctx->device));
  return update_links(g, m, eps, true);
}

int lqcd_solve_normal(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                      const lqcd_solve_opts* opts, lqcd_field* x, lqcd_solve_info* info) {
  LQCD_TRACE("lqcd_solve_normal");
  PdlSolverScope pdl_scope(g && pdl_solver_off((g->g.Vh + TILE - 1) / TILE));  // large: no PDL
  clear_error();
  if (!g || !src || !x) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_solve_opts o;
  lqcd_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.solver != LQCD_CG) return set_error(LQCD_EINVAL, "the normal equations are solved by CG");
  lqcd_engine* e = nullptr;
  LQCD_TRY(ctx_engine(g->ctx, o, 1, &e));
  const int rc = solve_normal_with(e, g, src, kappa, o.mu, tol, x, info);
  if (rc != LQCD_OK && rc != LQCD_ENOCONV && rc != LQCD_EBREAKDOWN && rc != LQCD_ENONFINITE)
    ctx_drop_engine(g->ctx);
  return rc;
}

void lqcd_hmc_params_default(lqcd_hmc_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->beta = 5.6;
  p->kappa = 0.156;
  p->mu = 0.0;
  p->tau = 1.0;
  p->nsteps = 10;
  p->ngauge = 4;
  p->scheme = LQCD_2MN;
  p->tol = 1e-10;
  p->accept_u = 0.0;
}

int lqcd_hmc_trajectory(lqcd_gauge* g, const lqcd_hmc_params* p, lqcd_mom* m, const lqcd_field* phi,
                        const lqcd_solve_opts* opts, lqcd_hmc_info* info) {
  LQCD_TRACE("lqcd_hmc_trajectory");
  PdlSolverScope pdl_scope(g && pdl_solver_off((g->g.Vh + TILE - 1) / TILE));  // large: no PDL
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (info) memset(info, 0, sizeof *info);
  LQCD_TRY(check_mom(g, m));
  if (!p || !phi) return set_error(LQCD_EINVAL, "NULL argument");
  if (phi->prec != LQCD_F64 || phi->subset != LQCD_FULL || memcmp(phi->g.L, g->g.L, sizeof g->g.L))
    return set_error(LQCD_EINVAL, "phi must be a FULL FP64 field of the gauge's lattice (even half used)");
  if (p->nsteps < 1 || p->ngauge < 1 || !(p->tau > 0) || !std::isfinite(p->tau) || !(p->tol > 0) ||
      (p->scheme != LQCD_LEAPFROG && p->scheme != LQCD_2MN) || !std::isfinite(p->beta) ||
      !std::isfinite(p->kappa) || !std::isfinite(p->mu) || p->chrono < 0 || p->chrono > 2)
    return set_error(LQCD_EINVAL, "bad HMC parameters");
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  lqcd_solve_opts o;
  lqcd_solve_opts_default(&o);
  if (opts) o = *opts;
  o.solver = LQCD_CG;
  o.mu = p->mu;
  int dims[4] = {g->g.L[0], g->g.L[1], g->g.L[2], g->g.L[3]};
  lqcd_field *x = nullptr, *y = nullptr, *xd = nullptr, *yd = nullptr;
  lqcd_field *xprev = nullptr, *guess = nullptr;  // chronological initial guesses
  lqcd_engine* e = nullptr;
  void* backup = nullptr;
  const size_t ubytes = gauge_copy_bytes(P_F64, 18, g->g.Vh);
  int rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &x);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &y);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_DF64, LQCD_FULL, &xd);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_DF64, LQCD_FULL, &yd);
  if (rc == LQCD_OK && p->chrono == 2) rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &xprev);
  if (rc == LQCD_OK && p->chrono == 2) rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &guess);
  if (rc == LQCD_OK) rc = ctx_engine(c, o, 1, &e);
  if (rc == LQCD_OK && p->accept_u > 0.0) {
    if (cudaMalloc(&backup, ubytes) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(LQCD_ENOMEM, "link backup");
    } else if (cudaMemcpyAsync(backup, g->copy[P_F64][0], ubytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
      rc = set_error(LQCD_ECUDA, "link backup copy");
    }
  }
  // energies at the start
  double kin0 = 0, kin1 = 0, plaq0 = 0, plaq1 = 0, sf0 = 0, sf1 = 0;
  if (rc == LQCD_OK) rc = kinetic_impl(m, &kin0);
  if (rc == LQCD_OK) rc = lqcd_plaquette(g, &plaq0);
  // kicks at the current links are merged until the links move
  double pend_f = 0.0, pend_g = 0.0;
  int force_evals = 0, solves_iters = 0;
  // the drifts move only the double-float copy; the master and the solver's copies are
  // rebuilt from it only where a fermion force, the plaquette or the caller reads them
  bool first_f = true, copies_stale = false;
  auto flush = [&]() -> int {
    if (pend_g != 0.0) LQCD_TRY(gauge_force_impl(g, p->beta, -pend_g, m));
    if (pend_f != 0.0) {
      if (copies_stale) LQCD_TRY(links_from_df(g));
      copies_stale = false;
      lqcd_solve_info si{};
      // initial guess: none, the last solution (chrono 1), or 2 X_last - X_before (chrono 2)
      const lqcd_field* x0 = nullptr;
      if (p->chrono >= 1 && force_evals >= 1) x0 = x;
      if (p->chrono == 2 && force_evals >= 2) {
        Work w = blank_work(g->g);
        w.in = x->half[0];
        w.y1 = xprev->half[0];
        w.out = guess->half[0];
        w.a = 2.0;
        w.c1 = -1.0;
        LQCD_CK(launch_blas(P_F64, B_AXPBY, single_launch(w, nullptr), 0, c->stream, P_F64));
        x0 = guess;
      }
      if (p->chrono == 2 && force_evals >= 1) LQCD_TRY(lqcd_field_copy(xprev, x, 1.0));
      LQCD_TRY(solve_normal_with(e, g, phi, p->kappa, p->mu, p->tol, x, &si, x0));
      solves_iters += si.iters;
      double s = 0.0;
      LQCD_TRY(fermion_force_from_x(g, p->kappa, p->mu, x, y, xd, yd, -pend_f, m, &s, phi));
      if (first_f) sf0 = s;
      first_f = false;
      sf1 = s;
      ++force_evals;
    }
    pend_f = pend_g = 0.0;
    return LQCD_OK;
  };
  auto drift = [&](double h) -> int {
    LQCD_TRY(flush());
    copies_stale = true;
    return update_links(g, m, h, false);
  };
  const double lam = 0.1931833275037836;
  auto inner = [&](double h) -> int {
    const double eg = h / p->ngauge;
    for (int k = 0; k < p->ngauge; ++k) {
      if (p->scheme == LQCD_LEAPFROG) {
        pend_g += 0.5 * eg;
        LQCD_TRY(drift(eg));
        pend_g += 0.5 * eg;
      } else {
        pend_g += lam * eg;
        LQCD_TRY(drift(0.5 * eg));
        pend_g += (1.0 - 2.0 * lam) * eg;
        LQCD_TRY(drift(0.5 * eg));
        pend_g += lam * eg;
      }
    }
    return LQCD_OK;
  };
  const double eps = p->tau / p->nsteps;
  for (int k = 0; k < p->nsteps && rc == LQCD_OK; ++k) {
    if (p->scheme == LQCD_LEAPFROG) {
      pend_f += 0.5 * eps;
      rc = inner(eps);
      pend_f += 0.5 * eps;
    } else {
      pend_f += lam * eps;
      rc = inner(0.5 * eps);
      if (rc == LQCD_OK) {
        pend_f += (1.0 - 2.0 * lam) * eps;
        rc = inner(0.5 * eps);
      }
      pend_f += lam * eps;
    }
  }
  if (rc == LQCD_OK) rc = flush();
  if (copies_stale) {  // also after a failure: the master must not stay behind the double-float copy
    const int r2 = links_from_df(g);
    if (rc == LQCD_OK) rc = r2;
  }
  if (rc == LQCD_OK) rc = kinetic_impl(m, &kin1);
  if (rc == LQCD_OK) rc = lqcd_plaquette(g, &plaq1);
  const double V = 2.0 * g->g.Vh;
  const double sg0 = p->beta * 6.0 * V * (1.0 - plaq0), sg1 = p->beta * 6.0 * V * (1.0 - plaq1);
  const double h0 = kin0 + sg0 + sf0, h1 = kin1 + sg1 + sf1;
  int accepted = 1;
  if (rc == LQCD_OK && p->accept_u > 0.0) {
    accepted = std::log(p->accept_u) <= -(h1 - h0) ? 1 : 0;
    if (!accepted) {
      if (cudaMemcpyAsync(g->copy[P_F64][0], backup, ubytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        rc = set_error(LQCD_ECUDA, "link restore");
      else
        rc = refresh_gauge_copies(g);
    }
  }
  if (backup) {
    cudaStreamSynchronize(c->stream);
    cudaFree(backup);
  }
  if (rc != LQCD_OK && e) ctx_drop_engine(c);  // a failure may leave a request in the engine
  for (lqcd_field* f : {x, y, xd, yd, xprev, guess}) lqcd_field_destroy(f);
  if (info) {
    info->dH = h1 - h0;
    info->H0 = h0;
    info->H1 = h1;
    info->kinetic0 = kin0;
    info->kinetic1 = kin1;
    info->gauge0 = sg0;
    info->gauge1 = sg1;
    info->fermion0 = sf0;
    info->fermion1 = sf1;
    info->plaquette = accepted ? plaq1 : plaq0;
    info->accepted = accepted;
    info->force_evals = force_evals;
    info->solver_iters = solves_iters;
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

}  // extern "C"
