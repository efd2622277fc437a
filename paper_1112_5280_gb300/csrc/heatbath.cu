// Pure-gauge SU(3) heatbath and plaquette (paper Section 3: the pure-gauge side needs an
// SU(3) heatbath, citing Creutz). The sweeps run on the gauge field's double-float copy
// (the matrix algebra in double-float on the FP32 pipes, the draws in FP64); the FP64 master
// is rebuilt from it at the end of the call.
//
// Wilson action S = beta sum_P (1 - Re Tr U_P / 3). A sweep updates the links class by
// class, mu = 0..3 and parity even, odd: the links U_mu(x) of one class share no staple,
// so one thread per link updates a class in one launch. Each link is updated by
// Cabibbo-Marinari over the SU(2) subgroups on index pairs (0,1), (1,2), (0,2): with
// V = U W (W the staple sum) and the subgroup block X of V, Re Tr(a X) = a.c for
// a = a0 + i a.sigma, k = |c|, v = c / k; b is drawn with density
// exp(beta k b0 / 3) on the 3-sphere by Creutz's method (b0 = 1 + ln(y) / alpha with y
// uniform in (exp(-2 alpha), 1], accepted with probability sqrt(1 - b0^2), uniform
// direction), a = b v, and U <- R U, R the embedding of a. Every sweep ends with a
// reunitarisation (Gram-Schmidt of rows 0, 1; row 2 = conj(row0 x row1)) when asked.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), key (seed, 0),
// counter (4 s + mu, sweep, subgroup, attempt) with s = x + Lx (y + Ly (z + Lz t)),
// u = ((r >> 11) + 1) 2^-53; four uniforms per attempt (b0, acceptance, cos theta,
// phi). So a sweep's result depends on (seed, sweep) and the links only, not on the
// launch shape. At most 1000 attempts per draw: a subgroup that never accepts is left
// unchanged and counted (the count is returned).
#include <cmath>
#include <cstring>

#include "gauge_field.cuh"
#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {
namespace {

using namespace gf;

constexpr int HB_THREADS = 128;
constexpr int HB_MAX_ATTEMPTS = 1000;

// ---------------------------------------------------------------- Philox4x64-10

__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// u = ((r >> 11) + 1) 2^-53 in (0, 1], built from its bits by integer operations (the same
// value as the FP64 expression, which would convert a 64-bit integer on the FP64 pipe)
__device__ __forceinline__ double unit_open0(uint64_t r) {
  const uint64_t k = (r >> 11) + 1;  // 1 .. 2^53
  const int p = 63 - __clzll((long long)k);
  if (p == 53) return 1.0;
  const uint64_t mant = (k << (52 - p)) & ((1ULL << 52) - 1);
  return __longlong_as_double((long long)(((uint64_t)(p + 970) << 52) | mant));
}
// the same u rounded toward zero to 24 bits (relative error below 2^-23), for FP32 work
__device__ __forceinline__ float unit_open0_f(uint64_t r) {
  const uint64_t k = (r >> 11) + 1;
  const int p = 63 - __clzll((long long)k);
  const unsigned m = (unsigned)(p >= 23 ? k >> (p - 23) : k << (23 - p));
  return __uint_as_float(((unsigned)(p + 74) << 23) | (m & 0x7fffffu));
}

// Creutz's SU(2) draw; false after HB_MAX_ATTEMPTS. The accept test u1^2 <= 1 - b0^2 is an
// FP64 decision; it is first evaluated in FP32 with t = 1 - b0 = -log1p(-u0 span) / alpha,
// 1 - b0^2 = t (2 - t), and taken from there only when the FP32 margin is beyond the FP32
// error (the bound: u's to 2^-23, span to ~2^-22, log1p conditioned by at most 150 while
// u0 span <= 1 - 2^-10, so |error of 1 - b0^2| < 2.2e-4 against a margin of 2^-11); every
// other attempt, and the accepted one's b, are computed in FP64 exactly as before.
__device__ __noinline__ bool su2_draw(double alpha, uint64_t seed, uint64_t c0, uint64_t c1, uint64_t c2, double b[4]) {
  const bool flat = alpha < 1e-12;  // uniform b0 in the alpha -> 0 limit
  const float af = (float)alpha;
  const float span_f = flat ? 0.0f : -expm1f(-2.0f * af);
  double span = -1.0;  // the FP64 1 - exp(-2 alpha), computed on first use
  for (int attempt = 0; attempt < HB_MAX_ATTEMPTS; ++attempt) {
    uint64_t r[4] = {c0, c1, c2, (uint64_t)attempt};
    philox4x64(r, seed, 0);
    int verdict = -1;  // 1 accept, 0 reject, -1 undecided in FP32
    {
      const float u0f = unit_open0_f(r[0]), u1f = unit_open0_f(r[1]);
      float s2f;
      bool ok = true;
      if (flat) {
        const float b0f = 1.0f - 2.0f * u0f;
        s2f = 1.0f - b0f * b0f;
      } else {
        const float xf = u0f * span_f;
        ok = xf <= 1.0f - 0x1.0p-10f;
        const float tf = -log1pf(-xf) / af;
        s2f = tf * (2.0f - tf);
      }
      const float d = u1f * u1f - s2f;
      if (ok && isfinite(d) && fabsf(d) > 0x1.0p-11f) verdict = d < 0.0f ? 1 : 0;
    }
    if (verdict == 0) continue;
    const double u0 = unit_open0(r[0]);
    double b0;
    if (flat) {
      b0 = 1.0 - 2.0 * u0;
    } else {
      if (span < 0.0) span = -expm1(-2.0 * alpha);
      b0 = 1.0 + log1p(-u0 * span) / alpha;
    }
    const double s2 = 1.0 - b0 * b0;
    if (verdict == -1) {
      const double u1 = unit_open0(r[1]);
      if (!(u1 * u1 <= s2)) continue;
    }
    const double u2 = unit_open0(r[2]), u3 = unit_open0(r[3]);
    const double rr = sqrt(fmax(s2, 0.0));
    const double ct = 2.0 * u2 - 1.0;
    const double st = sqrt(fmax(1.0 - ct * ct, 0.0));
    double sp, cp;
    sincospi(2.0 * u3, &sp, &cp);
    b[0] = b0;
    b[1] = rr * st * cp;
    b[2] = rr * st * sp;
    b[3] = rr * ct;
    return true;
  }
  return false;
}

// The SU(3) and SU(2) algebra (staple sum, V = U W, the subgroup projection c and its
// direction v = c / |c|, a = b v, the rotations of U and V) in double-float from the copy Ud
// on the FP32 pipes; the draw of b (Creutz) and |c| in FP64. The updated link goes to Ud
// only: the caller rebuilds the FP64 master from it.
// 3 CTAs of 128 threads per SM (168 registers, a 100-byte spill) against 2 (254 registers,
// no spill): measured on GB300 at 32^3x64 beta 6, 39.7 against 43.2 ms per sweep with the
// same chain; the update is latency bound, so the extra warps outweigh the spill. At 4 CTAs
// (128 registers) the spill grows and the sweep takes 40.1 ms.
#ifndef LQCD_HB_MIN_BLOCKS
#define LQCD_HB_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(HB_THREADS, LQCD_HB_MIN_BLOCKS) k_heatbath(float4* Ud, Geom g, int mu,
                                                                             int par, double beta, uint64_t seed,
                                                                             uint64_t sweep,
                                                                             unsigned long long* fails) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.Vh) return;
  const Site x = site_of(g, par, h);
  M3d u = load_link_df(Ud, g, x, mu);
  M3d V = mul_d<false, false>(u, staple_df(Ud, g, x, mu));
  const uint64_t s = (uint64_t)x.c[0] + (uint64_t)g.L[0] * ((uint64_t)x.c[1] + (uint64_t)g.L[1] *
                     ((uint64_t)x.c[2] + (uint64_t)g.L[2] * (uint64_t)x.c[3]));
  const uint64_t link_id = 4 * s + (uint64_t)mu;
  int nfail = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = k == 1 ? 1 : 0, j = k == 0 ? 1 : 2;  // (0,1), (1,2), (0,2)
    // c (the SU(2) projection of the block) and |c|^2 in double-float; k = |c|, 1 / k and
    // alpha = beta k / 3 in FP64 (the draw's input); v = c / k in double-float
    const C2d x00 = V.e[i * 3 + i], x01 = V.e[i * 3 + j], x10 = V.e[j * 3 + i], x11 = V.e[j * 3 + j];
    const df64 c[4] = {df_norm(df_add_u(x00.re, x11.re)), -df_norm(df_add_u(x01.im, x10.im)),
                       df_norm(df_add_u(x10.re, -x01.re)), -df_norm(df_add_u(x00.im, -x11.im))};
    df64 k2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) df_mac_u(k2, c[q], c[q]);
    const double kk = sqrt((double)df_norm(k2));
    df64 v[4] = {df64(1.0f, 0.0f), df64(0.0f, 0.0f), df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
    if (kk > 0.0) {
      const df64 ik = df_split_bits(1.0 / kk);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = c[q] * ik;
    }
    double bd[4];
    if (!su2_draw(beta * kk / 3.0, seed, link_id, sweep, (uint64_t)k, bd)) {
      ++nfail;
      continue;
    }
    const df64 b[4] = {df_split_bits(bd[0]), df_split_bits(bd[1]), df_split_bits(bd[2]), df_split_bits(bd[3])};
    // a = b v with mat(q) = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
    const C2d B[4] = {{b[0], b[3]}, {b[2], b[1]}, {-b[2], b[1]}, {b[0], -b[3]}};
    const C2d Vm[4] = {{v[0], v[3]}, {v[2], v[1]}, {-v[2], v[1]}, {v[0], -v[3]}};
    C2d A[4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q) A[r * 2 + q] = cmix_d(B[r * 2], Vm[q], B[r * 2 + 1], Vm[2 + q]);
    // U <- R U and V <- R V (rows i, j; V is not needed after the last subgroup)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const C2d ui = u.e[i * 3 + col], uj = u.e[j * 3 + col];
      u.e[i * 3 + col] = cmix_d(A[0], ui, A[1], uj);
      u.e[j * 3 + col] = cmix_d(A[2], ui, A[3], uj);
      if (k < 2) {
        const C2d vi = V.e[i * 3 + col], vj = V.e[j * 3 + col];
        V.e[i * 3 + col] = cmix_d(A[0], vi, A[1], vj);
        V.e[j * 3 + col] = cmix_d(A[2], vi, A[3], vj);
      }
    }
  }
  store_link_df(Ud, g, x, mu, u);
  if (nfail) atomicAdd(fails, (unsigned long long)nfail);
}

// FP64 master words from the double-float copy (hi + lo, exact in FP64)
__global__ void k_master_from_df(double2* U, const float4* Ud, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 d = Ud[i];
  U[i] = make_double2((double)d.x + (double)d.y, (double)d.z + (double)d.w);
}

// Gram-Schmidt of rows 0 and 1, row 2 = conj(row0 x row1), in double-float on the copy Ud
__global__ void k_reunitarise(float4* Ud, Geom g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (par, mu, h)
  if (i >= 8LL * g.Vh) return;
  const int h = (int)(i % g.Vh);
  const size_t base = (size_t)(i / g.Vh) * 9 * g.Vh + h;
  C2d r[9];
#pragma unroll
  for (int w = 0; w < 6; ++w) {
    const float4 d = Ud[base + (size_t)w * g.Vh];
    r[w] = {df64(d.x, d.y), df64(d.z, d.w)};
  }
  auto normalise_row = [&](int o) {
    df64 n(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      df_mac_u(n, r[o + c].re, r[o + c].re);
      df_mac_u(n, r[o + c].im, r[o + c].im);
    }
    const df64 s = df_rsqrt(df_norm(n));
#pragma unroll
    for (int c = 0; c < 3; ++c) r[o + c] = cscale_d(s, r[o + c]);
  };
  normalise_row(0);
  C2d p = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};  // <row0, row1> = sum row1 conj(row0)
#pragma unroll
  for (int c = 0; c < 3; ++c) p = cadd_d(p, cmul_d(r[3 + c], {r[c].re, -r[c].im}));
#pragma unroll
  for (int c = 0; c < 3; ++c) r[3 + c] = csub_d(r[3 + c], cmul_d(p, r[c]));
  normalise_row(3);
  // row 2 = conj(row0 x row1)
  auto cr = [&](int a, int b, int c, int d) {
    const C2d x = csub_d(cmul_d(r[a], r[b]), cmul_d(r[c], r[d]));
    return C2d{x.re, -x.im};
  };
  r[6] = cr(1, 5, 2, 4);
  r[7] = cr(2, 3, 0, 5);
  r[8] = cr(0, 4, 1, 3);
#pragma unroll
  for (int w = 0; w < 9; ++w)
    Ud[base + (size_t)w * g.Vh] = make_float4(r[w].re.hi, r[w].re.lo, r[w].im.hi, r[w].im.lo);
}

// per-CTA partial of sum_{x, mu<nu} Re Tr U_munu(x) over the sites of both parities
constexpr int PLAQ_THREADS = 256;
__global__ void __launch_bounds__(PLAQ_THREADS) k_plaquette(const double2* U, Geom g, double* partials) {
  __shared__ double red[PLAQ_THREADS];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (par, h)
  double acc = 0.0;
  if (i < 2LL * g.Vh) {
    const Site x = site_of(g, (int)(i / g.Vh), (int)(i % g.Vh));
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const M3 a = mul_nn(load_link(U, g, x, mu), load_link(U, g, shifted(g, x, mu, 1), nu));
        const M3 b = mul_nn(load_link(U, g, x, nu), load_link(U, g, shifted(g, x, nu, 1), mu));
        double tr = 0.0;
#pragma unroll
        for (int w = 0; w < 9; ++w) tr += a.e[w].re * b.e[w].re + a.e[w].im * b.e[w].im;  // Re Tr a b^dag
        acc += tr;
      }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = PLAQ_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// out = sum of n partials in a fixed order (one CTA, strided then tree)
__global__ void k_sum_ordered(const double* partials, int n, double* out) {
  __shared__ double red[PLAQ_THREADS];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += PLAQ_THREADS) acc += partials[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = PLAQ_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// FP64 18-real layout -> host AoS U[s][mu][row][col] (re, im)
__global__ void k_gauge_to_aos(const double2* U, Geom g, double2* aos) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (par, h)
  if (i >= 2LL * g.Vh) return;
  const Site x = site_of(g, (int)(i / g.Vh), (int)(i % g.Vh));
  const size_t s = (size_t)x.c[0] + (size_t)g.L[0] * (x.c[1] + (size_t)g.L[1] * (x.c[2] + (size_t)g.L[2] * x.c[3]));
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const size_t b = link_base(g, x, mu);
#pragma unroll
    for (int w = 0; w < 9; ++w) aos[(s * 4 + mu) * 9 + w] = U[b + (size_t)w * g.Vh];
  }
}

}  // namespace

// derived link copies follow the master after an update
// keep_df: the double-float copy is already current (the master was built from it)
int refresh_gauge_copies(lqcd_gauge* g, bool keep_df) {
  for (int p = 0; p < NPREC; ++p)
    for (int c = 0; c < 2; ++c) {
      if (p == P_F64 && c == 0) continue;
      if (keep_df && p == P_DF64 && c == 0) continue;
      if (!g->copy[p][c]) continue;
      LQCD_CK(gauge_convert(g->copy[P_F64][0], g->g, p, c ? 12 : 18, g->copy[p][c], g->ctx->stream));
    }
  return LQCD_OK;
}

int links_from_df(lqcd_gauge* g) {
  const float4* Ud = static_cast<const float4*>(g->copy[P_DF64][0]);
  if (!Ud) return set_error(LQCD_EINVAL, "the gauge field has no double-float copy");
  const long long n = 2LL * 4 * 9 * g->g.Vh;
  k_master_from_df<<<(unsigned)((n + 255) / 256), 256, 0, g->ctx->stream>>>(
      static_cast<double2*>(g->copy[P_F64][0]), Ud, n);
  g->ctx->launches++;
  LQCD_CK(cudaGetLastError());
  return refresh_gauge_copies(g, true);
}

cudaError_t links_to_aos(const double2* U, const Geom& g, double2* aos, cudaStream_t s) {
  k_gauge_to_aos<<<(unsigned)((2LL * g.Vh + 255) / 256), 256, 0, s>>>(U, g, aos);
  return cudaGetLastError();
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_heatbath(lqcd_gauge* g, double beta, int nsweeps, unsigned long long seed,
                  unsigned long long sweep0, int reunit, long long* fails_out) {
  LQCD_TRACE("lqcd_heatbath");
  clear_error();
  if (!g) return set_error(LQCD_EINVAL, "gauge is NULL");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return set_error(LQCD_EINVAL, "beta must be finite and >= 0");
  if (nsweeps < 0) return set_error(LQCD_EINVAL, "nsweeps %d", nsweeps);
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  LQCD_TRY(ctx_partials(c, 1));
  unsigned long long* d_fails = reinterpret_cast<unsigned long long*>(c->partials);
  LQCD_CK(cudaMemsetAsync(d_fails, 0, sizeof(unsigned long long), st));
  double2* U = static_cast<double2*>(g->copy[P_F64][0]);
  // the double-float copy the sweeps work on, rebuilt from the master at the start
  const void* dfbase;
  int dfnr;
  LQCD_TRY(gauge_links(g, P_DF64, &dfbase, &dfnr));
  float4* Ud = static_cast<float4*>(const_cast<void*>(dfbase));
  LQCD_CK(gauge_convert(U, g->g, P_DF64, 18, Ud, st));
  const unsigned grid = (unsigned)((g->g.Vh + HB_THREADS - 1) / HB_THREADS);
  const unsigned rgrid = (unsigned)((8LL * g->g.Vh + 255) / 256);
  for (int sw = 0; sw < nsweeps; ++sw) {
    const uint64_t sweep = (uint64_t)(sweep0 + (unsigned long long)sw);
    for (int mu = 0; mu < 4; ++mu)
      for (int par = 0; par < 2; ++par) {
        k_heatbath<<<grid, HB_THREADS, 0, st>>>(Ud, g->g, mu, par, beta, seed, sweep, d_fails);
        c->launches++;
      }
    if (reunit) {
      k_reunitarise<<<rgrid, 256, 0, st>>>(Ud, g->g);
      c->launches++;
    }
    LQCD_CK(cudaGetLastError());
  }
  LQCD_TRY(links_from_df(g));  // the sweeps moved the double-float copy only
  unsigned long long fails = 0;
  LQCD_CK(cudaMemcpyAsync(&fails, d_fails, sizeof fails, cudaMemcpyDeviceToHost, st));
  LQCD_CK(cudaStreamSynchronize(st));
  if (fails_out) *fails_out = (long long)fails;
  return LQCD_OK;
}

int lqcd_plaquette(const lqcd_gauge* g, double* plaq) {
  LQCD_TRACE("lqcd_plaquette");
  clear_error();
  if (!g || !plaq) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  const int nb = (int)((2LL * g->g.Vh + PLAQ_THREADS - 1) / PLAQ_THREADS);
  LQCD_TRY(ctx_partials(c, (size_t)nb + 1));
  k_plaquette<<<nb, PLAQ_THREADS, 0, st>>>(static_cast<const double2*>(g->copy[P_F64][0]), g->g, c->partials);
  k_sum_ordered<<<1, PLAQ_THREADS, 0, st>>>(c->partials, nb, c->partials + nb);
  c->launches += 2;
  LQCD_CK(cudaGetLastError());
  double sum = 0.0;
  LQCD_CK(cudaMemcpyAsync(&sum, c->partials + nb, sizeof sum, cudaMemcpyDeviceToHost, st));
  LQCD_CK(cudaStreamSynchronize(st));
  *plaq = sum / (18.0 * 2.0 * (double)g->g.Vh);
  return LQCD_OK;
}

int lqcd_gauge_download(const lqcd_gauge* g, double* host_U) {
  LQCD_TRACE("lqcd_gauge_download");
  clear_error();
  if (!g || !host_U) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  const size_t bytes = (size_t)2 * g->g.Vh * 4 * 18 * sizeof(double);
  LQCD_TRY(ctx_staging(c, bytes));
  LQCD_CK(links_to_aos(static_cast<const double2*>(g->copy[P_F64][0]), g->g,
                       reinterpret_cast<double2*>(c->staging), c->stream));
  c->launches++;
  LQCD_CK(cudaMemcpyAsync(host_U, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

}  // extern "C"
