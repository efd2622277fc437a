// SU(3) helpers shared by the pure-gauge kernels (heatbath.cu) and the HMC kernels
// (hmc.cu): complex 3x3 matrices in registers, site coordinates of the even-odd index,
// and loads / stores of links in the FP64 18-real layout [parity][mu][word][V/2] of
// double2 (word = row * 3 + column).
#pragma once

#include "dslash.cuh"

namespace lqcd {
namespace gf {

struct C2 {
  double re, im;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C2 cmulc(C2 a, C2 b) {  // a * conj(b)
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.re + b.re, a.im + b.im}; }

struct M3 {
  C2 e[9];
};

// ---------------------------------------------------------------- geometry and links

struct Site {
  int c[4];
};

__device__ __forceinline__ Site site_of(const Geom& g, int par, int h) {
  Site s;
  const unsigned r0 = geom_div(g, 0, (unsigned)h);
  const int xh = h - (int)r0 * g.Lxh;
  const unsigned r1 = geom_div(g, 1, r0);
  s.c[1] = (int)r0 - (int)r1 * g.L[1];
  const unsigned r2 = geom_div(g, 2, r1);
  s.c[2] = (int)r1 - (int)r2 * g.L[2];
  s.c[3] = (int)r2;
  s.c[0] = 2 * xh + ((par + s.c[1] + s.c[2] + s.c[3]) & 1);
  return s;
}
__device__ __forceinline__ Site shifted(const Geom& g, Site s, int mu, int d) {
  int v = s.c[mu] + d;
  v = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
  s.c[mu] = v;
  return s;
}
// double2 index of word 0 of link (site, mu) in the FP64 18-real layout
__device__ __forceinline__ size_t link_base(const Geom& g, const Site& s, int mu) {
  const int par = (s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1;
  const int h = (s.c[0] >> 1) + g.Lxh * (s.c[1] + g.L[1] * (s.c[2] + g.L[2] * s.c[3]));
  return (size_t)(par * 4 + mu) * 9 * g.Vh + h;
}
__device__ __forceinline__ M3 load_link(const double2* U, const Geom& g, const Site& s, int mu) {
  const size_t b = link_base(g, s, mu);
  M3 m;
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const double2 d = U[b + (size_t)w * g.Vh];
    m.e[w] = {d.x, d.y};
  }
  return m;
}
__device__ __forceinline__ void store_link(double2* U, const Geom& g, const Site& s, int mu, const M3& m) {
  const size_t b = link_base(g, s, mu);
#pragma unroll
  for (int w = 0; w < 9; ++w) U[b + (size_t)w * g.Vh] = make_double2(m.e[w].re, m.e[w].im);
}

__device__ __forceinline__ M3 mul_nn(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C2 s = cmul(a.e[i * 3], b.e[j]);
      s = cadd(s, cmul(a.e[i * 3 + 1], b.e[3 + j]));
      s = cadd(s, cmul(a.e[i * 3 + 2], b.e[6 + j]));
      c.e[i * 3 + j] = s;
    }
  return c;
}
__device__ __forceinline__ M3 mul_nd(const M3& a, const M3& b) {  // a b^dag
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C2 s = cmulc(a.e[i * 3], b.e[j * 3]);
      s = cadd(s, cmulc(a.e[i * 3 + 1], b.e[j * 3 + 1]));
      s = cadd(s, cmulc(a.e[i * 3 + 2], b.e[j * 3 + 2]));
      c.e[i * 3 + j] = s;
    }
  return c;
}
__device__ __forceinline__ M3 mul_dn(const M3& a, const M3& b) {  // a^dag b
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C2 s = cmulc(b.e[j], a.e[i]);
      s = cadd(s, cmulc(b.e[3 + j], a.e[3 + i]));
      s = cadd(s, cmulc(b.e[6 + j], a.e[6 + i]));
      c.e[i * 3 + j] = s;
    }
  return c;
}

// ---------------------------------------------------------------- double-float matrices
// The FP64 pipes of this part run at 1/64 of the FP32 rate, so the SU(3) products of the
// gauge kernels run in double-float (pairs of FP32, 48-bit significand) on the FP32 pipes,
// reading the gauge field's double-float copy (float4 = (re.hi, re.lo, im.hi, im.lo) per
// complex entry, the same word layout as the FP64 master). Products accumulate unnormalised
// and each entry is normalised once.

// A double as an (unnormalised) double-float pair by integer operations on its bits, for
// kernels where the conversion instructions would load the FP64 pipe (1/64 of the FP32
// rate on this part): hi keeps the top 24 significant bits (truncated), lo the next 24 of
// the remaining 29 (truncated), so hi + lo is within 2^-47 relative of x and |lo| < ulp(hi).
// Exponents outside +-60 (including zero, subnormals, inf and NaN) take the FP64 path.
__device__ __forceinline__ df64 df_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int E = (int)((hw >> 20) & 0x7ffu);
  if (E < 1023 - 60 || E > 1023 + 60) return df64(x);
  const unsigned sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const unsigned rem = lw & 0x1fffffffu;  // weight 2^(E - 1075) per unit
  if (rem == 0u) return df64(hi, 0.0f);
  const int top = 31 - __clz((int)rem);  // leading bit, <= 28
  const unsigned m = top >= 23 ? rem >> (top - 23) : rem << (23 - top);
  const float lo = __uint_as_float(sign | ((unsigned)(top + E - 948) << 23) | (m & 0x7fffffu));
  return df64(hi, lo);
}

struct C2d {
  df64 re, im;
};
struct M3d {
  C2d e[9];
};

__device__ __forceinline__ M3d load_link_df(const float4* U, const Geom& g, const Site& s, int mu) {
  const size_t b = link_base(g, s, mu);
  M3d m;
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const float4 d = U[b + (size_t)w * g.Vh];
    m.e[w] = {df64(d.x, d.y), df64(d.z, d.w)};
  }
  return m;
}
__device__ __forceinline__ void store_link_df(float4* U, const Geom& g, const Site& s, int mu, const M3d& m) {
  const size_t b = link_base(g, s, mu);
#pragma unroll
  for (int w = 0; w < 9; ++w) U[b + (size_t)w * g.Vh] = make_float4(m.e[w].re.hi, m.e[w].re.lo, m.e[w].im.hi, m.e[w].im.lo);
}
__device__ __forceinline__ M3d to_df(const M3& a) {
  M3d m;
#pragma unroll
  for (int w = 0; w < 9; ++w) m.e[w] = {df64(a.e[w].re), df64(a.e[w].im)};
  return m;
}
__device__ __forceinline__ M3 to_double(const M3d& a) {
  M3 m;
#pragma unroll
  for (int w = 0; w < 9; ++w) m.e[w] = {(double)a.e[w].re, (double)a.e[w].im};
  return m;
}

// complex double-float scalars
__device__ __forceinline__ C2d cmul_d(const C2d& a, const C2d& b) {
  df64 re(0.0f, 0.0f), im(0.0f, 0.0f);
  df_mac_u(re, a.re, b.re);
  df_mac_u(re, -a.im, b.im);
  df_mac_u(im, a.re, b.im);
  df_mac_u(im, a.im, b.re);
  return {df_norm(re), df_norm(im)};
}
__device__ __forceinline__ C2d cadd_d(const C2d& a, const C2d& b) {
  return {df_norm(df_add_u(a.re, b.re)), df_norm(df_add_u(a.im, b.im))};
}
__device__ __forceinline__ C2d csub_d(const C2d& a, const C2d& b) { return cadd_d(a, {-b.re, -b.im}); }
__device__ __forceinline__ C2d cscale_d(df64 f, const C2d& a) { return {f * a.re, f * a.im}; }

// a x + b y in double-float
__device__ __forceinline__ C2d cmix_d(const C2d& a, const C2d& x, const C2d& b, const C2d& y) {
  df64 re(0.0f, 0.0f), im(0.0f, 0.0f);
  df_mac_u(re, a.re, x.re);
  df_mac_u(re, -a.im, x.im);
  df_mac_u(re, b.re, y.re);
  df_mac_u(re, -b.im, y.im);
  df_mac_u(im, a.re, x.im);
  df_mac_u(im, a.im, x.re);
  df_mac_u(im, b.re, y.im);
  df_mac_u(im, b.im, y.re);
  return {df_norm(re), df_norm(im)};
}

// 1/sqrt(n) for n > 0 in double-float: the FP32 estimate and two Newton-Raphson steps
// y <- y + y (1 - n y^2) / 2, each of which squares the relative error
__device__ __forceinline__ df64 df_rsqrt(df64 n) {
  df64 y(rsqrtf(n.hi), 0.0f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df64 r = df64(1.0f, 0.0f) - n * (y * y);
    y = y + y * r * df64(0.5f, 0.0f);
  }
  return y;
}

// c = a op(b) with op(b) = b (DAGB false) or b^dag; a^dag b when DAGA
template <bool DAGA, bool DAGB>
__device__ __forceinline__ M3d mul_d(const M3d& a, const M3d& b) {
  M3d c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      df64 re(0.0f, 0.0f), im(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const C2d x = DAGA ? a.e[k * 3 + i] : a.e[i * 3 + k];
        const C2d y = DAGB ? b.e[j * 3 + k] : b.e[k * 3 + j];
        // x' y' with x' = conj(x) when DAGA, y' = conj(y) when DAGB
        const df64 xi = DAGA ? -x.im : x.im, yi = DAGB ? -y.im : y.im;
        df_mac_u(re, x.re, y.re);
        df_mac_u(re, -xi, yi);
        df_mac_u(im, x.re, yi);
        df_mac_u(im, xi, y.re);
      }
      c.e[i * 3 + j] = {df_norm(re), df_norm(im)};
    }
  return c;
}

// w += a op(b) in double-float: each entry accumulates unnormalised over k and is
// normalised once (the layout of mul_d, without the intermediate matrix)
template <bool DAGA, bool DAGB>
__device__ __forceinline__ void mac_d(M3d& w, const M3d& a, const M3d& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      df64 re = w.e[i * 3 + j].re, im = w.e[i * 3 + j].im;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const C2d x = DAGA ? a.e[k * 3 + i] : a.e[i * 3 + k];
        const C2d y = DAGB ? b.e[j * 3 + k] : b.e[k * 3 + j];
        const df64 xi = DAGA ? -x.im : x.im, yi = DAGB ? -y.im : y.im;
        df_mac_u(re, x.re, y.re);
        df_mac_u(re, -xi, yi);
        df_mac_u(im, x.re, yi);
        df_mac_u(im, xi, y.re);
      }
      w.e[i * 3 + j] = {df_norm(re), df_norm(im)};
    }
}

// m or m^dag, chosen at run time (selects on registers)
__device__ __forceinline__ M3d dagger_if(const M3d& m, bool dag) {
  M3d r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const C2d a = m.e[i * 3 + j], b = m.e[j * 3 + i];
      r.e[i * 3 + j] = dag ? C2d{b.re, -b.im} : a;
    }
  return r;
}

// coordinate nu of s and the site shifted by d in direction nu, for a direction known only
// at run time (selects, so that the site stays in registers)
__device__ __forceinline__ int coord(const Site& s, int nu) {
  return nu == 0 ? s.c[0] : (nu == 1 ? s.c[1] : (nu == 2 ? s.c[2] : s.c[3]));
}
__device__ __forceinline__ Site shifted_rt(const Geom& g, Site s, int nu, int d) {
  const int L = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
  int v = coord(s, nu) + d;
  v = v < 0 ? v + L : (v >= L ? v - L : v);
#pragma unroll
  for (int k = 0; k < 4; ++k) s.c[k] = (nu == k) ? v : s.c[k];
  return s;
}

// The staple sum W_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                                         + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
// for a direction mu known at run time, in double-float from the copy Ud. The six staples
// run through one loop body of two products
//   up (nu):   T = U_nu(x+mu) U_mu(x+nu)^dag,          W += T U_nu(x)^dag
//   down (nu): T = U_nu(x+mu-nu)^dag U_mu(x-nu)^dag,   W += T U_nu(x-nu)
// so that the instructions of the loop stay in the instruction cache (fully unrolled, at
// about 1400 instructions per double-float product, the staple sum did not).
__device__ __forceinline__ M3d staple_df(const float4* Ud, const Geom& g, const Site& x, int mu) {
  M3d W;
#pragma unroll
  for (int i = 0; i < 9; ++i) W.e[i] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
  const Site xp = shifted_rt(g, x, mu, 1);
#pragma unroll 1
  for (int t = 0; t < 6; ++t) {
    const int k = t >> 1, nu = k + (k >= mu ? 1 : 0);
    const bool up = (t & 1) == 0;
    const Site s0 = up ? xp : shifted_rt(g, xp, nu, -1);
    const Site s1 = shifted_rt(g, x, nu, up ? 1 : -1);
    const Site s2 = up ? x : s1;
    const M3d T = mul_d<false, true>(dagger_if(load_link_df(Ud, g, s0, nu), !up), load_link_df(Ud, g, s1, mu));
    mac_d<false, false>(W, T, dagger_if(load_link_df(Ud, g, s2, nu), up));
  }
  return W;
}

}  // namespace gf
}  // namespace lqcd
