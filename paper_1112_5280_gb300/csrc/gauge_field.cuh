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
  const int xh = h % g.Lxh;
  int r = h / g.Lxh;
  s.c[1] = r % g.L[1];
  r /= g.L[1];
  s.c[2] = r % g.L[2];
  s.c[3] = r / g.L[2];
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

// W_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
template <int mu>
__device__ __forceinline__ M3 staple(const double2* U, const Geom& g, const Site& x) {
  M3 W;
#pragma unroll
  for (int i = 0; i < 9; ++i) W.e[i] = {0.0, 0.0};
  const Site xp = shifted(g, x, mu, 1);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const Site xn = shifted(g, x, nu, 1), xm = shifted(g, x, nu, -1), xpm = shifted(g, xp, nu, -1);
    const M3 up = mul_nd(mul_nd(load_link(U, g, xp, nu), load_link(U, g, xn, mu)), load_link(U, g, x, nu));
    const M3 lo = mul_dn(mul_nn(load_link(U, g, xm, mu), load_link(U, g, xpm, nu)), load_link(U, g, xm, nu));
#pragma unroll
    for (int i = 0; i < 9; ++i) W.e[i] = cadd(W.e[i], cadd(up.e[i], lo.e[i]));
  }
  return W;
}

}  // namespace gf
}  // namespace lqcd
