// The even-odd Wilson hopping term at one output site.
//
// D_{pq} psi (x) = sum_mu [ eta (1 - g_mu) U_mu(x) psi(x+mu)
//                         + eta (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ],   x of parity p
// (paper Section 3: the even-odd preconditioned "dslash"; the operator itself
// is the textbook Wilson term with r = 1). eta = t_bc for hops across the t
// boundary, applied to the hop and never folded into the links, so the
// 12-real reconstruction stays valid. D^dag swaps the two projectors.
//
// Chiral basis: g_k = [[0, A_k], [A_k^dag, 0]] with A_k = -i sigma_k
// (mu = 0, 1, 2) and A_t = 1, so g5 = diag(1, 1, -1, -1). The projector
// (1 + s g_mu), s = +-1, has rank two:
//   (1 + s g) psi = [ h ; s A^dag h ],   h = psi_up + s A psi_dn,
// so each hop projects to a half spinor h (2 spin x 3 colour), multiplies the
// two colour vectors by the link, and rebuilds the lower spin components.
#pragma once

#include <type_traits>

#include "field.cuh"

namespace lqcd {

struct Geom {
  int L[4];  // Lx, Ly, Lz, Lt (all even)
  int Lxh;   // Lx / 2
  int Vh;    // V / 2 sites per parity
  int t_bc;  // +1 periodic, -1 antiperiodic in t
  // Division by the radices Lxh, Ly, Lz of the half-lattice index without a divide
  // instruction (Granlund and Montgomery, "Division by invariant integers using
  // multiplication", PLDI 1994, Figure 4.1): for divisor d with l = ceil(log2 d),
  // m = floor(2^32 (2^l - d) / d) + 1, and every 32-bit n,
  //   n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),  t = (m n) >> 32.
  unsigned dm[3];  // m for Lxh, Ly, Lz
  int dsh[3];      // min(l, 1) | max(l - 1, 0) << 8
};

// n / d for radix k (0: Lxh, 1: Ly, 2: Lz) of the geometry
__host__ __device__ __forceinline__ unsigned geom_div(const Geom& g, int k, unsigned n) {
#ifdef __CUDA_ARCH__
  const unsigned t = __umulhi(g.dm[k], n);
#else
  const unsigned t = (unsigned)(((unsigned long long)g.dm[k] * n) >> 32);
#endif
  return (t + ((n - t) >> (g.dsh[k] & 0xff))) >> (g.dsh[k] >> 8);
}

// the constants of geom_div for divisor d >= 1
inline void geom_set_divisor(Geom& g, int k, unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  g.dm[k] = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  g.dsh[k] = (l < 1 ? l : 1) | ((l > 1 ? l - 1 : 0) << 8);
}

// Half-lattice index h = xh + Lxh*(y + Ly*(z + Lz*t)) with x = 2 xh + ((p+y+z+t) & 1).
__device__ __forceinline__ void neighbours(const Geom& g, int h, int par, int nf[4], int nb[4],
                                           int& t) {
  const unsigned r0 = geom_div(g, 0, (unsigned)h);
  const int xh = h - (int)r0 * g.Lxh;
  const unsigned r1 = geom_div(g, 1, r0);
  const int y = (int)r0 - (int)r1 * g.L[1];
  const unsigned r2 = geom_div(g, 2, r1);
  const int z = (int)r1 - (int)r2 * g.L[2];
  t = (int)r2;
  const int x = 2 * xh + ((par + y + z + t) & 1);
  const int rest = h - xh;
  const int xp = (x + 1 == g.L[0]) ? 0 : x + 1;
  const int xm = (x == 0) ? g.L[0] - 1 : x - 1;
  nf[0] = rest + (xp >> 1);
  nb[0] = rest + (xm >> 1);
  const int sy = g.Lxh;
  nf[1] = (y + 1 == g.L[1]) ? h - (g.L[1] - 1) * sy : h + sy;
  nb[1] = (y == 0) ? h + (g.L[1] - 1) * sy : h - sy;
  const int sz = sy * g.L[1];
  nf[2] = (z + 1 == g.L[2]) ? h - (g.L[2] - 1) * sz : h + sz;
  nb[2] = (z == 0) ? h + (g.L[2] - 1) * sz : h - sz;
  const int st = sz * g.L[2];
  nf[3] = (t + 1 == g.L[3]) ? h - (g.L[3] - 1) * st : h + st;
  nb[3] = (t == 0) ? h + (g.L[3] - 1) * st : h - st;
}

template <typename R>
__device__ __forceinline__ Cx<R> sp(const R* v, int spin, int col) {
  return {v[sidx(spin, col)], v[sidx(spin, col) + 1]};
}
template <typename R>
__device__ __forceinline__ void acc_add(R* a, int spin, int col, Cx<R> w) {
  a[sidx(spin, col)] = f_add(a[sidx(spin, col)], w.re);
  a[sidx(spin, col) + 1] = f_add(a[sidx(spin, col) + 1], w.im);
}
// i * w
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> w) {
  return {-w.im, w.re};
}
// S * w for a compile-time sign S = +-1
template <int S, typename R>
__device__ __forceinline__ Cx<R> sgn(Cx<R> w) {
  if (S > 0) return w;
  return {-w.re, -w.im};
}

// Spin projection of one hop: h = psi_up + S A psi_dn (the rows of (1 + S g_MU) that carry
// information), times eta = +-1 (the t-boundary sign).
// a + S b for a compile-time sign S = +-1 (an add or a subtract, no product)
template <int S, typename R>
__device__ __forceinline__ R pm(R a, R b) {
  return S > 0 ? f_add(a, b) : f_sub(a, b);
}

template <int MU, int S, typename R>
__device__ __forceinline__ void project(const R psi[24], int eta, Cx<R> h0[3], Cx<R> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<R> p0 = sp(psi, 0, c), p1 = sp(psi, 1, c), p2 = sp(psi, 2, c), p3 = sp(psi, 3, c);
    if (MU == 0) {  // h = psi_up + S (-i sigma_1) psi_dn
      h0[c] = {pm<S>(p0.re, p3.im), pm<-S>(p0.im, p3.re)};
      h1[c] = {pm<S>(p1.re, p2.im), pm<-S>(p1.im, p2.re)};
    } else if (MU == 1) {  // -i sigma_2 = [[0,-1],[1,0]]
      h0[c] = {pm<-S>(p0.re, p3.re), pm<-S>(p0.im, p3.im)};
      h1[c] = {pm<S>(p1.re, p2.re), pm<S>(p1.im, p2.im)};
    } else if (MU == 2) {  // -i sigma_3 = diag(-i, i)
      h0[c] = {pm<S>(p0.re, p2.im), pm<-S>(p0.im, p2.re)};
      h1[c] = {pm<-S>(p1.re, p3.im), pm<S>(p1.im, p3.re)};
    } else {  // identity
      h0[c] = {pm<S>(p0.re, p2.re), pm<S>(p0.im, p2.im)};
      h1[c] = {pm<S>(p1.re, p3.re), pm<S>(p1.im, p3.im)};
    }
    if (MU == 3 && eta < 0) {
      h0[c] = sgn<-1>(h0[c]);
      h1[c] = sgn<-1>(h1[c]);
    }
  }
}

// The same projection on FP16 storage words, in packed half2 arithmetic: word c of a site
// holds colour c as (spin 0, 1, 2, 3) x (re, im) half2 pairs. One FP16 rounding per
// component of h; only the 6 complex numbers of h are then converted to FP32 (instead of
// the 12 of psi).
template <int MU, int S>
__device__ __forceinline__ void project_h2(const uint4 w[3], int eta, Cx<float> h0[3], Cx<float> h1[3]) {
  // (S, -S): multiplies the swapped pair (im, re) into S * (-i) * (re + i im) = S (im, -re)
  const __half2 mi = __floats2half2_rn(float(S), float(-S));
  const __half2 pi = __floats2half2_rn(float(-S), float(S));  // S * i * p = S (-im, re)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const __half2 p0 = *reinterpret_cast<const __half2*>(&w[c].x);
    const __half2 p1 = *reinterpret_cast<const __half2*>(&w[c].y);
    const __half2 p2 = *reinterpret_cast<const __half2*>(&w[c].z);
    const __half2 p3 = *reinterpret_cast<const __half2*>(&w[c].w);
    __half2 a, b;
    if (MU == 0) {
      a = __hfma2(__lowhigh2highlow(p3), mi, p0);
      b = __hfma2(__lowhigh2highlow(p2), mi, p1);
    } else if (MU == 1) {
      a = S > 0 ? __hsub2(p0, p3) : __hadd2(p0, p3);
      b = S > 0 ? __hadd2(p1, p2) : __hsub2(p1, p2);
    } else if (MU == 2) {
      a = __hfma2(__lowhigh2highlow(p2), mi, p0);
      b = __hfma2(__lowhigh2highlow(p3), pi, p1);
    } else {
      a = S > 0 ? __hadd2(p0, p2) : __hsub2(p0, p2);
      b = S > 0 ? __hadd2(p1, p3) : __hsub2(p1, p3);
    }
    if (MU == 3 && eta < 0) {
      a = __hneg2(a);
      b = __hneg2(b);
    }
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    h0[c] = {fa.x, fa.y};
    h1[c] = {fb.x, fb.y};
  }
}

// The rest of a hop: acc += (U or U^dag) h, lifted back to four spins by (1 + S g_MU).
template <int MU, int S, bool ADJ, typename R>
__device__ __forceinline__ void hop_half(const Cx<R> h0[3], const Cx<R> h1[3], const R u[18], R acc[24]) {
  // w = U h (or U^dag h) per spin row: for each product u h, re += u.re h.re - u.im h.im and
  // im += u.re h.im + u.im h.re, as four multiply-adds in this order
  Cx<R> w0[3], w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s0, s1;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<R> uab = ADJ ? Cx<R>{u[(b * 3 + a) * 2], -u[(b * 3 + a) * 2 + 1]}
                            : Cx<R>{u[(a * 3 + b) * 2], u[(a * 3 + b) * 2 + 1]};
      if (b == 0) {
        s0 = {f_mul(uab.re, h0[b].re), f_mul(uab.re, h0[b].im)};
        s1 = {f_mul(uab.re, h1[b].re), f_mul(uab.re, h1[b].im)};
      } else {
        s0 = {f_fma(uab.re, h0[b].re, s0.re), f_fma(uab.re, h0[b].im, s0.im)};
        s1 = {f_fma(uab.re, h1[b].re, s1.re), f_fma(uab.re, h1[b].im, s1.im)};
      }
      s0 = {f_fma(-uab.im, h0[b].im, s0.re), f_fma(uab.im, h0[b].re, s0.im)};
      s1 = {f_fma(-uab.im, h1[b].im, s1.re), f_fma(uab.im, h1[b].re, s1.im)};
    }
    w0[a] = s0;
    w1[a] = s1;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc_add(acc, 0, a, w0[a]);
    acc_add(acc, 1, a, w1[a]);
    if (MU == 0) {  // lower = S A^dag h, A^dag = [[0,i],[i,0]]
      acc_add(acc, 2, a, sgn<S>(mul_i(w1[a])));
      acc_add(acc, 3, a, sgn<S>(mul_i(w0[a])));
    } else if (MU == 1) {  // A^dag = [[0,1],[-1,0]]
      acc_add(acc, 2, a, sgn<S>(w1[a]));
      acc_add(acc, 3, a, sgn<-S>(w0[a]));
    } else if (MU == 2) {  // A^dag = diag(i, -i)
      acc_add(acc, 2, a, sgn<S>(mul_i(w0[a])));
      acc_add(acc, 3, a, sgn<-S>(mul_i(w1[a])));
    } else {
      acc_add(acc, 2, a, sgn<S>(w0[a]));
      acc_add(acc, 3, a, sgn<S>(w1[a]));
    }
  }
}

// One hop: acc += eta * (1 + S g_MU) (U or U^dag) psi, eta = +-1.
template <int MU, int S, bool ADJ, typename R>
__device__ __forceinline__ void hop(const R psi[24], const R u[18], int eta, R acc[24]) {
  Cx<R> h0[3], h1[3];
  project<MU, S>(psi, eta, h0, h1);
  hop_half<MU, S, ADJ>(h0, h1, u, acc);
}

// One hop from the raw storage words of the neighbour spinor: FP16 spinors are projected in
// half2 before conversion, every other precision is unpacked and projected in its arithmetic
// type. Every Dslash form calls this, so a site's arithmetic is the same in all of them.
template <int MU, int S, bool ADJ, int SP>
__device__ __forceinline__ void hop_words(const typename SpinorIO<SP>::Word w[SpinorIO<SP>::NW],
                                          const typename SpinorIO<SP>::Real u[18], int eta,
                                          typename SpinorIO<SP>::Real acc[24]) {
  if constexpr (SP == P_F16) {
    Cx<float> h0[3], h1[3];
    project_h2<MU, S>(w, eta, h0, h1);
    hop_half<MU, S, ADJ>(h0, h1, u, acc);
  } else {
    typename SpinorIO<SP>::Real psi[24];
    SpinorIO<SP>::unpack(w, psi);
    hop<MU, S, ADJ>(psi, u, eta, acc);
  }
}

// Link field of one parity: direction mu starts NR * Vh reals after direction mu-1.
template <int LP, int NR>
__device__ __forceinline__ const char* link_dir(const void* base, int Vh, int mu) {
  return reinterpret_cast<const char*>(base) + (size_t)mu * NR * Vh * prec_bytes(LP);
}

// Software-pipelined hop sequence. Hop K (0..7) is direction MU = K / 2,
// forward for even K and backward for odd K. The raw words (spinor and link)
// of hop K + D are loaded while hop K is computed, D = pipeline depth, so a
// thread keeps up to D hops of loads in flight instead of one; at small
// volumes, where every site already has a resident thread, this is what hides
// the memory latency.
// Depth per spinor precision: 3 (measured best on GB300) except double-float,
// whose wide words leave registers for one hop in flight only.
#ifndef LQCD_DSLASH_DEPTH
#define LQCD_DSLASH_DEPTH 3
#endif
#ifndef LQCD_DSLASH_DEPTH_HALF
#define LQCD_DSLASH_DEPTH_HALF LQCD_DSLASH_DEPTH
#endif
template <int SP>
struct DslashDepth {
  static constexpr int value =
      (SP == P_DF64) ? 1 : ((SP == P_F16 || SP == P_BF16) ? LQCD_DSLASH_DEPTH_HALF : LQCD_DSLASH_DEPTH);
};

template <int SP, int LP, int NR>
struct HopBuf {
  typename SpinorIO<SP>::Word s[SpinorIO<SP>::NW];
  typename LinkIO<LP, NR>::Word u[LinkIO<LP, NR>::NW];
};

template <int K, int SP, int LP, int NR>
__device__ __forceinline__ void issue_hop(const Geom& g, int h, const int nf[4], const int nb[4],
                                          const void* in, const void* Uout, const void* Uin,
                                          HopBuf<SP, LP, NR>& b) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  const int n = FWD ? nf[MU] : nb[MU];
  SpinorIO<SP>::load_raw(in, g.Vh, n, b.s);
  LinkIO<LP, NR>::load_raw(link_dir<LP, NR>(FWD ? Uout : Uin, g.Vh, MU), g.Vh, FWD ? h : n, b.u);
}

template <int K, int SP, int LP, int NR, bool DAG>
__device__ __forceinline__ void compute_hop(const Geom& g, int t, const HopBuf<SP, LP, NR>& b,
                                            typename SpinorIO<SP>::Real acc[24]) {
  using R = typename SpinorIO<SP>::Real;
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  R u[18];
  LinkIO<LP, NR>::unpack(b.u, u);
  if (NR == 12) reconstruct_row2(u);
  // forward: U_mu(x) psi(x + mu), projector (1 - g) for D, (1 + g) for D^dag
  // backward: U_mu(x - mu)^dag psi(x - mu), projector (1 + g) for D, (1 - g) for D^dag
  const int eta = (MU == 3 && t == (FWD ? g.L[3] - 1 : 0)) ? g.t_bc : 1;
  constexpr int S = FWD ? (DAG ? 1 : -1) : (DAG ? -1 : 1);
  hop_words<MU, S, !FWD, SP>(b.s, u, eta, acc);
}

template <int K, int D, int SP, int LP, int NR, bool DAG>
struct HopPipe {
  __device__ __forceinline__ static void run(const Geom& g, int h, int t, const int nf[4],
                                             const int nb[4], const void* in, const void* Uout,
                                             const void* Uin, HopBuf<SP, LP, NR> (&b)[D],
                                             typename SpinorIO<SP>::Real acc[24]) {
    compute_hop<K, SP, LP, NR, DAG>(g, t, b[K % D], acc);
    if (K + D < 8) issue_hop<(K + D < 8 ? K + D : 0), SP, LP, NR>(g, h, nf, nb, in, Uout, Uin, b[K % D]);
    HopPipe<K + 1, D, SP, LP, NR, DAG>::run(g, h, t, nf, nb, in, Uout, Uin, b, acc);
  }
};
template <int D, int SP, int LP, int NR, bool DAG>
struct HopPipe<8, D, SP, LP, NR, DAG> {
  __device__ __forceinline__ static void run(const Geom&, int, int, const int*, const int*,
                                             const void*, const void*, const void*,
                                             HopBuf<SP, LP, NR> (&)[D],
                                             typename SpinorIO<SP>::Real*) {}
};

template <int K, int D, int SP, int LP, int NR>
struct HopPrologue {
  __device__ __forceinline__ static void run(const Geom& g, int h, const int nf[4], const int nb[4],
                                             const void* in, const void* Uout, const void* Uin,
                                             HopBuf<SP, LP, NR> (&b)[D]) {
    issue_hop<K, SP, LP, NR>(g, h, nf, nb, in, Uout, Uin, b[K]);
    HopPrologue<K + 1, D, SP, LP, NR>::run(g, h, nf, nb, in, Uout, Uin, b);
  }
};
template <int D, int SP, int LP, int NR>
struct HopPrologue<D, D, SP, LP, NR> {
  __device__ __forceinline__ static void run(const Geom&, int, const int*, const int*, const void*,
                                             const void*, const void*, HopBuf<SP, LP, NR> (&)[D]) {}
};

// acc = (D_{p,1-p} in)(h) for output parity p. Uout: links of parity p, Uin: links of 1-p.
template <int SP, int LP, int NR, bool DAG>
__device__ __forceinline__ void dslash_site(const Geom& g, int h, int out_par, const void* in,
                                            const void* Uout, const void* Uin,
                                            typename SpinorIO<SP>::Real acc[24]) {
  int nf[4], nb[4], t;
  neighbours(g, h, out_par, nf, nb, t);
  constexpr int D = DslashDepth<SP>::value;
  HopBuf<SP, LP, NR> b[D];
  HopPrologue<0, D, SP, LP, NR>::run(g, h, nf, nb, in, Uout, Uin, b);
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0;
  HopPipe<0, D, SP, LP, NR, DAG>::run(g, h, t, nf, nb, in, Uout, Uin, b, acc);
}

// ---------------------------------------------------------------- colour-split form
// Three threads per output site, thread col computing output colour col for all
// four spins, multiplying by one row only: row col of U (forward) or of
// U^dag = conj(column col of U(x - mu)) (backward). The accumulator and the link
// data per thread shrink three-fold; this pays where the per-site work is latency
// bound at low occupancy (double-float), not where it is memory bound.

// The three threads of a site (colour col = 0, 1, 2, in different warps of the CTA) each
// need the projected half spinor h of all three colours of a neighbour. Each thread loads
// and projects only its own colour and publishes it in shared memory; after a barrier it
// reads the other two. Per hop that is one third of the spinor loads and projections of
// the unshared form, at the cost of one CTA barrier per hop (two buffers alternate, so one
// barrier per hop suffices). Every thread of the CTA must run all 8 hops: threads past
// the end of the lattice pass a clamped site and discard the result.

// one buffer: [colour][h0 | h1][tile site] of (re.hi, re.lo, im.hi, im.lo)
template <int NT>
struct ProjShare {
  float4 h[2][3][2][NT];
};

__device__ __forceinline__ float4 pack_c(const Cx<df64>& a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ Cx<df64> unpack_c(const float4& d) { return {df64(d.x, d.y), df64(d.z, d.w)}; }

template <int K, int LP, bool DAG, int NT>
__device__ __forceinline__ void hop3s_df(const Geom& g, int h, const int nf[4], const int nb[4], int t,
                                         const void* in, const void* Uout, const void* Uin, int col, int j,
                                         df64 acc[8], ProjShare<NT>& sh) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  constexpr int S = FWD ? (DAG ? 1 : -1) : (DAG ? -1 : 1);
  const int n = FWD ? nf[MU] : nb[MU];
  df64 v[8];
  SpinorIO<P_DF64>::load_colour(in, g.Vh, n, col, v);
  const Cx<df64> p0{v[0], v[1]}, p1{v[2], v[3]}, p2{v[4], v[5]}, p3{v[6], v[7]};
  Cx<df64> h0, h1;
  if (MU == 0) {
    h0 = {df_add_u(p0.re, S * p3.im), df_add_u(p0.im, S * -p3.re)};
    h1 = {df_add_u(p1.re, S * p2.im), df_add_u(p1.im, S * -p2.re)};
  } else if (MU == 1) {
    h0 = {df_add_u(p0.re, S * -p3.re), df_add_u(p0.im, S * -p3.im)};
    h1 = {df_add_u(p1.re, S * p2.re), df_add_u(p1.im, S * p2.im)};
  } else if (MU == 2) {
    h0 = {df_add_u(p0.re, S * p2.im), df_add_u(p0.im, S * -p2.re)};
    h1 = {df_add_u(p1.re, S * -p3.im), df_add_u(p1.im, S * p3.re)};
  } else {
    h0 = {df_add_u(p0.re, S * p2.re), df_add_u(p0.im, S * p2.im)};
    h1 = {df_add_u(p1.re, S * p3.re), df_add_u(p1.im, S * p3.im)};
  }
  float4 (&buf)[3][2][NT] = sh.h[K & 1];
  buf[col][0][j] = pack_c(h0);
  buf[col][1][j] = pack_c(h1);
  // row col of U (forward) or of U(x - mu)^dag (backward)
  df64 r[6];
  {
    const char* base = link_dir<LP, 18>(FWD ? Uout : Uin, g.Vh, MU);
    const int hl = FWD ? h : n;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int word = FWD ? (3 * col + b) : (3 * b + col);
      const float4 d = ld_stream(reinterpret_cast<const float4*>(base) + hl + (size_t)word * g.Vh);
      r[2 * b] = df64(d.x, d.y);
      r[2 * b + 1] = FWD ? df64(d.z, d.w) : df64(-d.z, -d.w);
    }
  }
  __syncthreads();
  Cx<df64> w0{df64(0.0f, 0.0f), df64(0.0f, 0.0f)}, w1 = w0;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const Cx<df64> hb0 = unpack_c(buf[b][0][j]), hb1 = unpack_c(buf[b][1][j]);
    const df64 rr = r[2 * b], ri = r[2 * b + 1];
    df_mac_u(w0.re, rr, hb0.re);
    df_mac_u(w0.re, -ri, hb0.im);
    df_mac_u(w0.im, rr, hb0.im);
    df_mac_u(w0.im, ri, hb0.re);
    df_mac_u(w1.re, rr, hb1.re);
    df_mac_u(w1.re, -ri, hb1.im);
    df_mac_u(w1.im, rr, hb1.im);
    df_mac_u(w1.im, ri, hb1.re);
  }
  const int eta = (MU == 3 && t == (FWD ? g.L[3] - 1 : 0)) ? g.t_bc : 1;
  if (MU == 3 && eta < 0) {
    w0 = sgn<-1>(w0);
    w1 = sgn<-1>(w1);
  }
  acc[0] = df_add_u(acc[0], w0.re); acc[1] = df_add_u(acc[1], w0.im);
  acc[2] = df_add_u(acc[2], w1.re); acc[3] = df_add_u(acc[3], w1.im);
  Cx<df64> l2, l3;
  if (MU == 0) { l2 = sgn<S>(mul_i(w1)); l3 = sgn<S>(mul_i(w0)); }
  else if (MU == 1) { l2 = sgn<S>(w1); l3 = sgn<-S>(w0); }
  else if (MU == 2) { l2 = sgn<S>(mul_i(w0)); l3 = sgn<-S>(mul_i(w1)); }
  else { l2 = sgn<S>(w0); l3 = sgn<S>(w1); }
  acc[4] = df_add_u(acc[4], l2.re); acc[5] = df_add_u(acc[5], l2.im);
  acc[6] = df_add_u(acc[6], l3.re); acc[7] = df_add_u(acc[7], l3.im);
}

// acc = colour col of (D_{p,1-p} in)(h) in double-float, 18-real double-float links; all
// 3 NT threads of the CTA call it together (thread j of colour col: site h)
template <int LP, bool DAG, int NT>
__device__ __forceinline__ void dslash_site3s_df(const Geom& g, int h, int out_par, const void* in,
                                                 const void* Uout, const void* Uin, int col, int j,
                                                 df64 acc[8], ProjShare<NT>& sh) {
  int nf[4], nb[4], t;
  neighbours(g, h, out_par, nf, nb, t);
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = df64(0.0f, 0.0f);
  hop3s_df<0, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<1, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<2, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<3, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<4, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<5, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<6, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
  hop3s_df<7, LP, DAG, NT>(g, h, nf, nb, t, in, Uout, Uin, col, j, acc, sh);
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = df_norm(acc[i]);
}

}  // namespace lqcd
