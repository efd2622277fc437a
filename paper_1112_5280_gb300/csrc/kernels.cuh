// Batched kernels: even-odd Dslash with fused epilogues, and the fused BLAS of
// the Krylov solvers. Instantiated per spinor precision in kernels_<prec>.cu.
#pragma once

#include "batch.cuh"

namespace lqcd {

// EPI_*_TW: the same epilogues with the twisted-mass factors of the Work (site-diagonal
// s (1 + i t g5) on the hopping term and on the operand vector); separate instantiations
// keep the Wilson kernels free of the twist code.
template <int EPI>
struct EpiTraits {
  static constexpr bool lin = (EPI == EPI_LIN || EPI == EPI_LIN_TW || EPI == EPI_PLAIN);
  static constexpr bool tw = (EPI == EPI_LIN_TW || EPI == EPI_CG_TW);
  static constexpr bool red = (EPI != EPI_PLAIN);
};

// Occupancy target (CTAs of TILE threads per SM) of the Dslash: 6 leaves 168
// registers per thread, room for a 3-deep hop pipeline (measured best on
// GB300 for batched and large lattices); a compile-time tunable.
#ifndef LQCD_DSLASH_MIN_BLOCKS
#define LQCD_DSLASH_MIN_BLOCKS 6
#endif
// FP16 / BF16 spinors: the same bytes in flight come from half the words, so the half
// precisions take a higher occupancy target: 10 CTAs per SM (96 registers). Measured on
// GB300 against 6: the plain operator at 32^3x64 unchanged (70.3 against 70.2 us), the
// solvers' linear epilogue 71.0 against 87.2 us despite a 148-byte spill, the 32^3x64 mixed
// CG 1.6% (FP16) and 2.0% (BF16) faster, twisted FP16 CG 4.6%.
#ifndef LQCD_DSLASH_MIN_BLOCKS_HALF
#define LQCD_DSLASH_MIN_BLOCKS_HALF 10
#endif
// Double-float needs the full 255 registers per thread (4 CTAs of 64 threads).
template <int SP>
struct DslashMinBlocks {
  static constexpr int value =
      (SP == P_DF64) ? 4 : ((SP == P_F16 || SP == P_BF16) ? LQCD_DSLASH_MIN_BLOCKS_HALF : LQCD_DSLASH_MIN_BLOCKS);
};
// The second register budget of the FP32 Dslash (launch form 3): 8 CTAs per SM, 128
// registers per thread. More warps with fewer hops in flight each; it pays where the
// launch is latency bound rather than at the HBM roofline (slots sharing links through
// L2), and the autotuner times it against the default.
constexpr int DSLASH_MIN_BLOCKS_HI = 8;

// Site sums with a fixed rounding sequence (f_fma; see field.cuh), as the Dslash forms share them.
template <typename R>
__device__ __forceinline__ double site_norm2(const R v[24]) {
  R s = f_mul(v[0], v[0]);
#pragma unroll
  for (int i = 1; i < 24; ++i) s = f_fma(v[i], v[i], s);
  return (double)s;
}

// <a, b> = sum conj(a) b over one site, (re, im)
template <typename R>
__device__ __forceinline__ void site_dot(const R a[24], const R b[24], double& re, double& im) {
  R sr = R(0), si = R(0);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    sr = f_fma(a[2 * i], b[2 * i], sr);
    sr = f_fma(a[2 * i + 1], b[2 * i + 1], sr);
    si = f_fma(a[2 * i], b[2 * i + 1], si);
    si = f_fma(-a[2 * i + 1], b[2 * i], si);
  }
  re = (double)sr;
  im = (double)si;
}

// Storage of the sloppy solution accumulator: that of an FP64-class solve, else FP32.
template <int SP>
struct XSloppy {
  static constexpr int P = (SP == P_F64 || SP == P_DF64) ? SP : P_F32;
};

// Conversions between the arithmetic types (double-float -> float rounds hi + lo).
template <typename To>
__device__ __forceinline__ To cvt(float x) { return To(x); }
template <typename To>
__device__ __forceinline__ To cvt(double x) { return To(x); }
template <typename To>
__device__ __forceinline__ To cvt(df64 x) { return To(x); }
template <>
__device__ __forceinline__ float cvt<float>(df64 x) { return __fadd_rn(x.hi, x.lo); }
template <>
__device__ __forceinline__ double cvt<double>(df64 x) { return (double)x; }
template <>
__device__ __forceinline__ df64 cvt<df64>(df64 x) { return x; }

// v <- s (1 + i t g5) v for the complex components of a site (colour-major order:
// component c has spin c % 4; g5 = +1 on spins 0, 1 and -1 on spins 2, 3).
template <typename R>
__device__ __forceinline__ void twist24(R v[24], double sd, double td) {
  const R s = R(sd), t = R(td);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const R re = v[2 * c], im = v[2 * c + 1];
    const R tt = (c % 4) < 2 ? t : -t;
    v[2 * c] = f_mul(s, f_fma(-tt, im, re));
    v[2 * c + 1] = f_mul(s, f_fma(tt, re, im));
  }
}
// the same for the 4 spins of one colour (v[2 spin], v[2 spin + 1])
template <typename R>
__device__ __forceinline__ void twist8(R v[8], double sd, double td) {
  const R s = R(sd), t = R(td);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    const R re = v[2 * sp], im = v[2 * sp + 1];
    const R tt = sp < 2 ? t : -t;
    v[2 * sp] = s * (re - tt * im);
    v[2 * sp + 1] = s * (im + tt * re);
  }
}

// Whole-CTA exit for a single-slot launch whose slot does not run.
__device__ __forceinline__ bool single_slot_idle(const Launch& L) {
  return L.nslots == 1 && !slot_runs(work_of(L, 0));
}

// Epilogue of the one-thread-per-site Dslash at site h of slot w, acc = D_{p,1-p} in at h:
//   out = a * acc + c1 * y1 + c2 * y2                                 (EPI_LIN, EPI_PLAIN)
//   r -= alpha (y1 + a * acc); x += alpha p                           (EPI_CG, CG step)
// (twisted: out = T(a acc) + c1 y1 + c2 T_y y2 and r -= alpha (T_y y1 + T(a acc)))
// and the site's contributions v0..v2 to the slot's reduction.
template <int SP, int EPI>
__device__ __forceinline__ void dslash_epilogue(const Work& w, int h, typename SpinorIO<SP>::Real acc[24],
                                                double& v0, double& v1, double& v2) {
  using R = typename SpinorIO<SP>::Real;
  const R a = (R)w.a;
  if constexpr (EpiTraits<EPI>::lin) {
    if (w.a != 1.0) {  // a plain hopping term (a = 1) keeps acc as it is, bit for bit
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] = f_mul(acc[i], a);
    }
    if constexpr (EpiTraits<EPI>::tw) twist24(acc, w.tw_s, w.tw_t);
    R y[24];
    if (w.y1) {
      SpinorIO<SP>::load(w.y1, w.g.Vh, h, y);
      const R c = (R)w.c1;
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] = f_fma(c, y[i], acc[i]);
    }
    if (w.y2) {
      R y2[24];
      SpinorIO<SP>::load(w.y2, w.g.Vh, h, y2);
      if constexpr (EpiTraits<EPI>::tw) twist24(y2, 1.0, w.ty_t);
      const R c = (R)w.c2;
#pragma unroll
      for (int i = 0; i < 24; ++i) acc[i] = f_fma(c, y2[i], acc[i]);
    }
    SpinorIO<SP>::store(w.out, w.g.Vh, h, acc);
    if (!EpiTraits<EPI>::red) {
    } else if (w.red == 1) {
      v0 = site_norm2(acc);
    } else if (w.red == 2) {
      R z[24];
      SpinorIO<SP>::load(w.zin, w.g.Vh, h, z);
      site_dot(z, acc, v0, v1);
    } else if (w.red == 3) {  // <out, y1>, |out|^2
      site_dot(acc, y, v0, v1);
      v2 = site_norm2(acc);
    }
  } else {
    const R alpha = (R)w.sc->alpha;
    R y[24], r[24];
    SpinorIO<SP>::load(w.y1, w.g.Vh, h, y);
    SpinorIO<SP>::load(w.out, w.g.Vh, h, r);
    if constexpr (EpiTraits<EPI>::tw) {
      twist24(acc, w.tw_s, w.tw_t);
      twist24(y, 1.0, w.ty_t);
    }
#pragma unroll
    for (int i = 0; i < 24; ++i) r[i] = f_fma(-alpha, f_fma(a, acc[i], y[i]), r[i]);
    SpinorIO<SP>::store(w.out, w.g.Vh, h, r);
    v0 = site_norm2(r);
    using XR = typename SpinorIO<XSloppy<SP>::P>::Real;
    R p[24];
    XR x[24];
    SpinorIO<SP>::load(w.zin, w.g.Vh, h, p);
    SpinorIO<XSloppy<SP>::P>::load(w.z, w.g.Vh, h, x);
#pragma unroll
    for (int i = 0; i < 24; ++i) x[i] = f_fma((XR)alpha, (XR)p[i], x[i]);
    SpinorIO<XSloppy<SP>::P>::store(w.z, w.g.Vh, h, x);
  }
}

// Batched Dslash: out = a * D_{p,1-p} in + c1 * y1 + c2 * y2      (EPI_LIN)
//                 r -= alpha (y1 + a * D in); x += alpha p      (EPI_CG, CG step)
// (twisted: out = T(a D in) + c1 y1 + c2 T_y y2 and r -= alpha (T_y y1 + T(a D in)))
// with the Work's reduction (norm / dots) and scalar finisher per slot.
template <int SP, int LP, int NR, bool DAG, int EPI>
__device__ __forceinline__ void dslash_tile(const Launch& L, int slot, int start) {
  using R = typename SpinorIO<SP>::Real;
  const Work& w = work_of(L, slot);
  const int h = start + threadIdx.x;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;
  if (h < w.g.Vh) {
    R acc[24];
    dslash_site<SP, LP, NR, DAG>(w.g, h, w.out_par, w.in, w.Uout, w.Uin, acc);
    dslash_epilogue<SP, EPI>(w, h, acc, v0, v1, v2);
  }
  if constexpr (EpiTraits<EPI>::red)
    tile_partial<TILE, std::is_same<R, float>::value>(w, start / TILE, v0, v1, v2, L.partials);
}

// The tile loop is written twice: over the running slots' tiles of a gated launch (slot
// view), and over all tiles otherwise, so that operator launches run the plain loop without
// the view's branches and without shared memory (measured: one loop with a static view cost
// 1.3% more instructions and 2-3% of the headline launch).
template <int SP, int LP, int NR, bool DAG, int EPI, int MB = DslashMinBlocks<SP>::value>
__global__ void __launch_bounds__(TILE, MB) k_dslash(const Launch L) {
  pdl_wait();
  if (single_slot_idle(L)) return;
  extern __shared__ int4 dyn_smem[];  // the slot view, launched with view_smem(L) bytes
  SlotView& sv = *reinterpret_cast<SlotView*>(dyn_smem);
  if (view_load(L, sv)) {
    for (int tile = blockIdx.x; tile < sv.total; tile += gridDim.x) {
      pdl_last_tile(tile, sv.total);
      int slot, start;
      view_tile(L, sv, tile, slot, start);
      dslash_tile<SP, LP, NR, DAG, EPI>(L, slot, start);
    }
    return;
  }
  for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x) {
    pdl_last_tile(tile, L.ntiles);
    int slot, start;
    tile_of(L, tile, slot, start);
    if (!slot_runs(work_of(L, slot))) continue;
    dslash_tile<SP, LP, NR, DAG, EPI>(L, slot, start);
  }
}

// ------------------------------------------------------------------ multi-right-hand-side form
// Every slot of the launch solves on the same gauge field (one lattice, one link copy): the
// 12 spin-colour point sources of a propagator (paper Section 4) or any set of solves on one
// configuration. A CTA takes one block of TILE sites and one group of slots. Each thread
// loads the 8 links of its site once and keeps them in shared memory, and then computes its
// site for every running slot of the group, in slot order, with k_dslash's hop arithmetic,
// epilogue and per-slot partial sums. So the links cross HBM once per site block for all
// slots instead of once per slot, and each slot's result is the same as in a launch of its
// own. 18-real links are kept whole (padded to 5 float4, 40 KB per CTA: 5 CTAs per SM);
// 12-real links keep their 12 stored reals (3 float4, 24 KB per CTA, 8 CTAs per SM at 128
// registers) and rebuild row 2 at each use, from the same reals and with the same
// operations as k_dslash, so the bits agree.
template <int NR>
struct Mrhs {
  static constexpr int W = NR == 12 ? 3 : 5;  // float4 words per link in shared memory
  static constexpr int MIN_BLOCKS = NR == 12 ? 8 : 5;
};

// the links of a thread's site: word q of hop k at s[(k * W + q) * TILE + thread]
template <int NR>
__device__ __forceinline__ void mrhs_store_link(float4* s, int k, const float u[18]) {
  constexpr int W = Mrhs<NR>::W;
#pragma unroll
  for (int q = 0; q < (NR == 12 ? 3 : 4); ++q)
    s[(k * W + q) * TILE] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
  if (NR == 18) s[(k * W + 4) * TILE] = make_float4(u[16], u[17], 0.0f, 0.0f);
}
template <int NR>
__device__ __forceinline__ void mrhs_load_link(const float4* s, int k, float u[18]) {
  constexpr int W = Mrhs<NR>::W;
#pragma unroll
  for (int q = 0; q < (NR == 12 ? 3 : 4); ++q) {
    const float4 d = s[(k * W + q) * TILE];
    u[4 * q] = d.x; u[4 * q + 1] = d.y; u[4 * q + 2] = d.z; u[4 * q + 3] = d.w;
  }
  if (NR == 18) {
    const float4 d = s[(k * W + 4) * TILE];
    u[16] = d.x; u[17] = d.y;
  } else {
    reconstruct_row2(u);
  }
}

template <int K, int LP, int NR>
__device__ __forceinline__ void mrhs_fetch_link(const Geom& g, int h, const int nb[4], const void* Uout,
                                                const void* Uin, float4* s) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  float u[18];
  LinkIO<LP, NR>::load(link_dir<LP, NR>(FWD ? Uout : Uin, g.Vh, MU), g.Vh, FWD ? h : nb[MU], u);
  mrhs_store_link<NR>(s, K, u);
}

// Hop K of D in at site h with the staged links; the spinor words of hop K + D are issued
// while hop K is computed (depth D), as in HopPipe.
template <int K, int D, int SP, int NR, bool DAG>
struct MrhsPipe {
  using IO = SpinorIO<SP>;
  __device__ __forceinline__ static void run(const Geom& g, int t, const int nf[4], const int nb[4],
                                             const void* in, const float4* s,
                                             typename IO::Word (&b)[D][IO::NW], float acc[24]) {
    constexpr int MU = K / 2;
    constexpr bool FWD = (K % 2) == 0;
    float u[18];
    mrhs_load_link<NR>(s, K, u);
    const int eta = (MU == 3 && t == (FWD ? g.L[3] - 1 : 0)) ? g.t_bc : 1;
    constexpr int S = FWD ? (DAG ? 1 : -1) : (DAG ? -1 : 1);
    hop_words<MU, S, !FWD, SP>(b[K % D], u, eta, acc);
    if (K + D < 8) {
      constexpr int KN = (K + D < 8) ? K + D : 0;
      IO::load_raw(in, g.Vh, (KN % 2 == 0) ? nf[KN / 2] : nb[KN / 2], b[K % D]);
    }
    MrhsPipe<K + 1, D, SP, NR, DAG>::run(g, t, nf, nb, in, s, b, acc);
  }
};
template <int D, int SP, int NR, bool DAG>
struct MrhsPipe<8, D, SP, NR, DAG> {
  __device__ __forceinline__ static void run(const Geom&, int, const int*, const int*, const void*,
                                             const float4*, typename SpinorIO<SP>::Word (&)[D][SpinorIO<SP>::NW],
                                             float*) {}
};

template <int SP, int LP, int NR, bool DAG, int EPI>
__global__ void __launch_bounds__(TILE, Mrhs<NR>::MIN_BLOCKS) k_dslash_mrhs(const Launch L) {
  pdl_wait();
  static_assert(SP == P_F32 || SP == P_F16 || SP == P_BF16, "multi-RHS form: FP32 arithmetic");
  using IO = SpinorIO<SP>;
  constexpr int D = DslashDepth<SP>::value;
  __shared__ float4 su[8 * Mrhs<NR>::W * TILE];
  __shared__ SlotView sv;
  const bool view = view_load(L, sv);
  float4* s = su + threadIdx.x;
  for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x) {
    pdl_last_tile(tile, L.ntiles);
    const int group = tile % L.mrhs_groups;
    const int block = tile / L.mrhs_groups;
    const int s0 = group * L.mrhs_group;
    const int s1 = min(L.nslots, s0 + L.mrhs_group);
    bool any = false;
    for (int si = s0; si < s1; ++si) any = any || slot_runs_v(sv, view, L, si);
    if (!any) continue;
    const Work& w0 = work_of(L, s0);  // lattice, parity and links are those of every slot
    const Geom& g = w0.g;
    const int h = block * TILE + threadIdx.x;
    const bool live = h < g.Vh;
    int nf[4], nb[4], t = 0;
    if (live) {
      neighbours(g, h, w0.out_par, nf, nb, t);
      mrhs_fetch_link<0, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<1, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<2, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<3, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<4, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<5, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<6, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
      mrhs_fetch_link<7, LP, NR>(g, h, nb, w0.Uout, w0.Uin, s);
    }
    for (int si = s0; si < s1; ++si) {
      if (!slot_runs_v(sv, view, L, si)) continue;  // uniform over the CTA
      const Work& w = work_of(L, si);
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      if (live) {
        typename IO::Word b[D][IO::NW];
#pragma unroll
        for (int k = 0; k < D; ++k) IO::load_raw(w.in, g.Vh, (k % 2 == 0) ? nf[k / 2] : nb[k / 2], b[k]);
        float acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0.0f;
        MrhsPipe<0, D, SP, NR, DAG>::run(g, t, nf, nb, w.in, s, b, acc);
        dslash_epilogue<SP, EPI>(w, h, acc, v0, v1, v2);
      }
      if constexpr (EpiTraits<EPI>::red) tile_partial<TILE, true>(w, block, v0, v1, v2, L.partials);
    }
  }
}

// Colour-split batched Dslash for 18-real double-float links: 3 * TILE threads per CTA,
// threads [c * TILE, (c + 1) * TILE) compute colour c of the tile's TILE sites, sharing
// each hop's projected half spinors through shared memory. Same epilogues, reductions
// and finishers as k_dslash (colour-local pieces of each site).
template <typename R>
__device__ __forceinline__ double colour_norm2(const R v[8]) {
  R s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += v[i] * v[i];
  return (double)s;
}
template <typename R>
__device__ __forceinline__ void colour_dot(const R a[8], const R b[8], double& re, double& im) {
  R sr = 0, si = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    sr += a[2 * i] * b[2 * i] + a[2 * i + 1] * b[2 * i + 1];
    si += a[2 * i] * b[2 * i + 1] - a[2 * i + 1] * b[2 * i];
  }
  re = (double)sr;
  im = (double)si;
}

#ifndef LQCD_DSLASH3_MIN_BLOCKS
#define LQCD_DSLASH3_MIN_BLOCKS 4
#endif
template <int SP, int LP, bool DAG, int EPI>
__global__ void __launch_bounds__(3 * TILE, LQCD_DSLASH3_MIN_BLOCKS) k_dslash3(const Launch L) {
  pdl_wait();
  using R = typename SpinorIO<SP>::Real;
  static_assert(SP == P_DF64 && LP == P_DF64, "the colour-split form is built for double-float");
  __shared__ ProjShare<TILE> sh;
  if (single_slot_idle(L)) return;
  __shared__ SlotView sv;
  const bool view = view_load(L, sv);
  const int ntiles = view ? sv.total : L.ntiles;
  const int col = threadIdx.x / TILE;
  const int j = threadIdx.x - col * TILE;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    pdl_last_tile(tile, ntiles);
    int slot, start;
    if (view) {
      view_tile(L, sv, tile, slot, start);
    } else {
      tile_of(L, tile, slot, start);
      if (!slot_runs(work_of(L, slot))) continue;
    }
    const Work& w = work_of(L, slot);
    const int h = start + j;
    const int Vh = w.g.Vh;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    // every thread runs the hops (they share projections through barriers); a thread
    // past the end of the lattice takes the last site and drops the result
    R acc[8];
    dslash_site3s_df<LP, DAG, TILE>(w.g, h < Vh ? h : Vh - 1, w.out_par, w.in, w.Uout, w.Uin, col, j, acc, sh);
    if (h < Vh) {
      const R a = (R)w.a;
      if constexpr (EpiTraits<EPI>::lin) {
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] *= a;
        if constexpr (EpiTraits<EPI>::tw) twist8(acc, w.tw_s, w.tw_t);
        R y[8];
        if (w.y1) {
          SpinorIO<SP>::load_colour(w.y1, Vh, h, col, y);
          const R c = (R)w.c1;
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] += c * y[i];
        }
        if (w.y2) {
          R y2[8];
          SpinorIO<SP>::load_colour(w.y2, Vh, h, col, y2);
          if constexpr (EpiTraits<EPI>::tw) twist8(y2, 1.0, w.ty_t);
          const R c = (R)w.c2;
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] += c * y2[i];
        }
        SpinorIO<SP>::store_colour(w.out, Vh, h, col, acc);
        if (!EpiTraits<EPI>::red) {
        } else if (w.red == 1) {
          v0 = colour_norm2(acc);
        } else if (w.red == 2) {
          R z[8];
          SpinorIO<SP>::load_colour(w.zin, Vh, h, col, z);
          colour_dot(z, acc, v0, v1);
        } else if (w.red == 3) {
          colour_dot(acc, y, v0, v1);
          v2 = colour_norm2(acc);
        }
      } else {
        const R alpha = (R)w.sc->alpha;
        R y[8], r[8];
        SpinorIO<SP>::load_colour(w.y1, Vh, h, col, y);
        SpinorIO<SP>::load_colour(w.out, Vh, h, col, r);
        if constexpr (EpiTraits<EPI>::tw) {
          twist8(acc, w.tw_s, w.tw_t);
          twist8(y, 1.0, w.ty_t);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] -= alpha * (y[i] + a * acc[i]);
        SpinorIO<SP>::store_colour(w.out, Vh, h, col, r);
        v0 = colour_norm2(r);
        using XR = typename SpinorIO<XSloppy<SP>::P>::Real;
        R p[8];
        XR x[8];
        SpinorIO<SP>::load_colour(w.zin, Vh, h, col, p);
        SpinorIO<XSloppy<SP>::P>::load_colour(w.z, Vh, h, col, x);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] += cvt<XR>(alpha) * cvt<XR>(p[i]);
        SpinorIO<XSloppy<SP>::P>::store_colour(w.z, Vh, h, col, x);
      }
    }
    if constexpr (EpiTraits<EPI>::red) tile_partial<3 * TILE>(w, start / TILE, v0, v1, v2, L.partials);
  }
}

// ------------------------------------------------------------------ fused BLAS

enum Blas {
  B_CG_P = 0,     // p(out) = r(in) + beta p
  B_RU_FOLD,      // x64(out) += sigma * xs(in) ; xs = 0          (SP = precision of xs)
  B_RU_CONVERT,   // r(out) = rho64(in) * res[5] ; p(z) = restart ? r : r + res[4] p
  B_NORM,         // |in|^2
  B_AXPBY,        // out(SP) = a * in(FP64) + c1 * y1(SP)
  B_ZERO,         // out = 0
  B_BICG_P,       // p(out) = r(in) + beta (p - omega v(y1))
  B_BICG_S,       // s(out) = r(in) - alpha v(y1)
  B_BICG_X,       // x(z) += alpha p(zin) + omega s(in) ; r(out) = s - omega t(y1) ; <r0(y2), r>, |r|^2
  B_FOLD64,       // x64(out) += a * xs(in) (SP) ; xs = 0
  B_TWIST,        // out = tw_s (1 + i tw_t g5) in
  B_RU_SCALE,     // out (SP) = in (TP) * res[2]
  B_RU_P,         // p(z) = restart ? r(in) : r + res[4] p
  B_RDOT,         // Re <in, y1>
};

// out = x + c * y (complex c)
template <typename R>
__device__ __forceinline__ void caxpy(R* out, const R* x, R cr, R ci, const R* y) {
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const R yr = y[2 * i], yi = y[2 * i + 1];
    out[2 * i] = x[2 * i] + cr * yr - ci * yi;
    out[2 * i + 1] = x[2 * i + 1] + cr * yi + ci * yr;
  }
}

// SP: precision of the sloppy / operated vectors; TP: precision of the
// FP64-class vectors (true residual, solution accumulator) in the mixed ops.
template <int SP, int OP, int TP = P_F64>
__global__ void __launch_bounds__(TILE) k_blas(const Launch L) {
  pdl_wait();
  using R = typename SpinorIO<SP>::Real;
  using TR = typename SpinorIO<TP>::Real;
  if (single_slot_idle(L)) return;
  __shared__ SlotView sv;
  const bool view = view_load(L, sv);
  const int ntiles = view ? sv.total : L.ntiles;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    pdl_last_tile(tile, ntiles);
    int slot, start;
    if (view) {
      view_tile(L, sv, tile, slot, start);
    } else {
      tile_of(L, tile, slot, start);
      if (!slot_runs(work_of(L, slot))) continue;
    }
    const Work& w = work_of(L, slot);
    const int h = start + threadIdx.x;
    const int Vh = w.g.Vh;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (h < Vh) {
      if (OP == B_CG_P) {
        const R beta = (R)w.sc->beta;
        R r[24], p[24];
        SpinorIO<SP>::load(w.in, Vh, h, r);
        SpinorIO<SP>::load(w.out, Vh, h, p);
#pragma unroll
        for (int i = 0; i < 24; ++i) p[i] = r[i] + beta * p[i];
        SpinorIO<SP>::store(w.out, Vh, h, p);
      } else if (OP == B_RU_FOLD || OP == B_FOLD64) {  // x (TP) += sigma * xs (SP); xs = 0
        const TR sg = TR((OP == B_RU_FOLD) ? w.sc->sigma : w.a);
        TR x[24];
        R xs[24];
        SpinorIO<TP>::load(w.out, Vh, h, x);
        SpinorIO<SP>::load(w.in, Vh, h, xs);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
          x[i] += sg * cvt<TR>(xs[i]);
          xs[i] = R(0);
        }
        SpinorIO<TP>::store(w.out, Vh, h, x);
        SpinorIO<SP>::store(const_cast<void*>(w.in), Vh, h, xs);
      } else if (OP == B_RU_CONVERT) {  // r (SP) = rho (TP) / sigma; p = restart ? r : r + c p
        const TR inv = TR(w.sc->res[5]);
        const double pc = w.sc->res[4];
        const int restart = w.sc->restart_p;
        TR rho[24];
        SpinorIO<TP>::load(w.in, Vh, h, rho);
        R r[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) r[i] = cvt<R>(rho[i] * inv);
        SpinorIO<SP>::store(w.out, Vh, h, r);
        R p[24];
        if (restart) {
#pragma unroll
          for (int i = 0; i < 24; ++i) p[i] = r[i];
        } else {
          SpinorIO<SP>::load(w.z, Vh, h, p);
#pragma unroll
          for (int i = 0; i < 24; ++i) p[i] = r[i] + (R)pc * p[i];
        }
        SpinorIO<SP>::store(w.z, Vh, h, p);
      } else if (OP == B_RU_SCALE) {  // sloppy copy of an FP64-class vector in the unit 1 / res[2]
        const TR sc = TR(w.sc->res[2]);
        TR u[24];
        SpinorIO<TP>::load(w.in, Vh, h, u);
        R q[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) q[i] = cvt<R>(u[i] * sc);
        SpinorIO<SP>::store(w.out, Vh, h, q);
      } else if (OP == B_RU_P) {
        R r[24], p[24];
        SpinorIO<SP>::load(w.in, Vh, h, r);
        if (w.sc->restart_p) {
#pragma unroll
          for (int i = 0; i < 24; ++i) p[i] = r[i];
        } else {
          const R pc = (R)w.sc->res[4];
          SpinorIO<SP>::load(w.z, Vh, h, p);
#pragma unroll
          for (int i = 0; i < 24; ++i) p[i] = r[i] + pc * p[i];
        }
        SpinorIO<SP>::store(w.z, Vh, h, p);
      } else if (OP == B_RDOT) {
        R a[24], b[24];
        SpinorIO<SP>::load(w.in, Vh, h, a);
        SpinorIO<SP>::load(w.y1, Vh, h, b);
        R acc = 0;
#pragma unroll
        for (int i = 0; i < 24; ++i) acc += a[i] * b[i];
        v0 = (double)acc;
      } else if (OP == B_NORM) {
        R v[24];
        SpinorIO<SP>::load(w.in, Vh, h, v);
        v0 = site_norm2(v);
      } else if (OP == B_AXPBY) {  // out (SP) = a * in (TP) [+ c1 * y1 (SP)]
        TR v[24];
        SpinorIO<TP>::load(w.in, Vh, h, v);
        const TR a = TR(w.a);
        R o[24];
        if (w.y1) {
          R y[24];
          SpinorIO<SP>::load(w.y1, Vh, h, y);
          const TR c1 = TR(w.c1);
#pragma unroll
          for (int i = 0; i < 24; ++i) o[i] = cvt<R>(a * v[i] + c1 * cvt<TR>(y[i]));
        } else {
#pragma unroll
          for (int i = 0; i < 24; ++i) o[i] = cvt<R>(a * v[i]);
        }
        SpinorIO<SP>::store(w.out, Vh, h, o);
        if (w.red == 1) v0 = site_norm2(o);
      } else if (OP == B_TWIST) {
        R v[24];
        SpinorIO<SP>::load(w.in, Vh, h, v);
        twist24(v, w.tw_s, w.tw_t);
        SpinorIO<SP>::store(w.out, Vh, h, v);
      } else if (OP == B_ZERO) {
        R v[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] = 0;
        SpinorIO<SP>::store(w.out, Vh, h, v);
      } else if (OP == B_BICG_P) {
        const R br = (R)w.sc->cres[6], bi = (R)w.sc->cres[7];
        const R omr = (R)w.sc->cres[4], omi = (R)w.sc->cres[5];
        R r[24], p[24], v[24], t[24];
        SpinorIO<SP>::load(w.in, Vh, h, r);
        SpinorIO<SP>::load(w.out, Vh, h, p);
        SpinorIO<SP>::load(w.y1, Vh, h, v);
        caxpy(t, p, -omr, -omi, v);  // p - omega v
        caxpy(p, r, br, bi, t);      // r + beta (p - omega v)
        SpinorIO<SP>::store(w.out, Vh, h, p);
      } else if (OP == B_BICG_S) {
        const R ar = (R)w.sc->cres[2], ai = (R)w.sc->cres[3];
        R r[24], v[24], s[24];
        SpinorIO<SP>::load(w.in, Vh, h, r);
        SpinorIO<SP>::load(w.y1, Vh, h, v);
        caxpy(s, r, -ar, -ai, v);
        SpinorIO<SP>::store(w.out, Vh, h, s);
      } else if (OP == B_BICG_X) {
        const R ar = (R)w.sc->cres[2], ai = (R)w.sc->cres[3];
        const R omr = (R)w.sc->cres[4], omi = (R)w.sc->cres[5];
        R s[24], t[24], p[24], x[24], r[24], r0[24];
        SpinorIO<SP>::load(w.in, Vh, h, s);
        SpinorIO<SP>::load(w.y1, Vh, h, t);
        SpinorIO<SP>::load(w.zin, Vh, h, p);
        SpinorIO<SP>::load(w.z, Vh, h, x);
        caxpy(x, x, ar, ai, p);
        caxpy(x, x, omr, omi, s);
        SpinorIO<SP>::store(w.z, Vh, h, x);
        caxpy(r, s, -omr, -omi, t);
        SpinorIO<SP>::store(w.out, Vh, h, r);
        SpinorIO<SP>::load(w.y2, Vh, h, r0);
        site_dot(r0, r, v0, v1);
        v2 = site_norm2(r);
      }
    }
    tile_partial<TILE>(w, start / TILE, v0, v1, v2, L.partials);
  }
}

}  // namespace lqcd
