// Storage formats of spinor and link fields in HBM, and their register loads.
//
// Half-lattice fields (one checkerboard, Vh = V/2 sites) are structure-of-
// arrays: the 24 reals of a spinor (4 spin x 3 colour x re/im) or the 18/12
// reals of a link are split into "chunks" of one vector word, and chunk c of
// every site is contiguous: word(c, h) = base[c * Vh + h]. A warp therefore
// reads 32 consecutive words per chunk, fully coalesced.
//
//   spinor, 16-byte words : F64 12 x double2, F32 6 x float4, F16/BF16 3 x uint4
//   link,   widest word that divides the link: F64 9/6 x double2,
//           F32 9 x float2 (18 reals) or 3 x float4 (12 reals),
//           F16 9 x half2 (18 reals) or 3 x 4 halves (12 reals)
//
// Links are stored per parity and direction: link(p, mu) occupies
// NR * Vh reals starting at base_p + mu * NR * Vh. RECONSTRUCT TWELVE (the
// paper's Section 3 cites it as the next memory optimisation) keeps rows 0
// and 1 and rebuilds row 2 = conj(row0 x row1) in registers, exact for
// det U = 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <vector>

namespace lqcd {

// Readers of the debug bounds-check words, one per translation unit (LQCD_DEBUG_BOUNDS).
inline std::vector<int (*)(unsigned long long*)>& bounds_word_readers() {
  static std::vector<int (*)(unsigned long long*)> readers;
  return readers;
}

// Storage precisions. P_DF64 stores each real as an (hi, lo) pair of floats
// (8 bytes, like FP64) and computes in double-float arithmetic (below).
enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3, P_DF64 = 4 };
constexpr int NPREC = 5;  // number of storage precisions (size of per-precision tables)

__host__ __device__ inline int prec_bytes(int p) {
  return (p == P_F64 || p == P_DF64) ? 8 : (p == P_F32 ? 4 : 2);
}

// ------------------------------------------------------------------ double-float
// A real as the unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, giving
// a 48-bit significand on the FP32 pipes (GB300's FP64 pipe is a small fraction
// of its FP32 rate). Addition uses Knuth's error-free two-sum of the high parts
// plus the low parts; multiplication the FMA error-free product (Dekker's
// product with the exact residual a*b - round(a*b) from one fused multiply-add).
// The _rn intrinsics keep the compiler from contracting or reassociating the
// error-free steps.
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __device__ df64(int v) : hi((float)v), lo(0.0f) {}
  __device__ df64(float v) : hi(v), lo(0.0f) {}
  __device__ df64(double v) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  }
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_renorm(float s, float e) {  // s + e -> (hi, lo)
  const float h = __fadd_rn(s, e);
  return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_renorm(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
// small integer factors (the +-1 of spin projections) without a full product
__device__ __forceinline__ df64 operator*(int s, df64 a) {
  return s == 1 ? a : (s == -1 ? -a : df64(s) * a);
}
__device__ __forceinline__ bool isfinite_df(df64 a) { return isfinite(a.hi); }

// Double-float sums left unnormalised inside a site's hop sums: the pair (hi, lo) still
// carries the exact sum of what went in, but |lo| may exceed ulp(hi) / 2 until df_norm.
// An add is a two-sum of the high words plus the low words (8 operations instead of 11);
// a multiply-accumulate feeds the exact product error into the low word (12 instead of
// 7 + 11). The low word only collects rounding errors, so it stays far below hi.
__device__ __forceinline__ df64 df_add_u(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return df64(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ void df_mac_u(df64& acc, df64 a, df64 b) {  // acc += a b
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
  const float s = __fadd_rn(acc.hi, p);
  const float v = __fsub_rn(s, acc.hi);
  const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  acc = df64(s, __fadd_rn(acc.lo, __fadd_rn(e, pe)));
}
// normalised form of an unnormalised pair (two-sum of hi and lo)
__device__ __forceinline__ df64 df_norm(df64 a) {
  const float s = __fadd_rn(a.hi, a.lo);
  const float v = __fsub_rn(s, a.hi);
  return df64(s, __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(a.lo, v)));
}

// Arithmetic with a fixed rounding sequence. nvcc fuses a * b + c into one FMA where it
// sees fit, and the same source inlined into two different kernels may be fused in two
// different ways, which round differently. The site arithmetic of the Dslash, which must
// give the same bits in every kernel form (one launch per slot, interleaved slots,
// shared-link multi-RHS), spells every product and multiply-add out with these: float and
// double map to the round-to-nearest intrinsics, which are never contracted or reordered;
// double-float keeps its own operators.
template <typename R>
__device__ __forceinline__ R f_fma(R a, R b, R c) { return a * b + c; }
template <>
__device__ __forceinline__ float f_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double f_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename R>
__device__ __forceinline__ R f_mul(R a, R b) { return a * b; }
template <>
__device__ __forceinline__ float f_mul<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double f_mul<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename R>
__device__ __forceinline__ R f_add(R a, R b) { return a + b; }
template <>
__device__ __forceinline__ float f_add<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double f_add<double>(double a, double b) { return __dadd_rn(a, b); }
template <typename R>
__device__ __forceinline__ R f_sub(R a, R b) { return a - b; }
template <>
__device__ __forceinline__ float f_sub<float>(float a, float b) { return __fsub_rn(a, b); }
template <>
__device__ __forceinline__ double f_sub<double>(double a, double b) { return __dsub_rn(a, b); }

// Device order of the 24 reals of a spinor: colour-major, so that the 8 reals
// (4 spin x re/im) of one colour are contiguous words:
//   real(spin, colour, re/im) = (colour * 4 + spin) * 2 + re/im
// (the host layout is spin-major; the upload / download kernels permute).
__host__ __device__ constexpr int sidx(int spin, int col) { return (col * 4 + spin) * 2; }

template <typename T>
struct Cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ Cx<T> cmulc(Cx<T> a, Cx<T> b) {  // conj(a) * b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// ------------------------------------------------------------------ debug bounds checks
// Built with -DLQCD_DEBUG_BOUNDS, every spinor and link access of the field IO below checks
// its half-lattice site index against the field's size. The first index outside it is
// recorded in an error word of the translation unit, (1 << 63) | (Vh << 32) | index, and
// the access goes to site 0 instead, so a faulty index reads and writes only inside the
// field (no trap, no fault). lqcd_debug_bounds() collects and clears the words of every
// translation unit. Without the flag the check compiles to nothing.
#ifdef LQCD_DEBUG_BOUNDS
static __device__ unsigned long long lqcd_bounds_word;
__device__ __forceinline__ int checked_site(int h, int Vh) {
  if ((unsigned)h < (unsigned)Vh) return h;
  atomicCAS(&lqcd_bounds_word, 0ull,
            (1ull << 63) | ((unsigned long long)(unsigned)Vh << 32) | (unsigned long long)(unsigned)h);
  return 0;
}
#define LQCD_SITE(h, Vh) ::lqcd::checked_site((h), (Vh))
// host side: the word of this translation unit, read and cleared (registered at load)
namespace {
int read_bounds_word(unsigned long long* out) {
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, lqcd_bounds_word, sizeof v) != cudaSuccess) return -1;
  if (v && cudaMemcpyToSymbol(lqcd_bounds_word, &z, sizeof z) != cudaSuccess) return -1;
  *out = v;
  return 0;
}
struct BoundsWordRegistration {
  BoundsWordRegistration() { bounds_word_readers().push_back(&read_bounds_word); }
} bounds_word_registration;
}  // namespace
#else
#define LQCD_SITE(h, Vh) (h)
#endif

// ------------------------------------------------------------------ raw loads
// Read-only data is loaded through the non-coherent path. Links are read
// exactly once per half-lattice sweep, so they bypass L1 allocation.

__device__ __forceinline__ double2 ld_ro(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float4 ld_ro(const float4* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_ro(const float2* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ld_ro(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ uint2 ld_ro(const uint2* p) { return __ldg(p); }
__device__ __forceinline__ unsigned ld_ro(const unsigned* p) { return __ldg(p); }

__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ld_stream(const unsigned* p) {
  unsigned v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// half2 / bfloat162 packed in a 32-bit word
__device__ __forceinline__ float2 unpack_h2(unsigned w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ float2 unpack_b2(unsigned w) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
  return __bfloat1622float2(h);
}
__device__ __forceinline__ unsigned pack_h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<unsigned*>(&h);
}
__device__ __forceinline__ unsigned pack_b2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<unsigned*>(&h);
}

// ------------------------------------------------------------------ spinors

template <int P>
struct SpinorIO;

template <>
struct SpinorIO<P_F64> {
  using Real = double;
  static constexpr int CHUNKS = 12;
  using Word = double2;
  static constexpr int NW = 12;
  __device__ static void load_raw(const void* base, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const double2* p = reinterpret_cast<const double2*>(base) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_ro(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], double v[24]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      v[2 * c] = w[c].x;
      v[2 * c + 1] = w[c].y;
    }
  }
  // the 8 reals of colour a: words 4a .. 4a+3
  __device__ static void load_colour(const void* base, int Vh, int h, int a, double v[8]) {
    h = LQCD_SITE(h, Vh);
    const double2* p = reinterpret_cast<const double2*>(base) + h + (size_t)(4 * a) * Vh;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double2 d = ld_ro(p + (size_t)c * Vh);
      v[2 * c] = d.x;
      v[2 * c + 1] = d.y;
    }
  }
  __device__ static void store_colour(void* base, int Vh, int h, int a, const double v[8]) {
    h = LQCD_SITE(h, Vh);
    double2* p = reinterpret_cast<double2*>(base) + h + (size_t)(4 * a) * Vh;
#pragma unroll
    for (int c = 0; c < 4; ++c) p[(size_t)c * Vh] = make_double2(v[2 * c], v[2 * c + 1]);
  }
  __device__ static void load(const void* base, int Vh, int h, double v[24]) {
    h = LQCD_SITE(h, Vh);
    const double2* p = reinterpret_cast<const double2*>(base) + h;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 d = ld_ro(p + (size_t)c * Vh);
      v[2 * c] = d.x;
      v[2 * c + 1] = d.y;
    }
  }
  __device__ static void store(void* base, int Vh, int h, const double v[24]) {
    h = LQCD_SITE(h, Vh);
    double2* p = reinterpret_cast<double2*>(base) + h;
#pragma unroll
    for (int c = 0; c < 12; ++c) p[(size_t)c * Vh] = make_double2(v[2 * c], v[2 * c + 1]);
  }
};

template <>
struct SpinorIO<P_F32> {
  using Real = float;
  static constexpr int CHUNKS = 6;
  using Word = float4;
  static constexpr int NW = 6;
  __device__ static void load_raw(const void* base, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_ro(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float v[24]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      v[4 * c] = w[c].x;
      v[4 * c + 1] = w[c].y;
      v[4 * c + 2] = w[c].z;
      v[4 * c + 3] = w[c].w;
    }
  }
  // the 8 reals of colour a: words 2a, 2a+1
  __device__ static void load_colour(const void* base, int Vh, int h, int a, float v[8]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base) + h + (size_t)(2 * a) * Vh;
    const float4 d0 = ld_ro(p), d1 = ld_ro(p + Vh);
    v[0] = d0.x; v[1] = d0.y; v[2] = d0.z; v[3] = d0.w;
    v[4] = d1.x; v[5] = d1.y; v[6] = d1.z; v[7] = d1.w;
  }
  __device__ static void store_colour(void* base, int Vh, int h, int a, const float v[8]) {
    h = LQCD_SITE(h, Vh);
    float4* p = reinterpret_cast<float4*>(base) + h + (size_t)(2 * a) * Vh;
    p[0] = make_float4(v[0], v[1], v[2], v[3]);
    p[Vh] = make_float4(v[4], v[5], v[6], v[7]);
  }
  __device__ static void load(const void* base, int Vh, int h, float v[24]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base) + h;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 d = ld_ro(p + (size_t)c * Vh);
      v[4 * c] = d.x;
      v[4 * c + 1] = d.y;
      v[4 * c + 2] = d.z;
      v[4 * c + 3] = d.w;
    }
  }
  __device__ static void store(void* base, int Vh, int h, const float v[24]) {
    h = LQCD_SITE(h, Vh);
    float4* p = reinterpret_cast<float4*>(base) + h;
#pragma unroll
    for (int c = 0; c < 6; ++c)
      p[(size_t)c * Vh] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  }
};

template <>
struct SpinorIO<P_DF64> {
  using Real = df64;
  static constexpr int CHUNKS = 12;
  using Word = float4;
  static constexpr int NW = 12;
  // the 8 reals of colour a (colour-major order): words 4a .. 4a+3
  __device__ static void load_colour(const void* base, int Vh, int h, int a, df64 v[8]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base) + h + (size_t)(4 * a) * Vh;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 d = ld_ro(p + (size_t)c * Vh);
      v[2 * c] = df64(d.x, d.y);
      v[2 * c + 1] = df64(d.z, d.w);
    }
  }
  __device__ static void store_colour(void* base, int Vh, int h, int a, const df64 v[8]) {
    h = LQCD_SITE(h, Vh);
    float4* p = reinterpret_cast<float4*>(base) + h + (size_t)(4 * a) * Vh;
#pragma unroll
    for (int c = 0; c < 4; ++c) p[(size_t)c * Vh] = make_float4(v[2 * c].hi, v[2 * c].lo, v[2 * c + 1].hi, v[2 * c + 1].lo);
  }
  __device__ static void load_raw(const void* base, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_ro(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], df64 v[24]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      v[2 * c] = df64(w[c].x, w[c].y);
      v[2 * c + 1] = df64(w[c].z, w[c].w);
    }
  }
  __device__ static void load(const void* base, int Vh, int h, df64 v[24]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base, Vh, h, w);
    unpack(w, v);
  }
  __device__ static void store(void* base, int Vh, int h, const df64 v[24]) {
    h = LQCD_SITE(h, Vh);
    float4* p = reinterpret_cast<float4*>(base) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c)
      p[(size_t)c * Vh] = make_float4(v[2 * c].hi, v[2 * c].lo, v[2 * c + 1].hi, v[2 * c + 1].lo);
  }
};

template <bool BF>
struct SpinorIO16 {
  using Real = float;
  static constexpr int CHUNKS = 3;
  using Word = uint4;
  static constexpr int NW = 3;
  __device__ static void load_raw(const void* base, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const uint4* p = reinterpret_cast<const uint4*>(base) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_ro(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float v[24]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      const float2 a = unpack(w[c].x), b = unpack(w[c].y), e = unpack(w[c].z), f = unpack(w[c].w);
      v[8 * c + 0] = a.x; v[8 * c + 1] = a.y; v[8 * c + 2] = b.x; v[8 * c + 3] = b.y;
      v[8 * c + 4] = e.x; v[8 * c + 5] = e.y; v[8 * c + 6] = f.x; v[8 * c + 7] = f.y;
    }
  }
  __device__ static float2 unpack(unsigned w) { return BF ? unpack_b2(w) : unpack_h2(w); }
  __device__ static unsigned pack(float a, float b) { return BF ? pack_b2(a, b) : pack_h2(a, b); }
  // the 8 reals of colour a: word a
  __device__ static void load_colour(const void* base, int Vh, int h, int a, float v[8]) {
    h = LQCD_SITE(h, Vh);
    const uint4 d = ld_ro(reinterpret_cast<const uint4*>(base) + h + (size_t)a * Vh);
    const float2 x = unpack(d.x), y = unpack(d.y), z = unpack(d.z), w = unpack(d.w);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y; v[4] = z.x; v[5] = z.y; v[6] = w.x; v[7] = w.y;
  }
  __device__ static void store_colour(void* base, int Vh, int h, int a, const float v[8]) {
    h = LQCD_SITE(h, Vh);
    uint4 d;
    d.x = pack(v[0], v[1]);
    d.y = pack(v[2], v[3]);
    d.z = pack(v[4], v[5]);
    d.w = pack(v[6], v[7]);
    reinterpret_cast<uint4*>(base)[h + (size_t)a * Vh] = d;
  }
  __device__ static void load(const void* base, int Vh, int h, float v[24]) {
    h = LQCD_SITE(h, Vh);
    const uint4* p = reinterpret_cast<const uint4*>(base) + h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 d = ld_ro(p + (size_t)c * Vh);
      float2 a = unpack(d.x), b = unpack(d.y), e = unpack(d.z), f = unpack(d.w);
      v[8 * c + 0] = a.x; v[8 * c + 1] = a.y; v[8 * c + 2] = b.x; v[8 * c + 3] = b.y;
      v[8 * c + 4] = e.x; v[8 * c + 5] = e.y; v[8 * c + 6] = f.x; v[8 * c + 7] = f.y;
    }
  }
  __device__ static void store(void* base, int Vh, int h, const float v[24]) {
    h = LQCD_SITE(h, Vh);
    uint4* p = reinterpret_cast<uint4*>(base) + h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 d;
      d.x = pack(v[8 * c + 0], v[8 * c + 1]);
      d.y = pack(v[8 * c + 2], v[8 * c + 3]);
      d.z = pack(v[8 * c + 4], v[8 * c + 5]);
      d.w = pack(v[8 * c + 6], v[8 * c + 7]);
      p[(size_t)c * Vh] = d;
    }
  }
};
template <>
struct SpinorIO<P_F16> : SpinorIO16<false> {};
template <>
struct SpinorIO<P_BF16> : SpinorIO16<true> {};

// ------------------------------------------------------------------ links

// Loads the NR stored reals of link (mu) at half-site h into u[18] (row-major,
// re/im interleaved) and rebuilds row 2 when NR == 12.
template <int LP, int NR>
struct LinkIO;

// Raw words of one link (loaded once, bypassing L1) and their unpacking.
template <int NR>
struct LinkIO<P_F64, NR> {
  using Real = double;
  using Word = double2;
  static constexpr int NW = NR / 2;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const double2* p = reinterpret_cast<const double2*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], double u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      u[2 * c] = w[c].x;
      u[2 * c + 1] = w[c].y;
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, double u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

template <int NR>
struct LinkIO<P_DF64, NR> {
  using Real = df64;
  using Word = float4;
  static constexpr int NW = NR / 2;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], df64 u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      u[2 * c] = df64(w[c].x, w[c].y);
      u[2 * c + 1] = df64(w[c].z, w[c].w);
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, df64 u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

template <>
struct LinkIO<P_F32, 18> {
  using Real = float;
  using Word = float2;
  static constexpr int NW = 9;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const float2* p = reinterpret_cast<const float2*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      u[2 * c] = w[c].x;
      u[2 * c + 1] = w[c].y;
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, float u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

template <>
struct LinkIO<P_F32, 12> {
  using Real = float;
  using Word = float4;
  static constexpr int NW = 3;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const float4* p = reinterpret_cast<const float4*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      u[4 * c] = w[c].x;
      u[4 * c + 1] = w[c].y;
      u[4 * c + 2] = w[c].z;
      u[4 * c + 3] = w[c].w;
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, float u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

template <>
struct LinkIO<P_F16, 18> {
  using Real = float;
  using Word = unsigned;
  static constexpr int NW = 9;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const unsigned* p = reinterpret_cast<const unsigned*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      const float2 d = unpack_h2(w[c]);
      u[2 * c] = d.x;
      u[2 * c + 1] = d.y;
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, float u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

template <>
struct LinkIO<P_F16, 12> {
  using Real = float;
  using Word = uint2;
  static constexpr int NW = 3;
  __device__ static void load_raw(const void* base_mu, int Vh, int h, Word w[NW]) {
    h = LQCD_SITE(h, Vh);
    const uint2* p = reinterpret_cast<const uint2*>(base_mu) + h;
#pragma unroll
    for (int c = 0; c < NW; ++c) w[c] = ld_stream(p + (size_t)c * Vh);
  }
  __device__ static void unpack(const Word w[NW], float u[18]) {
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      const float2 a = unpack_h2(w[c].x), b = unpack_h2(w[c].y);
      u[4 * c] = a.x;
      u[4 * c + 1] = a.y;
      u[4 * c + 2] = b.x;
      u[4 * c + 3] = b.y;
    }
  }
  __device__ static void load(const void* base_mu, int Vh, int h, float u[18]) {
    h = LQCD_SITE(h, Vh);
    Word w[NW];
    load_raw(base_mu, Vh, h, w);
    unpack(w, u);
  }
};

// a_i b_j - a_j b_i for complex a_i, b_j, a_j, b_i, in a fixed order of products and sums
template <typename R>
__device__ __forceinline__ Cx<R> cross_term(Cx<R> ai, Cx<R> bj, Cx<R> aj, Cx<R> bi) {
  R re = f_mul(ai.re, bj.re);
  re = f_fma(-ai.im, bj.im, re);
  re = f_fma(-aj.re, bi.re, re);
  re = f_fma(aj.im, bi.im, re);
  R im = f_mul(ai.re, bj.im);
  im = f_fma(ai.im, bj.re, im);
  im = f_fma(-aj.re, bi.im, im);
  im = f_fma(-aj.im, bi.re, im);
  return {re, im};
}

// row 2 = conj(row0 x row1)
template <typename R>
__device__ __forceinline__ void reconstruct_row2(R u[18]) {
  const Cx<R> a0{u[0], u[1]}, a1{u[2], u[3]}, a2{u[4], u[5]};
  const Cx<R> b0{u[6], u[7]}, b1{u[8], u[9]}, b2{u[10], u[11]};
  // c_k = a_i b_j - a_j b_i (k, i, j cyclic); row2_k = conj(c_k)
  const Cx<R> c0 = cross_term(a1, b2, a2, b1);
  const Cx<R> c1 = cross_term(a2, b0, a0, b2);
  const Cx<R> c2 = cross_term(a0, b1, a1, b0);
  u[12] = c0.re; u[13] = -c0.im;
  u[14] = c1.re; u[15] = -c1.im;
  u[16] = c2.re; u[17] = -c2.im;
}

template <int LP, int NR>
__device__ __forceinline__ void load_link(const void* base_mu, int Vh, int h,
                                          typename LinkIO<LP, NR>::Real u[18]) {
  LinkIO<LP, NR>::load(base_mu, Vh, h, u);
  if (NR == 12) reconstruct_row2(u);
}

// Number of reals stored per link and the word size of each link chunk.
__host__ __device__ inline int link_reals(int compress) { return compress == 12 ? 12 : 18; }

}  // namespace lqcd
