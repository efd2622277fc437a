// Layout kernels (gauge and spinor upload, even-odd split, precision
// conversion, link compression) and the host dispatch of batched launches.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "launch.h"

namespace lqcd {

// ------------------------------------------------------------------ scalar real access

template <int P>
__device__ __forceinline__ void st_real(void* base, size_t i, double v);
template <>
__device__ __forceinline__ void st_real<P_F64>(void* b, size_t i, double v) { ((double*)b)[i] = v; }
template <>
__device__ __forceinline__ void st_real<P_F32>(void* b, size_t i, double v) { ((float*)b)[i] = (float)v; }
template <>
__device__ __forceinline__ void st_real<P_F16>(void* b, size_t i, double v) { ((__half*)b)[i] = __double2half(v); }
template <>
__device__ __forceinline__ void st_real<P_BF16>(void* b, size_t i, double v) {
  ((__nv_bfloat16*)b)[i] = __double2bfloat16(v);
}

template <>
__device__ __forceinline__ void st_real<P_DF64>(void* b, size_t i, double v) {
  const float hi = __double2float_rn(v);
  ((float*)b)[2 * i] = hi;
  ((float*)b)[2 * i + 1] = __double2float_rn(v - (double)hi);
}

template <int P>
__device__ __forceinline__ double ld_real(const void* base, size_t i);
template <>
__device__ __forceinline__ double ld_real<P_DF64>(const void* b, size_t i) {
  return (double)((const float*)b)[2 * i] + (double)((const float*)b)[2 * i + 1];
}
template <>
__device__ __forceinline__ double ld_real<P_F64>(const void* b, size_t i) { return ((const double*)b)[i]; }
template <>
__device__ __forceinline__ double ld_real<P_F32>(const void* b, size_t i) { return ((const float*)b)[i]; }
template <>
__device__ __forceinline__ double ld_real<P_F16>(const void* b, size_t i) { return __half2float(((const __half*)b)[i]); }
template <>
__device__ __forceinline__ double ld_real<P_BF16>(const void* b, size_t i) {
  return __bfloat162float(((const __nv_bfloat16*)b)[i]);
}

// reals per storage word
__host__ __device__ inline int link_word(int p, int nr) {
  return (p == P_F64 || p == P_DF64) ? 2 : (nr == 18 ? 2 : 4);
}
__host__ __device__ inline int spinor_word(int p) { return 16 / prec_bytes(p); }

// offset (in reals) of real k of link (parity, mu, h)
__device__ __forceinline__ size_t link_off(int p, int nr, int Vh, int par, int mu, int h, int k) {
  const int W = link_word(p, nr);
  return (size_t)par * 4 * nr * Vh + (size_t)mu * nr * Vh + (size_t)(k / W) * Vh * W +
         (size_t)h * W + (k % W);
}
__device__ __forceinline__ size_t spinor_off(int p, int Vh, int h, int k) {
  const int W = spinor_word(p);
  return (size_t)(k / W) * Vh * W + (size_t)h * W + (k % W);
}

// host real k = (spin * 3 + colour) * 2 + re/im  ->  device position (colour-major)
__device__ __forceinline__ int dev_real(int k) {
  const int ri = k & 1, sc = k >> 1, spin = sc / 3, col = sc % 3;
  return sidx(spin, col) + ri;
}

__device__ __forceinline__ void full_coords(const Geom& g, long long s, int& par, int& h) {
  int x = (int)(s % g.L[0]);
  long long r = s / g.L[0];
  int y = (int)(r % g.L[1]);
  r /= g.L[1];
  int z = (int)(r % g.L[2]);
  int t = (int)(r / g.L[2]);
  par = (x + y + z + t) & 1;
  h = (int)(s >> 1);  // Lx even: (x >> 1) + Lxh * (y + Ly * (z + Lz * t))
}

// ------------------------------------------------------------------ gauge

template <int P, int NR>
__global__ void k_gauge_from_aos(const double* __restrict__ aos, Geom g, void* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // site * 4 + mu
  const long long V = 2LL * g.Vh;
  if (i >= 4 * V) return;
  const long long s = i >> 2;
  const int mu = (int)(i & 3);
  int par, h;
  full_coords(g, s, par, h);
  const double* src = aos + i * 18;
  for (int k = 0; k < NR; ++k) st_real<P>(out, link_off(P, NR, g.Vh, par, mu, h, k), src[k]);
}

template <int P, int NR>
__global__ void k_gauge_convert(const void* __restrict__ in64, Geom g, void* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (par, mu, h)
  const long long n = 8LL * g.Vh;
  if (i >= n) return;
  const int h = (int)(i % g.Vh);
  const int mu = (int)((i / g.Vh) & 3);
  const int par = (int)(i / (4LL * g.Vh));
  for (int k = 0; k < NR; ++k) {
    const double v = ld_real<P_F64>(in64, link_off(P_F64, 18, g.Vh, par, mu, h, k));
    st_real<P>(out, link_off(P, NR, g.Vh, par, mu, h, k), v);
  }
}

template <int P, int NR>
static cudaError_t go_gauge_from_aos(const double* a, const Geom& g, void* o, cudaStream_t s) {
  const long long n = 8LL * g.Vh;
  k_gauge_from_aos<P, NR><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, g, o);
  return cudaGetLastError();
}
template <int P, int NR>
static cudaError_t go_gauge_convert(const void* a, const Geom& g, void* o, cudaStream_t s) {
  const long long n = 8LL * g.Vh;
  k_gauge_convert<P, NR><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, g, o);
  return cudaGetLastError();
}

cudaError_t gauge_from_aos(const double* d_aos, const Geom& g, int prec, int nr, void* d_out,
                           cudaStream_t s) {
  if (prec == P_F64) return nr == 12 ? go_gauge_from_aos<P_F64, 12>(d_aos, g, d_out, s)
                                     : go_gauge_from_aos<P_F64, 18>(d_aos, g, d_out, s);
  if (prec == P_F32) return nr == 12 ? go_gauge_from_aos<P_F32, 12>(d_aos, g, d_out, s)
                                     : go_gauge_from_aos<P_F32, 18>(d_aos, g, d_out, s);
  if (prec == P_F16) return nr == 12 ? go_gauge_from_aos<P_F16, 12>(d_aos, g, d_out, s)
                                     : go_gauge_from_aos<P_F16, 18>(d_aos, g, d_out, s);
  if (prec == P_DF64) return nr == 12 ? go_gauge_from_aos<P_DF64, 12>(d_aos, g, d_out, s)
                                      : go_gauge_from_aos<P_DF64, 18>(d_aos, g, d_out, s);
  return cudaErrorInvalidValue;
}

cudaError_t gauge_convert(const void* d64, const Geom& g, int prec, int nr, void* d_out,
                          cudaStream_t s) {
  if (prec == P_F64) return nr == 12 ? go_gauge_convert<P_F64, 12>(d64, g, d_out, s)
                                     : go_gauge_convert<P_F64, 18>(d64, g, d_out, s);
  if (prec == P_F32) return nr == 12 ? go_gauge_convert<P_F32, 12>(d64, g, d_out, s)
                                     : go_gauge_convert<P_F32, 18>(d64, g, d_out, s);
  if (prec == P_F16) return nr == 12 ? go_gauge_convert<P_F16, 12>(d64, g, d_out, s)
                                     : go_gauge_convert<P_F16, 18>(d64, g, d_out, s);
  if (prec == P_DF64) return nr == 12 ? go_gauge_convert<P_DF64, 12>(d64, g, d_out, s)
                                      : go_gauge_convert<P_DF64, 18>(d64, g, d_out, s);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ spinors

template <int P>
__global__ void k_spinor_from_aos(const double* __restrict__ aos, Geom g, void* ev, void* od) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2LL * g.Vh) return;
  int par, h;
  full_coords(g, s, par, h);
  void* dst = par ? od : ev;
  if (!dst) return;
  const double* src = aos + s * 24;
  for (int k = 0; k < 24; ++k) st_real<P>(dst, spinor_off(P, g.Vh, h, dev_real(k)), src[k]);
}

template <int P>
__global__ void k_spinor_to_aos(const void* ev, const void* od, Geom g, double* __restrict__ aos) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2LL * g.Vh) return;
  int par, h;
  full_coords(g, s, par, h);
  const void* src = par ? od : ev;
  if (!src) return;
  double* dst = aos + s * 24;
  for (int k = 0; k < 24; ++k) dst[k] = ld_real<P>(src, spinor_off(P, g.Vh, h, dev_real(k)));
}

template <int PI, int PO>
__global__ void k_spinor_convert(const void* in, void* out, int Vh, double scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (h, k)
  if (i >= 24LL * Vh) return;
  const int h = (int)(i / 24), k = (int)(i % 24);
  st_real<PO>(out, spinor_off(PO, Vh, h, k), scale * ld_real<PI>(in, spinor_off(PI, Vh, h, k)));
}

template <int P>
static cudaError_t go_from_aos(const double* a, const Geom& g, void* e, void* o, cudaStream_t s) {
  const long long n = 2LL * g.Vh;
  k_spinor_from_aos<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, g, e, o);
  return cudaGetLastError();
}
template <int P>
static cudaError_t go_to_aos(const void* e, const void* o, const Geom& g, double* a, cudaStream_t s) {
  const long long n = 2LL * g.Vh;
  k_spinor_to_aos<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(e, o, g, a);
  return cudaGetLastError();
}

cudaError_t spinor_from_aos(const double* d_aos, const Geom& g, int prec, void* d_even,
                            void* d_odd, cudaStream_t s) {
  switch (prec) {
    case P_F64: return go_from_aos<P_F64>(d_aos, g, d_even, d_odd, s);
    case P_F32: return go_from_aos<P_F32>(d_aos, g, d_even, d_odd, s);
    case P_F16: return go_from_aos<P_F16>(d_aos, g, d_even, d_odd, s);
    case P_BF16: return go_from_aos<P_BF16>(d_aos, g, d_even, d_odd, s);
    case P_DF64: return go_from_aos<P_DF64>(d_aos, g, d_even, d_odd, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t spinor_to_aos(const void* d_even, const void* d_odd, const Geom& g, int prec,
                          double* d_aos, cudaStream_t s) {
  switch (prec) {
    case P_F64: return go_to_aos<P_F64>(d_even, d_odd, g, d_aos, s);
    case P_F32: return go_to_aos<P_F32>(d_even, d_odd, g, d_aos, s);
    case P_F16: return go_to_aos<P_F16>(d_even, d_odd, g, d_aos, s);
    case P_BF16: return go_to_aos<P_BF16>(d_even, d_odd, g, d_aos, s);
    case P_DF64: return go_to_aos<P_DF64>(d_even, d_odd, g, d_aos, s);
  }
  return cudaErrorInvalidValue;
}

template <int PI>
static cudaError_t go_convert_in(const void* in, void* out, int pout, int Vh, double sc,
                                 cudaStream_t s) {
  const long long n = 24LL * Vh;
  const unsigned nb = (unsigned)((n + 255) / 256);
  switch (pout) {
    case P_F64: k_spinor_convert<PI, P_F64><<<nb, 256, 0, s>>>(in, out, Vh, sc); break;
    case P_F32: k_spinor_convert<PI, P_F32><<<nb, 256, 0, s>>>(in, out, Vh, sc); break;
    case P_F16: k_spinor_convert<PI, P_F16><<<nb, 256, 0, s>>>(in, out, Vh, sc); break;
    case P_BF16: k_spinor_convert<PI, P_BF16><<<nb, 256, 0, s>>>(in, out, Vh, sc); break;
    case P_DF64: k_spinor_convert<PI, P_DF64><<<nb, 256, 0, s>>>(in, out, Vh, sc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t spinor_convert(const void* in, int pin, void* out, int pout, int Vh, double scale,
                           cudaStream_t s) {
  switch (pin) {
    case P_F64: return go_convert_in<P_F64>(in, out, pout, Vh, scale, s);
    case P_F32: return go_convert_in<P_F32>(in, out, pout, Vh, scale, s);
    case P_F16: return go_convert_in<P_F16>(in, out, pout, Vh, scale, s);
    case P_BF16: return go_convert_in<P_BF16>(in, out, pout, Vh, scale, s);
    case P_DF64: return go_convert_in<P_DF64>(in, out, pout, Vh, scale, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ dispatch

// the slots' reduction totals and scalar finishers of the launch just issued on s
static cudaError_t then_finish(cudaError_t err, const Launch& L, cudaStream_t s) {
  if (err != cudaSuccess || !L.finish) return err;
  return launch_finish(L, s);
}

cudaError_t launch_dslash(int sp, int nr, bool dag, int epi, const Launch& L, int grid,
                          cudaStream_t s, int form) {
  // no slot reduces or finishes: the instantiation without the reduction code (a batched
  // launch's finish flag covers its running slots; an inline Work says so itself)
  if (epi == EPI_LIN && !L.finish &&
      (L.works || (!L.inline_work.red && L.inline_work.fin == FIN_NONE)))
    epi = EPI_PLAIN;
  switch (sp) {
    case P_F64: return then_finish(launch_dslash_f64(nr, dag, epi, L, grid, s, form), L, s);
    case P_F32: return then_finish(launch_dslash_f32(nr, dag, epi, L, grid, s, form), L, s);
    case P_F16: return then_finish(launch_dslash_f16(nr, dag, epi, L, grid, s, form), L, s);
    case P_BF16: return then_finish(launch_dslash_bf16(nr, dag, epi, L, grid, s, form), L, s);
    case P_DF64: return then_finish(launch_dslash_df64(nr, dag, epi, L, grid, s, form), L, s);
  }
  return cudaErrorInvalidValue;
}

// Programmatic dependent launch of the batched kernels (each CTA lets the next grid launch
// when it starts its last tile). Measured on GB300: the batched 16^3x32 FP32 Dslash of ten
// slots per launch, applied back to back, 81.5 -> 80.5 us per launch; the solvers' step
// chains gain where their launches are small (up to PDL_SOLVER_MAX_TILES tiles) and lose
// where they are large (launch.h). So it is on for the operator launches (lqcd_dslash_eo,
// batches, M-hat) and the small solvers, and off in the large ones (PdlSolverScope);
// LQCD_PDL=1 turns it on everywhere, LQCD_PDL=0 off everywhere.
namespace {
thread_local int t_solver_depth = 0;
}
PdlSolverScope::PdlSolverScope(bool off) : off_(off) {
  if (off_) ++t_solver_depth;
}
PdlSolverScope::~PdlSolverScope() {
  if (off_) --t_solver_depth;
}

bool pdl_enabled() {
  static const int mode = [] {
    const char* v = std::getenv("LQCD_PDL");
    if (!v || !v[0]) return -1;
    return v[0] == '1' ? 1 : 0;
  }();
  if (mode >= 0) return mode == 1;
  return t_solver_depth == 0;
}

int dslash_occupancy(int sp, int nr, int form) {
  switch (sp) {
    case P_F64: return dslash_occupancy_f64(nr, form);
    case P_F32: return dslash_occupancy_f32(nr, form);
    case P_F16: return dslash_occupancy_f16(nr, form);
    case P_BF16: return dslash_occupancy_bf16(nr, form);
    case P_DF64: return dslash_occupancy_df64(nr, form);
  }
  return 0;
}

cudaError_t launch_blas(int sp, int op, const Launch& L, int grid, cudaStream_t s, int tp) {
  switch (sp) {
    case P_F64: return then_finish(launch_blas_f64(op, tp, L, grid, s), L, s);
    case P_F32: return then_finish(launch_blas_f32(op, tp, L, grid, s), L, s);
    case P_F16: return then_finish(launch_blas_f16(op, tp, L, grid, s), L, s);
    case P_BF16: return then_finish(launch_blas_bf16(op, tp, L, grid, s), L, s);
    case P_DF64: return then_finish(launch_blas_df64(op, tp, L, grid, s), L, s);
  }
  return cudaErrorInvalidValue;
}

namespace {
std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ;  // kernel -> resident CTAs per SM
int g_mult[4] = {0, 0, 0, 0};
int g_nsm = 0;
int g_nsm_dev = -1;
}  // namespace

int device_sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_occ_mu);
  if (g_nsm_dev != dev) {
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    g_nsm_dev = dev;
    g_occ.clear();
  }
  return g_nsm;
}

void set_grid_multiplier(int family, int mult) {
  if (family >= 0 && family < 4) g_mult[family] = mult;
}

namespace {
bool g_split[NPREC] = {false, false, false, false, true};
}  // namespace

bool dslash_colour_split(int prec) { return prec >= 0 && prec < NPREC && g_split[prec]; }
void set_dslash_colour_split(int prec, bool on) {
  if (prec >= 0 && prec < NPREC) g_split[prec] = on;
}

int kernel_occupancy(const void* fn, int block) {
  device_sm_count();  // resets the cache when the device changed
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto it = g_occ.find(fn);
  if (it != g_occ.end()) return it->second;
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, block, 0) != cudaSuccess || o < 1) {
    cudaGetLastError();
    o = 1;
  }
  g_occ[fn] = o;
  return o;
}

int grid_for(const void* fn, int ntiles, int family, int block, int ctas_per_sm) {
  const int nsm = device_sm_count();
  int occ = kernel_occupancy(fn, block);
  int m = (family >= 0 && family < 4) ? g_mult[family] : 0;
  if (m > 0 && m < occ) occ = m;
  if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
  long long grid = (long long)nsm * occ;
  if (grid > ntiles) grid = ntiles;
  return (int)(grid < 1 ? 1 : grid);
}

}  // namespace lqcd
