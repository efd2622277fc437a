// lqcd_alu_peak: the FMA throughput of this GPU in FP64 and FP32, measured.
//
// The FP64 Dslash (the paper's precision) and the double-float kernels are bound by
// arithmetic, not by HBM, on a part whose FP64 pipe is a small fraction of its FP32
// pipes; their rooflines need the two FMA rates of the device they run on, taken in
// the same process as the kernel times rather than from a datasheet.
#include <cuda_runtime.h>

#include "runtime.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (covers the FMA latency)
constexpr int kThreads = 256;  // per CTA
constexpr int kCtasPerSm = 8;  // 2048 resident threads per SM

__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }
__device__ __forceinline__ float fma_t(float x, float a, float b) { return __fmaf_rn(x, a, b); }

// Every thread runs kChains chains x <- x a + b for `iters` steps. a < 1 and b > 0 keep the
// values bounded and normal. The sum is written only on an impossible value, which keeps
// the chains live without a store per thread.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma_t(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == T(-1)) out[blockIdx.x] = s;
}

// The same with packed FP32 pairs (one fma.rn.f32x2 = two FMAs per lane).
__global__ void __launch_bounds__(kThreads) k_ffma2_peak(float* out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = make_float2((threadIdx.x + i) * 1e-3f, (threadIdx.x + 2 * i) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
  if (s == -1.0f) out[blockIdx.x] = s;
}

template <typename T, bool PACKED = false>
int measure(lqcd_ctx* c, int iters, double* tflops) {
  int sms = 0;
  LQCD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  const int grid = sms * kCtasPerSm;
  T* out = nullptr;
  LQCD_CK(cudaMalloc(&out, sizeof(T) * grid));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.0f;
  int rc = LQCD_OK;
  for (int rep = 0; rep < 6 && rc == LQCD_OK; ++rep) {  // the first run is a warm-up
    cudaEventRecord(e0, c->stream);
    if constexpr (PACKED)
      k_ffma2_peak<<<grid, kThreads, 0, c->stream>>>(out, iters, 0.9999999f, 1e-7f);
    else
      k_fma_peak<T><<<grid, kThreads, 0, c->stream>>>(out, iters, T(0.9999999), T(1e-7));
    cudaEventRecord(e1, c->stream);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) {
      rc = lqcd::set_error(LQCD_ECUDA, "FMA probe: %s", cudaGetErrorString(err));
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != LQCD_OK) return rc;
  const double flop = (PACKED ? 4.0 : 2.0) * kChains * (double)iters * grid * kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return LQCD_OK;
}

}  // namespace

extern "C" int lqcd_alu_peak(lqcd_ctx* ctx, int kind, double* tflops) {
  LQCD_TRACE("lqcd_alu_peak");
  using namespace lqcd;
  clear_error();
  if (!ctx || !tflops) return set_error(LQCD_EINVAL, "NULL argument");
  LQCD_CK(cudaSetDevice(ctx->device));
  // about 15 ms per run at the nominal rates
  if (kind == 0) return measure<double>(ctx, 4000, tflops);
  if (kind == 1) return measure<float>(ctx, 240000, tflops);
  if (kind == 2) return measure<float, true>(ctx, 120000, tflops);
  return set_error(LQCD_EINVAL, "kind %d (0: FP64 FMA, 1: FP32 FMA, 2: packed FP32 FMA)", kind);
}
