// lqcd_apply_Mhat_noalloc: the even-odd operator Mhat without any device
// allocation by the library.
//
// lqcd_apply_Mhat needs an odd-parity temporary t = D_oe in, which it takes
// from a context buffer that it grows with cudaMalloc on demand. Some callers
// cannot let a library allocate: an application that hands all device memory
// to its own pool (for instance PyTorch's caching allocator, or an arena with
// a fixed budget) sees a library cudaMalloc fail with out-of-memory while the
// pool still holds free blocks, and cudaMalloc / cudaFree synchronise the
// device, which stalls every other stream of a latency-sensitive caller. This
// entry point keeps the temporary in a fixed-size array that is part of the
// library image instead, so it never calls cudaMalloc, cudaFree or an
// allocating library routine.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "kernels.cuh"
#include "runtime.h"

namespace {

// Scratch for the odd temporary: 16 MiB, enough for FP32 fields up to
// V/2 = 174762 sites (16^3 x 32 and smaller) or FP64 up to V/2 = 87381.
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(16) << 20;
__device__ __align__(256) unsigned char g_mhat_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to

// Device address of the scratch array on `device` (which must be current).
// Looked up with cudaGetSymbolAddress at the first call on each device: in host
// code the name g_mhat_scratch is only a host-side stand-in and must never
// reach a kernel. The address belongs to the device's current context; if that
// context was destroyed and made again (cudaDeviceReset), the context's unique
// id changes and the address is looked up once more instead of reusing a dead one.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return lqcd::set_error(LQCD_EINVAL, "device %d beyond the %d supported by the scratch table",
                           device, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  // the two driver calls are fetched through the runtime, so that the library does not
  // need the driver library at load time (it loads on machines without a GPU)
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault) != cudaSuccess ||
        !f0 || !f1)
      return lqcd::set_error(LQCD_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
    get_current = reinterpret_cast<GetCurrentFn>(f0);
    get_id = reinterpret_cast<GetIdFn>(f1);
  }
  CUcontext cu = nullptr;
  unsigned long long ctx_id = 0;
  if (get_current(&cu) != CUDA_SUCCESS || !cu || get_id(cu, &ctx_id) != CUDA_SUCCESS)
    return lqcd::set_error(LQCD_ECUDA, "no current CUDA context on device %d", device);
  if (!g_scratch_addr[device] || g_scratch_ctx[device] != ctx_id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_mhat_scratch);
    if (e != cudaSuccess || !p)
      return lqcd::set_error(LQCD_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                             cudaGetErrorString(e));
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = ctx_id;
  }
  *out = g_scratch_addr[device];
  return LQCD_OK;
}

// out_p = a * D_{p,1-p} in + c1 * y1 with the gauge's existing link copy.
int dslash_noalloc(const lqcd_gauge* gauge, int prec, const void* links, int nr, const void* in,
                   void* out, const void* y1, double a, double c1, int out_par, bool dag) {
  using namespace lqcd;
  lqcd_ctx* c = gauge->ctx;
  const int lp = link_prec_for(prec);
  Work w = blank_work(gauge->g);
  w.out_par = out_par;
  w.in = in;
  w.out = out;
  w.Uout = parity_links(links, lp, nr, gauge->g.Vh, out_par);
  w.Uin = parity_links(links, lp, nr, gauge->g.Vh, 1 - out_par);
  w.y1 = y1;
  w.a = a;
  w.c1 = c1;
  w.sc = c->scratch_sc;  // no reduction and no finisher: never written
  LQCD_CK(launch_dslash(prec, nr, dag, EPI_LIN, single_launch(w, nullptr), 0, c->stream));
  c->launches++;
  return LQCD_OK;
}

}  // namespace

extern "C" int lqcd_apply_Mhat_noalloc(const lqcd_gauge* g, double kappa, const lqcd_field* in,
                                       lqcd_field* out, int dagger) {
  LQCD_TRACE("lqcd_apply_Mhat_noalloc");
  using namespace lqcd;
  clear_error();
  if (!g || !in || !out) return set_error(LQCD_EINVAL, "NULL argument");
  if (!std::isfinite(kappa)) return set_error(LQCD_EINVAL, "kappa must be finite");
  if (in->prec != out->prec) return set_error(LQCD_EINVAL, "fields differ in precision");
  if (in->ctx != g->ctx || out->ctx != g->ctx) return set_error(LQCD_EINVAL, "objects of different contexts");
  for (int mu = 0; mu < 4; ++mu)
    if (in->g.L[mu] != g->g.L[mu] || out->g.L[mu] != g->g.L[mu])
      return set_error(LQCD_EINVAL, "lattice mismatch");
  if (!in->half[0] || !out->half[0]) return set_error(LQCD_EINVAL, "fields must hold the even parity");
  if (in->half[0] == out->half[0]) return set_error(LQCD_EINVAL, "in and out must differ");
  const size_t need = half_spinor_bytes(in->prec, g->g.Vh);
  if (need > kScratchBytes)
    return set_error(LQCD_EINVAL,
                     "lqcd_apply_Mhat_noalloc: the odd temporary needs %zu bytes, more than its "
                     "fixed scratch of %zu bytes (use lqcd_apply_Mhat for this lattice)",
                     need, kScratchBytes);
  const int lp = link_prec_for(in->prec);
  // the copy lqcd_apply_Mhat would use: the gauge's compression, except double-float
  // links, which always keep 18 reals
  const int nr = (lp == P_DF64) ? 18 : g->compress;
  const void* links = g->copy[lp][nr == 12];
  if (!links)
    return set_error(LQCD_EINVAL,
                     "lqcd_apply_Mhat_noalloc: no resident %d-real link copy for this precision; "
                     "create it first with lqcd_gauge_add_copy(g, prec, %d)",
                     nr, nr);
  LQCD_CK(cudaSetDevice(g->ctx->device));
  void* tmp = nullptr;
  int rc = scratch_address(g->ctx->device, &tmp);
  if (rc != LQCD_OK) return rc;
  rc = dslash_noalloc(g, in->prec, links, nr, in->half[0], tmp, nullptr, 1.0, 0.0, 1, dagger != 0);
  if (rc != LQCD_OK) return rc;
  return dslash_noalloc(g, in->prec, links, nr, tmp, out->half[0], in->half[0], -kappa * kappa, 1.0,
                        0, dagger != 0);
}
