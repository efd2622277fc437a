// Reduction totals and scalar finishers of batched launches (k_finish).
//
// A reducing kernel leaves one FP64 partial per tile (per sum, strided by 3) at
// partials[slot.tile0 + tile]. k_finish, issued right after it on the same stream, adds
// each slot's partials in a fixed order and runs the slot's scalar program (run_fin). The
// kernel boundary orders the partials. A slot of n tiles is summed by
// G = min(16, ceil(n / 1024)) CTAs, fixed by n alone, so the result never depends on the
// batch or the grid: CTA q adds tiles [q c, (q + 1) c), c = ceil(n / G), thread t taking
// tiles q c + t, q c + t + 256, ... in that order, then a fixed tree; its sum replaces the
// group's first partial. With G > 1 the last group to finish (an atomic ticket on
// Scalars::ticket after a fence) adds the G group sums in order. The groups spread a large
// slot over several SMs (one SM adds FP64 at 2 per clock, and a 32^3x64 slot has 16 k
// partials), while a small slot keeps a single CTA and no ticket.
#include "launch.h"

namespace lqcd {
namespace {

constexpr int FINISH_THREADS = 256;
constexpr int FINISH_GROUPS = 16;     // most CTAs per slot
constexpr int FINISH_TILES = 1024;    // tiles per CTA before a slot takes another CTA

__device__ __forceinline__ int finish_groups(int ntiles) {
  const int g = (ntiles + FINISH_TILES - 1) / FINISH_TILES;
  return g < 1 ? 1 : (g > FINISH_GROUPS ? FINISH_GROUPS : g);
}

__global__ void __launch_bounds__(FINISH_THREADS) k_finish(const Launch L) {
  __shared__ double sh[FINISH_THREADS / 32];
  __shared__ int am_last;
  pdl_entry();
  const int slot = blockIdx.x, q = blockIdx.y;
  if (slot >= L.nslots) return;
  const Work& w = work_of(L, slot);
  if ((!w.red && w.fin == FIN_NONE) || !slot_runs(w)) return;
  const int G = finish_groups(w.ntiles);
  if (q >= G) return;
  const int ns = (w.red >= 2) ? 3 : 1;
  const int chunk = (w.ntiles + G - 1) / G;
  const int lo = q * chunk, hi = min(w.ntiles, lo + chunk);
  double* part = L.partials + 3 * (size_t)w.tile0;
  constexpr int UNR = 4;
  double acc[3] = {0, 0, 0};
  for (int i0 = lo + (int)threadIdx.x; i0 < hi; i0 += UNR * FINISH_THREADS) {
    double x[UNR][3];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int i = i0 + u * FINISH_THREADS;
      const double* src = part + 3 * (size_t)(i < hi ? i : lo);
#pragma unroll
      for (int k = 0; k < 3; ++k) x[u][k] = (k < ns) ? __ldcg(src + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
      if (i0 + u * FINISH_THREADS < hi)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < ns) acc[k] += x[u][k];
  }
  double tot[3] = {0, 0, 0};
  for (int k = 0; k < ns; ++k) tot[k] = block_sum<FINISH_THREADS>(acc[k], sh);
  if (G == 1) {
    if (threadIdx.x == 0) run_fin(w, tot);
    return;
  }
  if (threadIdx.x == 0) {
    if (lo < hi) {
      for (int k = 0; k < ns; ++k) part[3 * (size_t)lo + k] = tot[k];
    }
    __threadfence();
    const unsigned ticket = atomicAdd(&w.sc->ticket, 1u);
    am_last = (ticket == (unsigned)G - 1);
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double s[3] = {0, 0, 0};
    for (int g = 0; g < G; ++g) {
      const int glo = g * chunk;
      if (glo >= w.ntiles) break;
      for (int k = 0; k < ns; ++k) s[k] += __ldcg(part + 3 * (size_t)glo + k);
    }
    w.sc->ticket = 0;
    run_fin(w, s);
  }
}

}  // namespace

cudaError_t launch_finish(const Launch& L, cudaStream_t s) {
  if (L.nslots <= 0) return cudaSuccess;
  // enough groups for the largest slot (no slot has more tiles than the launch)
  int gy = (L.ntiles + FINISH_TILES - 1) / FINISH_TILES;
  gy = gy < 1 ? 1 : (gy > FINISH_GROUPS ? FINISH_GROUPS : gy);
  return launch_k(k_finish, dim3(L.nslots, gy), dim3(FINISH_THREADS), 0, s, L);
}

}  // namespace lqcd
