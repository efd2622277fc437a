// Host-side launch entry points of the batched kernels (one translation unit
// per spinor precision instantiates them).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "batch.cuh"

namespace lqcd {

// Link storage precision paired with a spinor precision.
inline int link_prec_for(int sp) { return (sp == P_F64 || sp == P_F32 || sp == P_DF64) ? sp : P_F16; }

// grid <= 0: persistent grid of the autotuned CTAs per SM (else the occupancy limit);
// form < 0: the autotuned Dslash form (else the default), 0 site, 1 colour split,
// 3 site at the second register budget (FP32 only; other precisions take form 0).
cudaError_t launch_dslash(int sp, int nr, bool dag, int epi, const Launch& L, int grid,
                          cudaStream_t s, int form = -1);
// tp: precision of the FP64-class operand of the mixed ops (P_F64 or P_DF64)
cudaError_t launch_blas(int sp, int op, const Launch& L, int grid, cudaStream_t s, int tp = P_F64);
// k_finish for a launch whose slots reduce or finish (finish.cu); launch_dslash and
// launch_blas issue it themselves when L.finish is set
cudaError_t launch_finish(const Launch& L, cudaStream_t s);

// per precision
#define LQCD_DECL(SFX)                                                                     \
  cudaError_t launch_dslash_##SFX(int nr, bool dag, int epi, const Launch& L, int grid,   \
                                  cudaStream_t s, int form);                               \
  int dslash_occupancy_##SFX(int nr, int form);                                            \
  cudaError_t launch_blas_##SFX(int op, int tp, const Launch& L, int grid, cudaStream_t s);
LQCD_DECL(f64)
LQCD_DECL(f32)
LQCD_DECL(f16)
LQCD_DECL(bf16)
LQCD_DECL(df64)
#undef LQCD_DECL

// Launches of the batched kernels, with programmatic stream serialization where enabled:
// the kernel may then be launched before the previous kernel on the stream completes, and
// waits for it itself (pdl_wait in batch.cuh). Enabled for operator launches and for the
// step chains of small solves; disabled while a PdlSolverScope(true) is alive on the calling
// thread, which the solvers open when their launches hold more than PDL_SOLVER_MAX_TILES
// tiles; LQCD_PDL=1 / 0 forces it on / off everywhere.
bool pdl_enabled();
struct PdlSolverScope {
  explicit PdlSolverScope(bool off);
  ~PdlSolverScope();
  PdlSolverScope(const PdlSolverScope&) = delete;
  PdlSolverScope& operator=(const PdlSolverScope&) = delete;
  bool off_;
};
// Measured on GB300: in solver step chains of up to about two tiles per resident CTA (8^4 to
// 16^3x32 one slot at a time, the 16^3x32 HMC) the programmatic launch hides launch latency
// (one-by-one small solves 9% faster, HMC 2%); in larger ones it costs up to 10% (the
// 32^3x64 double-float CG, the 64-lattice engine 6%).
constexpr long long PDL_SOLVER_MAX_TILES = 2048;
inline bool pdl_solver_off(long long tiles) { return tiles > PDL_SOLVER_MAX_TILES; }
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t dyn_smem, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = dyn_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Number of SMs of the current device and the persistent-grid multiplier.
int device_sm_count();
void set_grid_multiplier(int kernel_family, int mult);  // 0 = occupancy limit
// ctas_per_sm > 0 caps the grid below the occupancy limit (autotuned choice)
int grid_for(const void* kernel_fn, int ntiles, int family, int block, int ctas_per_sm = 0);
int kernel_occupancy(const void* kernel_fn, int block);
// resident CTAs per SM of the Dslash of this precision, link reals and form (0 if no such
// form): 0 one thread per site, 1 colour split (double-float), 2 shared-link multi-RHS,
// 3 one thread per site at 8 CTAs per SM (FP32)
int dslash_occupancy(int sp, int nr, int form);

// Autotuner table (tune.cu): the launch choice for Dslash launches of this precision and
// link reals whose tile count has the same floor(log2) as a tuned launch.
struct TuneChoice {
  int ctas_per_sm;  // 0: occupancy limit
  int form;         // 0 site, 1 colour split, 3 site at the second register budget
};
TuneChoice tune_choice(int sp, int nr, int ntiles);
// Shared-link choice for nrhs slots on one gauge field of `blocks` site blocks: the tuned
// slots per group (0: every slot loads its own links), with *ctas_per_sm the tuned grid
// (0: occupancy limit); -1 when nothing was tuned for the key.
int tune_shared_links(int sp, int nr, int nrhs, int blocks, int* ctas_per_sm);

// Whether the Dslash of spinor precision prec uses the colour-split form (double-float
// only; a runtime switch for measurement).
bool dslash_colour_split(int prec);
void set_dslash_colour_split(int prec, bool on);


// layout kernels (layout.cu)
cudaError_t gauge_from_aos(const double* d_aos, const Geom& g, int prec, int nr, void* d_out,
                           cudaStream_t s);
cudaError_t gauge_convert(const void* d_f64_18, const Geom& g, int prec, int nr, void* d_out,
                          cudaStream_t s);
cudaError_t spinor_from_aos(const double* d_aos, const Geom& g, int prec, void* d_even,
                            void* d_odd, cudaStream_t s);
cudaError_t spinor_to_aos(const void* d_even, const void* d_odd, const Geom& g, int prec,
                          double* d_aos, cudaStream_t s);
cudaError_t spinor_convert(const void* d_in, int pin, void* d_out, int pout, int Vh, double scale,
                           cudaStream_t s);

}  // namespace lqcd
