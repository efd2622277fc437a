// Host-side launch entry points of the batched kernels (one translation unit
// per spinor precision instantiates them).
#pragma once

#include <cuda_runtime.h>

#include "batch.cuh"

namespace lqcd {

// Link storage precision paired with a spinor precision.
inline int link_prec_for(int sp) { return (sp == P_F64 || sp == P_F32 || sp == P_DF64) ? sp : P_F16; }

// grid <= 0: persistent grid from the occupancy of the kernel (tuned multiplier).
cudaError_t launch_dslash(int sp, int nr, bool dag, int epi, const Launch& L, int grid,
                          cudaStream_t s);
// tp: precision of the FP64-class operand of the mixed ops (P_F64 or P_DF64)
cudaError_t launch_blas(int sp, int op, const Launch& L, int grid, cudaStream_t s, int tp = P_F64);

// per precision
#define LQCD_DECL(SFX)                                                                     \
  cudaError_t launch_dslash_##SFX(int nr, bool dag, int epi, const Launch& L, int grid,   \
                                  cudaStream_t s);                                         \
  cudaError_t launch_blas_##SFX(int op, int tp, const Launch& L, int grid, cudaStream_t s);
LQCD_DECL(f64)
LQCD_DECL(f32)
LQCD_DECL(f16)
LQCD_DECL(bf16)
LQCD_DECL(df64)
#undef LQCD_DECL

// Number of SMs of the current device and the persistent-grid multiplier.
int device_sm_count();
void set_grid_multiplier(int kernel_family, int mult);  // 0 = occupancy limit
int grid_for(const void* kernel_fn, int ntiles, int family, int block);

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
