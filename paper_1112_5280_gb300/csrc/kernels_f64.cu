// Batched Dslash and BLAS kernels, spinor storage F64.
#define LQCD_SP lqcd::P_F64
#define LQCD_SFX f64
#include "kernels_inst.cuh"
