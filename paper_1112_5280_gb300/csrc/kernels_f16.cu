// Batched Dslash and BLAS kernels, spinor storage F16.
#define LQCD_SP lqcd::P_F16
#define LQCD_SFX f16
#include "kernels_inst.cuh"
