// Batched Dslash and BLAS kernels, spinor storage F32.
#define LQCD_SP lqcd::P_F32
#define LQCD_SFX f32
#include "kernels_inst.cuh"
