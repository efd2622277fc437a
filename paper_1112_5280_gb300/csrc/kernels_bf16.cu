// Batched Dslash and BLAS kernels, spinor storage BF16.
#define LQCD_SP lqcd::P_BF16
#define LQCD_SFX bf16
#include "kernels_inst.cuh"
