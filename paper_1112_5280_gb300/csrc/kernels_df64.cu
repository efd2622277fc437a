// Batched Dslash and BLAS kernels, spinor storage DF64 (double-float pairs).
#define LQCD_SP lqcd::P_DF64
#define LQCD_SFX df64
#define LQCD_TW_EXTERN 1
#include "kernels_inst.cuh"
