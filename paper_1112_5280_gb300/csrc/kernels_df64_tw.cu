// Twisted-mass Dslash epilogues, spinor storage DF64 (double-float pairs), in a
// translation unit of their own (compiled in parallel with kernels_df64.cu).
#define LQCD_SP lqcd::P_DF64
#define LQCD_SFX df64
#define LQCD_TW_UNIT 1
#include "kernels_inst.cuh"
