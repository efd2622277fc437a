// Instantiates the batched kernels for one spinor precision LQCD_SP with
// launch-function suffix LQCD_SFX. Included by kernels_<prec>.cu.
#include "kernels.cuh"
#include "launch.h"

namespace lqcd {

#define LQCD_CAT2(a, b) a##b
#define LQCD_CAT(a, b) LQCD_CAT2(a, b)

namespace {
constexpr int SPX = LQCD_SP;
constexpr int LPX = (SPX == P_F64 || SPX == P_DF64 || SPX == P_F32) ? SPX : P_F16;

template <int NR, bool DAG, int EPI>
cudaError_t go_dslash(const Launch& L, int grid, cudaStream_t s) {
  if (L.ntiles <= 0) return cudaSuccess;
  if constexpr (SPX == P_DF64 && NR == 18) {
    if (dslash_colour_split(SPX)) {
      // double-float: the colour-split form (latency bound at one thread per site)
      auto fn3 = k_dslash3<SPX, LPX, DAG, EPI>;
      if (grid <= 0) grid = grid_for((const void*)fn3, L.ntiles, 0, 3 * TILE);
      fn3<<<grid, 3 * TILE, 0, s>>>(L);
      return cudaGetLastError();
    }
  }
  auto fn = k_dslash<SPX, LPX, NR, DAG, EPI>;
  if (grid <= 0) grid = grid_for((const void*)fn, L.ntiles, 0, TILE);
  fn<<<grid, TILE, 0, s>>>(L);
  return cudaGetLastError();
}

template <int OP, int P, int TP = P_F64>
cudaError_t go_blas(const Launch& L, int grid, cudaStream_t s) {
  auto fn = k_blas<P, OP, TP>;
  if (L.ntiles <= 0) return cudaSuccess;
  if (grid <= 0) grid = grid_for((const void*)fn, L.ntiles, 1, TILE);
  fn<<<grid, TILE, 0, s>>>(L);
  return cudaGetLastError();
}
}  // namespace

cudaError_t LQCD_CAT(launch_dslash_, LQCD_SFX)(int nr, bool dag, int epi, const Launch& L,
                                                int grid, cudaStream_t s) {
  if (nr == 18) {
    if (epi == EPI_LIN) return dag ? go_dslash<18, true, EPI_LIN>(L, grid, s)
                                   : go_dslash<18, false, EPI_LIN>(L, grid, s);
    if (dag) return go_dslash<18, true, EPI_CG>(L, grid, s);
  } else if (nr == 12) {
    if (epi == EPI_LIN) return dag ? go_dslash<12, true, EPI_LIN>(L, grid, s)
                                   : go_dslash<12, false, EPI_LIN>(L, grid, s);
    if (dag) return go_dslash<12, true, EPI_CG>(L, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t LQCD_CAT(launch_blas_, LQCD_SFX)(int op, int tp, const Launch& L, int grid,
                                              cudaStream_t s) {
  const bool df = (tp == P_DF64);
  switch (op) {
    case B_CG_P: return go_blas<B_CG_P, SPX>(L, grid, s);
    case B_NORM: return go_blas<B_NORM, SPX>(L, grid, s);
    case B_ZERO: return go_blas<B_ZERO, SPX>(L, grid, s);
    case B_TWIST: return go_blas<B_TWIST, SPX>(L, grid, s);
    case B_BICG_P: return go_blas<B_BICG_P, SPX>(L, grid, s);
    case B_BICG_S: return go_blas<B_BICG_S, SPX>(L, grid, s);
    case B_BICG_X: return go_blas<B_BICG_X, SPX>(L, grid, s);
    case B_RU_CONVERT:
      return df ? go_blas<B_RU_CONVERT, SPX, P_DF64>(L, grid, s) : go_blas<B_RU_CONVERT, SPX, P_F64>(L, grid, s);
    case B_AXPBY:
      return df ? go_blas<B_AXPBY, SPX, P_DF64>(L, grid, s) : go_blas<B_AXPBY, SPX, P_F64>(L, grid, s);
    case B_FOLD64:
    case B_RU_FOLD:
      if (SPX == P_F64 || SPX == P_F32 || SPX == P_DF64) {
        if (op == B_FOLD64)
          return df ? go_blas<B_FOLD64, SPX, P_DF64>(L, grid, s) : go_blas<B_FOLD64, SPX, P_F64>(L, grid, s);
        return df ? go_blas<B_RU_FOLD, SPX, P_DF64>(L, grid, s) : go_blas<B_RU_FOLD, SPX, P_F64>(L, grid, s);
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqcd
