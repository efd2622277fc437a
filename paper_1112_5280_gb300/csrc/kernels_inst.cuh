// Instantiates the batched kernels for one spinor precision LQCD_SP with
// launch-function suffix LQCD_SFX. Included by kernels_<prec>.cu.
//
// LQCD_TW_UNIT: this translation unit holds only the twisted-mass Dslash epilogues
// (launch_dslash_tw_<sfx>); LQCD_TW_EXTERN: the dispatcher of this unit forwards the
// twisted epilogues to such a unit. Double-float uses the pair, so that its two
// heaviest kernel sets compile in parallel.
#include "kernels.cuh"
#include "launch.h"

namespace lqcd {

#define LQCD_CAT2(a, b) a##b
#define LQCD_CAT(a, b) LQCD_CAT2(a, b)

namespace {
constexpr int SPX = LQCD_SP;
constexpr int LPX = (SPX == P_F64 || SPX == P_DF64 || SPX == P_F32) ? SPX : P_F16;

template <int NR, bool DAG, int EPI>
cudaError_t go_dslash(const Launch& L, int grid, cudaStream_t s, int form) {
  if (L.ntiles <= 0) return cudaSuccess;
  int cps = 0;
  if (form < 0 || grid <= 0) {
    const TuneChoice t = tune_choice(SPX, NR, L.ntiles);
    if (form < 0) form = t.form;
    cps = t.ctas_per_sm;
  }
  // shared-link multi-RHS launches (every slot on one gauge field): FP32-arithmetic
  // precisions, Wilson epilogues
  if (L.interleave == 2) {
    if constexpr ((SPX == P_F32 || SPX == P_F16 || SPX == P_BF16) && !EpiTraits<EPI>::tw) {
      auto fm = k_dslash_mrhs<SPX, LPX, NR, DAG, EPI>;
      if (grid <= 0) {
        int scps = 0;
        tune_shared_links(SPX, NR, L.nslots, L.ntiles / L.mrhs_groups, &scps);
        grid = grid_for((const void*)fm, L.ntiles, 0, TILE, scps);
      }
      return launch_k(fm, dim3(grid), dim3(TILE), 0, s, L);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  // twisted double-float runs the colour-split form alone (the one-thread-per-site form
  // is slower there and its twisted instantiations dominate the build)
  constexpr bool split_only = (SPX == P_DF64 && EpiTraits<EPI>::tw);
  if constexpr (SPX == P_DF64 && NR == 18) {
    if (form == 1 || split_only) {
      // double-float: the colour-split form (latency bound at one thread per site)
      auto fn3 = k_dslash3<SPX, LPX, DAG, EPI>;
      if (grid <= 0) grid = grid_for((const void*)fn3, L.ntiles, 0, 3 * TILE, cps);
      return launch_k(fn3, dim3(grid), dim3(3 * TILE), 0, s, L);
    }
  }
  if constexpr (SPX == P_F32) {
    if (form == 3) {  // the FP32 Dslash at the second register budget
      auto fh = k_dslash<SPX, LPX, NR, DAG, EPI, DSLASH_MIN_BLOCKS_HI>;
      if (grid <= 0) grid = grid_for((const void*)fh, L.ntiles, 0, TILE, cps);
      return launch_k(fh, dim3(grid), dim3(TILE), view_smem(L), s, L);
    }
  }
  if constexpr (!split_only) {
    auto fn = k_dslash<SPX, LPX, NR, DAG, EPI>;
    if (grid <= 0) grid = grid_for((const void*)fn, L.ntiles, 0, TILE, cps);
    return launch_k(fn, dim3(grid), dim3(TILE), view_smem(L), s, L);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int NR>
cudaError_t dispatch_tw(bool dag, int epi, const Launch& L, int grid, cudaStream_t s, int form) {
  switch (epi) {
    case EPI_LIN_TW: return dag ? go_dslash<NR, true, EPI_LIN_TW>(L, grid, s, form)
                                : go_dslash<NR, false, EPI_LIN_TW>(L, grid, s, form);
    case EPI_CG_TW: if (dag) return go_dslash<NR, true, EPI_CG_TW>(L, grid, s, form); break;
  }
  return cudaErrorInvalidValue;
}

template <int OP, int P, int TP = P_F64>
cudaError_t go_blas(const Launch& L, int grid, cudaStream_t s) {
  auto fn = k_blas<P, OP, TP>;
  if (L.ntiles <= 0) return cudaSuccess;
  if (grid <= 0) grid = grid_for((const void*)fn, L.ntiles, 1, TILE);
  return launch_k(fn, dim3(grid), dim3(TILE), 0, s, L);
}
}  // namespace

#ifdef LQCD_TW_UNIT

// double-float links always have 18 reals
cudaError_t LQCD_CAT(launch_dslash_tw_, LQCD_SFX)(int nr, bool dag, int epi, const Launch& L,
                                                   int grid, cudaStream_t s, int form) {
  if (nr != 18) return cudaErrorInvalidValue;
  return dispatch_tw<18>(dag, epi, L, grid, s, form);
}

#else

#ifdef LQCD_TW_EXTERN
cudaError_t LQCD_CAT(launch_dslash_tw_, LQCD_SFX)(int nr, bool dag, int epi, const Launch& L,
                                                   int grid, cudaStream_t s, int form);
#endif

namespace {
template <int NR>
cudaError_t dispatch_nr(bool dag, int epi, const Launch& L, int grid, cudaStream_t s, int form) {
  switch (epi) {
    case EPI_LIN: return dag ? go_dslash<NR, true, EPI_LIN>(L, grid, s, form)
                             : go_dslash<NR, false, EPI_LIN>(L, grid, s, form);
    case EPI_PLAIN: return dag ? go_dslash<NR, true, EPI_PLAIN>(L, grid, s, form)
                               : go_dslash<NR, false, EPI_PLAIN>(L, grid, s, form);
    case EPI_CG: if (dag) return go_dslash<NR, true, EPI_CG>(L, grid, s, form); break;
    case EPI_LIN_TW:
    case EPI_CG_TW:
#ifdef LQCD_TW_EXTERN
      return LQCD_CAT(launch_dslash_tw_, LQCD_SFX)(NR, dag, epi, L, grid, s, form);
#else
      return dispatch_tw<NR>(dag, epi, L, grid, s, form);
#endif
  }
  return cudaErrorInvalidValue;
}

// 12-real links for every precision but double-float (whose links always have 18)
template <int P>
cudaError_t dispatch_12(bool dag, int epi, const Launch& L, int grid, cudaStream_t s, int form) {
  if constexpr (P == P_DF64) {
    return cudaErrorInvalidValue;
  } else {
    return dispatch_nr<12>(dag, epi, L, grid, s, form);
  }
}
}  // namespace

cudaError_t LQCD_CAT(launch_dslash_, LQCD_SFX)(int nr, bool dag, int epi, const Launch& L,
                                                int grid, cudaStream_t s, int form) {
  // a twisted single-slot work needs the twisted epilogue (a batched launch's works live
  // on the device; their callers pick the epilogue from the slots they hold)
  if (!L.works && L.inline_work.twist && epi != EPI_LIN_TW && epi != EPI_CG_TW) return cudaErrorInvalidValue;
  if (nr == 18) return dispatch_nr<18>(dag, epi, L, grid, s, form);
  if (nr == 12) return dispatch_12<SPX>(dag, epi, L, grid, s, form);
  return cudaErrorInvalidValue;
}

namespace {
// a template, so that the colour-split kernel is instantiated for double-float only
template <int P>
int colour_split_occupancy(int nr) {
  if constexpr (P == P_DF64) {
    if (nr == 18) return kernel_occupancy((const void*)k_dslash3<P, LPX, false, EPI_LIN>, 3 * TILE);
  }
  return 0;
}
template <int P>
int site_occupancy_12() {
  if constexpr (P == P_DF64) {
    return 0;
  } else {
    return kernel_occupancy((const void*)k_dslash<P, LPX, 12, false, EPI_LIN>, TILE);
  }
}
}  // namespace

template <int P>
int shared_link_occupancy(int nr) {
  if constexpr (P == P_F32 || P == P_F16 || P == P_BF16) {
    if (nr == 18) return kernel_occupancy((const void*)k_dslash_mrhs<P, LPX, 18, false, EPI_LIN>, TILE);
    if (nr == 12) return kernel_occupancy((const void*)k_dslash_mrhs<P, LPX, 12, false, EPI_LIN>, TILE);
  }
  return 0;
}

namespace {
template <int P>
int second_budget_occupancy(int nr) {
  if constexpr (P == P_F32) {
    if (nr == 18) return kernel_occupancy((const void*)k_dslash<P, LPX, 18, false, EPI_LIN, DSLASH_MIN_BLOCKS_HI>, TILE);
    if (nr == 12) return kernel_occupancy((const void*)k_dslash<P, LPX, 12, false, EPI_LIN, DSLASH_MIN_BLOCKS_HI>, TILE);
  }
  return 0;
}
}  // namespace

int LQCD_CAT(dslash_occupancy_, LQCD_SFX)(int nr, int form) {
  if (form == 1) return colour_split_occupancy<SPX>(nr);
  if (form == 2) return shared_link_occupancy<SPX>(nr);
  if (form == 3) return second_budget_occupancy<SPX>(nr);
  if (form != 0) return 0;
  if (nr == 18) return kernel_occupancy((const void*)k_dslash<SPX, LPX, 18, false, EPI_LIN>, TILE);
  if (nr == 12) return site_occupancy_12<SPX>();
  return 0;
}

cudaError_t LQCD_CAT(launch_blas_, LQCD_SFX)(int op, int tp, const Launch& L, int grid,
                                              cudaStream_t s) {
  const bool df = (tp == P_DF64);
  switch (op) {
    case B_CG_P: return go_blas<B_CG_P, SPX>(L, grid, s);
    case B_NORM: return go_blas<B_NORM, SPX>(L, grid, s);
    case B_ZERO: return go_blas<B_ZERO, SPX>(L, grid, s);
    case B_TWIST: return go_blas<B_TWIST, SPX>(L, grid, s);
    case B_RU_P: return go_blas<B_RU_P, SPX>(L, grid, s);
    case B_RDOT: return go_blas<B_RDOT, SPX>(L, grid, s);
    case B_RU_SCALE:
      return df ? go_blas<B_RU_SCALE, SPX, P_DF64>(L, grid, s) : go_blas<B_RU_SCALE, SPX, P_F64>(L, grid, s);
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

#endif  // LQCD_TW_UNIT

}  // namespace lqcd
