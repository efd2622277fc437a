// Batched tile launches: one kernel launch covers many independent "slots"
// (a slot = one lattice problem: a single solve, one right-hand side of a
// multi-RHS solve, or one request of the serving loop).
//
// Work is cut into tiles of TILE consecutive half-lattice sites of one slot.
// A launch walks its tile list with a persistent grid (CTAs per SM chosen by
// the tuner). Norm reductions are deterministic and batch independent: every
// tile writes one FP64 partial at partial[slot.tile0 + tile_in_slot]; a second,
// small launch right after (k_finish in finish.cu) sums each slot's partials in
// tile order and runs the slot's scalar program (the "finisher"). So the
// result of a slot depends only on its own geometry, never on what else is in
// the batch or on the grid. (The kernel boundary orders the partials; a ticket
// inside the main kernel cost a fence and an atomic per tile and left one CTA
// summing all partials, about 90 us per launch at 16 k tiles.)
#pragma once

#include "dslash.cuh"

namespace lqcd {

#ifndef LQCD_TILE
#define LQCD_TILE 64
#endif
constexpr int TILE = LQCD_TILE;   // sites per tile (one tile per CTA pass of a batched kernel)
constexpr int MAX_SLOTS = 1024;   // slots in one launch

// Dslash epilogues. EPI_PLAIN: EPI_LIN for launches in which no slot reduces or runs a
// finisher (chosen by launch_dslash), compiled without the reduction code.
enum Epi { EPI_LIN = 0, EPI_CG = 1, EPI_LIN_TW = 2, EPI_CG_TW = 3, EPI_PLAIN = 4 };

// Slot state machine of the Krylov engine.
enum SlotState { S_RUNNING = 0, S_UPDATE = 1, S_DONE = 2, S_FAILED = 3, S_IDLE = 4 };
// run_if of a step that a slot never takes (the other reliable-update path)
constexpr int S_NEVER = 99;
// Status codes written into Scalars::status (mirrors the public LQCD_* codes).
enum SlotStatus { ST_OK = 0, ST_MAXITER = -3, ST_BREAKDOWN = -4, ST_NONFINITE = -5 };

// Scalar programs run by k_finish for a slot after a reduction.
enum Fin {
  FIN_NONE = 0,
  FIN_STORE0,    // res[0] = sum
  FIN_STORE1,    // res[1] = sum
  FIN_ALPHA,     // CG: qq = |Mhat p|^2, alpha = rr / qq
  FIN_BETA,      // CG: rr_new, beta, reliable-update / stop / maxiter decisions
  FIN_TRUERES,   // reliable update: |bhat - Mhat x|^2 -> converged?
  FIN_RHO,       // reliable update: |Mhat^dag u|^2 -> new sloppy scale and p coefficient
  FIN_RESUME,    // reliable update done: back to RUNNING
  FIN_RHO2,      // reliable update, sloppy rho = Mhat^dag (u / sigma_u): the same as FIN_RHO
  FIN_BICG_RHO,  // BiCGStab scalars (see solver.cu)
  FIN_BICG_ALPHA,
  FIN_BICG_OMEGA,
  FIN_BICG_RES,
};

// Per-slot solver state in device memory.
struct Scalars {
  double rr, rr_prev, alpha, beta, qq, rr_max;
  double stop_rr;   // sloppy rr at which the engine checks the true residual
  double delta2;    // reliable update when rr < delta2 * rr_max since the last update
  double target2;   // (tol * |b|)^2 for the FP64 true residual of Mhat
  double sigma;     // sloppy unit: true vector = sigma * stored vector
  double true_r2;   // last |bhat - Mhat x|^2 (FP64)
  double rho2;      // last |Mhat^dag u|^2 (FP64)
  double nreal;     // 24 * Vh, for the RMS normalisation of sloppy vectors
  double res[6];    // generic reduction results / coefficients
  double cres[8];   // complex scalars (BiCGStab): re, im pairs
  int state, status, iter, maxiter, last, n_updates, restart_p;
  int normal;       // 1: solve Mhat^dag Mhat x = phi; converged on |phi - Mhat^dag Mhat x|
  unsigned ticket;  // k_finish groups done (reset by the last)
  unsigned pad2[3];
};

// One slot's operands for one batched kernel.
struct Work {
  Geom g;
  int out_par;      // output parity (dslash) / parity of the half fields
  int run_if;       // run only when Scalars::state == run_if; -1: always
  int red;          // reduction: 0 none, 1 |out|^2, 2 <zin,out>, 3 <out,y1> and |out|^2,
                    //            4 <y2,out> and |out|^2 (complex dots as re, im)
  int fin;          // Fin program after the reduction
  int pad;
  const void* in;   // in-parity half field (dslash input)
  void* out;        // out-parity half field
  const void* Uout; // links of parity out_par (dslash)
  const void* Uin;  // links of parity 1 - out_par
  const void* y1;   // epilogue operands (out parity), may be null
  const void* y2;
  void* z;          // secondary output (CG: x_sloppy)
  const void* zin;  // secondary input (CG: p)
  double a, c1, c2; // out = a * D in + c1 * y1 + c2 * y2
  // Twisted mass (site-diagonal T(s, tau) = s (1 + i tau g5)): when `twist` is set, the
  // hopping term becomes T(tw_s, tw_t) (a D in) and the operand vector (y2 in the linear
  // epilogue, y1 in the CG step) is multiplied by T(1, ty_t) before its coefficient.
  int twist;
  int pad2;
  double tw_s, tw_t, ty_t;
  Scalars* sc;
  int tile0;        // first partial of this slot
  int ntiles;       // tiles of this slot = ceil(Vh / TILE)
};

// A launch: slots in device memory (works != nullptr) or one slot by value.
struct Launch {
  const Work* works;
  const int* tile_prefix;  // CONCAT mode: prefix sums of ntiles, nslots + 1 entries
  Work inline_work;
  int nslots;
  int ntiles;              // total tiles
  int interleave;          // 1: tile t -> (slot t % nslots, block t / nslots), equal Vh;
                           // 2: shared-link multi-RHS Dslash (all slots on one gauge field):
                           //    tile t -> (slot group t % mrhs_groups, block t / mrhs_groups)
  double* partials;
  int finish;              // 1: the slots' Works reduce or finish; k_finish follows the launch
  int mrhs_group;          // interleave 2: slots per group (group g holds [g G, (g + 1) G))
  int mrhs_groups;         // interleave 2: number of slot groups
  int gated;               // 1: some slot runs only in a given solver state (Work::run_if >= 0)
};

// Programmatic dependent launch. The batched kernels are launched with programmatic stream
// serialization (launch_k in launch.h) when it is enabled, so the next kernel on the stream
// may be launched while this one is still running. Each of them first waits for the grids
// before it to complete and their memory to be visible (griddepcontrol.wait, before any
// access to global memory, so any chain of dependent kernels stays ordered). A CTA lets the
// next grid launch (griddepcontrol.launch_dependents) when it starts its last tile, so the
// next grid's CTAs take the SM slots that this grid's tail leaves free, instead of a launch
// starting only after the last CTA ends. Without the launch attribute both instructions
// return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// kernels without a tile loop
__device__ __forceinline__ void pdl_entry() {
  pdl_wait();
  pdl_trigger();
}
// a persistent CTA about to take `tile`: its last one triggers the dependents
__device__ __forceinline__ void pdl_last_tile(int tile, int ntiles) {
  if (tile + (int)gridDim.x >= ntiles) pdl_trigger();
}

__device__ __forceinline__ const Work& work_of(const Launch& L, int slot) {
  return L.works ? L.works[slot] : L.inline_work;
}

// tile -> (slot, first site)
__device__ __forceinline__ void tile_of(const Launch& L, int tile, int& slot, int& start) {
  if (L.nslots == 1) {
    slot = 0;
    start = tile * TILE;
  } else if (L.interleave) {
    slot = tile % L.nslots;
    start = (tile / L.nslots) * TILE;
  } else {
    int lo = 0, hi = L.nslots;  // largest slot with prefix[slot] <= tile
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (__ldg(L.tile_prefix + mid) <= tile) lo = mid; else hi = mid;
    }
    slot = lo;
    start = (tile - __ldg(L.tile_prefix + lo)) * TILE;
  }
}

__device__ __forceinline__ bool slot_runs(const Work& w) {
  if (w.run_if < 0) return true;
  return *((volatile int*)&w.sc->state) == w.run_if;
}

// Per-CTA view of a solver launch (gated, 2..VIEW_SLOTS slots), staged in shared memory once
// per CTA: which slots run in this launch (a slot's state changes only in the finisher
// kernels between launches, never during one), compacted in slot order, with the prefix of
// their tile counts. The CTAs then stride over the running slots' tiles only, so a launch in
// which a few slots run (a reliable update that some slots take, slots waiting for one) is
// spread over every CTA; striding over all tiles and skipping idle slots' left the CTAs
// whose tiles fell on idle slots without work (with interleaved tiles a CTA meets only
// nslots / gcd(grid, nslots) slots). Each tile finds its slot in shared memory, instead of
// reading the slot state from global memory (a dependent L2 round trip) and binary-searching
// the tile prefix there. Which CTA computes a tile changes no result: each tile's partial
// sum goes to the slot's own tile index. Ungated launches (operators: every slot runs) and
// larger ones keep the plain path, without the prologue.
constexpr int VIEW_SLOTS = 128;
struct SlotView {
  int nact;                    // running slots
  int total;                   // their tiles
  unsigned runs[VIEW_SLOTS / 32];
  short act[VIEW_SLOTS];       // the running slots, in slot order
  int prefix[VIEW_SLOTS + 1];  // concatenated order: first tile of each running slot
};

// Dynamic shared memory of a one-thread-per-site Dslash launch: the slot view for gated
// launches, nothing otherwise (operator launches then keep the L1 carve-out of a kernel
// without shared memory).
inline size_t view_smem(const Launch& L) {
  return (L.gated && L.nslots > 1 && L.nslots <= VIEW_SLOTS) ? sizeof(SlotView) : 0;
}

// Called by every thread of the CTA (it ends in a barrier); false when the launch is not
// gated, has one slot or more than VIEW_SLOTS. Warp 0 compacts the running slots.
__device__ __forceinline__ bool view_load(const Launch& L, SlotView& v) {
  if (!L.gated || L.nslots <= 1 || L.nslots > VIEW_SLOTS) return false;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int base = 0, tiles = 0;
    for (int c = 0; c < L.nslots; c += 32) {
      const int i = c + lane;
      bool run = false;
      int cnt = 0;
      if (i < L.nslots) {
        run = slot_runs(work_of(L, i));
        if (run && !L.interleave) cnt = __ldg(L.tile_prefix + i + 1) - __ldg(L.tile_prefix + i);
      }
      const unsigned m = __ballot_sync(0xffffffffu, run);
      int sc = cnt;  // inclusive scan of the running slots' tile counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += y;
      }
      if (run) {
        const int k = base + __popc(m & ((1u << lane) - 1u));
        v.act[k] = (short)i;
        v.prefix[k] = tiles + sc - cnt;
      }
      if (lane == 0) v.runs[c >> 5] = m;
      tiles += __shfl_sync(0xffffffffu, sc, 31);
      base += __popc(m);
    }
    if (lane == 0) {
      v.nact = base;
      v.prefix[base] = tiles;
      v.total = L.interleave ? base * (L.ntiles / L.nslots) : tiles;
    }
  }
  __syncthreads();
  return true;
}

// running tile t (0 <= t < v.total) -> (slot, first site); interleave 1 or concatenated
__device__ __forceinline__ void view_tile(const Launch& L, const SlotView& v, int t, int& slot, int& start) {
  if (L.interleave) {
    const int k = t % v.nact;
    slot = v.act[k];
    start = (t / v.nact) * TILE;
  } else {
    int lo = 0, hi = v.nact;  // largest k with prefix[k] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (v.prefix[mid] <= t) lo = mid; else hi = mid;
    }
    slot = v.act[lo];
    start = (t - v.prefix[lo]) * TILE;
  }
}

__device__ __forceinline__ bool slot_runs_v(const SlotView& v, bool view, const Launch& L, int slot) {
  return view ? ((v.runs[slot >> 5] >> (slot & 31)) & 1u) != 0u : slot_runs(work_of(L, slot));
}

// Block-wide FP64 sum in a fixed order (NT threads). Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
  }
  __syncthreads();
  return s;
}

// The scalar programs. Run by one thread of k_finish for the slot.
__device__ __noinline__ static void run_fin_bicg(const Work& w, const double* v);

__device__ __noinline__ static void run_fin(const Work& w, const double* v) {
  Scalars* s = w.sc;
  const double sum = v[0];
  switch (w.fin) {
    case FIN_STORE0:
      s->res[0] = sum;
      break;
    case FIN_STORE1:
      s->res[1] = sum;
      break;
    case FIN_ALPHA:  // alpha = <r,r> / <p, Mhat^dag Mhat p> = rr / |Mhat p|^2
      s->qq = sum;
      if (!isfinite(sum)) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
      } else if (!(sum > 0.0)) {
        s->state = S_FAILED;
        s->status = ST_BREAKDOWN;
      } else {
        s->alpha = s->rr / sum;
      }
      break;
    case FIN_BETA: {  // new |r|^2: beta, and whether to leave for a reliable update
      s->rr_prev = s->rr;
      s->rr = sum;
      s->iter += 1;
      if (!isfinite(sum)) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
        break;
      }
      s->beta = sum / s->rr_prev;
      if (sum > s->rr_max) s->rr_max = sum;
      bool upd = (sum <= s->stop_rr) || (sum < s->delta2 * s->rr_max);
      if (s->iter >= s->maxiter) {
        upd = true;
        s->last = 1;
      }
      if (upd) s->state = S_UPDATE;
      break;
    }
    case FIN_TRUERES:  // FP64 |bhat - Mhat x|^2
      s->true_r2 = sum;
      s->n_updates += 1;
      if (!isfinite(sum)) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
      } else if (s->normal) {
        // normal equations: u = -Mhat x; the decision falls on rho = phi + Mhat^dag u
      } else if (sum <= s->target2) {
        s->state = S_DONE;
        s->status = ST_OK;
      } else if (s->last) {
        s->state = S_FAILED;
        s->status = ST_MAXITER;
      }
      // unit of the sloppy copy u / sigma_u taken by the sloppy-rho update path
      s->res[2] = sum > 0.0 ? sqrt(s->nreal / sum) : 0.0;
      break;
    case FIN_RHO2: {  // sum = |Mhat^dag (u / sigma_u)|^2 in the sloppy unit sigma_u
      const double sig_u = s->res[2] > 0.0 ? 1.0 / s->res[2] : 0.0;
      const double rho2 = sum * sig_u * sig_u;
      s->rho2 = rho2;
      if (!isfinite(sum) || !(sum > 0.0)) {
        s->state = S_FAILED;
        s->status = isfinite(sum) ? ST_BREAKDOWN : ST_NONFINITE;
        break;
      }
      double pc = 0.0;
      if (!s->restart_p) {  // beta of the replaced CG step (true units), p moved to the unit sig_u
        const double beta = rho2 / (s->sigma * s->sigma * s->rr_prev);
        pc = beta * s->sigma / sig_u;
      }
      s->res[4] = pc;
      const double c2 = s->true_r2 / rho2;
      s->sigma = sig_u;
      s->rr = sum;
      s->rr_max = sum;
      s->stop_rr = 0.5 * s->target2 / (c2 * sig_u * sig_u);
      break;
    }
    case FIN_RHO: {  // rho = Mhat^dag u: new sloppy unit, p coefficient, stop estimate
      s->rho2 = sum;
      if (s->normal && isfinite(sum)) {  // rho = phi - Mhat^dag Mhat x is the residual itself
        if (sum <= s->target2) {
          s->state = S_DONE;
          s->status = ST_OK;
          break;
        }
        if (s->last) {
          s->state = S_FAILED;
          s->status = ST_MAXITER;
          break;
        }
      }
      if (!isfinite(sum) || !(sum > 0.0)) {
        s->state = S_FAILED;
        s->status = isfinite(sum) ? ST_BREAKDOWN : ST_NONFINITE;
        break;
      }
      const double sig_new = sqrt(sum / s->nreal);
      double pc = 0.0;
      if (!s->restart_p) {
        // beta of the CG step replaced by this update, in true units, then
        // p rescaled from the old sloppy unit to the new one
        const double beta = sum / (s->sigma * s->sigma * s->rr_prev);
        pc = beta * s->sigma / sig_new;
      }
      s->res[4] = pc;
      s->res[5] = 1.0 / sig_new;
      // |u|^2 / |Mhat^dag u|^2 at this x (normal equations: the sloppy r is rho itself)
      const double c2 = s->normal ? 1.0 : s->true_r2 / sum;
      s->sigma = sig_new;
      s->rr = sum / (sig_new * sig_new);
      s->rr_max = s->rr;
      s->stop_rr = 0.5 * s->target2 / (c2 * sig_new * sig_new);
      break;
    }
    case FIN_RESUME:
      s->state = S_RUNNING;
      s->restart_p = 0;
      break;
    default:
      run_fin_bicg(w, v);
      break;
  }
}

// complex helpers for the BiCGStab scalars (re, im pairs in Scalars::cres)
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& r, double& i) {
  const double d = br * br + bi * bi;
  r = (ar * br + ai * bi) / d;
  i = (ai * br - ar * bi) / d;
}

// cres: [0,1] rho, [2,3] alpha, [4,5] omega, [6,7] beta; res[0] = |r|^2
__device__ __noinline__ static void run_fin_bicg(const Work& w, const double* v) {
  Scalars* s = w.sc;
  switch (w.fin) {
    case FIN_BICG_ALPHA: {  // alpha = rho / <r0, v>
      if (!isfinite(v[0]) || !isfinite(v[1])) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
      } else if (v[0] == 0.0 && v[1] == 0.0) {
        s->state = S_FAILED;
        s->status = ST_BREAKDOWN;
      } else {
        cdiv(s->cres[0], s->cres[1], v[0], v[1], s->cres[2], s->cres[3]);
      }
      break;
    }
    case FIN_BICG_OMEGA: {  // omega = <t, s> / <t, t>
      if (!isfinite(v[2]) || !isfinite(v[0])) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
      } else if (!(v[2] > 0.0)) {
        s->state = S_FAILED;
        s->status = ST_BREAKDOWN;
      } else {
        s->cres[4] = v[0] / v[2];
        s->cres[5] = v[1] / v[2];
      }
      break;
    }
    case FIN_BICG_RES: {  // rho_new = <r0, r>, |r|^2; beta = (rho_new / rho) (alpha / omega)
      s->iter += 1;
      s->res[0] = v[2];
      if (!isfinite(v[2]) || !isfinite(v[0])) {
        s->state = S_FAILED;
        s->status = ST_NONFINITE;
        break;
      }
      if (v[2] <= s->stop_rr) {
        s->state = S_DONE;
        break;
      }
      if (s->iter >= s->maxiter) {
        s->state = S_FAILED;
        s->status = ST_MAXITER;
        break;
      }
      double q1r, q1i, q2r, q2i;
      if ((s->cres[0] == 0.0 && s->cres[1] == 0.0) || (s->cres[4] == 0.0 && s->cres[5] == 0.0) ||
          (v[0] == 0.0 && v[1] == 0.0)) {
        s->state = S_FAILED;
        s->status = ST_BREAKDOWN;
        break;
      }
      cdiv(v[0], v[1], s->cres[0], s->cres[1], q1r, q1i);
      cdiv(s->cres[2], s->cres[3], s->cres[4], s->cres[5], q2r, q2i);
      s->cres[6] = q1r * q2r - q1i * q2i;
      s->cres[7] = q1r * q2i + q1i * q2r;
      s->cres[0] = v[0];
      s->cres[1] = v[1];
      break;
    }
    default:
      break;
  }
}

// The same for site values that are FP32 numbers (sloppy precisions): the warp stage adds
// in FP32 (FP64 runs at 1/64 of the FP32 rate here), the warps' sums are added in FP64.
template <int NT>
__device__ __forceinline__ double block_sum_f32(double v, double* sh) {
  float x = (float)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = (double)x;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
  }
  __syncthreads();
  return s;
}

// Called by all threads of the CTA after its tile: records the tile's partial sums
// (strided by 3: up to three sums per reduction) for k_finish. F32: the site values
// are FP32 sums (sloppy kernels).
template <int NT, bool F32 = false>
__device__ __forceinline__ void tile_partial(const Work& w, int tile_in_slot, double v0, double v1,
                                             double v2, double* partials) {
  __shared__ double sh[NT / 32];
  if (!w.red && w.fin == FIN_NONE) return;
  const int ns = (w.red >= 2) ? 3 : 1;
  auto bsum = [&](double v) { return F32 ? block_sum_f32<NT>(v, sh) : block_sum<NT>(v, sh); };
  double s[3];
  s[0] = bsum(v0);
  if (ns == 3) {
    s[1] = bsum(v1);
    s[2] = bsum(v2);
  }
  if (threadIdx.x == 0) {
    double* dst = partials + 3 * (size_t)(w.tile0 + tile_in_slot);
    for (int k = 0; k < ns; ++k) dst[k] = s[k];
  }
}

}  // namespace lqcd
