// Krylov engine: CG on the normal equations of the even-odd Schur system,
// Mhat^dag Mhat x_e = Mhat^dag bhat_e (paper Section 3: "inversion of the
// fermion matrix" with even-odd preconditioning), batched over slots.
//
// Mixed precision (defect correction with reliable updates):
//  * the Krylov vectors r, p, q, t live in the sloppy storage (FP32, FP16 or
//    BF16, arithmetic in FP32) in units of sigma (RMS 1 per real after each
//    update), the sloppy solution xs in FP32;
//  * an update folds sigma * xs into the FP64 solution x, recomputes the true
//    residual u = bhat - Mhat x in FP64-class arithmetic with FP64-class links,
//    then rho = Mhat^dag u (in the sloppy precision from u / |u|_rms for M x = b;
//    in FP64-class arithmetic for the normal equations), restarts r = rho / sigma_new
//    and keeps the search direction p (rescaled, with the CG beta of the replaced step);
//  * an update is triggered when |r| drops below delta * max|r| since the last
//    one, when the sloppy residual predicts convergence, or at maxiter. The
//    solve ends when |bhat - Mhat x| <= tol |b| in FP64; then x_o = b_o +
//    kappa D_oe x_e and the full ||b - M x|| is measured in FP64.
// With FP64 sloppy storage and delta = 0 this is the plain FP64 CG.
//
// Twisted mass (Section 3, M = A - kappa D with the site-diagonal A = 1 + i a g5,
// a = 2 kappa mu): the Schur operator becomes Mhat = A - kappa^2 D_eo A^-1 D_oe,
// Mhat^dag = A^dag - kappa^2 D^dag_eo A^-dag D^dag_oe, bhat = b_e + kappa D_eo A^-1 b_o
// and x_o = A^-1 (b_o + kappa D_oe x_e). A^-1 = (1 - i a g5) / (1 + a^2); every factor
// of A is applied inside the Dslash epilogues (twist fields of Work), so a twisted
// iteration has the launches and the HBM traffic of a Wilson one.
//
// Every slot runs its own scalar recurrences on the device (finishers in
// batch.cuh); the host replays CUDA graphs of `chunk` iterations and polls
// slot states between replays.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {

// RU_D2 / RU_RHO / RU_CONV: rho = Mhat^dag u in FP64-class arithmetic (normal-equation
// solves, whose convergence is decided on rho); RU_QS / RU_D2S / RU_RHOS / RU_PS: rho in
// the sloppy precision from the sloppy copy u / sigma_u (M x = b solves, whose convergence
// is decided on u; rho only restarts the sloppy recurrence).
enum Step { K1 = 0, K2, K3, K4, K6, RU_FOLD, RU_D1, RU_RES, RU_D2, RU_RHO, RU_CONV,
            RU_QS, RU_D2S, RU_RHOS, RU_PS, NSTEP };

__global__ void k_slot_init(Scalars* s, double tol2, double nreal, int maxiter, double delta2, int normal) {
  s->res[3] = s->res[0] + s->res[1];  // |b|^2 of the full source (normal equations: |phi_e|^2)
  s->normal = normal;
  s->target2 = tol2 * s->res[3];
  s->sigma = 1.0;
  s->nreal = nreal;
  s->maxiter = maxiter;
  s->delta2 = delta2;
  s->state = S_UPDATE;
  s->status = ST_OK;
  s->iter = 0;
  s->last = 0;
  s->n_updates = 0;
  s->restart_p = 1;
  s->rr = s->rr_prev = 1.0;
  s->alpha = s->beta = 0.0;
  s->rr_max = 0.0;
  s->stop_rr = 0.0;
  s->ticket = 0;
}

__global__ void k_slot_cancel(Scalars* s, int status) {
  if (s->state == S_RUNNING || s->state == S_UPDATE) {
    s->state = S_FAILED;
    s->status = status;
  }
}

struct SlotBuf {
  void* block = nullptr;
  size_t bytes = 0;
  void *be, *bo, *bhat, *x64, *u64, *t64;  // FP64 halves (t64 odd)
  void *r, *p, *q, *t;                     // sloppy halves (t odd)
  void* xs;                                // sloppy solution (FP32, or FP64 for an FP64 solve)
};

struct Request {
  long long id = 0;
  const lqcd_gauge* gauge = nullptr;
  Geom g{};
  double kappa = 0, tol = 0, mu = 0;
  bool normal = false;  // Mhat^dag Mhat x_e = src_e instead of M x = src
  int slot = -1;
  SlotBuf buf;
  int tile0 = 0, ntiles = 0;
  bool finished = false;
  lqcd_solve_info info{};
  std::chrono::steady_clock::time_point t0;
};

}  // namespace lqcd

using namespace lqcd;

struct lqcd_engine {
  lqcd_ctx* ctx = nullptr;
  bool holds_ctx = true;  // false for a context's cached engine
  lqcd_solve_opts opts{};
  int sp = P_F32, xp = P_F32, nr = 12;
  int tp = P_F64;  // FP64-class vectors and operator of the true residual: P_F64 or P_DF64
  double delta2 = 0.01;
  int ru_every = 8;
  size_t budget = 0;
  int max_slots = 0;
  Scalars* d_sc = nullptr;
  Scalars* h_sc = nullptr;
  Work* d_works = nullptr;  // NSTEP x max_slots
  int* d_prefix = nullptr;
  double* d_partials = nullptr;
  size_t partials_cap = 0;
  std::vector<int> free_slots;
  std::map<long long, Request> reqs;  // live and finished-not-collected
  std::vector<long long> active;      // ids in launch order
  std::vector<long long> done_ids;    // finished since last lqcd_engine_completed
  std::multimap<size_t, void*> pool;  // freed slot blocks by size
  size_t bytes_in_use = 0, bytes_pooled = 0;
  long long next_id = 1;
  bool dirty = true;
  int ntiles_total = 0;
  int interleave = 0;
  // shared-link multi-RHS Dslash for the sloppy steps (interleave mode 2): slots per group,
  // groups, and tiles (site blocks x groups); mrhs_groups == 0: not used
  int mrhs_group = 0, mrhs_groups = 0, mrhs_tiles = 0;
  bool any_twist = false;  // some active request has mu != 0
  bool any_normal = false, any_plain = false;  // active normal-equation / M x = b requests
  cudaGraphExec_t exec = nullptr;
  std::vector<Work> h_works;
};

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t slot_bytes(const lqcd_engine* e, int Vh) {
  return 6 * align256(half_spinor_bytes(e->tp, Vh)) + 4 * align256(half_spinor_bytes(e->sp, Vh)) +
         align256(half_spinor_bytes(e->xp, Vh));
}

void carve(SlotBuf& b, const lqcd_engine* e, int Vh) {
  char* p = static_cast<char*>(b.block);
  auto take = [&](int prec) {
    void* r = p;
    p += align256(half_spinor_bytes(prec, Vh));
    return r;
  };
  b.be = take(e->tp);
  b.bo = take(e->tp);
  b.bhat = take(e->tp);
  b.x64 = take(e->tp);
  b.u64 = take(e->tp);
  b.t64 = take(e->tp);
  b.r = take(e->sp);
  b.p = take(e->sp);
  b.q = take(e->sp);
  b.t = take(e->sp);
  b.xs = take(e->xp);
}

const void* sloppy_links(const lqcd_engine* e, const lqcd_gauge* g) {
  return g->copy[link_prec_for(e->sp)][e->nr == 12];
}

Work slot_work(const lqcd_engine* e, const Request& q) {
  Work w = blank_work(q.g);
  w.sc = e->d_sc + q.slot;
  w.tile0 = q.tile0;
  w.ntiles = q.ntiles;
  return w;
}

void step_works(const lqcd_engine* e, const Request& q, Work out[NSTEP]) {
  const int Vh = q.g.Vh;
  const double kk = q.kappa * q.kappa;
  const void* US = sloppy_links(e, q.gauge);
  const int lpS = link_prec_for(e->sp);
  const void* U64 = q.gauge->copy[e->tp][0];
  const int tp = e->tp;
  auto links = [&](Work& w, const void* U, int lp, int nr, int out_par) {
    w.out_par = out_par;
    w.Uout = parity_links(U, lp, nr, Vh, out_par);
    w.Uin = parity_links(U, lp, nr, Vh, 1 - out_par);
  };
  const SlotBuf& b = q.buf;
  for (int s = 0; s < NSTEP; ++s) out[s] = slot_work(e, q);
  // --- sloppy CG iteration
  Work& k1 = out[K1];
  links(k1, US, lpS, e->nr, 1);
  k1.in = b.p; k1.out = b.t; k1.a = 1.0; k1.run_if = S_RUNNING;
  Work& k2 = out[K2];
  links(k2, US, lpS, e->nr, 0);
  k2.in = b.t; k2.out = b.q; k2.y1 = b.p; k2.c1 = 1.0; k2.a = -kk;
  k2.red = 1; k2.fin = FIN_ALPHA; k2.run_if = S_RUNNING;
  Work& k3 = out[K3];
  links(k3, US, lpS, e->nr, 1);
  k3.in = b.q; k3.out = b.t; k3.a = 1.0; k3.run_if = S_RUNNING;
  Work& k4 = out[K4];
  links(k4, US, lpS, e->nr, 0);
  k4.in = b.t; k4.out = b.r; k4.y1 = b.q; k4.a = -kk; k4.z = b.xs; k4.zin = b.p;
  k4.red = 1; k4.fin = FIN_BETA; k4.run_if = S_RUNNING;
  Work& k6 = out[K6];
  k6.in = b.r; k6.out = b.p; k6.run_if = S_RUNNING;
  // --- FP64 reliable update
  Work& f = out[RU_FOLD];
  f.in = b.xs; f.out = b.x64; f.run_if = S_UPDATE;
  Work& d1 = out[RU_D1];
  links(d1, U64, tp, 18, 1);
  d1.in = b.x64; d1.out = b.t64; d1.a = 1.0; d1.run_if = S_UPDATE;
  Work& rs = out[RU_RES];
  links(rs, U64, tp, 18, 0);
  rs.in = b.t64; rs.out = b.u64; rs.y1 = b.bhat; rs.c1 = 1.0; rs.y2 = b.x64; rs.c2 = -1.0;
  rs.a = kk; rs.red = 1; rs.fin = FIN_TRUERES; rs.run_if = S_UPDATE;
  Work& d2 = out[RU_D2];
  links(d2, U64, tp, 18, 1);
  d2.in = b.u64; d2.out = b.t64; d2.a = 1.0; d2.run_if = S_UPDATE;
  Work& rh = out[RU_RHO];
  links(rh, U64, tp, 18, 0);
  rh.in = b.t64; rh.out = b.u64; rh.y1 = b.u64; rh.c1 = 1.0; rh.a = -kk;
  rh.red = 1; rh.fin = FIN_RHO; rh.run_if = S_UPDATE;
  Work& cv = out[RU_CONV];
  cv.in = b.u64; cv.out = b.r; cv.z = b.p; cv.fin = FIN_RESUME; cv.run_if = S_UPDATE;
  // sloppy rho path: q = u / sigma_u, t = D^dag_oe q, r = Mhat^dag q (+ norm), p = r + c p
  Work& qs = out[RU_QS];
  qs.in = b.u64; qs.out = b.q; qs.run_if = S_UPDATE;
  Work& d2s = out[RU_D2S];
  links(d2s, US, lpS, e->nr, 1);
  d2s.in = b.q; d2s.out = b.t; d2s.a = 1.0; d2s.run_if = S_UPDATE;
  Work& rhs = out[RU_RHOS];
  links(rhs, US, lpS, e->nr, 0);
  rhs.in = b.t; rhs.out = b.r; rhs.y1 = b.q; rhs.c1 = 1.0; rhs.a = -kk;
  rhs.red = 1; rhs.fin = FIN_RHO2; rhs.run_if = S_UPDATE;
  Work& ps = out[RU_PS];
  ps.in = b.r; ps.z = b.p; ps.fin = FIN_RESUME; ps.run_if = S_UPDATE;
  for (int st : {RU_D2, RU_RHO, RU_CONV}) out[st].run_if = q.normal ? S_UPDATE : S_NEVER;
  for (int st : {RU_QS, RU_D2S, RU_RHOS, RU_PS}) out[st].run_if = q.normal ? S_NEVER : S_UPDATE;
  if (q.normal) {  // rho = phi - Mhat^dag Mhat x = phi + Mhat^dag u with u = -Mhat x (bhat = 0)
    rh.y2 = b.be;
    rh.c2 = 1.0;
  }
  const double a = 2.0 * q.kappa * q.mu;
  if (a != 0.0) {
    const double s = 1.0 / (1.0 + a * a);
    set_twist(k1, s, -a, 0.0);  // t = A^-1 D_oe p
    k2.y1 = nullptr; k2.c1 = 0.0; k2.y2 = b.p; k2.c2 = 1.0;
    set_twist(k2, 1.0, 0.0, a);   // q = A p - k^2 D_eo t
    set_twist(k3, s, a, 0.0);     // t = A^-dag D^dag_oe q
    set_twist(k4, 1.0, 0.0, -a);  // r -= alpha (A^dag q - k^2 D^dag_eo t)
    set_twist(d1, s, -a, 0.0);
    set_twist(rs, 1.0, 0.0, a);   // u = bhat - A x + k^2 D_eo t
    set_twist(d2, s, a, 0.0);
    rh.y1 = q.normal ? b.be : nullptr; rh.c1 = q.normal ? 1.0 : 0.0; rh.y2 = b.u64; rh.c2 = 1.0;
    set_twist(rh, 1.0, 0.0, -a);  // rho = A^dag u - k^2 D^dag_eo t (+ phi)
    set_twist(d2s, s, a, 0.0);
    rhs.y1 = nullptr; rhs.c1 = 0.0; rhs.y2 = b.q; rhs.c2 = 1.0;
    set_twist(rhs, 1.0, 0.0, -a);  // r = A^dag q - k^2 D^dag_eo t
  }
}

struct StepKind {
  bool dslash;
  bool f64;
  bool dag;
  int epi_or_op;
};

StepKind kind_of(int s) {
  switch (s) {
    case K1: return {true, false, false, EPI_LIN};
    case K2: return {true, false, false, EPI_LIN};
    case K3: return {true, false, true, EPI_LIN};
    case K4: return {true, false, true, EPI_CG};
    case K6: return {false, false, false, B_CG_P};
    case RU_FOLD: return {false, false, false, B_RU_FOLD};
    case RU_D1: return {true, true, false, EPI_LIN};
    case RU_RES: return {true, true, false, EPI_LIN};
    case RU_D2: return {true, true, true, EPI_LIN};
    case RU_RHO: return {true, true, true, EPI_LIN};
    case RU_CONV: return {false, false, false, B_RU_CONVERT};
    case RU_QS: return {false, false, false, B_RU_SCALE};
    case RU_D2S: return {true, false, true, EPI_LIN};
    case RU_RHOS: return {true, false, true, EPI_LIN};
    case RU_PS: return {false, false, false, B_RU_P};
  }
  return {false, false, false, 0};
}

// tw: some slot of the launch is twisted (its Dslash steps take the twisted epilogues;
// untwisted slots carry the identity twist there and give the same bits)
cudaError_t issue(lqcd_engine* e, int s, const Launch& L, bool tw) {
  const StepKind k = kind_of(s);
  e->ctx->launches += L.finish ? 2 : 1;
  if (k.dslash) {
    const int epi = k.epi_or_op + (tw ? EPI_LIN_TW - EPI_LIN : 0);
    if (k.f64) return launch_dslash(e->tp, 18, k.dag, epi, L, 0, e->ctx->stream);
    return launch_dslash(e->sp, e->nr, k.dag, epi, L, 0, e->ctx->stream);
  }
  const int prec = (k.epi_or_op == B_RU_FOLD) ? e->xp : e->sp;
  return launch_blas(prec, k.epi_or_op, L, 0, e->ctx->stream, e->tp);
}

Launch batch_launch(const lqcd_engine* e, int s) {
  Launch L;
  memset(&L, 0, sizeof L);
  L.works = e->d_works + (size_t)s * e->max_slots;
  L.tile_prefix = e->d_prefix;
  L.nslots = (int)e->active.size();
  L.ntiles = e->ntiles_total;
  L.interleave = e->interleave;
  L.partials = e->d_partials;
  const StepKind k = kind_of(s);
  if (e->mrhs_groups > 0 && k.dslash && !k.f64) {
    L.interleave = 2;
    L.ntiles = e->mrhs_tiles;
    L.mrhs_group = e->mrhs_group;
    L.mrhs_groups = e->mrhs_groups;
  }
  // k_finish follows when any active slot's Work of this step reduces or runs a finisher
  for (int i = 0; i < L.nslots && !L.finish; ++i) {
    const Work& w = e->h_works[(size_t)s * e->max_slots + i];
    L.finish = ((w.red || w.fin != FIN_NONE) && w.run_if != S_NEVER) ? 1 : 0;
  }
  for (int i = 0; i < L.nslots && !L.gated; ++i)
    L.gated = e->h_works[(size_t)s * e->max_slots + i].run_if >= 0 ? 1 : 0;
  return L;
}

// the reliable-update steps for a launch holding normal-equation and / or M x = b slots
std::vector<int> ru_steps(bool normal, bool plain) {
  std::vector<int> v = {RU_FOLD, RU_D1, RU_RES};
  if (normal) v.insert(v.end(), {RU_D2, RU_RHO, RU_CONV});
  if (plain) v.insert(v.end(), {RU_QS, RU_D2S, RU_RHOS, RU_PS});
  return v;
}

cudaError_t issue_iteration_block(lqcd_engine* e, int iters) {
  for (int it = 0; it < iters; ++it) {
    for (int s : {K1, K2, K3, K4, K6}) {
      cudaError_t err = issue(e, s, batch_launch(e, s), e->any_twist);
      if (err != cudaSuccess) return err;
    }
    if ((it + 1) % e->ru_every == 0 || it + 1 == iters) {
      for (int s : ru_steps(e->any_normal, e->any_plain)) {
        cudaError_t err = issue(e, s, batch_launch(e, s), e->any_twist);
        if (err != cudaSuccess) return err;
      }
    }
  }
  return cudaSuccess;
}

int rebuild(lqcd_engine* e) {
  const int n = (int)e->active.size();
  e->dirty = false;
  if (n == 0) return LQCD_OK;
  // interleave tiles when every slot solves on the same gauge field (multi-RHS):
  // consecutive tiles then share links, which stream from HBM once per site block
  const lqcd_gauge* g0 = e->reqs[e->active[0]].gauge;
  bool same = true;
  e->any_twist = false;
  e->any_normal = e->any_plain = false;
  for (long long id : e->active) {
    same = same && e->reqs[id].gauge == g0;
    e->any_twist = e->any_twist || e->reqs[id].mu != 0.0;
    if (e->reqs[id].normal) e->any_normal = true;
    else e->any_plain = true;
  }
  e->interleave = (same && n > 1) ? 1 : 0;
  // Slots on one gauge field may share each site block's link loads in the sloppy Dslash
  // steps (k_dslash_mrhs): a CTA applies the block's links to a group of slots. The group
  // size is the autotuner's measured choice for this key. Without one the slots load their
  // own links: in the interleaved tile order consecutive CTAs read the same links, which L2
  // then serves, and at 24^3x48 with FP32-12 links the shared form measured no faster (the
  // own-link launch at 8 CTAs per SM is as fast). multi_rhs_links > 0 asks for the shared
  // form always: in the tuned group size when the tuner measured one, else in groups as
  // large as the lattice allows while the launch keeps at least 8 tiles per SM.
  e->mrhs_group = e->mrhs_groups = e->mrhs_tiles = 0;
  if (e->interleave && !e->any_twist && e->opts.multi_rhs_links >= 0 &&
      (e->sp == P_F32 || e->sp == P_F16 || e->sp == P_BF16)) {
    const int blocks = e->reqs[e->active[0]].ntiles;
    int gsize = tune_shared_links(e->sp, e->nr, n, blocks, nullptr);
    if (gsize <= 0 && e->opts.multi_rhs_links > 0) {
      const int want = 8 * device_sm_count();
      const int groups = std::min(n, std::max(1, (want + blocks - 1) / blocks));
      gsize = (n + groups - 1) / groups;
    }
    gsize = std::min(gsize, n);
    const int groups = gsize > 0 ? (n + gsize - 1) / gsize : 0;
    if (gsize > 1) {
      e->mrhs_group = gsize;
      e->mrhs_groups = groups;
      e->mrhs_tiles = blocks * groups;
    }
  }
  std::vector<int> prefix(n + 1, 0);
  e->h_works.assign((size_t)NSTEP * e->max_slots, Work{});
  for (int i = 0; i < n; ++i) {
    const Request& q = e->reqs[e->active[i]];
    Work w[NSTEP];
    step_works(e, q, w);
    for (int s = 0; s < NSTEP; ++s) e->h_works[(size_t)s * e->max_slots + i] = w[s];
    prefix[i + 1] = prefix[i] + q.ntiles;
  }
  e->ntiles_total = prefix[n];
  if (e->opts.ru_interval <= 0) {
    // A slot waiting for a reliable update idles until the next update block, and a
    // block costs six launches that skip when no slot needs them; measured on GB300
    // (8^4 to 32^3x64, FP16/FP32 sloppy) the solve time is flat in the interval
    // between 1 and 8 to within 3%, slightly lower at 4.
    e->ru_every = std::min(e->opts.chunk, 4);
  }
  cudaStream_t st = e->ctx->stream;
  LQCD_CK(cudaMemcpyAsync(e->d_works, e->h_works.data(), sizeof(Work) * e->h_works.size(),
                          cudaMemcpyHostToDevice, st));
  LQCD_CK(cudaMemcpyAsync(e->d_prefix, prefix.data(), sizeof(int) * (n + 1),
                          cudaMemcpyHostToDevice, st));
  LQCD_CK(cudaStreamSynchronize(st));  // host vectors are reused
  if (e->opts.use_graph) {
    cudaGraph_t graph = nullptr;
    LQCD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = issue_iteration_block(e, e->opts.chunk);
    cudaError_t err2 = cudaStreamEndCapture(st, &graph);
    if (err != cudaSuccess) return set_error(LQCD_ECUDA, "capture: %s", cudaGetErrorString(err));
    if (err2 != cudaSuccess) return set_error(LQCD_ECUDA, "end capture: %s", cudaGetErrorString(err2));
    if (e->exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(e->exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
      }
    }
    if (!e->exec) {
      cudaError_t ie = cudaGraphInstantiate(&e->exec, graph, 0);
      if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        e->exec = nullptr;
        return set_error(LQCD_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
      }
    }
    cudaGraphDestroy(graph);
  }
  return LQCD_OK;
}

int ensure_partials(lqcd_engine* e, size_t n) {
  if (e->partials_cap >= n) return LQCD_OK;
  LQCD_CK(cudaStreamSynchronize(e->ctx->stream));
  if (e->d_partials) cudaFree(e->d_partials);
  e->d_partials = nullptr;
  size_t cap = std::max(n, 2 * e->partials_cap);
  LQCD_CK(cudaMalloc(&e->d_partials, cap * sizeof(double)));
  e->partials_cap = cap;
  e->dirty = true;
  return LQCD_OK;
}

// tile ranges of live requests: first fit over the partials buffer
int assign_tiles(lqcd_engine* e, Request& q) {
  std::vector<std::pair<int, int>> used;
  for (auto& kv : e->reqs)
    if (kv.second.slot >= 0 && kv.first != q.id) used.push_back({kv.second.tile0, kv.second.ntiles});
  std::sort(used.begin(), used.end());
  int pos = 0;
  for (auto& u : used) {
    if (u.first - pos >= q.ntiles) break;
    pos = std::max(pos, u.first + u.second);
  }
  q.tile0 = pos;
  return ensure_partials(e, 3 * ((size_t)pos + q.ntiles));
}

int alloc_block(lqcd_engine* e, size_t bytes, void** out) {
  auto it = e->pool.find(bytes);
  if (it != e->pool.end()) {
    *out = it->second;
    e->pool.erase(it);
    e->bytes_pooled -= bytes;
    return LQCD_OK;
  }
  // free pooled blocks first when the budget would be exceeded
  while (e->budget && e->bytes_in_use + e->bytes_pooled + bytes > e->budget && !e->pool.empty()) {
    auto p = e->pool.begin();
    LQCD_CK(cudaStreamSynchronize(e->ctx->stream));
    cudaFree(p->second);
    e->bytes_pooled -= p->first;
    e->pool.erase(p);
  }
  cudaError_t err = cudaMalloc(out, bytes);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ENOMEM, "slot buffers (%zu bytes): %s", bytes, cudaGetErrorString(err));
  }
  return LQCD_OK;
}

// single-slot launches of the finishing steps (after DONE / FAILED)
int finalize_launch(lqcd_engine* e, Request& q) {
  if (q.normal) {  // x_e is the answer; no odd half
    LQCD_CK(cudaMemsetAsync(q.buf.t64, 0, half_spinor_bytes(e->tp, q.g.Vh), e->ctx->stream));
    return LQCD_OK;
  }
  const Geom& g = q.g;
  const int tp = e->tp;
  const void* U64 = q.gauge->copy[tp][0];
  const SlotBuf& b = q.buf;
  cudaStream_t st = e->ctx->stream;
  const double ta = 2.0 * q.kappa * q.mu, ts = 1.0 / (1.0 + ta * ta);
  // tw: 0 none, 1 the hopping term times A^-1, 2 the y2 operand times A
  auto lin = [&](int out_par, const void* in, void* out, const void* y1, double c1, const void* y2,
                 double c2, double a, int fin, int tw) -> int {
    Work w = slot_work(e, q);
    w.out_par = out_par;
    w.Uout = parity_links(U64, tp, 18, g.Vh, out_par);
    w.Uin = parity_links(U64, tp, 18, g.Vh, 1 - out_par);
    w.in = in; w.out = out; w.y1 = y1; w.c1 = c1; w.y2 = y2; w.c2 = c2; w.a = a;
    w.red = fin != FIN_NONE ? 1 : 0; w.fin = fin; w.run_if = -1;
    if (ta != 0.0 && tw == 1) set_twist(w, ts, -ta, 0.0);
    if (ta != 0.0 && tw == 2) set_twist(w, 1.0, 0.0, ta);
    Launch L = single_launch(w, e->d_partials);
    e->ctx->launches++;
    LQCD_CK(launch_dslash(tp, 18, false, w.twist ? EPI_LIN_TW : EPI_LIN, L, 0, st));
    return LQCD_OK;
  };
  int rc;
  const void* bo = b.bo;
  if (ta != 0.0) {
    // t = A^-1 b_o, then x_o = t + kappa A^-1 D_oe x_e
    Work w = slot_work(e, q);
    w.in = b.bo; w.out = b.t64; w.run_if = -1;
    set_twist(w, ts, -ta, 0.0);
    e->ctx->launches++;
    LQCD_CK(launch_blas(tp, B_TWIST, single_launch(w, e->d_partials), 0, st));
    bo = b.t64;
  }
  // x_o = A^-1 (b_o + kappa D_oe x_e)
  if ((rc = lin(1, b.x64, b.t64, bo, 1.0, nullptr, 0.0, q.kappa, FIN_NONE, 1))) return rc;
  // r_e = b_e - A x_e + kappa D_eo x_o ; r_o = b_o - A x_o + kappa D_oe x_e  (full M, FP64)
  if ((rc = lin(0, b.t64, b.u64, b.be, 1.0, b.x64, -1.0, q.kappa, FIN_STORE0, 2))) return rc;
  if ((rc = lin(1, b.x64, b.bhat, b.bo, 1.0, b.t64, -1.0, q.kappa, FIN_STORE1, 2))) return rc;
  return LQCD_OK;
}

int status_of(int st) { return st; }  // Scalars::status mirrors the public codes

}  // namespace

extern "C" {

void lqcd_solve_opts_default(lqcd_solve_opts* o) {
  if (!o) return;
  o->solver = LQCD_CG;
  o->sloppy_prec = LQCD_F32;
  o->sloppy_compress = 12;
  o->maxiter = 50000;
  o->delta = 0.0;
  // iterations per graph replay and host poll: measured on GB300 (16^3x32 and 32^3x64 mixed
  // CG, the 16^3x32 HMC), 8 against 32 saves the launches a converged solve would still
  // issue to the end of its chunk (5.63 -> 5.07 ms, 28.8 -> 27.9 ms, 430 -> 420 ms per
  // trajectory); the extra polls cost less
  o->chunk = 8;
  o->use_graph = 1;
  o->ru_interval = 0;
  o->true_prec = -1;
  o->mu = 0.0;
}

int lqcd_engine_create(lqcd_ctx* c, const lqcd_solve_opts* opts, size_t budget, int max_slots,
                       lqcd_engine** out) {
  clear_error();
  if (!c || !out) return set_error(LQCD_EINVAL, "NULL argument");
  *out = nullptr;
  if (max_slots < 1 || max_slots > MAX_SLOTS) return set_error(LQCD_EINVAL, "max_slots %d", max_slots);
  lqcd_solve_opts o;
  lqcd_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.solver != LQCD_CG) return set_error(LQCD_EINVAL, "the batched engine runs CG");
  if (o.sloppy_prec < LQCD_F64 || o.sloppy_prec > LQCD_DF64) return set_error(LQCD_EINVAL, "sloppy precision");
  if (o.true_prec != -1 && o.true_prec != LQCD_F64 && o.true_prec != LQCD_DF64)
    return set_error(LQCD_EINVAL, "true_prec must be LQCD_F64, LQCD_DF64 or -1");
  if (o.sloppy_compress != 12 && o.sloppy_compress != 18) return set_error(LQCD_EINVAL, "sloppy compress");
  if (o.maxiter < 1) o.maxiter = 50000;
  if (o.chunk < 1) o.chunk = 8;
  LQCD_CK(cudaSetDevice(c->device));
  lqcd_engine* e = new lqcd_engine();
  e->ctx = c;
  ctx_retain(c);
  e->opts = o;
  const bool fp64_class = (o.sloppy_prec == LQCD_F64 || o.sloppy_prec == LQCD_DF64);
  e->sp = o.sloppy_prec;
  e->xp = fp64_class ? o.sloppy_prec : P_F32;
  e->nr = fp64_class ? 18 : o.sloppy_compress;
  e->tp = (o.true_prec == -1) ? (o.sloppy_prec == LQCD_F64 ? P_F64 : P_DF64) : o.true_prec;
  // Default delta by sloppy storage, measured on GB300 (32^3x64 at kappa 0.155, tol 1e-10;
  // smaller delta: fewer FP64-class updates, until the sloppy residual recurrence drifts):
  // FP16 / BF16 0.01 (six updates, 39 / 45 iterations; at 0.003 BF16 took 944 iterations
  // and at 0.0003 FP16 269), FP32 0.001 (five updates, 40 iterations, 3% faster than at
  // 0.01; the 12-source 24^3x48 batch 4% faster). The FP64-class true residual decides
  // convergence in every case.
  const double delta = o.delta > 0 ? o.delta : (fp64_class ? 0.0 : (o.sloppy_prec == LQCD_F32 ? 0.001 : 0.01));
  e->delta2 = delta * delta;
  e->ru_every = o.ru_interval > 0 ? std::min(o.ru_interval, o.chunk) : 0;  // 0: per batch
  e->budget = budget;
  e->max_slots = max_slots;
  cudaError_t err = cudaMalloc(&e->d_sc, sizeof(Scalars) * max_slots);
  if (err == cudaSuccess) err = cudaMemset(e->d_sc, 0, sizeof(Scalars) * max_slots);
  if (err == cudaSuccess) err = cudaMallocHost(&e->h_sc, sizeof(Scalars) * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_works, sizeof(Work) * NSTEP * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_prefix, sizeof(int) * (max_slots + 1));
  if (err != cudaSuccess) {
    lqcd_engine_destroy(e);
    return set_error(LQCD_ENOMEM, "engine: %s", cudaGetErrorString(err));
  }
  for (int i = max_slots - 1; i >= 0; --i) e->free_slots.push_back(i);
  *out = e;
  return LQCD_OK;
}

void lqcd_engine_destroy(lqcd_engine* e) {
  if (!e) return;
  cudaSetDevice(e->ctx->device);
  cudaStreamSynchronize(e->ctx->stream);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  for (auto& kv : e->reqs)
    if (kv.second.buf.block) cudaFree(kv.second.buf.block);
  for (auto& kv : e->pool) cudaFree(kv.second);
  if (e->d_sc) cudaFree(e->d_sc);
  if (e->h_sc) cudaFreeHost(e->h_sc);
  if (e->d_works) cudaFree(e->d_works);
  if (e->d_prefix) cudaFree(e->d_prefix);
  if (e->d_partials) cudaFree(e->d_partials);
  lqcd_ctx* c = e->ctx;
  const bool release = e->holds_ctx;
  delete e;
  if (release) ctx_release(c);
}

size_t lqcd_engine_request_bytes(const lqcd_engine* e, const int dims[4]) {
  Geom g;
  if (!e || make_geom(dims, -1, g) != LQCD_OK) return 0;
  return slot_bytes(e, g.Vh);
}

int lqcd_engine_submit(lqcd_engine* e, const lqcd_gauge* gauge, const lqcd_field* src, double kappa,
                       double tol, long long* request_id) {
  LQCD_TRACE("lqcd_engine_submit");
  if (!e) {
    clear_error();
    return set_error(LQCD_EINVAL, "engine is NULL");
  }
  return lqcd_engine_submit_tm(e, gauge, src, kappa, e->opts.mu, tol, request_id);
}

static int submit_impl(lqcd_engine* e, const lqcd_gauge* gauge, const lqcd_field* src, double kappa,
                       double mu, double tol, bool normal, long long* request_id,
                       const lqcd_field* x0 = nullptr);

int lqcd_engine_submit_tm(lqcd_engine* e, const lqcd_gauge* gauge, const lqcd_field* src, double kappa,
                          double mu, double tol, long long* request_id) {
  LQCD_TRACE("lqcd_engine_submit_tm");
  return submit_impl(e, gauge, src, kappa, mu, tol, false, request_id);
}

int lqcd_engine_submit_normal(lqcd_engine* e, const lqcd_gauge* gauge, const lqcd_field* src, double kappa,
                              double mu, double tol, long long* request_id) {
  LQCD_TRACE("lqcd_engine_submit_normal");
  return submit_impl(e, gauge, src, kappa, mu, tol, true, request_id);
}

// x0 (may be NULL): the starting even half x_e (a FULL or EVEN FP64 field of the lattice);
// NULL starts from x = 0
static int submit_impl(lqcd_engine* e, const lqcd_gauge* gauge, const lqcd_field* src, double kappa,
                       double mu, double tol, bool normal, long long* request_id, const lqcd_field* x0) {
  PdlSolverScope pdl_scope(gauge && pdl_solver_off((gauge->g.Vh + TILE - 1) / TILE));  // large: no PDL
  clear_error();
  if (!e || !gauge || !src || !request_id) return set_error(LQCD_EINVAL, "NULL argument");
  if (x0 && (x0->prec != LQCD_F64 || !x0->half[0] || memcmp(x0->g.L, gauge->g.L, sizeof x0->g.L)))
    return set_error(LQCD_EINVAL, "the initial guess must be an FP64 field of the lattice holding the even parity");
  if (!std::isfinite(mu) || !std::isfinite(kappa)) return set_error(LQCD_EINVAL, "kappa and mu must be finite");
  if (src->prec != LQCD_F64 || src->subset != LQCD_FULL)
    return set_error(LQCD_EINVAL, "source must be a FULL FP64 field");
  if (memcmp(src->g.L, gauge->g.L, sizeof src->g.L)) return set_error(LQCD_EINVAL, "lattice mismatch");
  if (!(tol > 0) || !(kappa >= 0)) return set_error(LQCD_EINVAL, "tol must be > 0 and kappa >= 0");
  if (gauge->ctx != e->ctx || src->ctx != e->ctx) return set_error(LQCD_EINVAL, "context mismatch");
  lqcd_ctx* c = e->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  const size_t need = slot_bytes(e, gauge->g.Vh);
  if (e->budget && need > e->budget) return set_error(LQCD_ENOMEM, "request needs %zu bytes > budget %zu", need, e->budget);
  if (e->free_slots.empty()) return set_error(LQCD_EBUSY, "no free slot");
  if (e->budget && e->bytes_in_use + need > e->budget)
    return set_error(LQCD_EBUSY, "budget: %zu in use + %zu > %zu", e->bytes_in_use, need, e->budget);
  // sloppy and true-residual link copies
  if (e->sp != P_F64) {
    int rc = lqcd_gauge_add_copy(const_cast<lqcd_gauge*>(gauge), e->sp, e->nr);
    if (rc != LQCD_OK) return rc;
  }
  if (e->tp != P_F64) {
    int rc = lqcd_gauge_add_copy(const_cast<lqcd_gauge*>(gauge), e->tp, 18);
    if (rc != LQCD_OK) return rc;
  }
  Request q;
  q.id = e->next_id++;
  q.gauge = gauge;
  q.g = gauge->g;
  q.kappa = kappa;
  q.tol = tol;
  q.mu = mu;
  q.normal = normal;
  q.ntiles = (q.g.Vh + TILE - 1) / TILE;
  q.t0 = std::chrono::steady_clock::now();
  int rc = alloc_block(e, need, &q.buf.block);
  if (rc != LQCD_OK) return rc;
  q.buf.bytes = need;
  carve(q.buf, e, q.g.Vh);
  q.slot = e->free_slots.back();
  e->free_slots.pop_back();
  e->bytes_in_use += need;
  e->reqs[q.id] = q;
  Request& R = e->reqs[q.id];
  rc = assign_tiles(e, R);
  cudaStream_t st = c->stream;
  const size_t hb = half_spinor_bytes(e->tp, q.g.Vh);
  Scalars* sc = e->d_sc + R.slot;
  if (rc == LQCD_OK) {
    cudaError_t err = spinor_convert(src->half[0], P_F64, R.buf.be, e->tp, q.g.Vh, 1.0, st);
    if (err == cudaSuccess) {
      if (normal) err = cudaMemsetAsync(R.buf.bo, 0, hb, st);  // only phi_e counts
      else err = spinor_convert(src->half[1], P_F64, R.buf.bo, e->tp, q.g.Vh, 1.0, st);
    }
    if (err == cudaSuccess)
      err = x0 ? spinor_convert(x0->half[0], P_F64, R.buf.x64, e->tp, q.g.Vh, 1.0, st)
               : cudaMemsetAsync(R.buf.x64, 0, hb, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(R.buf.xs, 0, half_spinor_bytes(e->xp, q.g.Vh), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc, 0, sizeof(Scalars), st);
    if (err != cudaSuccess) rc = set_error(LQCD_ECUDA, "submit copies: %s", cudaGetErrorString(err));
  }
  if (rc == LQCD_OK) {
    // |b|^2 (both halves) and bhat_e = b_e + kappa D_eo b_o, in FP64
    Work w = slot_work(e, R);
    w.red = 1;
    w.in = R.buf.be;
    w.fin = FIN_STORE0;
    cudaError_t err = launch_blas(e->tp, B_NORM, single_launch(w, e->d_partials), 0, st);
    w.in = R.buf.bo;
    w.fin = FIN_STORE1;
    if (err == cudaSuccess) err = launch_blas(e->tp, B_NORM, single_launch(w, e->d_partials), 0, st);
    if (err == cudaSuccess) {
      k_slot_init<<<1, 1, 0, st>>>(sc, tol * tol, 24.0 * q.g.Vh, e->opts.maxiter, e->delta2, normal ? 1 : 0);
      err = cudaGetLastError();
    }
    const double ta = 2.0 * kappa * mu;
    if (err == cudaSuccess && normal) {
      // normal equations: bhat = 0, so the update computes u = -Mhat x and rho = phi + Mhat^dag u
      err = cudaMemsetAsync(R.buf.bhat, 0, hb, st);
    }
    if (err == cudaSuccess && ta != 0.0 && !normal) {
      // t = A^-1 b_o
      Work w3 = slot_work(e, R);
      w3.in = R.buf.bo;
      w3.out = R.buf.t64;
      set_twist(w3, 1.0 / (1.0 + ta * ta), -ta, 0.0);
      err = launch_blas(e->tp, B_TWIST, single_launch(w3, e->d_partials), 0, st);
      c->launches++;
    }
    if (err == cudaSuccess && !normal) {
      // bhat_e = b_e + kappa D_eo A^-1 b_o
      Work d = slot_work(e, R);
      const void* U64 = gauge->copy[e->tp][0];
      d.out_par = 0;
      d.Uout = parity_links(U64, e->tp, 18, q.g.Vh, 0);
      d.Uin = parity_links(U64, e->tp, 18, q.g.Vh, 1);
      d.in = ta != 0.0 ? R.buf.t64 : R.buf.bo;
      d.out = R.buf.bhat;
      d.y1 = R.buf.be;
      d.c1 = 1.0;
      d.a = kappa;
      err = launch_dslash(e->tp, 18, false, EPI_LIN, single_launch(d, e->d_partials), 0, st);
    }
    if (err == cudaSuccess) {
      // first true residual and restart (state UPDATE, restart_p = 1). With x = 0 the update's
      // fold and its two FP64-class Dslash would compute u = bhat - Mhat 0 from zero fields:
      // u = bhat exactly, so it is an exact copy (a = 1) with its norm and the same finisher,
      // followed by the rest of the update.
      // From an initial guess the whole update runs (u = bhat - Mhat x0).
      Work w2[NSTEP];
      step_works(e, R, w2);
      if (!x0) {
        Work cu = slot_work(e, R);
        cu.in = R.buf.bhat;
        cu.out = R.buf.u64;
        cu.a = 1.0;
        cu.red = 1;
        cu.fin = FIN_TRUERES;
        cu.run_if = S_UPDATE;
        err = launch_blas(e->tp, B_AXPBY, single_launch(cu, e->d_partials), 0, st, e->tp);
      }
      for (int s : ru_steps(normal, !normal)) {
        if (err != cudaSuccess) break;
        if (!x0 && (s == RU_FOLD || s == RU_D1 || s == RU_RES)) continue;
        err = issue(e, s, single_launch(w2[s], e->d_partials), mu != 0.0);
      }
    }
    c->launches += 4;
    if (err != cudaSuccess) rc = set_error(LQCD_ECUDA, "submit kernels: %s", cudaGetErrorString(err));
  }
  if (rc != LQCD_OK) {
    e->free_slots.push_back(R.slot);
    e->bytes_in_use -= need;
    cudaFree(R.buf.block);
    e->reqs.erase(q.id);
    return rc;
  }
  e->active.push_back(q.id);
  e->dirty = true;
  *request_id = q.id;
  return LQCD_OK;
}

// tiles of the launches over the engine's active solves (the programmatic-launch rule)
static long long engine_active_tiles(const lqcd_engine* e) {
  long long t = 0;
  if (e)
    for (long long id : e->active) t += e->reqs.at(id).ntiles;
  return t;
}

int lqcd_engine_step(lqcd_engine* e, int* n_active) {
  LQCD_TRACE("lqcd_engine_step");
  PdlSolverScope pdl_scope(pdl_solver_off(engine_active_tiles(e)));  // large launches: no PDL
  clear_error();
  if (!e) return set_error(LQCD_EINVAL, "engine is NULL");
  lqcd_ctx* c = e->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  if (!e->active.empty()) {
    if (e->dirty) {
      int rc = rebuild(e);
      if (rc != LQCD_OK) return rc;
    }
    if (e->opts.use_graph) {
      LQCD_CK(cudaGraphLaunch(e->exec, st));
      c->launches += (long long)e->opts.chunk * 5 +
                     ((e->opts.chunk + e->ru_every - 1) / e->ru_every) *
                         (long long)ru_steps(e->any_normal, e->any_plain).size();
    } else {
      cudaError_t err = issue_iteration_block(e, e->opts.chunk);
      if (err != cudaSuccess) return set_error(LQCD_ECUDA, "iteration: %s", cudaGetErrorString(err));
    }
    int maxslot = 0;
    for (long long id : e->active) maxslot = std::max(maxslot, e->reqs[id].slot + 1);
    LQCD_CK(cudaMemcpyAsync(e->h_sc, e->d_sc, sizeof(Scalars) * maxslot, cudaMemcpyDeviceToHost, st));
    LQCD_CK(cudaStreamSynchronize(st));
    std::vector<long long> fin;
    for (long long id : e->active) {
      const Scalars& s = e->h_sc[e->reqs[id].slot];
      if (s.state == S_DONE || s.state == S_FAILED) fin.push_back(id);
    }
    if (!fin.empty()) {
      for (long long id : fin) {
        int rc = finalize_launch(e, e->reqs[id]);
        if (rc != LQCD_OK) return rc;
      }
      LQCD_CK(cudaMemcpyAsync(e->h_sc, e->d_sc, sizeof(Scalars) * maxslot, cudaMemcpyDeviceToHost, st));
      LQCD_CK(cudaStreamSynchronize(st));
      const auto now = std::chrono::steady_clock::now();
      for (long long id : fin) {
        Request& q = e->reqs[id];
        const Scalars& s = e->h_sc[q.slot];
        q.finished = true;
        q.info.status = status_of(s.status);
        q.info.iters = s.iter;
        q.info.reliable_updates = s.n_updates;
        const double r2 = q.normal ? s.rho2 : s.res[0] + s.res[1];
        q.info.true_resid = s.res[3] > 0 ? sqrt(r2 / s.res[3]) : 0.0;
        q.info.ms = std::chrono::duration<double, std::milli>(now - q.t0).count();
        if (q.info.status == LQCD_OK && !(q.info.true_resid <= q.tol)) {
          // the Schur residual met the tolerance but the full one did not
          q.info.status = LQCD_ENOCONV;
        }
        e->done_ids.push_back(id);
        e->active.erase(std::find(e->active.begin(), e->active.end(), id));
      }
      e->dirty = true;
    }
  }
  if (n_active) *n_active = (int)e->active.size();
  return LQCD_OK;
}

int lqcd_engine_completed(lqcd_engine* e, long long* ids, int max, int* n) {
  clear_error();
  if (!e || !n || (max > 0 && !ids)) return set_error(LQCD_EINVAL, "NULL argument");
  int k = 0;
  while (k < max && k < (int)e->done_ids.size()) {
    ids[k] = e->done_ids[k];
    ++k;
  }
  e->done_ids.erase(e->done_ids.begin(), e->done_ids.begin() + k);
  *n = k;
  return LQCD_OK;
}

int lqcd_engine_result(lqcd_engine* e, long long id, lqcd_field* x, lqcd_solve_info* info) {
  LQCD_TRACE("lqcd_engine_result");
  clear_error();
  if (!e) return set_error(LQCD_EINVAL, "engine is NULL");
  auto it = e->reqs.find(id);
  if (it == e->reqs.end()) return set_error(LQCD_EINVAL, "unknown request %lld", id);
  Request& q = it->second;
  PdlSolverScope pdl_scope(pdl_solver_off(q.ntiles));  // large launches: no PDL
  if (!q.finished) return set_error(LQCD_EBUSY, "request %lld still running", id);
  LQCD_CK(cudaSetDevice(e->ctx->device));
  if (x) {
    if (x->subset != LQCD_FULL || memcmp(x->g.L, q.g.L, sizeof q.g.L))
      return set_error(LQCD_EINVAL, "x must be a FULL field of the request's lattice");
    LQCD_CK(spinor_convert(q.buf.x64, e->tp, x->half[0], x->prec, q.g.Vh, 1.0, e->ctx->stream));
    LQCD_CK(spinor_convert(q.buf.t64, e->tp, x->half[1], x->prec, q.g.Vh, 1.0, e->ctx->stream));
  }
  if (info) *info = q.info;
  const int rc = q.info.status;
  // release the slot
  LQCD_CK(cudaStreamSynchronize(e->ctx->stream));
  e->pool.insert({q.buf.bytes, q.buf.block});
  e->bytes_pooled += q.buf.bytes;
  e->bytes_in_use -= q.buf.bytes;
  e->free_slots.push_back(q.slot);
  e->reqs.erase(it);
  return rc;
}

int lqcd_engine_cancel(lqcd_engine* e, long long id, int status) {
  clear_error();
  if (!e) return set_error(LQCD_EINVAL, "engine is NULL");
  auto it = e->reqs.find(id);
  if (it == e->reqs.end()) return set_error(LQCD_EINVAL, "unknown request %lld", id);
  if (status >= 0) return set_error(LQCD_EINVAL, "cancel status must be a negative LQCD_E* code");
  if (it->second.finished) return LQCD_OK;
  LQCD_CK(cudaSetDevice(e->ctx->device));
  k_slot_cancel<<<1, 1, 0, e->ctx->stream>>>(e->d_sc + it->second.slot, status);
  LQCD_CK(cudaGetLastError());
  return LQCD_OK;
}

int lqcd_engine_stats(const lqcd_engine* e, int* active, size_t* bytes) {
  if (!e) return set_error(LQCD_EINVAL, "engine is NULL");
  if (active) *active = (int)e->active.size();
  if (bytes) *bytes = e->bytes_in_use;
  return LQCD_OK;
}

// ------------------------------------------------------------------ one-shot solves

}  // extern "C"

namespace lqcd {

static bool same_opts(const lqcd_solve_opts& a, const lqcd_solve_opts& b) {
  return a.solver == b.solver && a.sloppy_prec == b.sloppy_prec && a.sloppy_compress == b.sloppy_compress &&
         a.maxiter == b.maxiter && a.delta == b.delta && a.chunk == b.chunk && a.use_graph == b.use_graph &&
         a.ru_interval == b.ru_interval && a.true_prec == b.true_prec &&
         a.multi_rhs_links == b.multi_rhs_links;  // mu is per request
}

void ctx_drop_engine(lqcd_ctx* c) {
  if (c->engine_cache) lqcd_engine_destroy(c->engine_cache);
  c->engine_cache = nullptr;
}

int ctx_engine(lqcd_ctx* c, const lqcd_solve_opts& o, int n, lqcd_engine** out) {
  lqcd_engine* e = c->engine_cache;
  if (e && same_opts(c->engine_opts, o) && e->max_slots >= n && e->active.empty() && e->reqs.empty()) {
    *out = e;
    return LQCD_OK;
  }
  ctx_drop_engine(c);
  int rc = lqcd_engine_create(c, &o, 0, std::max(n, 16), &e);
  if (rc != LQCD_OK) return rc;
  e->holds_ctx = false;  // the context owns this engine
  ctx_release(c);        // undo the reference lqcd_engine_create took
  c->engine_cache = e;
  c->engine_opts = o;
  *out = e;
  return LQCD_OK;
}

int engine_submit_normal_guess(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* src,
                               const lqcd_field* x0, double kappa, double mu, double tol, long long* id) {
  return submit_impl(e, g, src, kappa, mu, tol, true, id, x0);
}

void engine_trim_pool(lqcd_engine* e, size_t keep_bytes) {
  if (e->bytes_pooled <= keep_bytes) return;
  cudaStreamSynchronize(e->ctx->stream);
  // free the smallest blocks first; the largest (most recent lattice) usually stays
  while (e->bytes_pooled > keep_bytes && !e->pool.empty()) {
    auto it = e->pool.begin();
    cudaFree(it->second);
    e->bytes_pooled -= it->first;
    e->pool.erase(it);
  }
}

}  // namespace lqcd

extern "C" {

static int run_engine(lqcd_engine* e, int n, const long long* ids, lqcd_field* const* xs,
                      lqcd_solve_info* infos) {
  int active = n;
  while (active > 0) {
    int rc = lqcd_engine_step(e, &active);
    if (rc != LQCD_OK) return rc;
  }
  int first_bad = LQCD_OK;
  for (int i = 0; i < n; ++i) {
    lqcd_solve_info info{};
    int rc = lqcd_engine_result(e, ids[i], xs[i], &info);
    if (infos) infos[i] = info;
    if (rc != LQCD_OK && first_bad == LQCD_OK) first_bad = rc;
  }
  return first_bad;
}

int lqcd_solve_fields(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                      const lqcd_solve_opts* opts, lqcd_field* x, lqcd_solve_info* info) {
  LQCD_TRACE("lqcd_solve_fields");
  const lqcd_field* s[1] = {src};
  lqcd_field* xx[1] = {x};
  return lqcd_solve_multi(g, 1, s, kappa, tol, opts, xx, info);
}

int lqcd_solve_multi(const lqcd_gauge* g, int n, const lqcd_field* const* srcs, double kappa,
                     double tol, const lqcd_solve_opts* opts, lqcd_field* const* xs,
                     lqcd_solve_info* infos) {
  LQCD_TRACE("lqcd_solve_multi");
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (!g || n < 1 || n > MAX_SLOTS || !srcs || !xs) return set_error(LQCD_EINVAL, "bad arguments");
  lqcd_solve_opts o;
  lqcd_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.solver == LQCD_BICGSTAB) {
    int first_bad = LQCD_OK;
    for (int i = 0; i < n; ++i) {
      lqcd_solve_info inf{};
      int rc = bicgstab_solve(g, srcs[i], kappa, tol, &o, xs[i], &inf);
      if (infos) infos[i] = inf;
      if (rc != LQCD_OK && first_bad == LQCD_OK) first_bad = rc;
    }
    return first_bad;
  }
  lqcd_engine* e = nullptr;
  int rc = ctx_engine(g->ctx, o, n, &e);
  if (rc != LQCD_OK) return rc;
  std::vector<long long> ids(n);
  int submitted = 0;
  for (int i = 0; i < n && rc == LQCD_OK; ++i) {
    rc = lqcd_engine_submit_tm(e, g, srcs[i], kappa, o.mu, tol, &ids[i]);
    if (rc == LQCD_OK) ++submitted;
  }
  if (rc == LQCD_OK) rc = run_engine(e, n, ids.data(), xs, infos);
  if (rc != LQCD_OK && !(rc == LQCD_ENOCONV || rc == LQCD_EBREAKDOWN || rc == LQCD_ENONFINITE)) {
    ctx_drop_engine(g->ctx);  // a failed submit or launch may leave requests behind
  } else {
    engine_trim_pool(e, (size_t)8 << 30);
  }
  (void)submitted;
  if (infos && rc != LQCD_ECUDA && rc != LQCD_EINVAL) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (n == 1) infos[0].ms = ms;
  }
  return rc;
}

int lqcd_solve_batch(int n, const lqcd_gauge* const* gauges, const lqcd_field* const* srcs,
                     const double* kappas, const double* tols, const lqcd_solve_opts* opts,
                     lqcd_field* const* xs, lqcd_solve_info* infos) {
  LQCD_TRACE("lqcd_solve_batch");
  clear_error();
  if (n < 1 || n > MAX_SLOTS || !gauges || !srcs || !kappas || !tols || !xs)
    return set_error(LQCD_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i) {
    if (!gauges[i] || !srcs[i] || !xs[i]) return set_error(LQCD_EINVAL, "NULL entry %d", i);
    if (gauges[i]->ctx != gauges[0]->ctx) return set_error(LQCD_EINVAL, "gauges of different contexts");
  }
  lqcd_solve_opts o;
  lqcd_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.solver == LQCD_BICGSTAB) {
    int first_bad = LQCD_OK;
    for (int i = 0; i < n; ++i) {
      lqcd_solve_info inf{};
      int rc = bicgstab_solve(gauges[i], srcs[i], kappas[i], tols[i], &o, xs[i], &inf);
      if (infos) infos[i] = inf;
      if (rc != LQCD_OK && first_bad == LQCD_OK) first_bad = rc;
    }
    return first_bad;
  }
  lqcd_ctx* c = gauges[0]->ctx;
  lqcd_engine* e = nullptr;
  int rc = ctx_engine(c, o, n, &e);
  if (rc != LQCD_OK) return rc;
  std::vector<long long> ids(n);
  for (int i = 0; i < n && rc == LQCD_OK; ++i)
    rc = lqcd_engine_submit_tm(e, gauges[i], srcs[i], kappas[i], o.mu, tols[i], &ids[i]);
  if (rc == LQCD_OK) rc = run_engine(e, n, ids.data(), xs, infos);
  if (rc != LQCD_OK && !(rc == LQCD_ENOCONV || rc == LQCD_EBREAKDOWN || rc == LQCD_ENONFINITE)) {
    ctx_drop_engine(c);  // a failed submit or launch may leave requests behind
  } else {
    engine_trim_pool(e, (size_t)8 << 30);
  }
  return rc;
}

int lqcd_solve(const lqcd_gauge* g, const double* host_src, double kappa, double tol,
               const lqcd_solve_opts* opts, double* host_x, lqcd_solve_info* info) {
  LQCD_TRACE("lqcd_solve");
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (!g || !host_src || !host_x) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = g->ctx;
  int dims[4] = {g->g.L[0], g->g.L[1], g->g.L[2], g->g.L[3]};
  lqcd_field *b = nullptr, *x = nullptr;
  lqcd_solve_info inf{};
  int rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &b);
  if (rc == LQCD_OK) rc = lqcd_field_create(c, dims, LQCD_F64, LQCD_FULL, &x);
  if (rc == LQCD_OK) rc = lqcd_field_upload(b, host_src);
  int src_rc = rc;
  if (rc == LQCD_OK) rc = lqcd_solve_fields(g, b, kappa, tol, opts, x, &inf);
  if (src_rc == LQCD_OK && (rc == LQCD_OK || rc == LQCD_ENOCONV || rc == LQCD_EBREAKDOWN ||
                            rc == LQCD_ENONFINITE)) {
    int rc2 = lqcd_field_download(x, host_x);
    if (rc2 != LQCD_OK) rc = rc2;
  }
  lqcd_field_destroy(b);
  lqcd_field_destroy(x);
  inf.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return rc;
}

}  // extern "C"
