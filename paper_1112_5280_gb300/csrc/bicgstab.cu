// BiCGStab (van der Vorst) on the even-odd Schur operator Mhat
// (paper Section 3: inversion of the even-odd preconditioned fermion matrix).
//
// Inner iterations run in the sloppy precision (FP64 or FP32 storage and
// arithmetic); an FP64 defect-correction loop wraps them: u = bhat - Mhat x
// (FP64 links), r = u / |u|, inner BiCGStab to |r| <= delta_inner, then
// x += |u| e. The scalar recurrences (rho, alpha, omega, beta) run on the
// device in the slot's finishers; the host only polls the state between
// chunks of iterations.
//
// Twisted mass (a = 2 kappa mu != 0): Mhat = A - kappa^2 D_eo A^-1 D_oe with
// A = 1 + i a g5; A^-1 multiplies the odd-target Dslash in its epilogue and A the
// operand vector of the even-target one (twist fields of Work).
#include <chrono>
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {

__global__ void k_bicg_init(Scalars* s, double delta2, int maxiter) {
  const double rr = s->res[0];  // |r|^2 of the normalised restart residual (r0 = r)
  s->cres[0] = rr;              // rho = <r0, r>
  s->cres[1] = 0.0;
  s->cres[2] = 1.0;  // alpha
  s->cres[3] = 0.0;
  s->cres[4] = 1.0;  // omega
  s->cres[5] = 0.0;
  s->cres[6] = 0.0;  // beta (p = r on the first iteration)
  s->cres[7] = 0.0;
  s->stop_rr = delta2 * rr;
  s->iter = 0;
  s->maxiter = maxiter;
  s->state = S_RUNNING;
  s->status = ST_OK;
  s->ticket = 0;
}

}  // namespace lqcd

using namespace lqcd;

namespace {

struct BicgBufs {
  void* block = nullptr;
  void *be, *bo, *bhat, *x64, *u64, *t64;
  void *r, *r0, *p, *v, *s, *t, *o, *xs;
};

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int lqcd::bicgstab_solve(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                              const lqcd_solve_opts* o, lqcd_field* x, lqcd_solve_info* info) {
  PdlSolverScope pdl_scope(g && pdl_solver_off((g->g.Vh + TILE - 1) / TILE));  // large: no PDL
  const auto t0 = std::chrono::steady_clock::now();
  if (info) memset(info, 0, sizeof *info);
  if (!g || !src || !x || !o) return set_error(LQCD_EINVAL, "NULL argument");
  if (src->prec != LQCD_F64 || src->subset != LQCD_FULL || x->subset != LQCD_FULL)
    return set_error(LQCD_EINVAL, "source must be FULL FP64 and x FULL");
  const int sp = o->sloppy_prec;
  if (sp != LQCD_F64 && sp != LQCD_F32 && sp != LQCD_DF64)
    return set_error(LQCD_EINVAL, "BiCGStab runs with FP64, DF64 or FP32 inner precision");
  // FP64-class vectors and operator of the outer defect correction
  const int tp = (o->true_prec == -1) ? (sp == LQCD_F64 ? P_F64 : P_DF64) : o->true_prec;
  if (tp != P_F64 && tp != P_DF64) return set_error(LQCD_EINVAL, "true_prec");
  if (!(tol > 0)) return set_error(LQCD_EINVAL, "tol must be > 0");
  if (!std::isfinite(o->mu) || !std::isfinite(kappa)) return set_error(LQCD_EINVAL, "kappa and mu must be finite");
  const double ta = 2.0 * kappa * o->mu, ts = 1.0 / (1.0 + ta * ta);
  // hopping term times A^-1 (odd targets) / operand y2 times A (even targets)
  auto tw_inv = [&](Work& w) { if (ta != 0.0) set_twist(w, ts, -ta, 0.0); };
  auto tw_a = [&](Work& w) { if (ta != 0.0) set_twist(w, 1.0, 0.0, ta); };
  lqcd_ctx* c = g->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  const Geom gm = g->g;
  const int Vh = gm.Vh;
  const int nr = (sp == LQCD_F64 || sp == LQCD_DF64) ? 18 : o->sloppy_compress;
  if (sp != LQCD_F64) {
    int rc = lqcd_gauge_add_copy(const_cast<lqcd_gauge*>(g), sp, nr);
    if (rc != LQCD_OK) return rc;
  }
  if (tp != P_F64) {
    int rc = lqcd_gauge_add_copy(const_cast<lqcd_gauge*>(g), tp, 18);
    if (rc != LQCD_OK) return rc;
  }
  const void* US = g->copy[link_prec_for(sp)][nr == 12];
  const void* U64 = g->copy[tp][0];
  const size_t h64 = a256(half_spinor_bytes(tp, Vh)), hs = a256(half_spinor_bytes(sp, Vh));
  BicgBufs b;
  // the vectors live on the context between calls: repeated solves allocate nothing
  if (ctx_work(c, 6 * h64 + 8 * hs) != LQCD_OK) {
    const std::string why = lqcd_last_error();
    return set_error(LQCD_ENOMEM, "BiCGStab buffers: %s", why.c_str());
  }
  cudaError_t err = cudaSuccess;
  b.block = c->work;
  {
    char* p = static_cast<char*>(b.block);
    void** f64[] = {&b.be, &b.bo, &b.bhat, &b.x64, &b.u64, &b.t64};
    for (void** q : f64) { *q = p; p += h64; }
    void** fs[] = {&b.r, &b.r0, &b.p, &b.v, &b.s, &b.t, &b.o, &b.xs};
    for (void** q : fs) { *q = p; p += hs; }
  }
  Scalars* sc = c->scratch_sc + 1;
  int rc = ctx_partials(c, 3 * (size_t)((Vh + TILE - 1) / TILE));
  auto base = [&]() {
    Work w = blank_work(gm);
    w.sc = sc;
    return w;
  };
  auto links = [&](Work& w, const void* U, int lp, int n, int out_par) {
    w.out_par = out_par;
    w.Uout = parity_links(U, lp, n, Vh, out_par);
    w.Uin = parity_links(U, lp, n, Vh, 1 - out_par);
  };
  auto dsl = [&](int prec, const Work& w, bool dag) {
    c->launches++;
    return launch_dslash(prec, prec == tp ? 18 : nr, dag, w.twist ? EPI_LIN_TW : EPI_LIN,
                         single_launch(w, c->partials), 0, st);
  };
  auto blas = [&](int prec, int op, const Work& w) {
    c->launches++;
    return launch_blas(prec, op, single_launch(w, c->partials), 0, st, tp);
  };
  auto read_sc = [&](Scalars* h) -> int {
    LQCD_CK(cudaMemcpyAsync(h, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    LQCD_CK(cudaStreamSynchronize(st));
    return LQCD_OK;
  };
  Scalars* hs_ = c->host_sc + 1;
  int status = LQCD_OK, iters = 0, outer = 0;
  double bnorm2 = 0;
  if (rc == LQCD_OK) {
    err = spinor_convert(src->half[0], P_F64, b.be, tp, Vh, 1.0, st);
    if (err == cudaSuccess) err = spinor_convert(src->half[1], P_F64, b.bo, tp, Vh, 1.0, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(b.x64, 0, h64, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc, 0, sizeof(Scalars), st);
    // |b|^2
    Work w = base();
    w.red = 1;
    w.fin = FIN_STORE0;
    w.in = b.be;
    if (err == cudaSuccess) err = blas(tp, B_NORM, w);
    w.fin = FIN_STORE1;
    w.in = b.bo;
    if (err == cudaSuccess) err = blas(tp, B_NORM, w);
    // t = A^-1 b_o ; bhat = b_e + kappa D_eo t
    if (ta != 0.0 && err == cudaSuccess) {
      Work tw = base();
      tw.in = b.bo; tw.out = b.t64;
      tw_inv(tw);
      err = blas(tp, B_TWIST, tw);
    }
    Work d = base();
    links(d, U64, tp, 18, 0);
    d.in = ta != 0.0 ? b.t64 : b.bo; d.out = b.bhat; d.y1 = b.be; d.c1 = 1.0; d.a = kappa;
    if (err == cudaSuccess) err = dsl(tp, d, false);
    if (err == cudaSuccess) rc = read_sc(hs_);
    else rc = set_error(LQCD_ECUDA, "BiCGStab setup: %s", cudaGetErrorString(err));
    bnorm2 = hs_->res[0] + hs_->res[1];
  }
  const double target2 = tol * tol * bnorm2;
  const int max_outer = 200;
  while (rc == LQCD_OK && status == LQCD_OK) {
    // FP64 true residual u = bhat - Mhat x
    Work d1 = base();
    links(d1, U64, tp, 18, 1);
    d1.in = b.x64; d1.out = b.t64; d1.a = 1.0;
    tw_inv(d1);
    Work d2 = base();
    links(d2, U64, tp, 18, 0);
    d2.in = b.t64; d2.out = b.u64; d2.y1 = b.bhat; d2.c1 = 1.0; d2.y2 = b.x64; d2.c2 = -1.0;
    d2.a = kappa * kappa; d2.red = 1; d2.fin = FIN_STORE0;
    tw_a(d2);
    err = dsl(tp, d1, false);
    if (err == cudaSuccess) err = dsl(tp, d2, false);
    if (err != cudaSuccess) { rc = set_error(LQCD_ECUDA, "residual: %s", cudaGetErrorString(err)); break; }
    if ((rc = read_sc(hs_)) != LQCD_OK) break;
    const double u2 = hs_->res[0];
    if (!std::isfinite(u2)) { status = LQCD_ENONFINITE; break; }
    if (u2 <= target2) break;
    if (outer >= max_outer || iters >= o->maxiter) { status = LQCD_ENOCONV; break; }
    ++outer;
    const double sigma = std::sqrt(u2);
    // restart: r = r0 = u / sigma, p = v = xs = 0
    Work cv = base();
    cv.in = b.u64; cv.out = b.r; cv.a = 1.0 / sigma; cv.red = 1; cv.fin = FIN_STORE0;
    err = blas(sp, B_AXPBY, cv);
    cv.out = b.r0; cv.red = 0; cv.fin = FIN_NONE;
    if (err == cudaSuccess) err = blas(sp, B_AXPBY, cv);
    if (err == cudaSuccess) err = cudaMemsetAsync(b.p, 0, hs, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(b.v, 0, hs, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(b.xs, 0, hs, st);
    // inner target: the remaining defect, limited by the sloppy precision
    double rel = 0.5 * std::sqrt(target2) / sigma;
    if (sp == LQCD_F32) rel = std::max(rel, 1e-5);
    if (sp == LQCD_DF64 && tp == P_F64) rel = std::max(rel, 1e-12);
    if (err == cudaSuccess) {
      k_bicg_init<<<1, 1, 0, st>>>(sc, rel * rel, o->maxiter - iters);
      err = cudaGetLastError();
    }
    if (err != cudaSuccess) { rc = set_error(LQCD_ECUDA, "restart: %s", cudaGetErrorString(err)); break; }
    // iteration kernels
    const double kk = kappa * kappa;
    Work w1 = base();  // p = r + beta (p - omega v)
    w1.in = b.r; w1.out = b.p; w1.y1 = b.v; w1.run_if = S_RUNNING;
    Work w2 = base();  // o = D_oe p
    links(w2, US, link_prec_for(sp), nr, 1);
    w2.in = b.p; w2.out = b.o; w2.a = 1.0; w2.run_if = S_RUNNING;
    tw_inv(w2);
    Work w3 = base();  // v = p - k^2 D_eo o ; alpha = rho / <r0, v>
    links(w3, US, link_prec_for(sp), nr, 0);
    w3.in = b.o; w3.out = b.v; w3.y1 = b.p; w3.c1 = 1.0; w3.a = -kk; w3.zin = b.r0;
    w3.red = 2; w3.fin = FIN_BICG_ALPHA; w3.run_if = S_RUNNING;
    if (ta != 0.0) {  // v = A p - k^2 D_eo o
      w3.y1 = nullptr; w3.c1 = 0.0; w3.y2 = b.p; w3.c2 = 1.0;
      tw_a(w3);
    }
    Work w4 = base();  // s = r - alpha v
    w4.in = b.r; w4.out = b.s; w4.y1 = b.v; w4.run_if = S_RUNNING;
    Work w5 = w2;      // o = D_oe s
    w5.in = b.s;
    Work w6 = base();  // t = s - k^2 D_eo o ; omega = <t, s> / <t, t>
    links(w6, US, link_prec_for(sp), nr, 0);
    w6.in = b.o; w6.out = b.t; w6.y1 = b.s; w6.c1 = 1.0; w6.a = -kk;
    w6.red = 3; w6.fin = FIN_BICG_OMEGA; w6.run_if = S_RUNNING;
    if (ta != 0.0) {  // t = A s - k^2 D_eo o; y1 = s stays (weight 0) for <t, s>
      w6.c1 = 0.0; w6.y2 = b.s; w6.c2 = 1.0;
      tw_a(w6);
    }
    Work w7 = base();  // x += alpha p + omega s ; r = s - omega t ; rho_new, |r|^2
    w7.in = b.s; w7.y1 = b.t; w7.zin = b.p; w7.z = b.xs; w7.out = b.r; w7.y2 = b.r0;
    w7.red = 4; w7.fin = FIN_BICG_RES; w7.run_if = S_RUNNING;
    const int chunk = 8;
    for (;;) {
      for (int it = 0; it < chunk && err == cudaSuccess; ++it) {
        err = blas(sp, B_BICG_P, w1);
        if (err == cudaSuccess) err = dsl(sp, w2, false);
        if (err == cudaSuccess) err = dsl(sp, w3, false);
        if (err == cudaSuccess) err = blas(sp, B_BICG_S, w4);
        if (err == cudaSuccess) err = dsl(sp, w5, false);
        if (err == cudaSuccess) err = dsl(sp, w6, false);
        if (err == cudaSuccess) err = blas(sp, B_BICG_X, w7);
      }
      if (err != cudaSuccess) { rc = set_error(LQCD_ECUDA, "iteration: %s", cudaGetErrorString(err)); break; }
      if ((rc = read_sc(hs_)) != LQCD_OK) break;
      if (hs_->state != S_RUNNING) break;
    }
    if (rc != LQCD_OK) break;
    iters += hs_->iter;
    const int inner_state = hs_->state, inner_status = hs_->status;
    // x += sigma * xs (FP64), whatever the inner outcome: the iterate is still a correction
    Work f = base();
    f.in = b.xs; f.out = b.x64; f.a = sigma;
    err = blas(sp, B_FOLD64, f);
    if (err != cudaSuccess) { rc = set_error(LQCD_ECUDA, "fold: %s", cudaGetErrorString(err)); break; }
    if (inner_state == S_FAILED) {
      if (inner_status == ST_NONFINITE) status = LQCD_ENONFINITE;
      else if (inner_status == ST_MAXITER) status = LQCD_ENOCONV;
      else if (hs_->iter == 0) status = LQCD_EBREAKDOWN;  // no progress since the restart
      // a breakdown after progress: restart from the new true residual
    }
  }
  double true_res = -1;
  if (rc == LQCD_OK) {
    // x_o = A^-1 (b_o + kappa D_oe x_e), full FP64 residual, copy out
    err = cudaSuccess;
    if (ta != 0.0) {
      Work tw = base();
      tw.in = b.bo; tw.out = b.t64;
      tw_inv(tw);
      err = blas(tp, B_TWIST, tw);
    }
    Work a = base();
    links(a, U64, tp, 18, 1);
    a.in = b.x64; a.out = b.t64; a.y1 = ta != 0.0 ? b.t64 : b.bo; a.c1 = 1.0; a.a = kappa;
    tw_inv(a);
    Work re = base();
    links(re, U64, tp, 18, 0);
    re.in = b.t64; re.out = b.u64; re.y1 = b.be; re.c1 = 1.0; re.y2 = b.x64; re.c2 = -1.0;
    re.a = kappa; re.red = 1; re.fin = FIN_STORE0;
    tw_a(re);
    Work ro = base();
    links(ro, U64, tp, 18, 1);
    ro.in = b.x64; ro.out = b.bhat; ro.y1 = b.bo; ro.c1 = 1.0; ro.y2 = b.t64; ro.c2 = -1.0;
    ro.a = kappa; ro.red = 1; ro.fin = FIN_STORE1;
    tw_a(ro);
    if (err == cudaSuccess) err = dsl(tp, a, false);
    if (err == cudaSuccess) err = dsl(tp, re, false);
    if (err == cudaSuccess) err = dsl(tp, ro, false);
    if (err == cudaSuccess) err = spinor_convert(b.x64, tp, x->half[0], x->prec, Vh, 1.0, st);
    if (err == cudaSuccess) err = spinor_convert(b.t64, tp, x->half[1], x->prec, Vh, 1.0, st);
    if (err != cudaSuccess) rc = set_error(LQCD_ECUDA, "reconstruction: %s", cudaGetErrorString(err));
    else if ((rc = read_sc(hs_)) == LQCD_OK)
      true_res = bnorm2 > 0 ? std::sqrt((hs_->res[0] + hs_->res[1]) / bnorm2) : 0.0;
    if (rc == LQCD_OK && status == LQCD_OK && !(true_res <= tol)) status = LQCD_ENOCONV;
  }
  cudaStreamSynchronize(st);
  if (info) {
    info->status = rc != LQCD_OK ? rc : status;
    info->iters = iters;
    info->reliable_updates = outer;
    info->true_resid = true_res;
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc != LQCD_OK ? rc : status;
}
