// Host-side objects behind the C ABI handles.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdarg>
#include <string>

#include "lqcd.h"
#include "launch.h"

struct lqcd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;      // stream all work is issued on
  cudaStream_t own_stream = nullptr;  // created by the context
  double* partials = nullptr;         // reduction partials of one-off launches
  size_t partials_cap = 0;            // in doubles
  lqcd::Scalars* scratch_sc = nullptr;  // scalar blocks for one-off reductions
  lqcd::Scalars* host_sc = nullptr;     // pinned mirror
  void* tmp = nullptr;                // operator temporaries (odd half fields)
  size_t tmp_bytes = 0;
  double* staging = nullptr;          // host-layout FP64 staging on the device
  size_t staging_bytes = 0;
  void* work = nullptr;               // solver vectors of the one-shot BiCGStab
  size_t work_bytes = 0;
  long long launches = 0;
  // engine reused by the one-shot solves (lqcd_solve*, the HMC driver) while their options
  // match; it holds no reference to the context and is destroyed with it
  struct lqcd_engine* engine_cache = nullptr;
  lqcd_solve_opts engine_opts{};
  // The context handle and every gauge, field and engine made from it hold one
  // reference; lqcd_ctx_destroy drops the handle's and the context is freed
  // when the last object goes, so objects may outlive the handle.
  std::atomic<int> refs{1};
};

struct lqcd_gauge {
  lqcd_ctx* ctx = nullptr;
  lqcd::Geom g{};
  int prec = 0;
  int compress = 18;
  void* copy[lqcd::NPREC][2] = {};  // [link precision][compress == 12]
  size_t bytes = 0;
};

// HMC momenta / forces: traceless anti-Hermitian 3x3 per link, FP64, in the link layout
// [parity][mu][word][V/2] of double2 (word = row * 3 + column)
struct lqcd_mom {
  lqcd_ctx* ctx = nullptr;
  lqcd::Geom g{};
  double2* d = nullptr;
  size_t bytes = 0;
};

struct lqcd_field {
  lqcd_ctx* ctx = nullptr;
  lqcd::Geom g{};
  int prec = 0;
  int subset = LQCD_FULL;
  void* half[2] = {nullptr, nullptr};
  size_t half_bytes = 0;
};

namespace lqcd {

int set_error(int code, const char* fmt, ...);
void ctx_retain(lqcd_ctx* c);
void ctx_release(lqcd_ctx* c);
void clear_error();

#define LQCD_CK(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ::lqcd::set_error(LQCD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// An NVTX range over a library call, named after the entry point: profilers (Nsight Systems,
// ncu --nvtx) attribute kernels to the call that issued them. Without an attached tool the
// push and pop return at once; the header-only NVTX needs no library at link time.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define LQCD_TRACE(name) ::lqcd::TraceRange lqcd_trace_range_(name)

#define LQCD_TRY(x)                 \
  do {                              \
    int rc_ = (x);                  \
    if (rc_ != LQCD_OK) return rc_; \
  } while (0)

int make_geom(const int dims[4], int t_bc, Geom& g);
size_t half_spinor_bytes(int prec, int Vh);
size_t gauge_copy_bytes(int prec, int nr, int Vh);

// device buffers of the context, grown on demand (synchronises when growing)
int ctx_partials(lqcd_ctx* c, size_t n);
int ctx_tmp(lqcd_ctx* c, size_t bytes);
int ctx_work(lqcd_ctx* c, size_t bytes);
int ctx_staging(lqcd_ctx* c, size_t bytes);

// link copy for fields of precision field_prec (created on first use)
int gauge_links(const lqcd_gauge* g, int field_prec, const void** base, int* nr);
inline const void* parity_links(const void* base, int lp, int nr, int Vh, int par) {
  return static_cast<const char*>(base) + (size_t)par * gauge_copy_bytes(lp, nr, Vh) / 2;
}

// out_p = T(ds, dt) (a D_{p,1-p} in) + c1 y1_p + c2 T(1, yt) y2_p on the context stream,
// T(s, t) = s (1 + i t g5); half fields of precision prec (capi.cu)
int dslash_tw(const lqcd_gauge* gauge, int prec, const void* in, void* out, const void* y1,
              const void* y2, double a, double c1, double c2, int out_par, bool dag, double ds,
              double dt, double yt);

// pure gauge (heatbath.cu): derived link copies rebuilt from the FP64 master; FP64
// link layout -> host AoS layout on the device
int refresh_gauge_copies(lqcd_gauge* g, bool keep_df = false);
// the FP64 master rebuilt from the double-float copy, then the other copies from the master
int links_from_df(lqcd_gauge* g);
cudaError_t links_to_aos(const double2* U, const Geom& g, double2* aos, cudaStream_t s);

// the context's cached engine for options o and at least n slots (engine.cu)
int ctx_engine(lqcd_ctx* c, const lqcd_solve_opts& o, int n, lqcd_engine** out);
void ctx_drop_engine(lqcd_ctx* c);
// after a one-shot solve: free pooled slot blocks beyond keep_bytes
void engine_trim_pool(lqcd_engine* e, size_t keep_bytes);

// a normal-equation request of the engine starting from x0 (FP64, even half used; engine.cu)
int engine_submit_normal_guess(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* src,
                               const lqcd_field* x0, double kappa, double mu, double tol, long long* id);

// BiCGStab on Mhat (bicgstab.cu)
int bicgstab_solve(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                   const lqcd_solve_opts* opts, lqcd_field* x, lqcd_solve_info* info);

// a single-slot launch description
Launch single_launch(const Work& w, double* partials);
Work blank_work(const Geom& g);
// Twisted-mass factors of a Work: the hopping term times ds (1 + i dt g5), the operand
// vector (y2 of the linear epilogue, y1 of the CG step) times (1 + i yt g5).
inline void set_twist(Work& w, double ds, double dt, double yt) {
  w.twist = 1;
  w.tw_s = ds;
  w.tw_t = dt;
  w.ty_t = yt;
}

}  // namespace lqcd

static_assert(LQCD_DF64 == lqcd::P_DF64 && LQCD_BF16 == lqcd::P_BF16 && LQCD_F16 == lqcd::P_F16 &&
                  LQCD_F32 == lqcd::P_F32 && LQCD_F64 == lqcd::P_F64 && lqcd::NPREC == LQCD_DF64 + 1,
              "public precision codes index the per-precision tables");
