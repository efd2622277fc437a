// C ABI: contexts, gauge and spinor fields, and the Wilson-Dirac operators.
#include <cstdio>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

int make_geom(const int dims[4], int t_bc, Geom& g) {
  if (!dims) return set_error(LQCD_EINVAL, "dims is NULL");
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || (dims[mu] & 1))
      return set_error(LQCD_EINVAL, "extent %d of direction %d must be even and >= 2", dims[mu], mu);
    g.L[mu] = dims[mu];
    V *= dims[mu];
  }
  if (V / 2 >= (1LL << 31) / 24) return set_error(LQCD_EINVAL, "lattice too large (V = %lld)", V);
  if (t_bc != 1 && t_bc != -1) return set_error(LQCD_EINVAL, "t_bc must be +1 or -1");
  g.Lxh = dims[0] / 2;
  g.Vh = (int)(V / 2);
  g.t_bc = t_bc;
  const int radix[3] = {g.Lxh, g.L[1], g.L[2]};
  for (int k = 0; k < 3; ++k) {
    geom_set_divisor(g, k, (unsigned)radix[k]);
    // the method is exact for every 32-bit numerator; check the ends of the used range
    const unsigned d = (unsigned)radix[k];
    for (unsigned n : {0u, 1u, d - 1, d, d + 1, (unsigned)g.Vh - 1, (unsigned)g.Vh, 0x7fffffffu}) {
      const unsigned q = geom_div(g, k, n);
      if (q != n / d) return set_error(LQCD_EINVAL, "division constants for %u failed at %u", d, n);
    }
  }
  return LQCD_OK;
}

size_t half_spinor_bytes(int prec, int Vh) { return (size_t)24 * prec_bytes(prec) * Vh; }
size_t gauge_copy_bytes(int prec, int nr, int Vh) { return (size_t)2 * 4 * nr * prec_bytes(prec) * Vh; }

int ctx_partials(lqcd_ctx* c, size_t n) {
  if (c->partials_cap >= n) return LQCD_OK;
  LQCD_CK(cudaStreamSynchronize(c->stream));
  if (c->partials) cudaFree(c->partials);
  c->partials = nullptr;
  c->partials_cap = 0;
  LQCD_CK(cudaMalloc(&c->partials, n * sizeof(double)));
  c->partials_cap = n;
  return LQCD_OK;
}

int ctx_tmp(lqcd_ctx* c, size_t bytes) {
  if (c->tmp_bytes >= bytes) return LQCD_OK;
  LQCD_CK(cudaStreamSynchronize(c->stream));
  if (c->tmp) cudaFree(c->tmp);
  c->tmp = nullptr;
  c->tmp_bytes = 0;
  LQCD_CK(cudaMalloc(&c->tmp, bytes));
  c->tmp_bytes = bytes;
  return LQCD_OK;
}

int ctx_work(lqcd_ctx* c, size_t bytes) {
  if (c->work_bytes >= bytes) return LQCD_OK;
  LQCD_CK(cudaStreamSynchronize(c->stream));
  if (c->work) cudaFree(c->work);
  c->work = nullptr;
  c->work_bytes = 0;
  LQCD_CK(cudaMalloc(&c->work, bytes));
  c->work_bytes = bytes;
  return LQCD_OK;
}

int ctx_staging(lqcd_ctx* c, size_t bytes) {
  if (c->staging_bytes >= bytes) return LQCD_OK;
  LQCD_CK(cudaStreamSynchronize(c->stream));
  if (c->staging) cudaFree(c->staging);
  c->staging = nullptr;
  c->staging_bytes = 0;
  LQCD_CK(cudaMalloc(&c->staging, bytes));
  c->staging_bytes = bytes;
  return LQCD_OK;
}

int gauge_links(const lqcd_gauge* gc, int field_prec, const void** base, int* nr) {
  lqcd_gauge* g = const_cast<lqcd_gauge*>(gc);
  const int lp = link_prec_for(field_prec);
  if (lp < 0 || lp >= NPREC) return set_error(LQCD_EINVAL, "link precision %d", lp);
  const int n = (lp == P_DF64) ? 18 : g->compress;  // double-float links keep 18 reals
  void*& slot = g->copy[lp][n == 12];
  if (!slot) {
    size_t b = gauge_copy_bytes(lp, n, g->g.Vh);
    LQCD_CK(cudaMalloc(&slot, b));
    g->bytes += b;
    LQCD_CK(gauge_convert(g->copy[P_F64][0], g->g, lp, n, slot, g->ctx->stream));
  }
  *base = slot;
  *nr = n;
  return LQCD_OK;
}

Work blank_work(const Geom& g) {
  Work w;
  memset(&w, 0, sizeof w);
  w.g = g;
  w.run_if = -1;
  w.fin = FIN_NONE;
  w.ntiles = (g.Vh + TILE - 1) / TILE;
  w.tw_s = 1.0;
  return w;
}

Launch single_launch(const Work& w, double* partials) {
  Launch L;
  memset(&L, 0, sizeof L);
  L.works = nullptr;
  L.inline_work = w;
  L.nslots = 1;
  L.ntiles = w.ntiles;
  L.partials = partials;
  L.finish = (partials && (w.red || w.fin != FIN_NONE)) ? 1 : 0;
  return L;
}

}  // namespace lqcd

using namespace lqcd;

static int ctx_set_device(lqcd_ctx* c) {
  LQCD_CK(cudaSetDevice(c->device));
  return LQCD_OK;
}

extern "C" {

const char* lqcd_status_string(int s) {
  switch (s) {
    case LQCD_OK: return "ok";
    case LQCD_EINVAL: return "invalid argument";
    case LQCD_ENOMEM: return "out of device memory / over budget";
    case LQCD_ENOCONV: return "not converged (maxiter)";
    case LQCD_EBREAKDOWN: return "Krylov breakdown";
    case LQCD_ENONFINITE: return "non-finite residual";
    case LQCD_ETIMEOUT: return "timeout";
    case LQCD_ECUDA: return "CUDA error";
    case LQCD_EBUSY: return "engine busy";
  }
  return "unknown status";
}

const char* lqcd_last_error(void) { return g_err.c_str(); }
const char* lqcd_version(void) { return "lqcd-gb300 0.1 (sm_103a)"; }

int lqcd_ctx_create(lqcd_ctx** out, int device, void* stream) {
  clear_error();
  if (!out) return set_error(LQCD_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  LQCD_CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return set_error(LQCD_EINVAL, "device %d of %d", device, n);
  lqcd_ctx* c = new lqcd_ctx();
  c->device = device;
  int rc = ctx_set_device(c);
  if (rc == LQCD_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = set_error(LQCD_ECUDA, "stream: %s", cudaGetErrorString(e));
  }
  if (rc == LQCD_OK) {
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    cudaError_t e = cudaMalloc(&c->scratch_sc, 16 * sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMemset(c->scratch_sc, 0, 16 * sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_sc, 16 * sizeof(Scalars));
    if (e != cudaSuccess) rc = set_error(LQCD_ECUDA, "scratch: %s", cudaGetErrorString(e));
  }
  if (rc != LQCD_OK) {
    lqcd_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return LQCD_OK;
}

void lqcd_ctx_destroy(lqcd_ctx* c) {
  if (!c) return;
  ctx_release(c);
}

}  // extern "C"

namespace lqcd {

void ctx_retain(lqcd_ctx* c) { c->refs.fetch_add(1); }

void ctx_release(lqcd_ctx* c) {
  if (c->refs.fetch_sub(1) != 1) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  ctx_drop_engine(c);
  if (c->partials) cudaFree(c->partials);
  if (c->scratch_sc) cudaFree(c->scratch_sc);
  if (c->host_sc) cudaFreeHost(c->host_sc);
  if (c->tmp) cudaFree(c->tmp);
  if (c->staging) cudaFree(c->staging);
  if (c->work) cudaFree(c->work);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

}  // namespace lqcd

extern "C" {

int lqcd_ctx_set_stream(lqcd_ctx* c, void* stream) {
  clear_error();
  if (!c) return set_error(LQCD_EINVAL, "ctx is NULL");
  LQCD_TRY(ctx_set_device(c));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return LQCD_OK;
}

void* lqcd_ctx_stream(const lqcd_ctx* c) { return c ? (void*)c->stream : nullptr; }

int lqcd_ctx_sync(lqcd_ctx* c) {
  clear_error();
  if (!c) return set_error(LQCD_EINVAL, "ctx is NULL");
  LQCD_TRY(ctx_set_device(c));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

long long lqcd_ctx_launch_count(const lqcd_ctx* c) { return c ? c->launches : 0; }

int lqcd_debug_bounds(lqcd_ctx* c, unsigned long long* word) {
  clear_error();
  if (!c || !word) return set_error(LQCD_EINVAL, "NULL argument");
  *word = 0;
#ifdef LQCD_DEBUG_BOUNDS
  LQCD_TRY(ctx_set_device(c));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  for (auto read : bounds_word_readers()) {
    unsigned long long v = 0;
    if (read(&v) != 0) return set_error(LQCD_ECUDA, "reading a bounds-check word failed");
    if (v && !*word) *word = v;
  }
  return LQCD_OK;
#else
  return set_error(LQCD_EINVAL, "the library was built without LQCD_DEBUG_BOUNDS");
#endif
}

int lqcd_ctx_release_cache(lqcd_ctx* c) {
  clear_error();
  if (!c) return set_error(LQCD_EINVAL, "NULL context");
  LQCD_CK(cudaSetDevice(c->device));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  ctx_drop_engine(c);
  void** bufs[] = {&c->tmp, &c->work, reinterpret_cast<void**>(&c->staging)};
  size_t* caps[] = {&c->tmp_bytes, &c->work_bytes, &c->staging_bytes};
  for (int i = 0; i < 3; ++i) {
    if (*bufs[i]) cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
    *caps[i] = 0;
  }
  return LQCD_OK;
}

void lqcd_set_grid_multiplier(int family, int mult) { set_grid_multiplier(family, mult); }

int lqcd_set_dslash_form(int prec, int form) {
  clear_error();
  if (prec != LQCD_DF64 || (form != 0 && form != 1))
    return set_error(LQCD_EINVAL, "the Dslash form is selectable for LQCD_DF64 only (0 site, 1 colour split)");
  set_dslash_colour_split(prec, form == 1);
  return LQCD_OK;
}



// ------------------------------------------------------------------ gauge

static int gauge_upload_impl(lqcd_ctx* c, const int dims[4], const double* U, bool dev, int prec,
                             int compress, int t_bc, lqcd_gauge** out) {
  clear_error();
  if (!c || !U || !out) return set_error(LQCD_EINVAL, "NULL argument");
  *out = nullptr;
  if (prec < LQCD_F64 || prec > LQCD_DF64) return set_error(LQCD_EINVAL, "precision %d", prec);
  if (compress != 18 && compress != 12) return set_error(LQCD_EINVAL, "compress must be 18 or 12");
  Geom g;
  LQCD_TRY(make_geom(dims, t_bc, g));
  LQCD_TRY(ctx_set_device(c));
  const size_t aos_bytes = (size_t)2 * g.Vh * 4 * 18 * sizeof(double);
  const double* src = U;
  if (!dev) {
    LQCD_TRY(ctx_staging(c, aos_bytes));
    LQCD_CK(cudaMemcpyAsync(c->staging, U, aos_bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->staging;
  }
  lqcd_gauge* gg = new lqcd_gauge();
  gg->ctx = c;
  ctx_retain(c);
  gg->g = g;
  gg->prec = prec;
  gg->compress = compress;
  const size_t b64 = gauge_copy_bytes(P_F64, 18, g.Vh);
  cudaError_t e = cudaMalloc(&gg->copy[P_F64][0], b64);
  if (e != cudaSuccess) {
    delete gg;
    return set_error(LQCD_ENOMEM, "gauge field: %s", cudaGetErrorString(e));
  }
  gg->bytes = b64;
  e = gauge_from_aos(src, g, P_F64, 18, gg->copy[P_F64][0], c->stream);
  int rc = (e == cudaSuccess) ? LQCD_OK : set_error(LQCD_ECUDA, "gauge layout: %s", cudaGetErrorString(e));
  if (rc == LQCD_OK) {
    const void* base;
    int nr;
    rc = gauge_links(gg, prec, &base, &nr);
  }
  if (rc == LQCD_OK) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = set_error(LQCD_ECUDA, "gauge upload: %s", cudaGetErrorString(e));
  }
  if (rc != LQCD_OK) {
    lqcd_gauge_destroy(gg);
    return rc;
  }
  *out = gg;
  return LQCD_OK;
}

int lqcd_gauge_upload(lqcd_ctx* c, const int dims[4], const double* U, int prec, int compress,
                      int t_bc, lqcd_gauge** out) {
  LQCD_TRACE("lqcd_gauge_upload");
  return gauge_upload_impl(c, dims, U, false, prec, compress, t_bc, out);
}

int lqcd_gauge_upload_dev(lqcd_ctx* c, const int dims[4], const double* U, int prec, int compress,
                          int t_bc, lqcd_gauge** out) {
  LQCD_TRACE("lqcd_gauge_upload_dev");
  return gauge_upload_impl(c, dims, U, true, prec, compress, t_bc, out);
}

int lqcd_gauge_add_copy(lqcd_gauge* g, int prec, int compress) {
  clear_error();
  if (!g) return set_error(LQCD_EINVAL, "gauge is NULL");
  if (prec < LQCD_F64 || prec > LQCD_DF64) return set_error(LQCD_EINVAL, "precision %d", prec);
  if (compress != 18 && compress != 12) return set_error(LQCD_EINVAL, "compress must be 18 or 12");
  LQCD_TRY(ctx_set_device(g->ctx));
  const int lp = link_prec_for(prec);
  if (lp < 0 || lp >= NPREC) return set_error(LQCD_EINVAL, "link precision %d", lp);
  if (lp == P_DF64) compress = 18;  // double-float links keep 18 reals
  void*& slot = g->copy[lp][compress == 12];
  if (slot) return LQCD_OK;
  const size_t b = gauge_copy_bytes(lp, compress, g->g.Vh);
  cudaError_t e = cudaMalloc(&slot, b);
  if (e != cudaSuccess) {
    slot = nullptr;
    return set_error(LQCD_ENOMEM, "gauge copy: %s", cudaGetErrorString(e));
  }
  g->bytes += b;
  LQCD_CK(gauge_convert(g->copy[P_F64][0], g->g, lp, compress, slot, g->ctx->stream));
  return LQCD_OK;
}

size_t lqcd_gauge_bytes(const lqcd_gauge* g) { return g ? g->bytes : 0; }

void lqcd_gauge_destroy(lqcd_gauge* g) {
  if (!g) return;
  cudaSetDevice(g->ctx->device);
  cudaStreamSynchronize(g->ctx->stream);
  for (auto& row : g->copy)
    for (auto& p : row)
      if (p) cudaFree(p);
  lqcd_ctx* c = g->ctx;
  delete g;
  ctx_release(c);
}

// ------------------------------------------------------------------ fields

int lqcd_field_create(lqcd_ctx* c, const int dims[4], int prec, int subset, lqcd_field** out) {
  clear_error();
  if (!c || !out) return set_error(LQCD_EINVAL, "NULL argument");
  *out = nullptr;
  if (prec < LQCD_F64 || prec > LQCD_DF64) return set_error(LQCD_EINVAL, "precision %d", prec);
  if (subset < LQCD_EVEN || subset > LQCD_FULL) return set_error(LQCD_EINVAL, "subset %d", subset);
  Geom g;
  LQCD_TRY(make_geom(dims, -1, g));
  LQCD_TRY(ctx_set_device(c));
  lqcd_field* f = new lqcd_field();
  f->ctx = c;
  ctx_retain(c);
  f->g = g;
  f->prec = prec;
  f->subset = subset;
  f->half_bytes = half_spinor_bytes(prec, g.Vh);
  for (int p = 0; p < 2; ++p) {
    if (subset != LQCD_FULL && subset != p) continue;
    cudaError_t e = cudaMalloc(&f->half[p], f->half_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->half[p], 0, f->half_bytes, c->stream);
    if (e != cudaSuccess) {
      lqcd_field_destroy(f);
      return set_error(LQCD_ENOMEM, "field: %s", cudaGetErrorString(e));
    }
  }
  *out = f;
  return LQCD_OK;
}

size_t lqcd_field_bytes(const lqcd_field* f) {
  return f ? f->half_bytes * ((f->half[0] ? 1 : 0) + (f->half[1] ? 1 : 0)) : 0;
}

void lqcd_field_destroy(lqcd_field* f) {
  if (!f) return;
  cudaSetDevice(f->ctx->device);
  cudaStreamSynchronize(f->ctx->stream);
  for (auto& p : f->half)
    if (p) cudaFree(p);
  lqcd_ctx* c = f->ctx;
  delete f;
  ctx_release(c);
}

static int field_upload_impl(lqcd_field* f, const double* psi, bool dev) {
  clear_error();
  if (!f || !psi) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = f->ctx;
  LQCD_TRY(ctx_set_device(c));
  const size_t bytes = (size_t)2 * f->g.Vh * 24 * sizeof(double);
  const double* src = psi;
  if (!dev) {
    LQCD_TRY(ctx_staging(c, bytes));
    LQCD_CK(cudaMemcpyAsync(c->staging, psi, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->staging;
  }
  LQCD_CK(spinor_from_aos(src, f->g, f->prec, f->half[0], f->half[1], c->stream));
  if (!dev) LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

int lqcd_field_upload(lqcd_field* f, const double* psi) {
  LQCD_TRACE("lqcd_field_upload"); return field_upload_impl(f, psi, false); }
int lqcd_field_upload_dev(lqcd_field* f, const double* psi) {
  LQCD_TRACE("lqcd_field_upload_dev"); return field_upload_impl(f, psi, true); }

int lqcd_field_download_dev(const lqcd_field* f, double* psi) {
  LQCD_TRACE("lqcd_field_download_dev");
  clear_error();
  if (!f || !psi) return set_error(LQCD_EINVAL, "NULL argument");
  LQCD_TRY(ctx_set_device(f->ctx));
  LQCD_CK(spinor_to_aos(f->half[0], f->half[1], f->g, f->prec, psi, f->ctx->stream));
  return LQCD_OK;
}

int lqcd_field_download(const lqcd_field* f, double* psi) {
  LQCD_TRACE("lqcd_field_download");
  clear_error();
  if (!f || !psi) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = f->ctx;
  LQCD_TRY(ctx_set_device(c));
  const size_t V = (size_t)2 * f->g.Vh;
  const size_t bytes = V * 24 * sizeof(double);
  LQCD_TRY(ctx_staging(c, bytes));
  LQCD_CK(spinor_to_aos(f->half[0], f->half[1], f->g, f->prec, c->staging, c->stream));
  if (f->subset == LQCD_FULL) {
    LQCD_CK(cudaMemcpyAsync(psi, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
    LQCD_CK(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
  }
  std::vector<double> tmp(V * 24);
  LQCD_CK(cudaMemcpyAsync(tmp.data(), c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  const int* L = f->g.L;
  for (size_t s = 0; s < V; ++s) {
    size_t r = s;
    const int x = (int)(r % L[0]);
    r /= L[0];
    const int y = (int)(r % L[1]);
    r /= L[1];
    const int z = (int)(r % L[2]);
    const int t = (int)(r / L[2]);
    if (((x + y + z + t) & 1) == f->subset) memcpy(psi + s * 24, tmp.data() + s * 24, 24 * sizeof(double));
  }
  return LQCD_OK;
}

int lqcd_field_copy(lqcd_field* dst, const lqcd_field* src, double scale) {
  clear_error();
  if (!dst || !src) return set_error(LQCD_EINVAL, "NULL argument");
  if (dst->g.Vh != src->g.Vh || memcmp(dst->g.L, src->g.L, sizeof dst->g.L))
    return set_error(LQCD_EINVAL, "lattice mismatch");
  LQCD_TRY(ctx_set_device(dst->ctx));
  int n = 0;
  for (int p = 0; p < 2; ++p) {
    if (!dst->half[p] || !src->half[p]) continue;
    LQCD_CK(spinor_convert(src->half[p], src->prec, dst->half[p], dst->prec, dst->g.Vh, scale,
                           dst->ctx->stream));
    ++n;
  }
  if (!n) return set_error(LQCD_EINVAL, "fields share no parity");
  return LQCD_OK;
}

int lqcd_field_zero(lqcd_field* f) {
  clear_error();
  if (!f) return set_error(LQCD_EINVAL, "field is NULL");
  LQCD_TRY(ctx_set_device(f->ctx));
  for (auto p : f->half)
    if (p) LQCD_CK(cudaMemsetAsync(p, 0, f->half_bytes, f->ctx->stream));
  return LQCD_OK;
}

int lqcd_field_norm2(const lqcd_field* f, double* out) {
  clear_error();
  if (!f || !out) return set_error(LQCD_EINVAL, "NULL argument");
  lqcd_ctx* c = f->ctx;
  LQCD_TRY(ctx_set_device(c));
  Work w = blank_work(f->g);
  LQCD_TRY(ctx_partials(c, 3 * (size_t)w.ntiles));
  double total = 0;
  for (int p = 0; p < 2; ++p) {
    if (!f->half[p]) continue;
    w.in = f->half[p];
    w.red = 1;
    w.fin = FIN_STORE0;
    w.sc = c->scratch_sc;
    Launch L = single_launch(w, c->partials);
    LQCD_CK(launch_blas(f->prec, B_NORM, L, 0, c->stream));
    c->launches++;
    LQCD_CK(cudaMemcpyAsync(c->host_sc, c->scratch_sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                            c->stream));
    LQCD_CK(cudaStreamSynchronize(c->stream));
    total += c->host_sc->res[0];
  }
  *out = total;
  return LQCD_OK;
}

// ------------------------------------------------------------------ operators

static int check_pair(const lqcd_gauge* g, const lqcd_field* a, const lqcd_field* b) {
  if (!g || !a || !b) return set_error(LQCD_EINVAL, "NULL argument");
  if (a->prec != b->prec) return set_error(LQCD_EINVAL, "fields differ in precision");
  if (a->ctx != g->ctx || b->ctx != g->ctx) return set_error(LQCD_EINVAL, "objects of different contexts");
  if (memcmp(a->g.L, g->g.L, sizeof g->g.L) || memcmp(b->g.L, g->g.L, sizeof g->g.L))
    return set_error(LQCD_EINVAL, "lattice mismatch");
  return LQCD_OK;
}

}  // extern "C"

// out_p = T(ds, dt) (a * D_{p,1-p} in) + c1 * y1_p + c2 T(1, yt) y2_p, T(s, t) = s (1 + i t g5)
int lqcd::dslash_tw(const lqcd_gauge* gauge, int prec, const void* in, void* out, const void* y1,
                     const void* y2, double a, double c1, double c2, int out_par, bool dag,
                     double ds, double dt, double yt) {
  lqcd_ctx* c = gauge->ctx;
  const void* base;
  int nr;
  LQCD_TRY(gauge_links(gauge, prec, &base, &nr));
  const int lp = link_prec_for(prec);
  Work w = blank_work(gauge->g);
  w.out_par = out_par;
  w.in = in;
  w.out = out;
  w.Uout = parity_links(base, lp, nr, gauge->g.Vh, out_par);
  w.Uin = parity_links(base, lp, nr, gauge->g.Vh, 1 - out_par);
  w.y1 = y1;
  w.y2 = y2;
  w.a = a;
  w.c1 = c1;
  w.c2 = c2;
  if (dt != 0.0 || ds != 1.0 || yt != 0.0) set_twist(w, ds, dt, yt);
  w.sc = c->scratch_sc;
  Launch L = single_launch(w, c->partials);
  LQCD_CK(launch_dslash(prec, nr, dag, w.twist ? EPI_LIN_TW : EPI_LIN, L, 0, c->stream));
  c->launches++;
  return LQCD_OK;
}

extern "C" {

// out_p = a * D_{p,1-p} in + c1 * y1_p
static int dslash_lin(const lqcd_gauge* gauge, int prec, const void* in, void* out, const void* y1,
                      double a, double c1, int out_par, bool dag) {
  return dslash_tw(gauge, prec, in, out, y1, nullptr, a, c1, 0.0, out_par, dag, 1.0, 0.0, 0.0);
}

int lqcd_dslash_eo(const lqcd_gauge* g, const lqcd_field* in, lqcd_field* out, int out_parity,
                   int dagger) {
  LQCD_TRACE("lqcd_dslash_eo");
  clear_error();
  LQCD_TRY(check_pair(g, in, out));
  if (out_parity != 0 && out_parity != 1) return set_error(LQCD_EINVAL, "parity %d", out_parity);
  if (!in->half[1 - out_parity] || !out->half[out_parity])
    return set_error(LQCD_EINVAL, "fields do not hold the needed parities");
  if (in == out && in->subset == LQCD_FULL) {
    // in and out use different halves of the same field: allowed
  }
  LQCD_TRY(ctx_set_device(g->ctx));
  return dslash_lin(g, in->prec, in->half[1 - out_parity], out->half[out_parity], nullptr, 1.0, 0.0,
                    out_parity, dagger != 0);
}

}  // extern "C"

struct lqcd_dslash_batch {
  lqcd_ctx* ctx = nullptr;
  int prec = 0, nr = 18, dagger = 0, n = 0;
  Launch L{};
  Work* d_works = nullptr;
  int* d_prefix = nullptr;
};

extern "C" {

int lqcd_dslash_batch_create(int n, const lqcd_gauge* const* g, const lqcd_field* const* in,
                             lqcd_field* const* out, int out_parity, int dagger,
                             lqcd_dslash_batch** batch) {
  clear_error();
  if (!batch || !g || !in || !out || n < 1 || n > MAX_SLOTS)
    return set_error(LQCD_EINVAL, "bad batch arguments (n = %d)", n);
  *batch = nullptr;
  if (out_parity != 0 && out_parity != 1) return set_error(LQCD_EINVAL, "parity %d", out_parity);
  lqcd_ctx* c = g[0] ? g[0]->ctx : nullptr;
  if (!c) return set_error(LQCD_EINVAL, "NULL gauge");
  const int prec = in[0] ? in[0]->prec : -1;
  int nr = -1;
  std::vector<Work> w(n);
  std::vector<int> prefix(n + 1, 0);
  bool same_vh = true;
  LQCD_TRY(ctx_set_device(c));
  for (int i = 0; i < n; ++i) {
    LQCD_TRY(check_pair(g[i], in[i], out[i]));
    if (g[i]->ctx != c || in[i]->prec != prec) return set_error(LQCD_EINVAL, "batch mixes contexts or precisions");
    if (!in[i]->half[1 - out_parity] || !out[i]->half[out_parity])
      return set_error(LQCD_EINVAL, "entry %d: fields do not hold the needed parities", i);
    const void* base;
    int nri;
    LQCD_TRY(gauge_links(g[i], prec, &base, &nri));
    if (nr < 0) nr = nri;
    if (nri != nr) return set_error(LQCD_EINVAL, "batch mixes 12- and 18-real links");
    const int lp = link_prec_for(prec);
    Work& x = w[i];
    x = blank_work(g[i]->g);
    x.out_par = out_parity;
    x.in = in[i]->half[1 - out_parity];
    x.out = out[i]->half[out_parity];
    x.Uout = parity_links(base, lp, nr, g[i]->g.Vh, out_parity);
    x.Uin = parity_links(base, lp, nr, g[i]->g.Vh, 1 - out_parity);
    x.a = 1.0;
    x.sc = c->scratch_sc;
    x.tile0 = prefix[i];
    prefix[i + 1] = prefix[i] + x.ntiles;
    same_vh = same_vh && g[i]->g.Vh == g[0]->g.Vh;
  }
  lqcd_dslash_batch* b = new lqcd_dslash_batch();
  b->ctx = c;
  b->prec = prec;
  b->nr = nr;
  b->dagger = dagger != 0;
  b->n = n;
  cudaError_t e = cudaMalloc(&b->d_works, sizeof(Work) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_prefix, sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_works, w.data(), sizeof(Work) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_prefix, prefix.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (b->d_works) cudaFree(b->d_works);
    if (b->d_prefix) cudaFree(b->d_prefix);
    delete b;
    return set_error(LQCD_ENOMEM, "dslash batch: %s", cudaGetErrorString(e));
  }
  memset(&b->L, 0, sizeof b->L);
  b->L.works = b->d_works;
  b->L.tile_prefix = b->d_prefix;
  b->L.nslots = n;
  b->L.ntiles = prefix[n];
  b->L.interleave = (same_vh && n > 1) ? 1 : 0;
  b->L.partials = nullptr;  // no reduction
  if (n == 1) {
    b->L.works = nullptr;
    b->L.inline_work = w[0];
  }
  ctx_retain(c);
  *batch = b;
  return LQCD_OK;
}

int lqcd_dslash_batch_apply(lqcd_dslash_batch* b) {
  LQCD_TRACE("lqcd_dslash_batch_apply");
  clear_error();
  if (!b) return set_error(LQCD_EINVAL, "batch is NULL");
  LQCD_TRY(ctx_set_device(b->ctx));
  LQCD_CK(launch_dslash(b->prec, b->nr, b->dagger != 0, EPI_LIN, b->L, 0, b->ctx->stream));
  b->ctx->launches++;
  return LQCD_OK;
}

void lqcd_dslash_batch_destroy(lqcd_dslash_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  cudaStreamSynchronize(b->ctx->stream);
  cudaFree(b->d_works);
  cudaFree(b->d_prefix);
  lqcd_ctx* c = b->ctx;
  delete b;
  ctx_release(c);
}

int lqcd_apply_Mhat(const lqcd_gauge* g, double kappa, const lqcd_field* in, lqcd_field* out,
                    int dagger) {
  return lqcd_apply_Mhat_tm(g, kappa, 0.0, in, out, dagger);
}

int lqcd_apply_M(const lqcd_gauge* g, double kappa, const lqcd_field* in, lqcd_field* out,
                 int dagger) {
  return lqcd_apply_M_tm(g, kappa, 0.0, in, out, dagger);
}

int lqcd_apply_Mhat_tm(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* in,
                       lqcd_field* out, int dagger) {
  LQCD_TRACE("lqcd_apply_Mhat_tm");
  clear_error();
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return set_error(LQCD_EINVAL, "kappa and mu must be finite");
  LQCD_TRY(check_pair(g, in, out));
  if (!in->half[0] || !out->half[0]) return set_error(LQCD_EINVAL, "fields must hold the even parity");
  if (in->half[0] == out->half[0]) return set_error(LQCD_EINVAL, "in and out must differ");
  lqcd_ctx* c = g->ctx;
  LQCD_TRY(ctx_set_device(c));
  LQCD_TRY(ctx_tmp(c, half_spinor_bytes(in->prec, g->g.Vh)));
  if (mu == 0.0) {
    LQCD_TRY(dslash_lin(g, in->prec, in->half[0], c->tmp, nullptr, 1.0, 0.0, 1, dagger != 0));
    return dslash_lin(g, in->prec, c->tmp, out->half[0], in->half[0], -kappa * kappa, 1.0, 0,
                      dagger != 0);
  }
  // tmp = A^-1 D_oe in (A^-dag D^dag_oe), out = A in - k^2 D_eo tmp (A^dag, D^dag)
  const double a = (dagger ? -2.0 : 2.0) * kappa * mu;
  LQCD_TRY(dslash_tw(g, in->prec, in->half[0], c->tmp, nullptr, nullptr, 1.0, 0.0, 0.0, 1,
                     dagger != 0, 1.0 / (1.0 + a * a), -a, 0.0));
  return dslash_tw(g, in->prec, c->tmp, out->half[0], nullptr, in->half[0], -kappa * kappa, 0.0, 1.0,
                   0, dagger != 0, 1.0, 0.0, a);
}

int lqcd_apply_M_tm(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* in,
                    lqcd_field* out, int dagger) {
  LQCD_TRACE("lqcd_apply_M_tm");
  clear_error();
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return set_error(LQCD_EINVAL, "kappa and mu must be finite");
  LQCD_TRY(check_pair(g, in, out));
  if (in->subset != LQCD_FULL || out->subset != LQCD_FULL)
    return set_error(LQCD_EINVAL, "apply_M needs FULL fields");
  if (in == out) return set_error(LQCD_EINVAL, "in and out must differ");
  LQCD_TRY(ctx_set_device(g->ctx));
  const double a = (dagger ? -2.0 : 2.0) * kappa * mu;  // A (A^dag)
  for (int p = 0; p < 2; ++p) {
    if (mu == 0.0)
      LQCD_TRY(dslash_lin(g, in->prec, in->half[1 - p], out->half[p], in->half[p], -kappa, 1.0, p,
                          dagger != 0));
    else
      LQCD_TRY(dslash_tw(g, in->prec, in->half[1 - p], out->half[p], nullptr, in->half[p], -kappa,
                         0.0, 1.0, p, dagger != 0, 1.0, 0.0, a));
  }
  return LQCD_OK;
}

}  // extern "C"
