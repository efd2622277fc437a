// Launch autotuner of the batched Dslash: for a given set of gauge fields (one slot
// each, as in a multi-RHS or multi-lattice launch) it times every distinct persistent
// grid (CTAs per SM from 1 to the occupancy limit) of every compiled kernel form and
// keeps the fastest in a table keyed by (spinor precision, link reals,
// floor(log2(tiles))). Every later Dslash launch whose key matches takes the tuned
// choice; the table can be saved to and loaded from a text file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {
namespace {

struct Entry {
  int ntiles = 0, ctas_per_sm = 0, form = 0, candidates = 0;
  double us_best = 0, us_default = 0;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int>, Entry> g_table;  // (prec, nr, bucket)

int bucket_of(int ntiles) {
  int b = 0;
  while (b < 30 && (ntiles >> (b + 1)) > 0) ++b;
  return b;
}

std::string device_tag() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string n = p.name;
  for (char& ch : n)
    if (ch == ' ') ch = '_';
  return n + "_sm" + std::to_string(p.multiProcessorCount);
}

}  // namespace

TuneChoice tune_choice(int sp, int nr, int ntiles) {
  TuneChoice c{0, dslash_colour_split(sp) ? 1 : 0};
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find({sp, nr, bucket_of(ntiles)});
  if (it != g_table.end()) {
    c.ctas_per_sm = it->second.ctas_per_sm;
    c.form = it->second.form;
  }
  return c;
}

}  // namespace lqcd

using namespace lqcd;

static void fill_result(lqcd_tune_result* r, int prec, int nr, const Entry& e) {
  r->prec = prec;
  r->nr = nr;
  r->ntiles = e.ntiles;
  r->ctas_per_sm = e.ctas_per_sm;
  r->form = e.form;
  r->candidates = e.candidates;
  r->us_best = e.us_best;
  r->us_default = e.us_default;
}

extern "C" {

int lqcd_autotune_dslash(int n, const lqcd_gauge* const* g, int prec, int compress, lqcd_tune_result* out) {
  clear_error();
  if (n < 1 || n > MAX_SLOTS || !g || !g[0]) return set_error(LQCD_EINVAL, "bad gauge list (n = %d)", n);
  if (prec < LQCD_F64 || prec > LQCD_DF64) return set_error(LQCD_EINVAL, "precision %d", prec);
  if (compress != 0 && compress != 12 && compress != 18) return set_error(LQCD_EINVAL, "compress %d", compress);
  lqcd_ctx* c = g[0]->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  int nr = -1;
  std::vector<Work> w(n);
  std::vector<int> prefix(n + 1, 0);
  std::vector<size_t> off(n + 1, 0);
  bool same_vh = true;
  for (int i = 0; i < n; ++i) {
    if (!g[i] || g[i]->ctx != c) return set_error(LQCD_EINVAL, "gauge %d: NULL or another context", i);
    const void* base;
    int nri;
    int rc;
    if (compress == 0) {
      rc = gauge_links(g[i], prec, &base, &nri);
    } else {
      const int lp = link_prec_for(prec);
      nri = (lp == P_DF64) ? 18 : compress;
      rc = lqcd_gauge_add_copy(const_cast<lqcd_gauge*>(g[i]), prec, nri);
      base = g[i]->copy[lp][nri == 12];
    }
    if (rc != LQCD_OK) return rc;
    if (nr < 0) nr = nri;
    if (nri != nr) return set_error(LQCD_EINVAL, "gauge list mixes 12- and 18-real links");
    const int Vh = g[i]->g.Vh;
    Work& x = w[i];
    x = blank_work(g[i]->g);
    x.out_par = 0;
    x.Uout = parity_links(base, link_prec_for(prec), nr, Vh, 0);
    x.Uin = parity_links(base, link_prec_for(prec), nr, Vh, 1);
    x.a = 1.0;
    x.sc = c->scratch_sc;
    x.tile0 = prefix[i];
    prefix[i + 1] = prefix[i] + x.ntiles;
    off[i + 1] = off[i] + 2 * ((half_spinor_bytes(prec, Vh) + 255) & ~(size_t)255);
    same_vh = same_vh && Vh == g[0]->g.Vh;
  }
  const int ntiles = prefix[n];
  // scratch spinors (in: odd half, out: even half per slot) and the work list
  char* buf = nullptr;
  Work* d_works = nullptr;
  int* d_prefix = nullptr;
  cudaError_t err = cudaMalloc(&buf, off[n]);
  if (err == cudaSuccess) err = cudaMemsetAsync(buf, 0, off[n], st);
  for (int i = 0; i < n; ++i) {
    const size_t hb = (off[i + 1] - off[i]) / 2;
    w[i].in = buf + off[i];
    w[i].out = buf + off[i] + hb;
  }
  if (err == cudaSuccess && n > 1) err = cudaMalloc(&d_works, sizeof(Work) * n);
  if (err == cudaSuccess && n > 1) err = cudaMalloc(&d_prefix, sizeof(int) * (n + 1));
  if (err == cudaSuccess && n > 1)
    err = cudaMemcpyAsync(d_works, w.data(), sizeof(Work) * n, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess && n > 1)
    err = cudaMemcpyAsync(d_prefix, prefix.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
  Launch L;
  memset(&L, 0, sizeof L);
  if (n == 1) {
    L.inline_work = w[0];
  } else {
    L.works = d_works;
    L.tile_prefix = d_prefix;
  }
  L.nslots = n;
  L.ntiles = ntiles;
  L.interleave = (same_vh && n > 1) ? 1 : 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const int nsm = device_sm_count();
  const int def_form = dslash_colour_split(prec) ? 1 : 0;
  // time `reps` launches of one configuration: best average of three trials (us)
  auto time_cfg = [&](int grid, int form, double* us) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_dslash(prec, nr, false, EPI_LIN, L, grid, st, form);
    if (e != cudaSuccess) return e;
    int reps = 5;
    double best = 1e30;
    for (int trial = 0; trial < 3; ++trial) {
      e = cudaEventRecord(e0, st);
      for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch_dslash(prec, nr, false, EPI_LIN, L, grid, st, form);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return e;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = 1e3 * ms / reps;
      best = std::min(best, per);
      if (trial == 0) reps = std::max(5, std::min(100, (int)(2000.0 / std::max(per, 1.0))));  // ~2 ms a trial
    }
    *us = best;
    return cudaSuccess;
  };
  Entry ent;
  ent.ntiles = ntiles;
  double best_us = 1e30, def_us = 0;
  int best_cps = 0, best_form = def_form;
  for (int form = 0; form < 2 && err == cudaSuccess; ++form) {
    const int occ = dslash_occupancy(prec, nr, form);
    if (occ < 1) continue;
    int last_grid = -1;
    for (int cps = 1; cps <= occ && err == cudaSuccess; ++cps) {
      const int grid = std::max(1, std::min(nsm * cps, ntiles));
      if (grid == last_grid) continue;  // small launches: the same grid again
      last_grid = grid;
      double us = 0;
      err = time_cfg(grid, form, &us);
      if (err != cudaSuccess) break;
      ++ent.candidates;
      if (form == def_form && (cps == occ || grid == ntiles)) def_us = us;
      if (us < best_us) {
        best_us = us;
        best_cps = (cps == occ || grid == ntiles) ? 0 : cps;
        best_form = form;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (d_works) cudaFree(d_works);
  if (d_prefix) cudaFree(d_prefix);
  if (err != cudaSuccess) return set_error(LQCD_ECUDA, "autotune: %s", cudaGetErrorString(err));
  // keep the default unless the best is more than 2% faster (timing noise)
  if (def_us > 0 && def_us <= 1.02 * best_us) {
    best_cps = 0;
    best_form = def_form;
    best_us = def_us;
  }
  ent.ctas_per_sm = best_cps;
  ent.form = best_form;
  ent.us_best = best_us;
  ent.us_default = def_us;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[{prec, nr, bucket_of(ntiles)}] = ent;
  }
  if (out) fill_result(out, prec, nr, ent);
  return LQCD_OK;
}

int lqcd_tune_entries(lqcd_tune_result* out, int max, int* n) {
  clear_error();
  if (!n || (max > 0 && !out)) return set_error(LQCD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  int k = 0;
  for (auto& kv : g_table) {
    if (k >= max) break;
    fill_result(out + k, std::get<0>(kv.first), std::get<1>(kv.first), kv.second);
    ++k;
  }
  *n = (int)g_table.size();
  return LQCD_OK;
}

void lqcd_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
}

int lqcd_tune_save(const char* path) {
  clear_error();
  if (!path) return set_error(LQCD_EINVAL, "NULL path");
  FILE* f = fopen(path, "w");
  if (!f) return set_error(LQCD_EINVAL, "cannot write %s", path);
  std::lock_guard<std::mutex> lk(g_mu);
  fprintf(f, "lqcd-tune 1 %s\n", device_tag().c_str());
  for (auto& kv : g_table) {
    const Entry& e = kv.second;
    fprintf(f, "dslash %d %d %d %d %d %d %d %.3f %.3f\n", std::get<0>(kv.first), std::get<1>(kv.first),
            std::get<2>(kv.first), e.ntiles, e.ctas_per_sm, e.form, e.candidates, e.us_best, e.us_default);
  }
  const bool ok = fclose(f) == 0;
  return ok ? LQCD_OK : set_error(LQCD_EINVAL, "write error on %s", path);
}

int lqcd_tune_load(const char* path) {
  clear_error();
  if (!path) return set_error(LQCD_EINVAL, "NULL path");
  FILE* f = fopen(path, "r");
  if (!f) return set_error(LQCD_EINVAL, "cannot read %s", path);
  char tag[256] = {0};
  int ver = 0;
  if (fscanf(f, "lqcd-tune %d %255s", &ver, tag) != 2 || ver != 1) {
    fclose(f);
    return set_error(LQCD_EINVAL, "%s: not a tune file", path);
  }
  if (device_tag() != tag) {
    fclose(f);
    return set_error(LQCD_EINVAL, "%s was tuned on %s, this device is %s", path, tag, device_tag().c_str());
  }
  std::map<std::tuple<int, int, int>, Entry> add;
  int prec, nr, b;
  Entry e;
  while (fscanf(f, " dslash %d %d %d %d %d %d %d %lf %lf", &prec, &nr, &b, &e.ntiles, &e.ctas_per_sm,
                &e.form, &e.candidates, &e.us_best, &e.us_default) == 9) {
    const bool valid = prec >= LQCD_F64 && prec <= LQCD_DF64 && (nr == 12 || nr == 18) && b >= 0 && b <= 30 &&
                       e.ctas_per_sm >= 0 && e.ctas_per_sm <= 64 && (e.form == 0 || e.form == 1) &&
                       dslash_occupancy(prec, nr, e.form) > 0;
    if (!valid) {
      fclose(f);
      return set_error(LQCD_EINVAL, "%s: bad entry", path);
    }
    add[{prec, nr, b}] = e;
  }
  const bool at_end = feof(f) != 0;
  fclose(f);
  if (!at_end) return set_error(LQCD_EINVAL, "%s: unreadable line", path);
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : add) g_table[kv.first] = kv.second;
  return LQCD_OK;
}

}  // extern "C"
