// Launch autotuner of the batched Dslash. For a given set of gauge fields (one slot
// each, as in a multi-RHS or multi-lattice launch) it times every distinct persistent
// grid (CTAs per SM from 1 to the occupancy limit) of every compiled kernel form (one
// thread per site at the default register budget; colour split for double-float; one
// thread per site at 8 CTAs per SM, 128 registers, for FP32) and keeps the fastest in a
// table keyed by (spinor precision, link reals, floor(log2(tiles))).
// When every slot is on the same gauge field (n right-hand sides), it also times the
// shared-link form, which loads each site block's links once for a group of slots, for
// several group sizes and grids, against the slots loading their own links, and keeps the
// better under the key (precision, link reals, n, floor(log2(site blocks))). Every later
// launch whose key matches takes the tuned choice; the table can be saved to and loaded
// from a JSON file tagged with the device name and SM count.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
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
  int ntiles = 0, ctas_per_sm = 0, form = 0, group = 0, candidates = 0;
  double us_best = 0, us_default = 0;
};

// (prec, nr, nrhs, bucket): nrhs 0 for the launch-shape entries of every Dslash launch,
// nrhs >= 2 for the shared-link choice of n slots on one gauge field (bucket of site blocks)
using Key = std::tuple<int, int, int, int>;
std::mutex g_mu;
std::map<Key, Entry> g_table;

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

bool shared_link_prec(int p) { return p == P_F32 || p == P_F16 || p == P_BF16; }

// ------------------------------------------------------------------ a small JSON reader
// Enough of JSON for the table file: objects, arrays, strings without escapes other than
// \" and \\, numbers, true, false, null. Values are kept as text (numbers) or nested.
struct JVal {
  enum T { NUL, NUM, STR, ARR, OBJ, BOOL } t = NUL;
  double num = 0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal* get(const char* k) const {
    for (auto& kv : obj)
      if (kv.first == k) return &kv.second;
    return nullptr;
  }
};

struct JParser {
  const char* p;
  const char* end;
  bool ok = true;
  void ws() {
    while (p < end && std::isspace((unsigned char)*p)) ++p;
  }
  bool lit(const char* s) {
    const size_t n = strlen(s);
    if ((size_t)(end - p) >= n && !strncmp(p, s, n)) {
      p += n;
      return true;
    }
    return false;
  }
  bool string(std::string& out) {
    if (p >= end || *p != '"') return false;
    ++p;
    while (p < end && *p != '"') {
      if (*p == '\\') {
        ++p;
        if (p >= end || (*p != '"' && *p != '\\')) return false;
      }
      out.push_back(*p++);
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool value(JVal& v, int depth) {
    if (depth > 8) return false;
    ws();
    if (p >= end) return false;
    if (*p == '{') {
      ++p;
      v.t = JVal::OBJ;
      ws();
      if (p < end && *p == '}') {
        ++p;
        return true;
      }
      for (;;) {
        ws();
        std::string k;
        if (!string(k)) return false;
        ws();
        if (p >= end || *p != ':') return false;
        ++p;
        JVal x;
        if (!value(x, depth + 1)) return false;
        v.obj.emplace_back(k, std::move(x));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == '}') {
          ++p;
          return true;
        }
        return false;
      }
    }
    if (*p == '[') {
      ++p;
      v.t = JVal::ARR;
      ws();
      if (p < end && *p == ']') {
        ++p;
        return true;
      }
      for (;;) {
        JVal x;
        if (!value(x, depth + 1)) return false;
        v.arr.push_back(std::move(x));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == ']') {
          ++p;
          return true;
        }
        return false;
      }
    }
    if (*p == '"') {
      v.t = JVal::STR;
      return string(v.str);
    }
    if (lit("true") || lit("false")) {
      v.t = JVal::BOOL;
      return true;
    }
    if (lit("null")) return true;
    char* q = nullptr;
    v.num = strtod(p, &q);
    if (q == p || q > end) return false;
    p = q;
    v.t = JVal::NUM;
    return true;
  }
};

bool get_int(const JVal& o, const char* k, int& out) {
  const JVal* v = o.get(k);
  if (!v || v->t != JVal::NUM || v->num != std::floor(v->num) || std::fabs(v->num) > 1e9) return false;
  out = (int)v->num;
  return true;
}
bool get_num(const JVal& o, const char* k, double& out) {
  const JVal* v = o.get(k);
  if (!v || v->t != JVal::NUM) return false;
  out = v->num;
  return true;
}

}  // namespace

TuneChoice tune_choice(int sp, int nr, int ntiles) {
  TuneChoice c{0, dslash_colour_split(sp) ? 1 : 0};
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find({sp, nr, 0, bucket_of(ntiles)});
  if (it != g_table.end()) {
    c.ctas_per_sm = it->second.ctas_per_sm;
    c.form = it->second.form;
  }
  return c;
}

int tune_shared_links(int sp, int nr, int nrhs, int blocks, int* ctas_per_sm) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find({sp, nr, nrhs, bucket_of(blocks)});
  if (it == g_table.end()) return -1;
  if (ctas_per_sm) *ctas_per_sm = it->second.ctas_per_sm;
  return it->second.group;
}

}  // namespace lqcd

using namespace lqcd;

static void fill_result(lqcd_tune_result* r, const Key& k, const Entry& e) {
  r->prec = std::get<0>(k);
  r->nr = std::get<1>(k);
  r->ntiles = e.ntiles;
  r->ctas_per_sm = e.ctas_per_sm;
  r->form = e.form;
  r->candidates = e.candidates;
  r->us_best = e.us_best;
  r->us_default = e.us_default;
  r->nrhs = std::get<2>(k);
  r->group = e.group;
}

extern "C" {

int lqcd_autotune_dslash(int n, const lqcd_gauge* const* g, int prec, int compress, lqcd_tune_result* out) {
  LQCD_TRACE("lqcd_autotune_dslash");
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
  bool same_vh = true, same_gauge = true;
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
    same_gauge = same_gauge && g[i] == g[0];
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
  auto time_cfg = [&](const Launch& LL, int grid, int form, double* us) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_dslash(prec, nr, false, EPI_LIN, LL, grid, st, form);
    if (e != cudaSuccess) return e;
    int reps = 5;
    double best = 1e30;
    for (int trial = 0; trial < 3; ++trial) {
      e = cudaEventRecord(e0, st);
      for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch_dslash(prec, nr, false, EPI_LIN, LL, grid, st, form);
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
  // 1. grid and form of the launch with every slot loading its own links
  Entry ent;
  ent.ntiles = ntiles;
  double best_us = 1e30, def_us = 0;
  int best_cps = 0, best_form = def_form;
  for (int form : {0, 1, 3}) {
    if (err != cudaSuccess) break;
    const int occ = dslash_occupancy(prec, nr, form);
    if (occ < 1) continue;
    int last_grid = -1;
    for (int cps = 1; cps <= occ && err == cudaSuccess; ++cps) {
      const int grid = std::max(1, std::min(nsm * cps, ntiles));
      if (grid == last_grid) continue;  // small launches: the same grid again
      last_grid = grid;
      double us = 0;
      err = time_cfg(L, grid, form, &us);
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
  // 2. n slots on one gauge field: the shared-link form, slots per group and grid, against
  //    the own-link launch just tuned
  Entry sh;
  const bool try_shared = err == cudaSuccess && same_gauge && n > 1 && shared_link_prec(prec);
  if (try_shared) {
    const int blocks = w[0].ntiles;
    const int occ = dslash_occupancy(prec, nr, 2);
    sh.ntiles = ntiles;
    sh.us_default = best_us;  // the own-link launch
    double sh_best = 1e30;
    int sh_group = 0, sh_cps = 0;
    std::vector<int> groups_tried;
    for (int d = 1; d <= n && err == cudaSuccess; ++d) {
      const int gsize = (n + d - 1) / d;
      if (gsize < 2 || std::find(groups_tried.begin(), groups_tried.end(), gsize) != groups_tried.end()) continue;
      groups_tried.push_back(gsize);
      Launch LS = L;
      LS.interleave = 2;
      LS.mrhs_group = gsize;
      LS.mrhs_groups = (n + gsize - 1) / gsize;
      LS.ntiles = blocks * LS.mrhs_groups;
      int last_grid = -1;
      for (int cps = 1; cps <= occ && err == cudaSuccess; ++cps) {
        const int grid = std::max(1, std::min(nsm * cps, LS.ntiles));
        if (grid == last_grid) continue;
        last_grid = grid;
        double us = 0;
        err = time_cfg(LS, grid, 0, &us);
        if (err != cudaSuccess) break;
        ++sh.candidates;
        if (us < sh_best) {
          sh_best = us;
          sh_group = gsize;
          sh_cps = (cps == occ || grid == LS.ntiles) ? 0 : cps;
        }
      }
    }
    if (err == cudaSuccess) {
      // shared links only when more than 2% faster than every slot loading its own
      const bool take = sh_group > 0 && sh_best < best_us / 1.02;
      sh.group = take ? sh_group : 0;
      sh.form = take ? 2 : best_form;
      sh.ctas_per_sm = take ? sh_cps : best_cps;
      sh.us_best = take ? sh_best : best_us;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (d_works) cudaFree(d_works);
  if (d_prefix) cudaFree(d_prefix);
  if (err != cudaSuccess) return set_error(LQCD_ECUDA, "autotune: %s", cudaGetErrorString(err));
  const Key k0{prec, nr, 0, bucket_of(ntiles)};
  const Key ks{prec, nr, n, bucket_of(w[0].ntiles)};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[k0] = ent;
    if (try_shared) g_table[ks] = sh;
  }
  if (out) {
    if (try_shared) fill_result(out, ks, sh);
    else fill_result(out, k0, ent);
  }
  return LQCD_OK;
}

int lqcd_tune_entries(lqcd_tune_result* out, int max, int* n) {
  clear_error();
  if (!n || (max > 0 && !out)) return set_error(LQCD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  int k = 0;
  for (auto& kv : g_table) {
    if (k >= max) break;
    fill_result(out + k, kv.first, kv.second);
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
  fprintf(f, "{\"format\": \"lqcd-tune\", \"version\": 2, \"device\": \"%s\", \"entries\": [",
          device_tag().c_str());
  bool first = true;
  for (auto& kv : g_table) {
    const Entry& e = kv.second;
    fprintf(f,
            "%s\n  {\"prec\": %d, \"nr\": %d, \"nrhs\": %d, \"bucket\": %d, \"ntiles\": %d, "
            "\"ctas_per_sm\": %d, \"form\": %d, \"group\": %d, \"candidates\": %d, "
            "\"us_best\": %.3f, \"us_default\": %.3f}",
            first ? "" : ",", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
            std::get<3>(kv.first), e.ntiles, e.ctas_per_sm, e.form, e.group, e.candidates, e.us_best,
            e.us_default);
    first = false;
  }
  fprintf(f, "\n]}\n");
  const bool ok = fclose(f) == 0;
  return ok ? LQCD_OK : set_error(LQCD_EINVAL, "write error on %s", path);
}

int lqcd_tune_load(const char* path) {
  clear_error();
  if (!path) return set_error(LQCD_EINVAL, "NULL path");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(LQCD_EINVAL, "cannot read %s", path);
  std::string text;
  char chunk[4096];
  size_t got;
  while ((got = fread(chunk, 1, sizeof chunk, f)) > 0 && text.size() < (16u << 20)) text.append(chunk, got);
  fclose(f);
  JVal root;
  JParser jp{text.data(), text.data() + text.size()};
  const bool parsed = jp.value(root, 0);
  jp.ws();
  if (!parsed || jp.p != jp.end || root.t != JVal::OBJ) return set_error(LQCD_EINVAL, "%s: not a JSON tune file", path);
  const JVal* fmt = root.get("format");
  int ver = 0;
  if (!fmt || fmt->t != JVal::STR || fmt->str != "lqcd-tune" || !get_int(root, "version", ver) || ver != 2)
    return set_error(LQCD_EINVAL, "%s: not a tune file (format lqcd-tune, version 2)", path);
  const JVal* dev = root.get("device");
  if (!dev || dev->t != JVal::STR) return set_error(LQCD_EINVAL, "%s: no device tag", path);
  if (device_tag() != dev->str)
    return set_error(LQCD_EINVAL, "%s was tuned on %s, this device is %s", path, dev->str.c_str(),
                     device_tag().c_str());
  const JVal* ents = root.get("entries");
  if (!ents || ents->t != JVal::ARR) return set_error(LQCD_EINVAL, "%s: no entries", path);
  std::map<Key, Entry> add;
  for (const JVal& o : ents->arr) {
    int prec, nr, nrhs, b;
    Entry e;
    const bool read = o.t == JVal::OBJ && get_int(o, "prec", prec) && get_int(o, "nr", nr) &&
                      get_int(o, "nrhs", nrhs) && get_int(o, "bucket", b) && get_int(o, "ntiles", e.ntiles) &&
                      get_int(o, "ctas_per_sm", e.ctas_per_sm) && get_int(o, "form", e.form) &&
                      get_int(o, "group", e.group) && get_int(o, "candidates", e.candidates) &&
                      get_num(o, "us_best", e.us_best) && get_num(o, "us_default", e.us_default);
    const bool valid = read && prec >= LQCD_F64 && prec <= LQCD_DF64 && (nr == 12 || nr == 18) && b >= 0 &&
                       b <= 30 && e.ctas_per_sm >= 0 && e.ctas_per_sm <= 64 && e.form >= 0 && e.form <= 3 &&
                       dslash_occupancy(prec, nr, e.form) > 0 &&
                       (nrhs == 0 ? (e.form != 2 && e.group == 0)
                                  : (nrhs >= 2 && nrhs <= MAX_SLOTS &&
                                     (e.form == 2 ? (e.group >= 2 && e.group <= nrhs) : e.group == 0)));
    if (!valid) return set_error(LQCD_EINVAL, "%s: bad entry", path);
    add[{prec, nr, nrhs, b}] = e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : add) g_table[kv.first] = kv.second;
  return LQCD_OK;
}

}  // extern "C"
