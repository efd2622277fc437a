// Meson two-point functions from a point-source propagator (paper Section 4,
// eq. 4.1):  C_Gamma(x) = - Tr[ S^dag(x) g5 Gamma S(x) Gamma g5 ],  trace over
// spin and colour, S(x) the 12 x 12 matrix whose column (beta, b) is the
// solution for the point source of spin beta, colour b, read at site x; and
// C_Gamma(t) = sum of C_Gamma(x) over the spatial sites of time slice t.
//
// In the chiral basis every Gamma used here, and so A = g5 Gamma and
// B = Gamma g5, has one non-zero per row and column: A[al][pi(al)] = a_al,
// B[rho(be)][be] = b_be. Then
//   C(x) = - sum_{al, a, be, b} conj(S[al a][be b]) a_al b_be S[pi(al) a][rho(be) b],
// a sum of 144 products per Gamma. The requested Gammas fall into a few classes
// of equal permutations (pi, rho) (three for the sixteen of the chiral basis: the
// identity for 1 and g5, and two pairings for g_x, g_y / g_z, g_t and their g5
// partners), so per class and site the "spin Gram" entries
//   G[al][be] = sum_{a, b} conj(S[al a][be b]) S[pi(al) a][rho(be) b]
// are formed once and each Gamma is C(x) = - sum a_al b_be G[al][be]. A CTA stages
// the 12 solutions of its 32 sites in shared memory; four threads per site (one
// per source spin be) form G[.][be] for every class. Each CTA covers sites of one
// time slice and writes one partial per Gamma; a second kernel sums the partials
// of each slice in a fixed order.
#include <array>
#include <complex>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"

namespace lqcd {

namespace {

constexpr int CSITES = 32;  // sites per CTA (one warp)
constexpr int MAXG = 16;

struct Monomial {  // one non-zero per row: M[r][col[r]] = (re[r], im[r])
  int col[4];
  double re[4], im[4];
};
struct GammaTab {
  Monomial A[MAXG], Bt[MAXG];  // A = g5 Gamma (by rows), B^T = (Gamma g5)^T (by columns of B)
  int cls[MAXG];               // permutation class of each Gamma
  int pi[MAXG][4], rho[MAXG][4];  // permutations of each class
  int nclass;
};

__constant__ GammaTab c_gamma;

using cd = std::complex<double>;
using M4 = std::array<std::array<cd, 4>, 4>;

M4 mat_mul(const M4& a, const M4& b) {
  M4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) c[i][j] += a[i][k] * b[k][j];
  return c;
}

// chiral basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z), g_t = [[0, 1], [1, 0]]
M4 chiral_gamma(int mu) {
  const cd I(0, 1);
  const cd s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  M4 g{};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      if (mu < 3) {
        g[a][2 + b] = -I * s[mu][a][b];
        g[2 + a][b] = I * s[mu][a][b];
      } else if (a == b) {
        g[a][2 + b] = 1;
        g[2 + a][b] = 1;
      }
    }
  return g;
}

M4 gamma_of(int code) {
  M4 g5 = mat_mul(mat_mul(chiral_gamma(0), chiral_gamma(1)), mat_mul(chiral_gamma(2), chiral_gamma(3)));
  if (code == 0) {
    M4 one{};
    for (int i = 0; i < 4; ++i) one[i][i] = 1;
    return one;
  }
  if (code == 1) return g5;
  if (code >= 2 && code <= 5) return chiral_gamma(code - 2);
  return mat_mul(g5, chiral_gamma(code - 6));
}

bool monomial_rows(const M4& m, Monomial& out) {
  for (int r = 0; r < 4; ++r) {
    int n = 0;
    for (int c = 0; c < 4; ++c)
      if (std::abs(m[r][c]) > 1e-12) {
        out.col[r] = c;
        out.re[r] = m[r][c].real();
        out.im[r] = m[r][c].imag();
        ++n;
      }
    if (n != 1) return false;
  }
  return true;
}

constexpr int CTHREADS = 4 * CSITES;  // four threads (source spins) per site

// S[j][src][comp]: comp = device real pair index (colour-major: (a * 4 + al))
__global__ void __launch_bounds__(CTHREADS) k_meson(const double2* const* props, Geom g, int ngam,
                                                    int tiles_per_slice, double* partials) {
  extern __shared__ double2 sm[];  // [CSITES][12 sources][12 components]
  __shared__ double red[CTHREADS / 32][2 * MAXG];
  const int S3 = g.L[0] * g.L[1] * g.L[2];
  const int t = blockIdx.x / tiles_per_slice;
  const int k = blockIdx.x % tiles_per_slice;
  // staging: thread i loads components of site i % CSITES
  for (int i = threadIdx.x; i < CSITES * 12; i += CTHREADS) {
    const int j = i % CSITES, src = i / CSITES;
    const int s3 = k * CSITES + j;
    if (s3 >= S3) continue;
    const long long s = (long long)t * S3 + s3;
    const int x = (int)(s % g.L[0]);
    const long long r = s / g.L[0];
    const int y = (int)(r % g.L[1]), z = (int)((r / g.L[1]) % g.L[2]);
    const int par = (x + y + z + t) & 1;
    const int h = (int)(s >> 1);
    const double2* base = props[2 * src + par];
    double2* my = sm + (size_t)j * 144 + src * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) my[c] = base[(size_t)c * g.Vh + h];
  }
  __syncthreads();
  const int j = threadIdx.x % CSITES, be = threadIdx.x / CSITES;
  const bool active = k * CSITES + j < S3;
  const double2* my = sm + (size_t)j * 144;
  double acc[2 * MAXG];
#pragma unroll
  for (int q = 0; q < 2 * MAXG; ++q) acc[q] = 0.0;
  if (active) {
    for (int cl = 0; cl < c_gamma.nclass; ++cl) {
      const int rb = c_gamma.rho[cl][be];
      double gr[4], gi[4];
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        const int pa = c_gamma.pi[cl][al];
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double2* c1 = my + (3 * be + b) * 12;
          const double2* c2 = my + (3 * rb + b) * 12;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const double2 u = c1[a * 4 + al];  // S[al a][be b]
            const double2 v = c2[a * 4 + pa];  // S[pi(al) a][rho(be) b]
            sr += u.x * v.x + u.y * v.y;       // conj(u) v
            si += u.x * v.y - u.y * v.x;
          }
        }
        gr[al] = sr;
        gi[al] = si;
      }
      for (int gm = 0; gm < ngam; ++gm) {
        if (c_gamma.cls[gm] != cl) continue;
        const Monomial& A = c_gamma.A[gm];
        const double br = c_gamma.Bt[gm].re[be], bi = c_gamma.Bt[gm].im[be];
        double cr = 0.0, ci = 0.0;
#pragma unroll
        for (int al = 0; al < 4; ++al) {  // a_al G[al][be]
          cr += A.re[al] * gr[al] - A.im[al] * gi[al];
          ci += A.re[al] * gi[al] + A.im[al] * gr[al];
        }
        acc[2 * gm] += br * cr - bi * ci;  // times b_be
        acc[2 * gm + 1] += br * ci + bi * cr;
      }
    }
  }
  // fixed-order reduction: warp shuffles, then the warps in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 2 * ngam; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * ngam) {
    double v = 0.0;
    for (int w = 0; w < CTHREADS / 32; ++w) v += red[w][threadIdx.x];
    partials[(size_t)blockIdx.x * 2 * ngam + threadIdx.x] = -v;
  }
}

// corr[gm][t] = sum over the tiles of slice t of the partials, in tile order
__global__ void k_meson_slices(const double* partials, int ngam, int tiles_per_slice, int lt, double* corr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (gm, t, re/im)
  if (i >= 2 * ngam * lt) return;
  const int q = i % (2 * ngam), t = i / (2 * ngam);
  double v = 0.0;
  for (int k = 0; k < tiles_per_slice; ++k) v += partials[((size_t)t * tiles_per_slice + k) * 2 * ngam + q];
  const int gm = q / 2, ri = q % 2;
  corr[((size_t)gm * lt + t) * 2 + ri] = v;
}

}  // namespace
}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_meson_correlator(const lqcd_field* const* props, int ngamma, const int* gammas,
                                     double* host_corr) {
  LQCD_TRACE("lqcd_meson_correlator");
  clear_error();
  if (!props || !gammas || !host_corr || ngamma < 1 || ngamma > MAXG)
    return set_error(LQCD_EINVAL, "bad arguments (ngamma = %d, at most %d)", ngamma, MAXG);
  const lqcd_field* f0 = props[0];
  if (!f0) return set_error(LQCD_EINVAL, "NULL propagator field");
  for (int i = 0; i < 12; ++i) {
    const lqcd_field* f = props[i];
    if (!f || f->prec != LQCD_F64 || f->subset != LQCD_FULL || f->ctx != f0->ctx ||
        memcmp(f->g.L, f0->g.L, sizeof f->g.L))
      return set_error(LQCD_EINVAL, "propagator %d: need 12 FULL FP64 fields of one lattice", i);
  }
  GammaTab tab;
  memset(&tab, 0, sizeof tab);
  const M4 g5 = gamma_of(1);
  for (int i = 0; i < ngamma; ++i) {
    if (gammas[i] < 0 || gammas[i] > 9) return set_error(LQCD_EINVAL, "gamma code %d", gammas[i]);
    const M4 G = gamma_of(gammas[i]);
    const M4 A = mat_mul(g5, G), B = mat_mul(G, g5);
    M4 Bt{};
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) Bt[c][r] = B[r][c];
    if (!monomial_rows(A, tab.A[i]) || !monomial_rows(Bt, tab.Bt[i]))
      return set_error(LQCD_EINVAL, "gamma code %d is not monomial", gammas[i]);
    // permutation class: pi from the rows of A, rho from the columns of B
    int cl = 0;
    for (; cl < tab.nclass; ++cl)
      if (!memcmp(tab.pi[cl], tab.A[i].col, sizeof tab.pi[cl]) && !memcmp(tab.rho[cl], tab.Bt[i].col, sizeof tab.rho[cl]))
        break;
    if (cl == tab.nclass) {
      memcpy(tab.pi[cl], tab.A[i].col, sizeof tab.pi[cl]);
      memcpy(tab.rho[cl], tab.Bt[i].col, sizeof tab.rho[cl]);
      ++tab.nclass;
    }
    tab.cls[i] = cl;
  }
  lqcd_ctx* c = f0->ctx;
  LQCD_CK(cudaSetDevice(c->device));
  const Geom& g = f0->g;
  const int S3 = g.L[0] * g.L[1] * g.L[2];
  const int tps = (S3 + CSITES - 1) / CSITES;
  const int nblk = tps * g.L[3];
  const size_t npart = (size_t)nblk * ngamma * 2;
  std::vector<const double2*> hp(24);
  for (int i = 0; i < 12; ++i)
    for (int p = 0; p < 2; ++p) hp[2 * i + p] = static_cast<const double2*>(props[i]->half[p]);
  LQCD_CK(cudaMemcpyToSymbolAsync(c_gamma, &tab, sizeof tab, 0, cudaMemcpyHostToDevice, c->stream));
  const size_t ncorr = (size_t)2 * ngamma * g.L[3];
  const size_t nd = ((npart + ncorr + 31) / 32) * 32;
  int rc = ctx_staging(c, nd * sizeof(double) + 24 * sizeof(void*) + 256);
  if (rc != LQCD_OK) return rc;
  double* d_part = c->staging;
  const double2** d_props = reinterpret_cast<const double2**>(d_part + nd);
  LQCD_CK(cudaMemcpyAsync(d_props, hp.data(), 24 * sizeof(void*), cudaMemcpyHostToDevice, c->stream));
  const size_t smem = (size_t)CSITES * 144 * sizeof(double2);
  LQCD_CK(cudaFuncSetAttribute(k_meson, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  double* d_corr = d_part + npart;  // ngamma x Lt complex, after the partials
  k_meson<<<nblk, CTHREADS, smem, c->stream>>>(d_props, g, ngamma, tps, d_part);
  const int nout = 2 * ngamma * g.L[3];
  k_meson_slices<<<(nout + 127) / 128, 128, 0, c->stream>>>(d_part, ngamma, tps, g.L[3], d_corr);
  LQCD_CK(cudaGetLastError());
  c->launches += 2;
  LQCD_CK(cudaMemcpyAsync(host_corr, d_corr, (size_t)nout * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQCD_CK(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}
