/* FP64 CPU oracle of the pure-gauge SU(3) heatbath and the plaquette.
 *
 * TEST INFRASTRUCTURE ONLY: the correctness reference of the CUDA heatbath.
 * Only the tests, the smoke check and the benchmark's CPU baseline may load it;
 * it shares no code, header, table or constant with the library.
 *
 * The paper (Section 3) names an SU(3) heatbath for pure gauge theory, citing
 * Creutz, and gives no algorithm. This oracle takes the standard reading:
 *
 *   Action      S = beta sum_P (1 - Re Tr U_P / 3), Wilson plaquette action.
 *   Staple      W_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
 *                                          + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ],
 *               so the weight of U = U_mu(x) is exp((beta/3) Re Tr(U W)).
 *   Update      Cabibbo-Marinari: for the SU(2) subgroups on index pairs
 *               (0,1), (1,2), (0,2) in turn, U <- R U with R in the subgroup
 *               drawn from the heatbath distribution of Re Tr(R U W).
 *   SU(2) draw  Creutz: the subgroup block X of V = U W gives the 4-vector c
 *               with Re Tr(a X) = a.c for a = a0 + i a.sigma; k = |c|, v = c/k,
 *               alpha = beta k / 3. b is drawn with density
 *               ~ exp(alpha b0) sqrt(1 - b0^2) on [-1, 1] (b0 = 1 + ln y / alpha,
 *               y uniform in (exp(-2 alpha), 1], accepted with probability
 *               sqrt(1 - b0^2)) and a uniform direction for (b1, b2, b3); then
 *               a = b v (so a.v = b0) and R embeds a.
 *   Order       per sweep: mu = 0..3, parity = even, odd; the links of one
 *               (mu, parity) class are independent of each other. After the
 *               sweep every link is reunitarised (Gram-Schmidt of rows 0, 1,
 *               row 2 = conj(row0 x row1)) when reunit != 0.
 *   Randomness  Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), key
 *               (seed, 0), counter (4 link_id + mu, sweep,
 *               subgroup, attempt) with link_id the lexicographic site index;
 *               u = (r >> 11 + 1) 2^-53 in (0, 1]. Four uniforms per attempt:
 *               u0 -> b0, u1 -> accept (u1^2 <= 1 - b0^2), u2 -> cos(theta) =
 *               2 u2 - 1, u3 -> phi = 2 pi u3. For alpha < 1e-12, b0 = 1 - 2 u0.
 *               At most 1000 attempts; a subgroup that never accepts is left
 *               unchanged and counted.
 *
 * Layout as wilson_oracle.h: U[s][mu][row][col] complex double, site
 * s = x + Lx*(y + Ly*(z + Lz*t)), all extents even.
 *
 * Pins (tests/test_oracle_heatbath.py): Philox against numpy's Philox bit
 * generator; the SU(2) draw against the exact moments I2(alpha)/I1(alpha) and
 * a Kolmogorov-Smirnov test against the density; single-link equilibrium
 * against a brute-force Haar-measure integral; Haar moments at beta = 0; the
 * strong-coupling plaquette beta/18 + beta^2/216; unitarity.
 */
#ifndef LQCD_HEATBATH_ORACLE_H
#define LQCD_HEATBATH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* out = Philox4x64-10(counter, key) */
void oracle_philox4x64(const uint64_t counter[4], const uint64_t key[2], uint64_t out[4]);

/* n SU(2) draws b (4 reals each) with density ~ exp(alpha b0) on the 3-sphere, the
 * i-th from counters (i, 0, 0, attempt) under key (seed, 0).
 * Returns the number of draws that hit the attempt limit (left as b = (1, 0, 0, 0)). */
long long oracle_su2_draws(double alpha, uint64_t seed, long long n, double* out);

/* Average plaquette sum_{x, mu<nu} Re Tr U_munu(x) / (18 V). */
double oracle_plaquette(const int dims[4], const double* U);

/* Staple sum W_mu(x) (3x3 complex) of the link at lexicographic site s. */
void oracle_staple(const int dims[4], const double* U, long long s, int mu, double* W);

/* One heatbath update of the single link U_mu(s) (three subgroups, counters of
 * sweep `sweep`). Returns the number of subgroups left unchanged. */
int oracle_heatbath_link(const int dims[4], double* U, double beta, uint64_t seed, uint64_t sweep,
                         long long s, int mu);

/* nsweeps full sweeps, sweep numbers sweep0, sweep0 + 1, ...; returns the number of
 * subgroup updates that hit the attempt limit, or -1 for bad arguments. */
long long oracle_heatbath(const int dims[4], double* U, double beta, uint64_t seed, uint64_t sweep0,
                          int nsweeps, int reunit);

/* Reunitarise every link (Gram-Schmidt of rows 0, 1; row 2 = conj(row0 x row1)). */
void oracle_reunitarise(const int dims[4], double* U);

#ifdef __cplusplus
}
#endif
#endif
