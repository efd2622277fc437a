/* FP64 CPU oracle for the Wilson-Dirac fermion matrix and its Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY. This code is the correctness reference for the
 * CUDA library. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library never calls it, and it shares no code,
 * header, table or constant with the library.
 *
 * The paper (Sections 3 and 4) names the even-odd preconditioned Wilson
 * hopping term ("dslash") and the inversion of the fermion matrix as the hot
 * path, without writing the operator down. This oracle states it in the
 * textbook form, r = 1, kappa normalisation:
 *
 *   (M psi)(x) = psi(x) - kappa * sum_mu [ eta+ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                        + eta- (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *
 * with chiral gamma matrices g_k = [[0, -i s_k], [i s_k, 0]] (mu = 0,1,2 for
 * k = 1,2,3) and g_4 = [[0, 1], [1, 0]] (mu = 3), so g5 = diag(1, 1, -1, -1);
 * eta = t_bc on hops that cross the t boundary, else 1.
 *
 * Layout: site s = x + Lx*(y + Ly*(z + Lz*t)); links U[s][mu][row][col];
 * spinors psi[s][spin][colour]; all complex double (re, im interleaved).
 * Even-odd vectors are full-lattice arrays whose other-parity sites are zero.
 *
 * Parity pins (see tests/test_oracle_*.py): free-field plane-wave eigenvalues,
 * constant field with periodic links, gamma5-hermiticity, adjointness of the
 * dagger, gauge covariance, a dense brute-force matrix on 2^4 and 2x2x2x4,
 * dense LAPACK solves on 2^4 and 4^4, and an FFT solve of the free field.
 */
#ifndef WILSON_ORACLE_H
#define WILSON_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* status of a solve */
enum { ORACLE_OK = 0, ORACLE_MAXITER = 1, ORACLE_BREAKDOWN = 2, ORACLE_BADARG = -1 };

void oracle_set_threads(int n);
int  oracle_get_threads(void);

/* out = D psi (hopping term alone), full lattice. dagger != 0 gives D^dag. */
int oracle_hop(const int dims[4], int t_bc, const double* U, const double* psi,
               double* out, int dagger);

/* out(x) = (D psi)(x) at sites of parity out_parity, 0 elsewhere (D_{pq}). */
int oracle_hop_eo(const int dims[4], int t_bc, const double* U, const double* psi,
                  double* out, int out_parity, int dagger);

/* out[i] = (D psi)(sites[i]) for a list of sites; out is nsites x 12 complex. */
int oracle_hop_sites(const int dims[4], int t_bc, const double* U, const double* psi,
                     const long long* sites, long long nsites, double* out, int dagger);

/* out = M psi = psi - kappa D psi + 2 i kappa mu g5 psi (full lattice): the Wilson
 * operator for mu = 0, the N_f = 2 twisted-mass operator (paper Section 3, one flavour;
 * the other has -mu) otherwise. dagger gives M^dag. */
int oracle_apply_M(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                   const double* psi, double* out, int dagger);

/* Schur complement on the even sites, A = 1 + 2 i kappa mu g5 the site-diagonal part:
 * out_e = A psi_e - kappa^2 D_eo A^-1 D_oe psi_e, 0 on odd sites (mu = 0: 1 - k^2 D_eo D_oe).
 * dagger gives its adjoint. */
int oracle_apply_Mhat(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                      const double* psi, double* out, int dagger);

/* Solve M x = b.
 *   method 0: CG on M^dag M (full lattice)
 *   method 1: even-odd: CG on Mhat^dag Mhat for x_e, then x_o = A^-1 (b_o + kappa D_oe x_e)
 *   method 2: even-odd: BiCGStab on Mhat, then the same reconstruction
 * (bhat_e = b_e + kappa D_eo A^-1 b_o; A = 1 for mu = 0)
 * Stops when ||b - M x|| <= tol ||b|| (full, unpreconditioned M, FP64).
 * x is overwritten (start value 0). info[0] = iterations, info[1] = final
 * true relative residual. Returns ORACLE_OK, ORACLE_MAXITER or ORACLE_BREAKDOWN. */
int oracle_solve(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                 const double* b, double* x, double tol, int maxiter, int method,
                 double* info);

/* ||b - M x|| / ||b|| with the full operator. */
double oracle_true_residual(const int dims[4], int t_bc, const double* U, double kappa, double mu,
                            const double* b, const double* x);

#ifdef __cplusplus
}
#endif
#endif
