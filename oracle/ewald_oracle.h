/*
 * Exact Ewald decomposition of the three Stokes potentials (stokeslet S, rotlet Omega,
 * stresslet T) with D = 3, 2, 1 or 0 periodic directions, in plain FP64 on the host.
 *
 * TEST INFRASTRUCTURE ONLY. This is the oracle that the CUDA path of the library is
 * checked against. Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference
 * arm of bench.py may load it. The library itself never calls it and shares no code
 * with it.
 *
 * Conventions (Bagge & Tornberg, "Fast Ewald summation for Stokes flow with arbitrary
 * periodicity", Sec. 2):
 *   - mu = 1, kernels exactly as Eq. (stokes-kernels), no 1/(8 pi) factor.
 *   - positions x[n*3 + i] lie in the primary cell [0,L1) x [0,L2) x [0,L3);
 *     the first D directions are periodic (Eq. periodic-images).
 *   - strengths: S and Omega f[n*3 + l]; T f[n*6 + 0..2] = q, f[n*6 + 3..5] = nu with
 *     f_lm = q_l nu_m (Sec. 2, stresslet source).
 *   - targets t[m*3 + i]; t == NULL selects the star form (targets = sources, the n = m,
 *     p = 0 term omitted, Eq. periodic-potential-star). With explicit targets, a pair at
 *     exactly zero separation is skipped in real space, and orc_self adds the self term
 *     for it, so both forms give the same number.
 *   - every routine ADDS into u[m*3 + j].
 * Return value: 0 on success, -1 on a bad argument.
 */
#ifndef EWALD_ORACLE_H
#define EWALD_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_STOKESLET = 1, ORC_ROTLET = 2, ORC_STRESSLET = 4 };

/* Real-space part, Eq. (real-space-potential-Dp) with the kernels of Eqs.
 * (stokeslet-real), (rotlet-real), (stresslet-real); all images p in P_{DP} with
 * |x - x_n + p| < rc. */
int orc_real(int D, const double L[3], double xi, double rc, int kernel, long N,
             const double* x, const double* f, long Nt, const double* t, double* u);

/* Triply periodic Fourier part for k != 0, Eq. (fourier-space-potential-3p), summed
 * directly over all k with |k| <= kmax, with G^F from Eqs. (stokeslet-fourier) ... */
int orc_fourier3p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u);

/* The non-periodic stresslet zero-mode term of the triply periodic sum,
 * Eq. (k0-stresslet-3p). Uses the coordinates as given (in [0,L)). */
int orc_k0_stresslet3p(const double L[3], long N, const double* x, const double* f,
                       long Nt, const double* t, double* u);

/* Doubly periodic Fourier part: Eq. (2p-evaluated-integrals-nonzero) with the
 * App. A tensors Q^{2P} for all (k1,k2) != 0 with |k| <= kmax, plus the k^P = 0 mode,
 * Eq. (2p-evaluated-integrals-k0) with Q^{2P,(0)}. */
int orc_fourier2p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u);

/* Singly periodic Fourier part: Eq. (1p-evaluated-integrals-nonzero) with the App. B
 * tensors Q^{1P} for k1 != 0, |k1| <= kmax, plus the k1 = 0 mode with Q^{1P,(0)}
 * (gauge l_B = 1 for the stokeslet, Eq. 1p-stokeslet-Q0). */
int orc_fourier1p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u);

/* Free-space potential by direct summation of Eq. (periodic-potential) with D = 0,
 * skipping pairs at zero separation. */
int orc_direct0p(int kernel, long N, const double* x, const double* f, long Nt,
                 const double* t, double* u);

/* Self term Eq. (self-term)/(3p-stokeslet-self-term): -(4 xi / sqrt(pi)) f for the
 * stokeslet, zero for the rotlet and stresslet; added for every target that coincides
 * exactly with a source (every target in the star form). */
int orc_self(double xi, int kernel, long N, const double* x, const double* f, long Nt,
             const double* t, double* u);

/* Special functions, exposed for the tests. */
double orc_Knu(int nu, double a, double b);  /* Eq. (Knu-def), a > 0, b >= 0 */
double orc_En(int n, double x);              /* exponential integral E_n, x > 0 */

/* App. A / App. B tensors, exposed for the tests. Output: 27 entries G[j*9 + l*3 + m]
 * for the stresslet, 9 entries G[j*3 + l] for the stokeslet and rotlet. */
int orc_Q2p(int kernel, double xi, double k1, double k2, double r3, double* re, double* im);
int orc_Q2p0(int kernel, double xi, double r3, double* re);
int orc_Q1p(int kernel, double xi, double k1, double r2, double r3, double* re, double* im);
int orc_Q1p0(int kernel, double xi, double r2, double r3, double* re);

/* Fourier-space kernel G^F(k; xi) of Eqs. (stokeslet-fourier)-(stresslet-fourier) at a
 * nonzero k, exposed for the tests (same output layout as above). */
int orc_GF(int kernel, double xi, const double* k, double* re, double* im);

/* Harmonic (Laplace) potential phi(x) = sum_n q_n / |x - x_n| (kernel H = 1/r, Sec. 2.1):
 * one strength q[n] per source, one output u[m] per target (added into). Ewald split with
 * the Ewald screening function; zero-mode conventions: 3P zero mean over the cell
 * (orc_h_k0_3p adds the constant that this needs), 2P the k^P = 0 kernel -2 pi |r_3|
 * (App. A), 1P the k_1 = 0 kernel -2 log(rho) (App. B, gauge l_H = 1), 0P direct sum. */
int orc_h_real(int D, const double L[3], double xi, double rc, long N, const double* x,
               const double* q, long Nt, const double* t, double* u);
int orc_h_fourier3p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u);
int orc_h_k0_3p(const double L[3], double xi, long N, const double* q, long Nt, double* u);
int orc_h_fourier2p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u);
int orc_h_fourier1p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u);
int orc_h_direct0p(long N, const double* x, const double* q, long Nt, const double* t, double* u);
int orc_h_self(double xi, long N, const double* x, const double* q, long Nt, const double* t,
               double* u);

#ifdef __cplusplus
}
#endif
#endif
