/*
 * lbm_vn.h -- C ABI for the linear (von Neumann) stability analysis of the
 * D2V16 MRT-FD scheme, Sec. IV.
 *
 * About a uniform state (rho, u, v, T) a small Fourier disturbance
 * Delta f_i = F_i exp(i k.x) of the populations grows by F <- G F per step,
 *
 *   G_ij = delta_ij [a0_i + aE_i e^{i k_x dx} + aW_i e^{-i k_x dx}
 *                         + aN_i e^{i k_y dy} + aS_i e^{-i k_y dy}]
 *          + d(Delta f_i^coll) / d f_j,
 *
 * the first term the Lax-Wendroff update of Eq. A.1 (a* its weights: a0 = 1 -
 * a_x^2 - a_y^2, aE = (a_x^2 - a_x)/2, ..., a_x = v_ix dt/dx) and the second
 * the Jacobian of the Eq. 3 collision -dt M^-1 S_hat (M - dfhat^eq/df) at
 * the state, which Sec. IV writes out. The scheme is von Neumann stable at the
 * state when max |omega| <= 1 over the eigenvalues omega of G for every k.
 *
 * On the device: the collision Jacobian is obtained per case by forward-mode
 * differentiation (dual numbers) of the same per-node collision code that the
 * step kernels run; G's eigenvalues come from a Householder reduction to
 * Hessenberg form followed by single-shift complex QR iterations (Wilkinson
 * shifts, deflation on negligible subdiagonals), all in FP64, one matrix per
 * 16 threads.
 *
 * Layouts. Complex numbers are two doubles (re, im), as C99 double complex.
 * A 16 x 16 matrix is row-major: entry (i, j) at index 16 i + j; row i is
 * population i in the order of Eq. 4 used by lbm.h. Case c and wave vector q
 * make item c * nk + q.
 *
 * Pointers. With on_device = 0 every array is in host memory and the call
 * synchronises; with on_device = 1 every array is in device memory and the
 * call is asynchronous on cuda_stream (NULL: the legacy default stream).
 * Inputs are read during the call only; outputs are caller-owned.
 *
 * Convergence. The QR iteration is bounded (30 sweeps per eigenvalue on
 * average, as LAPACK's complex Hessenberg QR allows): a matrix that has not
 * converged by then gets NaN eigenvalues and radius. If nonconverged is not
 * NULL (a host pointer) the call synchronises and stores how many matrices
 * did not converge.
 *
 * Errors: LBM_ERR_INVALID for counts < 1, non-finite or non-positive
 * spacings or time step, a case with rho <= 0, T <= 0 or a non-finite entry,
 * a non-finite wave vector, or NULL required arrays; LBM_ERR_OOM /
 * LBM_ERR_CUDA for allocation or launch failures (text: lbm_vn_last_error()).
 * With on_device = 1 the cases are not read on the host: a case that fails
 * those checks gets NaN results instead (counted in nonconverged).
 */
#ifndef LBM_VN_H
#define LBM_VN_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One stability case: the uniform state and the 16 relaxation rates
 * s_1..s_16 of S_hat (s_1..s_4 multiply zero rows and have no effect). */
typedef struct {
  double rho, u, v, T;
  double s[16];
} lbm_vn_case;

/* G for every (case, wave vector) pair: cases[ncases], k[nk][2] = (k_x, k_y)
 * in inverse length units, G[ncases * nk][16][16] complex (output). */
int lbm_vn_matrices(const lbm_vn_case* cases, int ncases, const double* k, int nk, double dx,
                    double dy, double dt, double* G, int on_device, void* cuda_stream);

/* The eigenvalues of G for every (case, wave vector) pair: radius[ncases * nk]
 * = max |omega| (output, may be NULL), omega[ncases * nk][16] complex
 * (output, may be NULL; order unspecified). */
int lbm_vn_spectrum(const lbm_vn_case* cases, int ncases, const double* k, int nk, double dx,
                    double dy, double dt, double* radius, double* omega, int on_device,
                    void* cuda_stream, long long* nonconverged);

/* Eigenvalues of n arbitrary complex 16 x 16 matrices A[n][16][16] by the same
 * device solver: omega[n][16] complex (may be NULL), radius[n] = max |omega|
 * (may be NULL). A matrix with a non-finite entry gets NaN results. */
int lbm_eig16(const double* A, long long n, double* omega, double* radius, int on_device,
              void* cuda_stream, long long* nonconverged);

/* One-line reason for the last failing call of this header on this thread. */
const char* lbm_vn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_VN_H */
