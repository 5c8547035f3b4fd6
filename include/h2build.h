/*
 * libh2build -- native helpers of the host-side H^2 constructor (setup only).
 *
 * Stage I of the minimal-rank construction (Omar & Jiao, Sec. III.B, Eqs.
 * 5-6): adaptive cross approximation with partial pivoting of the grouped
 * admissible block G^t of one cluster, for the pulse-basis E-field VIE kernel
 *
 *   K_mn = dV k^2 g(R) [(1 - j/kR - 1/kR^2) I + (-1 + 3j/kR + 3/kR^2) R^R^],
 *   g(R) = e^{-jkR} / (4 pi R),   K_mm = self * I,
 *
 * between voxel centres (3 unknowns per voxel, component-minor).
 *
 * Conventions: complex numbers are interleaved (re, im) doubles; matrices are
 * column-major; all arrays are caller-owned host memory; the functions are
 * thread-safe (no global state) and allocate only internal scratch.
 */
#ifndef LIBH2_H2BUILD_H
#define LIBH2_H2BUILD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * ACA of G = K[rows, cols] (m = 3 m_vox rows, n = 3 n_vox columns):
 * G ~ U V^T with U (m x k), V (n x k). Each step takes the residual row of the
 * current pivot row, its largest entry as pivot column, the residual column,
 * and the next pivot row as the largest entry of that column among unused
 * rows; it stops when |u_k| |v_k| <= eps * sqrt(sum_l |u_l|^2 |v_l|^2) (the usual
 * estimate of ||U V^T||_F) on two consecutive steps.
 *
 * centres: [3 * n_all] voxel centres (x, y, z); rows_vox / cols_vox: voxel
 * indices into centres; U_out: [2 * m * kmax] doubles; V_out: [2 * n * kmax].
 * piv_rows (may be NULL): [kmax] the pivot row (unknown index in 0..m) of
 * each term; piv_vals (may be NULL): [2 * kmax] the pivot entry of each term,
 * so that row piv_rows[l] of G equals piv_vals[l] v_l + sum_{p<l} U[piv_rows[l], p] v_p
 * (the cross/skeleton form of the approximation).
 * Writes the rank to *k_out. Returns 0 on success, 1 if kmax steps were taken
 * without meeting the stopping rule (U, V hold kmax terms), -1 on bad
 * arguments.
 */
int h2c_aca_vie(const double *centres, double dv, double k, double self_re, double self_im,
                const int64_t *rows_vox, int32_t m_vox, const int64_t *cols_vox, int32_t n_vox,
                double eps, int32_t kmax, double *U_out, double *V_out, int32_t *k_out,
                int64_t *piv_rows, double *piv_vals);

/*
 * Dense block K[rows, cols] (3 m_vox x 3 n_vox, column-major, complex
 * interleaved doubles) scaled on the right by diag(colscale) (one complex
 * factor per voxel, may be NULL for 1) and multiplied by `alpha`:
 * out = alpha * K[rows, cols] * diag(colscale).
 */
int h2c_block_vie(const double *centres, double dv, double k, double self_re, double self_im,
                  const int64_t *rows_vox, int32_t m_vox, const int64_t *cols_vox, int32_t n_vox,
                  const double *colscale, double alpha_re, double alpha_im, double *out);

#ifdef __cplusplus
}
#endif
#endif /* LIBH2_H2BUILD_H */
