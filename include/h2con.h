/*
 * libh2con -- GPU kernels of the H^2 constructor for the pulse-basis E-field
 * VIE (setup, not on the timed path; driven by construct_gpu.py).
 *
 * Operator: K_mn = dV k^2 G(r_m - r_n) with the dyadic Green's function
 * G(R) = g(R) [(1 - j/kR - 1/(kR)^2) I + (-1 + 3j/kR + 3/(kR)^2) R^R^],
 * g = e^{-jkR} / (4 pi R) (Sec. II.A, Eq. 1), and the self term K_mm = s I
 * (s passed by the caller). Unknown 3 p + c is field component c of the voxel
 * at tree position p; `centres` holds the voxel centres in tree order
 * (FP64, [nv][3]). Entries are formed with FP64 geometry and phase reduction
 * and FP32 arithmetic after it; every output is complex64.
 *
 * Every pointer below is a DEVICE pointer unless marked host; every call is
 * asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy
 * default stream) and returns 0, or -1 for an invalid argument, or the CUDA
 * error code of a failed launch. The caller owns every buffer.
 */
#ifndef LIBH2_H2CON_H
#define LIBH2_H2CON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of the VIE kernel entries. */
typedef struct {
    double k;        /* wavenumber */
    double dv;       /* voxel volume */
    double self_re;  /* self term s: K_mm = s I */
    double self_im;
} h2c_vie;

/* One near-field block Z^{t,s} = delta_ts I - K^{t,s} diag(chi_s) of the
   system matrix Z = I - K diag(chi) (Sec. II; the near blocks of Sec. IV.A),
   stored column-major, 3 row_nv x 3 col_nv complex64 at Z + out_off. */
typedef struct {
    int32_t row_v0, row_nv;   /* rows: voxels [row_v0, row_v0 + row_nv) (tree positions) */
    int32_t col_v0, col_nv;   /* columns */
    int64_t out_off;          /* element offset of the block */
    int32_t diag;             /* 1: add the identity (t == s) */
    int32_t pad_;
} h2c_near_desc;

/* chi: complex64 per voxel (tree order). One thread block per descriptor. */
int h2c_near_blocks(const double *centres, h2c_vie vie, const float *chi, const h2c_near_desc *desc,
                    int64_t ndesc, float *Z, void *stream);

/* One Stage I job (Sec. III.B, Eq. 6): adaptive cross approximation with
   partial pivoting of the grouped block G^t = K[rows of t, cols] ~ U V^T,
   with the rows the unknowns of the voxels [row_v0, row_v0 + row_nv) and the
   columns the unknowns of the voxels colvox[col_off .. col_off + col_nv).
   U is stored column by column, [kmax][3 row_nv] at U + u_off; V likewise
   [kmax][3 col_nv] at V + v_off, each column scaled by 1 / pivot so that row
   piv_row[l] of the block equals piv_val[l] v_l + sum_{p<l} U[piv_row[l], p] v_p.
   `used` holds 3 row_nv bytes of scratch at used_off; pivots are written at
   piv_off. Stops when |u_k| |v_k| <= eps (sum_l |u_l|^2 |v_l|^2)^{1/2} on two
   consecutive steps. */
typedef struct {
    int32_t row_v0, row_nv;
    int32_t col_nv, kmax;
    int64_t col_off;
    int64_t u_off, v_off, used_off, piv_off;
} h2c_aca_job;

/* k_out[j] = rank reached; status[j] = 0 converged (or the block is exhausted:
   k = min(m, n)), 1 stopped at kmax before converging. kmax is clamped to
   4096. One thread block per job. */
int h2c_aca(const double *centres, h2c_vie vie, const int32_t *colvox, const h2c_aca_job *jobs, int32_t njobs,
            float eps, float *U, float *V, uint8_t *used, int32_t *piv_row, float *piv_val, int32_t *k_out,
            int32_t *status, void *stream);

/* Operand forms of the grouped GEMM. */
enum { H2C_N = 0, H2C_T = 1, H2C_C = 2 /* conjugate transpose */, H2C_R = 3 /* conjugate */ };

/* One complex product C = alpha op(A) op(B) (+ C when beta = 1), C m x n,
   op(A) m x k, op(B) k x n, all column-major complex64 (A, B) with leading
   dimensions lda, ldb, ldc. */
typedef struct {
    const float *A;
    const float *B;
    void *C;
    int32_t m, n, k;
    int32_t opa, opb, beta;
    int64_t lda, ldb, ldc;
    float alpha_re, alpha_im;
} h2c_gemm;

/* Many independent products in one launch. out_f64 = 0: C complex64 with FP32
   accumulation; 1: C complex128 with FP64 accumulation (used for the Gram
   matrices whose eigenvalues are truncated at eps^2, Eqs. 11 and 15). Products
   of one call must not write overlapping outputs. desc: device array.
   tile_prob, tile_idx: device arrays of ntiles entries (problem of each 64x64
   output tile and its index within the problem, column-major over tiles). */
int h2c_gemm_grouped(const h2c_gemm *desc, const int32_t *tile_prob, const int32_t *tile_idx, int64_t ntiles,
                     int32_t out_f64, void *stream);

/* One coupling product Q = V^{sH} K[rows of s, pivots of t] (Sec. III.C,
   Eq. 18, with the pivot rows of t's Stage I cross approximation standing for
   its row factor), Q k_s x kp column-major at Q (leading dimension ldq); the
   kernel entries are generated inside the product. Vs: the expanded basis of
   s, n_s x k_s column-major (leading dimension ldv), n_s = 3 s_nv. piv: kp
   pivot unknowns (3 p + c, tree positions). */
typedef struct {
    const float *Vs;
    const int32_t *piv;
    float *Q;
    int64_t ldv, ldq;
    int32_t s_v0, s_nv;
    int32_t ks, kp;
} h2c_couple;

int h2c_couple_grouped(const double *centres, h2c_vie vie, const h2c_couple *desc, const int32_t *tile_prob,
                       const int32_t *tile_idx, int64_t ntiles, void *stream);

/* For every pair (t, s) listed: M = (S^{t,s} + (S^{s,t})^T) / 2, then
   S^{t,s} = M and S^{s,t} = M^T (Eq. 8 with one basis per cluster: the
   couplings of the complex-symmetric kernel satisfy S^{s,t} = (S^{t,s})^T).
   off_ts / off_st: element offsets of the two column-major blocks (k_t x k_s
   and k_s x k_t). One thread block per pair. */
int h2c_sym_average(float *S, const int64_t *off_ts, const int64_t *off_st, const int32_t *kt, const int32_t *ks,
                    int64_t npairs, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBH2_H2CON_H */
