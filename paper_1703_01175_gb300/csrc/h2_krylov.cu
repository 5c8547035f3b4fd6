// Restarted GMRES(m) around the H^2 product, on the device, one right-hand
// side at a time.
//
// The paper solves with BiCGStab (Sec. V); here the Krylov solver is restarted
// GMRES (Saad & Schultz 1986) with the FP64 Arnoldi process of h2_arnoldi.cu
// (classical Gram-Schmidt with selective reorthogonalisation, Givens rotations
// and the least-squares solve on the device) and the H^2 product in FP32 (c64)
// inside the Arnoldi steps. With `refine` every restart residual r = b - A x
// is formed with the FP64-accumulated product, so that the outer loop is an
// iterative refinement of the FP32 inner solves. With a preconditioner loaded
// the solver is flexible GMRES (Saad 1993): z_j = M(v_j) is kept and the
// product acts on z_j; a cycle that reduces the residual by less than 5 %
// switches the rest of the solve to plain GMRES.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "h2_internal.h"

using namespace h2;

void h2_free_krylov(h2_handle *h)
{
    arn_free(reinterpret_cast<ArnWork *>(h->krylov));
    h->krylov = nullptr;
}

// r = b - A x (x, b: c128); FP64-accumulated product when `refine`, else the FP32 product.
static h2_status true_residual(h2_handle *h, ArnWork *w, const double2 *b, const double2 *x, bool x_zero, bool refine,
                               cudaStream_t st)
{
    const int n = h->n;
    if (x_zero) return arn_residual(w, b, n, nullptr, st);
    h2_status s;
    if (refine) {
        const h2_prec acc = w->mode != ARN_FP64 ? H2_PREC_DFACC : H2_PREC_FP64ACC;
        if ((s = h2_matvec(h, x, w->tmp, 1, n, acc, st)) != H2_OK) return s;
    } else {
        if ((s = arn_c128_to_c64(w, x, n, w->x32, st)) != H2_OK) return s;
        if ((s = h2_matvec(h, w->x32, w->y32, 1, n, H2_PREC_FP32, st)) != H2_OK) return s;
        if ((s = arn_c64_to_c128(w, w->y32, w->tmp, st)) != H2_OK) return s;
    }
    return arn_residual(w, b, n, w->tmp, st);
}

extern "C" {

h2_status h2_gmres(h2_handle *h, const void *b_, void *x_, int32_t nrhs, int64_t ld, const h2_solve_opts *opts,
                   h2_solve_info *info, void *stream)
{
    if (!h || !b_ || !x_ || !opts) return (set_error("h2_gmres: NULL argument"), H2_ERR_ARG);
    if (nrhs < 1 || (nrhs > 1 && ld < h->n)) return (set_error("h2_gmres: bad nrhs/ld"), H2_ERR_ARG);
    const int m = opts->restart;
    if (m < 1 || m > 1024 || opts->maxit < 1 || !(opts->tol > 0.0))
        return (set_error("h2_gmres: need 1 <= restart <= 1024, maxit >= 1, tol > 0"), H2_ERR_ARG);
    const bool flexible = opts->precond != 0;
    if (flexible && !h->precond)
        return (set_error("h2_gmres: no preconditioner loaded (h2_set_preconditioner)"), H2_ERR_STATE);
    h2::DeviceGuard dev_guard(h->device);
    if (dev_guard.err != cudaSuccess) return (set_error("h2_gmres: cudaSetDevice failed"), H2_ERR_CUDA);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ArnWork *w = reinterpret_cast<ArnWork *>(h->krylov);
    h2_status s = arn_get(&w, h->n, m, 1, flexible ? m : 0, opts->arnoldi);
    h->krylov = w;
    if (s != H2_OK) return s;
    if ((s = arn_set_eta(w, opts->reorth_eta)) != H2_OK) return s;
    const int n = h->n;
    h2_status worst = H2_OK;
    for (int32_t c = 0; c < nrhs; ++c) {
        const double2 *b = reinterpret_cast<const double2 *>(b_) + (int64_t)c * ld;
        double2 *x = reinterpret_cast<double2 *>(x_) + (int64_t)c * ld;
        h2_solve_info inf{};
        // ||b||
        if ((s = arn_residual(w, b, n, nullptr, st)) != H2_OK) return s;
        if ((s = arn_read(w, st)) != H2_OK) return s;
        const double bnorm = w->h_scal[0];
        if (!opts->x0_given || bnorm == 0.0)
            if (cudaMemsetAsync(x, 0, sizeof(double2) * n, st) != cudaSuccess)
                return (set_error("h2_gmres: cudaMemsetAsync failed"), H2_ERR_CUDA);
        if (bnorm == 0.0) {
            inf.status = H2_OK;
            if (info) info[c] = inf;
            continue;
        }
        if ((s = true_residual(h, w, b, x, !opts->x0_given, opts->refine != 0, st)) != H2_OK) return s;
        if ((s = arn_read(w, st)) != H2_OK) return s;
        double beta = w->h_scal[0];
        int it = 0;
        h2_status rs = H2_OK;
        bool pc = flexible;  // preconditioned cycles until one stagnates, then plain GMRES
        while (beta / bnorm > opts->tol && it < opts->maxit) {
            const double beta_start = beta;
            if ((s = arn_start(w, st)) != H2_OK) return s;
            if (pc && ((s = arn_basis_c128(w, 0, w->tmp, st)) != H2_OK ||
                       (s = h2_apply_precond(h, w->tmp, w->Z, w->x32, st)) != H2_OK))
                return s;
            int k = 0;
            for (int j = 0; j < m && it < opts->maxit; ++j) {
                if ((s = h2_matvec(h, pc ? w->x32 : arn_input(w, j), w->y32, 1, n, H2_PREC_FP32, st)) != H2_OK) return s;
                if ((s = arn_step(w, j, st)) != H2_OK) return s;
                ++it;
                k = j + 1;
                if (w->reorth[0]) ++inf.reorth_steps;
                if (w->bad[0]) {
                    rs = H2_ERR_BREAKDOWN;
                    break;
                }
                const double est = w->est[0];
                const bool lucky = w->beta[0] <= 1e-14 * bnorm;
                if (est <= 0.5 * opts->tol * bnorm || lucky) break;
                if (pc && j + 1 < m &&
                    ((s = arn_basis_c128(w, j + 1, w->tmp, st)) != H2_OK ||
                     (s = h2_apply_precond(h, w->tmp, w->Z + (size_t)(j + 1) * n, w->x32, st)) != H2_OK))
                    return s;
            }
            if (rs != H2_OK) break;
            w->h_kact[0] = k;
            if ((s = arn_finish(w, pc ? w->Z : w->K.V, x, n, st)) != H2_OK) return s;
            ++inf.restarts;
            if (pc) ++inf.precond_cycles;
            if ((s = true_residual(h, w, b, x, false, opts->refine != 0, st)) != H2_OK) return s;
            if ((s = arn_read(w, st)) != H2_OK) return s;
            beta = w->h_scal[0];
            if (!std::isfinite(beta)) {
                rs = H2_ERR_BREAKDOWN;
                break;
            }
            if (pc && beta > 0.95 * beta_start) pc = false;  // stagnating: fall back to plain GMRES
        }
        inf.iterations = it;
        inf.rel_res = beta / bnorm;
        if (rs == H2_OK && !(inf.rel_res <= opts->tol)) rs = H2_ERR_NOT_CONVERGED;
        inf.status = rs;
        if (info) info[c] = inf;
        if (rs != H2_OK && worst == H2_OK) worst = rs;
    }
    return worst;
}

}  // extern "C"
