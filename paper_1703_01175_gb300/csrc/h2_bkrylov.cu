// Batched restarted GMRES(m): R right-hand sides advance in lockstep, so every
// Arnoldi step needs ONE multi-RHS H^2 product (FP32 CUDA-core GEMMs or the
// split-bf16 tensor-core path) instead of R single products. Each right-hand
// side keeps its own Krylov basis, Hessenberg matrix and Givens rotations; the
// FP64 Arnoldi kernels of h2_arnoldi.cu are batched over the right-hand sides.
// Restart residuals are recomputed with the FP64-accumulated product when
// `refine` (iterative refinement), else with the batched FP32 product.
// With the learned preconditioner (flexible GMRES, Saad 1993) the network is
// applied to the basis vectors of all right-hand sides in one batched pass;
// a right-hand side whose preconditioned cycle reduces its true residual by
// less than 5 % continues with plain GMRES.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "h2_internal.h"

using namespace h2;

void h2_free_bkrylov(h2_handle *h)
{
    arn_free(reinterpret_cast<ArnWork *>(h->bkrylov));
    h->bkrylov = nullptr;
}

// rr = b - A x for all right-hand sides; |rr| -> scal
static h2_status bk_true_residual(h2_handle *h, ArnWork *w, const double2 *b, int64_t ldb, const double2 *x,
                                  int64_t ldx, bool refine, h2_prec prec, cudaStream_t st)
{
    const int n = h->n, R = w->R;
    h2_status s;
    if (refine) {
        const h2_prec acc = w->mode != ARN_FP64 ? H2_PREC_DFACC : H2_PREC_FP64ACC;
        for (int r = 0; r < R; ++r)
            if ((s = h2_matvec(h, x + (size_t)r * ldx, w->tmp + (size_t)r * n, 1, n, acc, st)) != H2_OK)
                return s;
    } else {
        if ((s = arn_c128_to_c64(w, x, ldx, w->x32, st)) != H2_OK) return s;
        if ((s = h2_matvec(h, w->x32, w->y32, R, n, prec, st)) != H2_OK) return s;
        if ((s = arn_c64_to_c128(w, w->y32, w->tmp, st)) != H2_OK) return s;
    }
    return arn_residual(w, b, ldb, w->tmp, st);
}

extern "C" h2_status h2_gmres_batched(h2_handle *h, const void *b_, void *x_, int32_t nrhs, int64_t ld,
                                      const h2_solve_opts *opts, h2_prec prec, h2_solve_info *info, void *stream)
{
    if (!h || !b_ || !x_ || !opts || nrhs < 1 || ld < h->n) return (set_error("h2_gmres_batched: bad argument"), H2_ERR_ARG);
    const int m = opts->restart;
    if (m < 1 || m > 1024 || opts->maxit < 1 || !(opts->tol > 0.0))
        return (set_error("h2_gmres_batched: need 1 <= restart <= 1024, maxit >= 1, tol > 0"), H2_ERR_ARG);
    if (prec != H2_PREC_FP32 && prec != H2_PREC_SPLITBF16)
        return (set_error("h2_gmres_batched: products must be H2_PREC_FP32 or H2_PREC_SPLITBF16"), H2_ERR_ARG);
    const bool flexible = opts->precond != 0;
    if (flexible && !h->precond)
        return (set_error("h2_gmres_batched: no preconditioner loaded (h2_set_preconditioner)"), H2_ERR_STATE);
    h2::DeviceGuard dev_guard(h->device);
    if (dev_guard.err != cudaSuccess) return (set_error("h2_gmres_batched: cudaSetDevice failed"), H2_ERR_CUDA);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ArnWork *w = reinterpret_cast<ArnWork *>(h->bkrylov);
    h2_status s = arn_get(&w, h->n, m, nrhs, flexible ? m : 0, opts->arnoldi);
    h->bkrylov = w;
    if (s != H2_OK) return s;
    if ((s = arn_set_eta(w, opts->reorth_eta)) != H2_OK) return s;
    const int n = h->n, R = nrhs;
    const double2 *b = reinterpret_cast<const double2 *>(b_);
    double2 *x = reinterpret_cast<double2 *>(x_);

    // |b|
    if ((s = arn_residual(w, b, ld, nullptr, st)) != H2_OK) return s;
    if ((s = arn_read(w, st)) != H2_OK) return s;
    std::vector<double> bnorm(R), beta(R);
    std::vector<h2_solve_info> inf(R);
    for (int r = 0; r < R; ++r) bnorm[r] = w->h_scal[8 * r];
    if (!opts->x0_given)
        for (int r = 0; r < R; ++r)
            if (cudaMemsetAsync(x + (size_t)r * ld, 0, sizeof(double2) * n, st) != cudaSuccess)
                return (set_error("h2_gmres_batched: cudaMemsetAsync failed"), H2_ERR_CUDA);
    // with x0 = 0 the residual is b itself, already in rr with |b| (no product)
    if (opts->x0_given) {
        if ((s = bk_true_residual(h, w, b, ld, x, ld, opts->refine != 0, prec, st)) != H2_OK) return s;
        if ((s = arn_read(w, st)) != H2_OK) return s;
    }
    std::vector<char> active(R);
    auto update_active = [&]() {
        int na = 0;
        for (int r = 0; r < R; ++r) {
            beta[r] = w->h_scal[8 * r];
            const double rel = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
            inf[r].rel_res = rel;
            if (!std::isfinite(beta[r])) {
                inf[r].status = H2_ERR_BREAKDOWN;
                active[r] = 0;
            } else {
                active[r] = rel > opts->tol;
            }
            na += active[r];
        }
        return na;
    };
    int it = 0;
    std::vector<int> conv(R);
    std::vector<char> pc(R, flexible ? 1 : 0);   // right-hand sides still preconditioned
    // z_j = M(v_j) for every right-hand side in one pass of the network (the
    // identity for those that fell back to plain GMRES); x32 = c64(z_j) is the
    // product's input
    auto precond_col = [&](int j) -> h2_status {
        h2_status ps;
        if ((ps = arn_basis_c128(w, j, w->tmp, st)) != H2_OK) return ps;
        double2 *zc = w->Z + (size_t)j * R * n;
        if ((ps = h2_apply_precond_batched(h, w->tmp, n, R, zc, n, w->x32, st)) != H2_OK) return ps;
        bool any_off = false;
        for (int r = 0; r < R; ++r)
            if (!pc[r]) {
                any_off = true;
                if (cudaMemcpyAsync(zc + (size_t)r * n, w->tmp + (size_t)r * n, sizeof(double2) * n,
                                    cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return (set_error("h2_gmres_batched: cudaMemcpyAsync failed"), H2_ERR_CUDA);
            }
        return any_off ? arn_c128_to_c64(w, zc, n, w->x32, st) : H2_OK;
    };
    std::vector<double> beta_start(R);
    while (update_active() > 0 && it < opts->maxit) {
        if ((s = arn_start(w, st)) != H2_OK) return s;
        for (int r = 0; r < R; ++r) beta_start[r] = beta[r];
        if (flexible && (s = precond_col(0)) != H2_OK) return s;
        std::fill(conv.begin(), conv.end(), -1);
        int k = 0;
        for (int j = 0; j < m && it < opts->maxit; ++j) {
            if ((s = h2_matvec(h, flexible ? w->x32 : arn_input(w, j), w->y32, R, n, prec, st)) != H2_OK) return s;
            if ((s = arn_step(w, j, st)) != H2_OK) return s;
            ++it;
            k = j + 1;
            bool all = true;
            for (int r = 0; r < R; ++r) {
                if (!active[r] || conv[r] >= 0) continue;
                if (w->reorth[r]) ++inf[r].reorth_steps;
                const bool lucky = w->beta[r] <= 1e-14 * bnorm[r];
                if (w->bad[r] || w->est[r] <= 0.5 * opts->tol * bnorm[r] || lucky) conv[r] = k;
                else all = false;
            }
            if (all) break;
            if (flexible && j + 1 < m && (s = precond_col(j + 1)) != H2_OK) return s;
        }
        for (int r = 0; r < R; ++r) {
            w->h_kact[r] = active[r] ? (conv[r] >= 0 ? conv[r] : k) : 0;
            if (active[r]) {
                inf[r].iterations += w->h_kact[r];
                ++inf[r].restarts;
                if (pc[r]) ++inf[r].precond_cycles;
            }
        }
        if ((s = arn_finish(w, flexible ? w->Z : w->K.V, x, ld, st)) != H2_OK) return s;
        if ((s = bk_true_residual(h, w, b, ld, x, ld, opts->refine != 0, prec, st)) != H2_OK) return s;
        if ((s = arn_read(w, st)) != H2_OK) return s;
        for (int r = 0; r < R; ++r)   // a stagnating preconditioned cycle: plain GMRES for this right-hand side
            if (pc[r] && active[r] && w->h_scal[8 * r] > 0.95 * beta_start[r]) pc[r] = 0;
    }
    update_active();
    h2_status worst = H2_OK;
    for (int r = 0; r < R; ++r) {
        if (inf[r].status == H2_OK && !(inf[r].rel_res <= opts->tol)) inf[r].status = H2_ERR_NOT_CONVERGED;
        if (inf[r].status != H2_OK && worst == H2_OK) worst = (h2_status)inf[r].status;
        if (info) info[r] = inf[r];
    }
    return worst;
}
