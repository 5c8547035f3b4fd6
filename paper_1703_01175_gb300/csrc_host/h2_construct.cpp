// Native helpers of the host-side H^2 constructor: VIE kernel entries and the
// adaptive cross approximation of Stage I (Sec. III.B, Eq. 6).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "h2build.h"

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

struct Kern {
    const double *c;
    double dv, k;
    cd self;
    // row `a` of the 3x3 block K(p, q): out[0..2]
    inline void row(int64_t p, int a, int64_t q, cd *out) const
    {
        const double rx = c[3 * p] - c[3 * q], ry = c[3 * p + 1] - c[3 * q + 1], rz = c[3 * p + 2] - c[3 * q + 2];
        const double r2 = rx * rx + ry * ry + rz * rz;
        if (r2 == 0.0) {
            out[0] = out[1] = out[2] = 0.0;
            out[a] = self;
            return;
        }
        const double r = std::sqrt(r2), kr = k * r, inv = 1.0 / kr;
        const double sc = dv * k * k / (4.0 * kPi * r);
        const cd g(sc * std::cos(kr), -sc * std::sin(kr));
        const cd ca = g * cd(1.0 - inv * inv, -inv);
        const cd cb = g * cd(-1.0 + 3.0 * inv * inv, 3.0 * inv);
        const double h[3] = {rx / r, ry / r, rz / r};
        for (int b = 0; b < 3; ++b) out[b] = cb * (h[a] * h[b]);
        out[a] += ca;
    }
};

}  // namespace

extern "C" int h2c_aca_vie(const double *centres, double dv, double k, double self_re, double self_im,
                           const int64_t *rows_vox, int32_t m_vox, const int64_t *cols_vox, int32_t n_vox,
                           double eps, int32_t kmax, double *U_out, double *V_out, int32_t *k_out,
                           int64_t *piv_rows, double *piv_vals)
{
    if (!centres || !rows_vox || !cols_vox || !U_out || !V_out || !k_out || m_vox <= 0 || n_vox <= 0 || kmax <= 0)
        return -1;
    const Kern K{centres, dv, k, cd(self_re, self_im)};
    const int64_t m = 3 * (int64_t)m_vox, n = 3 * (int64_t)n_vox;
    // factors kept as separate real / imaginary planes (vectorisable loops),
    // copied to the interleaved outputs at the end
    std::vector<double> Ur((size_t)m * kmax), Ui((size_t)m * kmax), Vr((size_t)n * kmax), Vi((size_t)n * kmax);
    std::vector<double> rr(n), ri(n), ur(m), ui(m);
    std::vector<cd> tmp(std::max(n, m));
    std::vector<char> used(m, 0);
    int64_t i = 0;
    int32_t kk = 0, small = 0;
    double norm2 = 0.0;  // sum_l |u_l|^2 |v_l|^2, the usual estimate of ||U V^T||_F^2
    while (kk < kmax) {
        // residual row i
        const int64_t pv = rows_vox[i / 3];
        const int a = (int)(i % 3);
        for (int64_t q = 0; q < n_vox; ++q) K.row(pv, a, cols_vox[q], &tmp[3 * q]);
        for (int64_t j = 0; j < n; ++j) {
            rr[j] = tmp[j].real();
            ri[j] = tmp[j].imag();
        }
        for (int l = 0; l < kk; ++l) {
            const double ar = Ur[(size_t)l * m + i], ai = Ui[(size_t)l * m + i];
            const double *vr = &Vr[(size_t)l * n], *vi = &Vi[(size_t)l * n];
            for (int64_t j = 0; j < n; ++j) {
                rr[j] -= ar * vr[j] - ai * vi[j];
                ri[j] -= ar * vi[j] + ai * vr[j];
            }
        }
        used[i] = 1;
        int64_t jp = 0;
        double best = -1.0;
        for (int64_t j = 0; j < n; ++j) {
            const double v = rr[j] * rr[j] + ri[j] * ri[j];
            if (v > best) {
                best = v;
                jp = j;
            }
        }
        if (best <= 0.0) {
            int64_t f = -1;
            for (int64_t q = 0; q < m; ++q)
                if (!used[q]) {
                    f = q;
                    break;
                }
            if (f < 0) break;
            i = f;
            continue;
        }
        const cd piv(rr[jp], ri[jp]);
        // residual column jp (K symmetric: column of G = row of K for the column unknown)
        const int64_t qv = cols_vox[jp / 3];
        const int b = (int)(jp % 3);
        for (int64_t p = 0; p < m_vox; ++p) K.row(qv, b, rows_vox[p], &tmp[3 * p]);
        for (int64_t q = 0; q < m; ++q) {
            ur[q] = tmp[q].real();
            ui[q] = tmp[q].imag();
        }
        for (int l = 0; l < kk; ++l) {
            const double br = Vr[(size_t)l * n + jp], bi = Vi[(size_t)l * n + jp];
            const double *xr = &Ur[(size_t)l * m], *xi = &Ui[(size_t)l * m];
            for (int64_t q = 0; q < m; ++q) {
                ur[q] -= xr[q] * br - xi[q] * bi;
                ui[q] -= xr[q] * bi + xi[q] * br;
            }
        }
        if (piv_rows) piv_rows[kk] = i;
        if (piv_vals) {
            piv_vals[2 * kk] = piv.real();
            piv_vals[2 * kk + 1] = piv.imag();
        }
        const cd inv = 1.0 / piv;
        double *vr = &Vr[(size_t)kk * n], *vi = &Vi[(size_t)kk * n];
        double nu2 = 0, nv2 = 0;
        for (int64_t j = 0; j < n; ++j) {
            vr[j] = rr[j] * inv.real() - ri[j] * inv.imag();
            vi[j] = rr[j] * inv.imag() + ri[j] * inv.real();
            nv2 += vr[j] * vr[j] + vi[j] * vi[j];
        }
        double *xr = &Ur[(size_t)kk * m], *xi = &Ui[(size_t)kk * m];
        for (int64_t q = 0; q < m; ++q) {
            xr[q] = ur[q];
            xi[q] = ui[q];
            nu2 += ur[q] * ur[q] + ui[q] * ui[q];
        }
        norm2 += nu2 * nv2;
        ++kk;
        if (std::sqrt(nu2 * nv2) <= eps * std::sqrt(norm2)) {
            if (++small >= 2) break;
        } else {
            small = 0;
        }
        int64_t nx = -1;
        double bu = -1.0;
        for (int64_t q = 0; q < m; ++q) {
            const double v = ur[q] * ur[q] + ui[q] * ui[q];
            if (!used[q] && v > bu) {
                bu = v;
                nx = q;
            }
        }
        if (nx < 0) break;
        i = nx;
    }
    for (int l = 0; l < kk; ++l) {
        for (int64_t q = 0; q < m; ++q) {
            U_out[2 * ((size_t)l * m + q)] = Ur[(size_t)l * m + q];
            U_out[2 * ((size_t)l * m + q) + 1] = Ui[(size_t)l * m + q];
        }
        for (int64_t j = 0; j < n; ++j) {
            V_out[2 * ((size_t)l * n + j)] = Vr[(size_t)l * n + j];
            V_out[2 * ((size_t)l * n + j) + 1] = Vi[(size_t)l * n + j];
        }
    }
    *k_out = kk;
    return (kk >= kmax && small < 2) ? 1 : 0;
}

extern "C" int h2c_block_vie(const double *centres, double dv, double k, double self_re, double self_im,
                             const int64_t *rows_vox, int32_t m_vox, const int64_t *cols_vox, int32_t n_vox,
                             const double *colscale, double alpha_re, double alpha_im, double *out)
{
    if (!centres || !rows_vox || !cols_vox || !out || m_vox < 0 || n_vox < 0) return -1;
    const Kern K{centres, dv, k, cd(self_re, self_im)};
    const int64_t m = 3 * (int64_t)m_vox;
    cd *O = reinterpret_cast<cd *>(out);
    const cd alpha(alpha_re, alpha_im);
    cd row3[3];
    for (int64_t q = 0; q < n_vox; ++q) {
        const cd sc = alpha * (colscale ? cd(colscale[2 * q], colscale[2 * q + 1]) : cd(1.0, 0.0));
        for (int64_t p = 0; p < m_vox; ++p)
            for (int a = 0; a < 3; ++a) {
                K.row(rows_vox[p], a, cols_vox[q], row3);
                for (int b = 0; b < 3; ++b) O[(3 * q + b) * m + 3 * p + a] = row3[b] * sc;
            }
    }
    return 0;
}
