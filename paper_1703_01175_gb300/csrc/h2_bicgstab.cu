// BiCGStab (van der Vorst 1992), the paper's solver (Sec. V), around the H^2
// product: FP32 products (c64) inside the iteration, FP64 vectors and inner
// products on the device. With `refine`, a recursive residual below tol is
// checked against the true residual b - A x formed with the accumulated
// product (FP64, or double-float when opts->arnoldi = 1); if that is still
// above tol the iteration restarts from x with a new shadow residual.
//
// One iteration is two products and five vector kernels:
//   p = r + beta (p - omega v), p32            (beta from the device scalars)
//   v = A p;  alpha = rho / (rhat, v)
//   s = r - alpha v, s32
//   t = A s;  omega = (t, s) / (t, t)
//   x += alpha p + omega s;  r = s - omega t;  rho' = (rhat, r), |r|^2
// Every inner product is combined in a fixed order by the last block to
// finish, which also updates the scalars, so the host reads only |r| and the
// breakdown flag once per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "h2_internal.h"
#include "h2_reduce.cuh"

namespace h2 {
namespace {

constexpr int BT = 256;

// scalars (complex) of the iteration
enum { S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_RNORM2, S_FLAG, S_COUNT };

struct BG {
    double2 *r, *rhat, *p, *v, *s, *t;
    double2 *part;      // [2][nblk] partial sums
    unsigned *ticket;   // [4]
    double2 *sc;        // [S_COUNT]
    float2 *x32, *y32;
    int n, nblk, rows;
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    const double d = b.x * b.x + b.y * b.y;
    return d > 0 ? make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d) : make_double2(0, 0);
}
// conj(a) * b
__device__ __forceinline__ double2 cj(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }

// sums NV partial values of every block in fixed order (last block only)
template <int NV>
__device__ void finish(const BG &K, double2 *out)
{
    for (int q = 0; q < NV; ++q) {
        double2 acc = make_double2(0, 0);
        const volatile double2 *p = K.part + (size_t)q * K.nblk;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += BT) acc = zsum2(acc, make_double2(p[b].x, p[b].y));
        const double2 t = block_sum2<BT>(acc);
        if (threadIdx.x == 0) out[q] = t;
    }
}

// r = b - y (y NULL: r = b); rhat = r; |r|^2; scalars reset for a new start
__global__ void __launch_bounds__(BT) bg_start(BG K, const double2 *__restrict__ b, const double2 *__restrict__ y)
{
    const int i0 = blockIdx.x * K.rows, i1 = min(K.n, i0 + K.rows);
    double nrm = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += BT) {
        double2 v = b[i];
        if (y) v = make_double2(v.x - y[i].x, v.y - y[i].y);
        K.r[i] = v;
        K.rhat[i] = v;
        K.p[i] = make_double2(0, 0);
        K.v[i] = make_double2(0, 0);
        nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
    }
    const double2 tot = block_sum2<BT>(make_double2(nrm, 0));
    if (threadIdx.x == 0) K.part[blockIdx.x] = tot;
    if (!last_block(K.ticket + 0)) return;
    __shared__ double2 out[1];
    finish<1>(K, out);
    if (threadIdx.x == 0) {
        K.sc[S_RNORM2] = out[0];
        K.sc[S_RHO] = out[0];  // (rhat, r) = |r|^2
        K.sc[S_RHO_OLD] = make_double2(1, 0);
        K.sc[S_ALPHA] = make_double2(1, 0);
        K.sc[S_OMEGA] = make_double2(1, 0);
        K.sc[S_FLAG] = make_double2(0, 0);
    }
}

// p = r + beta (p - omega v), p32 = c64(p)
__global__ void bg_p(BG K)
{
    const double2 beta = cm(cdiv(K.sc[S_RHO], K.sc[S_RHO_OLD]), cdiv(K.sc[S_ALPHA], K.sc[S_OMEGA]));
    const double2 om = K.sc[S_OMEGA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 q = cm(om, K.v[i]);
        const double2 d = make_double2(K.p[i].x - q.x, K.p[i].y - q.y);
        const double2 bd = cm(beta, d);
        const double2 p = make_double2(K.r[i].x + bd.x, K.r[i].y + bd.y);
        K.p[i] = p;
        K.x32[i] = make_float2((float)p.x, (float)p.y);
    }
}

// v = c128(y32); alpha = rho / (rhat, v)
__global__ void __launch_bounds__(BT) bg_v(BG K)
{
    const int i0 = blockIdx.x * K.rows, i1 = min(K.n, i0 + K.rows);
    double2 acc = make_double2(0, 0);
    for (int i = i0 + threadIdx.x; i < i1; i += BT) {
        const double2 v = make_double2(K.y32[i].x, K.y32[i].y);
        K.v[i] = v;
        acc = zsum2(acc, cj(K.rhat[i], v));
    }
    const double2 tot = block_sum2<BT>(acc);
    if (threadIdx.x == 0) K.part[blockIdx.x] = tot;
    if (!last_block(K.ticket + 1)) return;
    __shared__ double2 out[1];
    finish<1>(K, out);
    if (threadIdx.x == 0) {
        const double2 d = out[0];
        if (d.x == 0.0 && d.y == 0.0) K.sc[S_FLAG] = make_double2(1, 0);
        K.sc[S_ALPHA] = cdiv(K.sc[S_RHO], d);
    }
}

// s = r - alpha v, s32 = c64(s)
__global__ void bg_s(BG K)
{
    const double2 al = K.sc[S_ALPHA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 q = cm(al, K.v[i]);
        const double2 s = make_double2(K.r[i].x - q.x, K.r[i].y - q.y);
        K.s[i] = s;
        K.x32[i] = make_float2((float)s.x, (float)s.y);
    }
}

// t = c128(y32); omega = (t, s) / (t, t)
__global__ void __launch_bounds__(BT) bg_t(BG K)
{
    const int i0 = blockIdx.x * K.rows, i1 = min(K.n, i0 + K.rows);
    double2 ts = make_double2(0, 0);
    double tt = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += BT) {
        const double2 t = make_double2(K.y32[i].x, K.y32[i].y);
        K.t[i] = t;
        ts = zsum2(ts, cj(t, K.s[i]));
        tt = fma(t.x, t.x, fma(t.y, t.y, tt));
    }
    const double2 a = block_sum2<BT>(ts);
    const double2 b = block_sum2<BT>(make_double2(tt, 0));
    if (threadIdx.x == 0) {
        K.part[blockIdx.x] = a;
        K.part[K.nblk + blockIdx.x] = b;
    }
    if (!last_block(K.ticket + 2)) return;
    __shared__ double2 out[2];
    finish<2>(K, out);
    if (threadIdx.x == 0) {
        const double den = out[1].x;
        K.sc[S_OMEGA] = den > 0 ? make_double2(out[0].x / den, out[0].y / den) : make_double2(0, 0);
        if (!(den > 0)) K.sc[S_FLAG] = make_double2(1, 0);
    }
}

// x += alpha p + omega s; r = s - omega t; rho' = (rhat, r); |r|^2
__global__ void __launch_bounds__(BT) bg_x(BG K, double2 *__restrict__ x)
{
    const double2 al = K.sc[S_ALPHA], om = K.sc[S_OMEGA];
    const int i0 = blockIdx.x * K.rows, i1 = min(K.n, i0 + K.rows);
    double2 rho = make_double2(0, 0);
    double nrm = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += BT) {
        const double2 s = K.s[i];
        const double2 ap = cm(al, K.p[i]), os = cm(om, s), ot = cm(om, K.t[i]);
        x[i] = make_double2(x[i].x + ap.x + os.x, x[i].y + ap.y + os.y);
        const double2 r = make_double2(s.x - ot.x, s.y - ot.y);
        K.r[i] = r;
        rho = zsum2(rho, cj(K.rhat[i], r));
        nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
    }
    const double2 a = block_sum2<BT>(rho);
    const double2 b = block_sum2<BT>(make_double2(nrm, 0));
    if (threadIdx.x == 0) {
        K.part[blockIdx.x] = a;
        K.part[K.nblk + blockIdx.x] = b;
    }
    if (!last_block(K.ticket + 3)) return;
    __shared__ double2 out[2];
    finish<2>(K, out);
    if (threadIdx.x == 0) {
        K.sc[S_RHO_OLD] = K.sc[S_RHO];
        K.sc[S_RHO] = out[0];
        K.sc[S_RNORM2] = out[1];
        if (out[0].x == 0.0 && out[0].y == 0.0) K.sc[S_FLAG] = make_double2(1, 0);
    }
}

}  // namespace
}  // namespace h2

using namespace h2;

struct BGWork {
    int n = 0;
    BG K{};
    double2 *tmp = nullptr;
    double2 *h_sc = nullptr;  // pinned copy of the scalars
    void *block = nullptr;
};

void h2_free_bicgstab(h2_handle *h)
{
    BGWork *w = reinterpret_cast<BGWork *>(h->bicgstab);
    if (!w) return;
    cudaFree(w->block);
    cudaFreeHost(w->h_sc);
    delete w;
    h->bicgstab = nullptr;
}

#define BGC(call)                                                                     \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

static h2_status bg_get(h2_handle *h, BGWork **out)
{
    BGWork *w = reinterpret_cast<BGWork *>(h->bicgstab);
    if (w) {
        *out = w;
        return H2_OK;
    }
    w = new BGWork();
    const int n = h->n;
    w->n = n;
    BG &K = w->K;
    K.n = n;
    K.nblk = std::max(1, std::min((n + BT - 1) / BT, 4 * 152));
    K.rows = ((n + K.nblk - 1) / K.nblk + 31) / 32 * 32;
    K.nblk = (n + K.rows - 1) / K.rows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    size_t ov[7];
    for (int q = 0; q < 7; ++q) ov[q] = take(sizeof(double2) * n);  // r rhat p v s t tmp
    const size_t op = take(sizeof(double2) * 2 * K.nblk);
    const size_t ot = take(sizeof(unsigned) * 4);
    const size_t osc = take(sizeof(double2) * S_COUNT);
    const size_t ox = take(sizeof(float2) * n), oy = take(sizeof(float2) * n);
    if (cudaMalloc(&w->block, off) != cudaSuccess || cudaMallocHost(&w->h_sc, sizeof(double2) * S_COUNT) != cudaSuccess) {
        cudaGetLastError();  // clear the out-of-memory result
        cudaFree(w->block);
        delete w;
        set_error("h2_bicgstab: workspace allocation failed");
        return H2_ERR_ALLOC;
    }
    char *base = reinterpret_cast<char *>(w->block);
    double2 **vec[7] = {&K.r, &K.rhat, &K.p, &K.v, &K.s, &K.t, &w->tmp};
    for (int q = 0; q < 7; ++q) *vec[q] = reinterpret_cast<double2 *>(base + ov[q]);
    K.part = reinterpret_cast<double2 *>(base + op);
    K.ticket = reinterpret_cast<unsigned *>(base + ot);
    K.sc = reinterpret_cast<double2 *>(base + osc);
    K.x32 = reinterpret_cast<float2 *>(base + ox);
    K.y32 = reinterpret_cast<float2 *>(base + oy);
    if (cudaMemset(K.ticket, 0, sizeof(unsigned) * 4) != cudaSuccess) {
        h->bicgstab = w;
        h2_free_bicgstab(h);
        return H2_ERR_CUDA;
    }
    h->bicgstab = w;
    *out = w;
    return H2_OK;
}

static h2_status bg_read(BGWork *w, cudaStream_t st)
{
    BGC(cudaMemcpyAsync(w->h_sc, w->K.sc, sizeof(double2) * S_COUNT, cudaMemcpyDeviceToHost, st));
    BGC(cudaStreamSynchronize(st));
    return H2_OK;
}

extern "C" h2_status h2_bicgstab(h2_handle *h, const void *b_, void *x_, int32_t nrhs, int64_t ld,
                                 const h2_solve_opts *opts, h2_solve_info *info, void *stream)
{
    if (!h || !b_ || !x_ || !opts) return (set_error("h2_bicgstab: NULL argument"), H2_ERR_ARG);
    if (nrhs < 1 || (nrhs > 1 && ld < h->n)) return (set_error("h2_bicgstab: bad nrhs/ld"), H2_ERR_ARG);
    if (opts->maxit < 1 || !(opts->tol > 0.0)) return (set_error("h2_bicgstab: need maxit >= 1, tol > 0"), H2_ERR_ARG);
    if (opts->precond) return (set_error("h2_bicgstab: no preconditioner in BiCGStab"), H2_ERR_ARG);
    if (opts->arnoldi != ARN_FP64 && opts->arnoldi != ARN_DF)
        return (set_error("h2_bicgstab: unknown residual arithmetic"), H2_ERR_ARG);
    h2::DeviceGuard dev_guard(h->device);
    BGC(dev_guard.err);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BGWork *w = nullptr;
    h2_status s = bg_get(h, &w);
    if (s != H2_OK) return s;
    BG &K = w->K;
    const int n = h->n;
    const dim3 vg(std::min(1024, (n + 255) / 256));
    const h2_prec acc = opts->arnoldi == ARN_DF ? H2_PREC_DFACC : H2_PREC_FP64ACC;
    h2_status worst = H2_OK;
    for (int32_t c = 0; c < nrhs; ++c) {
        const double2 *b = reinterpret_cast<const double2 *>(b_) + (int64_t)c * ld;
        double2 *x = reinterpret_cast<double2 *>(x_) + (int64_t)c * ld;
        h2_solve_info inf{};
        bg_start<<<K.nblk, BT, 0, st>>>(K, b, nullptr);
        BGC(cudaGetLastError());
        if ((s = bg_read(w, st)) != H2_OK) return s;
        const double bnorm = std::sqrt(w->h_sc[S_RNORM2].x);
        if (!opts->x0_given || bnorm == 0.0) BGC(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
        if (bnorm == 0.0) {
            if (info) info[c] = inf;
            continue;
        }
        // r = b - A x (or b)
        auto true_start = [&](bool x_zero) -> h2_status {
            if (x_zero) {
                bg_start<<<K.nblk, BT, 0, st>>>(K, b, nullptr);
            } else {
                h2_status e = h2_matvec(h, x, w->tmp, 1, n, acc, st);
                if (e != H2_OK) return e;
                bg_start<<<K.nblk, BT, 0, st>>>(K, b, w->tmp);
            }
            BGC(cudaGetLastError());
            return bg_read(w, st);
        };
        if ((s = true_start(!opts->x0_given)) != H2_OK) return s;
        double rel = std::sqrt(w->h_sc[S_RNORM2].x) / bnorm;
        int it = 0;
        h2_status rs = H2_OK;
        while (rel > opts->tol && it < opts->maxit) {
            bg_p<<<vg, 256, 0, st>>>(K);
            BGC(cudaGetLastError());
            if ((s = h2_matvec(h, K.x32, K.y32, 1, n, H2_PREC_FP32, st)) != H2_OK) return s;
            bg_v<<<K.nblk, BT, 0, st>>>(K);
            bg_s<<<vg, 256, 0, st>>>(K);
            BGC(cudaGetLastError());
            if ((s = h2_matvec(h, K.x32, K.y32, 1, n, H2_PREC_FP32, st)) != H2_OK) return s;
            bg_t<<<K.nblk, BT, 0, st>>>(K);
            bg_x<<<K.nblk, BT, 0, st>>>(K, x);
            BGC(cudaGetLastError());
            if ((s = bg_read(w, st)) != H2_OK) return s;
            ++it;
            rel = std::sqrt(w->h_sc[S_RNORM2].x) / bnorm;
            if (!std::isfinite(rel)) {
                rs = H2_ERR_BREAKDOWN;
                break;
            }
            const bool breakdown = w->h_sc[S_FLAG].x != 0.0;
            if (rel <= opts->tol || breakdown) {
                // decide by the true residual; restart from x when it is not small enough
                if (opts->refine || breakdown) {
                    if ((s = true_start(false)) != H2_OK) return s;
                    rel = std::sqrt(w->h_sc[S_RNORM2].x) / bnorm;
                    ++inf.restarts;
                }
            }
        }
        inf.iterations = it;
        inf.rel_res = rel;
        if (rs == H2_OK && !(rel <= opts->tol)) rs = H2_ERR_NOT_CONVERGED;
        inf.status = rs;
        if (info) info[c] = inf;
        if (rs != H2_OK && worst == H2_OK) worst = rs;
    }
    return worst;
}
