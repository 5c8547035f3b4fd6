// Batched restarted GMRES(m): R right-hand sides advance in lockstep, so every
// Arnoldi step needs ONE multi-RHS H^2 product (FP32 CUDA-core GEMMs or the
// split-bf16 tensor-core path) instead of R single products. Each right-hand
// side keeps its own Krylov basis, Hessenberg matrix and Givens rotations;
// the Gram-Schmidt passes (CGS2), the rotations and the back-substitution run
// in FP64 on the device in kernels batched over the right-hand sides
// (blockIdx.y = right-hand side). Restart residuals are recomputed with the
// FP64-accumulated product when `refine` (iterative refinement), else with the
// batched FP32 product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "h2_internal.h"

namespace h2 {
namespace {

constexpr int BT = 256;

__device__ __forceinline__ double2 bmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 bcmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ double2 badd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 bsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 bwsum(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

struct BK {
    double2 *V;       // [(m+1)][R][n]
    double2 *w;       // [R][n]
    double2 *part;    // [R][nblk][m+2]
    unsigned *ticket; // [R][3]
    double2 *H;       // [R][(m+1) m]
    double *cs;       // [R][m]
    double2 *sn;      // [R][m]
    double2 *g;       // [R][m+1]
    double2 *h1, *h2; // [R][m+1]
    double *scal;     // [R][4]: beta, estimate, flag
    int *kact;        // [R]: columns used at the end of a cycle
    int n, m, R, nblk, rows;
    __device__ double2 *Vc(int l, int r) const { return V + ((size_t)l * R + r) * n; }
    __device__ double2 *P(int r) const { return part + (size_t)r * nblk * (m + 2); }
};

__device__ void bdots(const BK &K, int r, const double2 *ws, int r0, int nr, int ncols, double2 *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = 0; l < ncols; ++l) {
        const double2 *Vl = K.Vc(l, r) + r0;
        double2 acc = make_double2(0, 0);
        for (int i = threadIdx.x; i < nr; i += BT) acc = badd(acc, bcmul(Vl[i], ws[i]));
        acc = bwsum(acc);
        if (lane == 0) red[warp * (K.m + 2) + l] = acc;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < ncols; l += BT) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < BT / 32; ++q) s = badd(s, red[q * (K.m + 2) + l]);
        K.P(r)[(size_t)blockIdx.x * (K.m + 2) + l] = s;
    }
}

__device__ bool blast(const BK &K, int r, int which, int ncols, double2 *out)
{
    __shared__ bool last;
    unsigned *ticket = K.ticket + 3 * r + which;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int l = threadIdx.x; l < ncols; l += BT) {
        double2 s = make_double2(0, 0);
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const volatile double2 *p = K.P(r) + (size_t)b * (K.m + 2) + l;
            s.x += p->x;
            s.y += p->y;
        }
        out[l] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__global__ void __launch_bounds__(BT) bk_dot1(BK K, const float2 *__restrict__ y32, int j)
{
    extern __shared__ double2 sm[];
    const int r = blockIdx.y;
    double2 *ws = sm, *red = sm + K.rows;
    const int r0 = blockIdx.x * K.rows, nr = max(0, min(K.rows, K.n - r0));
    double2 *w = K.w + (size_t)r * K.n;
    const float2 *y = y32 + (size_t)r * K.n;
    for (int i = threadIdx.x; i < nr; i += BT) {
        const float2 v = y[r0 + i];
        const double2 d = make_double2(v.x, v.y);
        ws[i] = d;
        w[r0 + i] = d;
    }
    __syncthreads();
    bdots(K, r, ws, r0, nr, j + 1, red);
    blast(K, r, 0, j + 1, K.h1 + (size_t)r * (K.m + 1));
}

template <bool SECOND>
__global__ void __launch_bounds__(BT) bk_update(BK K, int j)
{
    extern __shared__ double2 sm[];
    const int r = blockIdx.y;
    const int m = K.m;
    double2 *ws = sm, *red = sm + K.rows, *hs = red + (BT / 32) * (m + 2);
    const double2 *h = (SECOND ? K.h2 : K.h1) + (size_t)r * (m + 1);
    for (int l = threadIdx.x; l <= j; l += BT) hs[l] = h[l];
    __syncthreads();
    const int r0 = blockIdx.x * K.rows, nr = max(0, min(K.rows, K.n - r0));
    double2 *w = K.w + (size_t)r * K.n;
    double nrm = 0;
    for (int i = threadIdx.x; i < nr; i += BT) {
        double2 acc = w[r0 + i];
        for (int l = 0; l <= j; ++l) acc = bsub(acc, bmul(K.Vc(l, r)[r0 + i], hs[l]));
        w[r0 + i] = acc;
        ws[i] = acc;
        nrm += acc.x * acc.x + acc.y * acc.y;
    }
    __syncthreads();
    if (!SECOND) {
        bdots(K, r, ws, r0, nr, j + 1, red);
        blast(K, r, 1, j + 1, K.h2 + (size_t)r * (m + 1));
        return;
    }
    double2 v = bwsum(make_double2(nrm, 0.0));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < BT / 32; ++q) s += red[q].x;
        K.P(r)[(size_t)blockIdx.x * (m + 2)] = make_double2(s, 0.0);
    }
    __shared__ double2 tot;
    if (!blast(K, r, 2, 1, &tot)) return;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double2 *Hj = K.H + (size_t)r * (m + 1) * m + (size_t)j * (m + 1);
    const double2 *h1 = K.h1 + (size_t)r * (m + 1), *h2 = K.h2 + (size_t)r * (m + 1);
    double *cs = K.cs + (size_t)r * m;
    double2 *sn = K.sn + (size_t)r * m, *g = K.g + (size_t)r * (m + 1);
    double *sc = K.scal + 4 * r;
    for (int l = 0; l <= j; ++l) Hj[l] = badd(h1[l], h2[l]);
    const double beta = sqrt(tot.x);
    sc[0] = beta;
    for (int l = 0; l < j; ++l) {
        const double c = cs[l];
        const double2 s = sn[l], a = Hj[l], b = Hj[l + 1];
        Hj[l] = badd(make_double2(c * a.x, c * a.y), bmul(s, b));
        Hj[l + 1] = bsub(make_double2(c * b.x, c * b.y), bcmul(s, a));
    }
    const double2 a = Hj[j];
    const double na = hypot(a.x, a.y);
    double c;
    double2 s;
    if (beta == 0.0) {
        c = 1.0;
        s = make_double2(0, 0);
    } else if (na == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
    } else {
        const double nr2 = hypot(na, beta);
        c = na / nr2;
        s = make_double2(a.x / na * beta / nr2, a.y / na * beta / nr2);
    }
    cs[j] = c;
    sn[j] = s;
    Hj[j] = badd(make_double2(c * a.x, c * a.y), make_double2(s.x * beta, s.y * beta));
    Hj[j + 1] = make_double2(0, 0);
    const double2 gj = g[j];
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
    sc[1] = hypot(g[j + 1].x, g[j + 1].y);
    sc[2] = (!isfinite(beta) || !isfinite(sc[1])) ? 1.0 : 0.0;
}

__global__ void bk_normalize(BK K, int jn, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[4 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    double2 *Vn = K.Vc(jn, r);
    const double2 *w = K.w + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 q = make_double2(w[i].x * inv, w[i].y * inv);
        Vn[i] = q;
        x[i] = make_float2((float)q.x, (float)q.y);
    }
}

// rr = b - y (y may be NULL); |rr| -> scal[4 r]
__global__ void __launch_bounds__(BT) bk_residual(BK K, const double2 *__restrict__ b, int64_t ldb,
                                                  const double2 *__restrict__ y, double2 *__restrict__ rr)
{
    __shared__ double2 red[BT / 32];
    const int r = blockIdx.y;
    double nrm = 0;
    for (int i = blockIdx.x * BT + threadIdx.x; i < K.n; i += gridDim.x * BT) {
        double2 v = b[(size_t)r * ldb + i];
        if (y) v = bsub(v, y[(size_t)r * K.n + i]);
        rr[(size_t)r * K.n + i] = v;
        nrm += v.x * v.x + v.y * v.y;
    }
    double2 s = bwsum(make_double2(nrm, 0));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < BT / 32; ++q) t += red[q].x;
        K.P(r)[(size_t)blockIdx.x * (K.m + 2)] = make_double2(t, 0);
    }
    __shared__ double2 tot;
    if (!blast(K, r, 2, 1, &tot)) return;
    __syncthreads();
    if (threadIdx.x == 0) K.scal[4 * r] = sqrt(tot.x);
}

__global__ void bk_start(BK K, const double2 *__restrict__ rr, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[4 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    double2 *V0 = K.Vc(0, r);
    const double2 *v = rr + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 q = make_double2(v[i].x * inv, v[i].y * inv);
        V0[i] = q;
        x[i] = make_float2((float)q.x, (float)q.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double2 *g = K.g + (size_t)r * (K.m + 1);
        for (int l = 0; l <= K.m; ++l) g[l] = make_double2(0, 0);
        g[0] = make_double2(beta, 0);
    }
}

__global__ void bk_backsolve(BK K)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= K.R) return;
    const int m = K.m, k = K.kact[r];
    const double2 *H = K.H + (size_t)r * (m + 1) * m, *g = K.g + (size_t)r * (m + 1);
    double2 *y = K.h1 + (size_t)r * (m + 1);
    for (int i = k - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int l = i + 1; l < k; ++l) s = bsub(s, bmul(H[(size_t)l * (m + 1) + i], y[l]));
        const double2 d = H[(size_t)i * (m + 1) + i];
        const double den = d.x * d.x + d.y * d.y;
        y[i] = den > 0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                       : make_double2(0, 0);
    }
}

__global__ void bk_xupdate(BK K, double2 *__restrict__ x, int64_t ldx)
{
    extern __shared__ double2 ys[];
    const int r = blockIdx.y;
    const int k = K.kact[r];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = K.h1[(size_t)r * (K.m + 1) + l];
    __syncthreads();
    if (k == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        double2 acc = x[(size_t)r * ldx + i];
        for (int l = 0; l < k; ++l) acc = badd(acc, bmul(K.Vc(l, r)[i], ys[l]));
        x[(size_t)r * ldx + i] = acc;
    }
}

__global__ void bk_to_c64(const double2 *__restrict__ a, int64_t lda, float2 *__restrict__ b, int n)
{
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 v = a[(size_t)r * lda + i];
        b[(size_t)r * n + i] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void bk_to_c128(const float2 *__restrict__ a, double2 *__restrict__ b, int n)
{
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 v = a[(size_t)r * n + i];
        b[(size_t)r * n + i] = make_double2(v.x, v.y);
    }
}

}  // namespace
}  // namespace h2

using namespace h2;

struct BKWork {
    int n = 0, m = 0, R = 0;
    BK K{};
    double2 *rr = nullptr, *tmp = nullptr;
    float2 *x32 = nullptr, *y32 = nullptr;
    double *h_scal = nullptr;
    int *h_kact = nullptr;
    void *block = nullptr;
};

static void bk_free(BKWork *w)
{
    if (!w) return;
    cudaFree(w->block);
    cudaFreeHost(w->h_scal);
    cudaFreeHost(w->h_kact);
    delete w;
}

void h2_free_bkrylov(h2_handle *h)
{
    bk_free(reinterpret_cast<BKWork *>(h->bkrylov));
    h->bkrylov = nullptr;
}

static h2_status bk_get(h2_handle *h, int m, int R, BKWork **out)
{
    BKWork *w = reinterpret_cast<BKWork *>(h->bkrylov);
    if (w && w->m == m && w->R == R) {
        *out = w;
        return H2_OK;
    }
    h2_free_bkrylov(h);
    w = new BKWork();
    const int n = h->n;
    w->n = n;
    w->m = m;
    w->R = R;
    int nblk = std::max(1, std::min((n + BT - 1) / BT, 2 * 152));
    int rows = (n + nblk - 1) / nblk;
    if (rows > 2048) rows = 2048;
    rows = (rows + 31) / 32 * 32;
    nblk = (n + rows - 1) / rows;
    BK &K = w->K;
    K.n = n;
    K.m = m;
    K.R = R;
    K.nblk = nblk;
    K.rows = rows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oV = take(sizeof(double2) * (size_t)n * (m + 1) * R);
    const size_t ow = take(sizeof(double2) * (size_t)n * R);
    const size_t op = take(sizeof(double2) * (size_t)nblk * (m + 2) * R);
    const size_t ot = take(sizeof(unsigned) * 3 * R);
    const size_t oH = take(sizeof(double2) * (size_t)(m + 1) * m * R);
    const size_t oc = take(sizeof(double) * (size_t)m * R);
    const size_t os = take(sizeof(double2) * (size_t)m * R);
    const size_t og = take(sizeof(double2) * (size_t)(m + 1) * R);
    const size_t o1 = take(sizeof(double2) * (size_t)(m + 1) * R);
    const size_t o2 = take(sizeof(double2) * (size_t)(m + 1) * R);
    const size_t osc = take(sizeof(double) * 4 * R);
    const size_t ok = take(sizeof(int) * R);
    const size_t orr = take(sizeof(double2) * (size_t)n * R);
    const size_t otm = take(sizeof(double2) * (size_t)n * R);
    const size_t ox = take(sizeof(float2) * (size_t)n * R);
    const size_t oy = take(sizeof(float2) * (size_t)n * R);
    if (cudaMalloc(&w->block, off) != cudaSuccess || cudaMallocHost(&w->h_scal, 4 * sizeof(double) * R) != cudaSuccess ||
        cudaMallocHost(&w->h_kact, sizeof(int) * R) != cudaSuccess) {
        bk_free(w);
        set_error("h2_gmres_batched: workspace allocation failed (" + std::to_string(off >> 20) + " MiB)");
        return H2_ERR_ALLOC;
    }
    char *base = reinterpret_cast<char *>(w->block);
    K.V = reinterpret_cast<double2 *>(base + oV);
    K.w = reinterpret_cast<double2 *>(base + ow);
    K.part = reinterpret_cast<double2 *>(base + op);
    K.ticket = reinterpret_cast<unsigned *>(base + ot);
    K.H = reinterpret_cast<double2 *>(base + oH);
    K.cs = reinterpret_cast<double *>(base + oc);
    K.sn = reinterpret_cast<double2 *>(base + os);
    K.g = reinterpret_cast<double2 *>(base + og);
    K.h1 = reinterpret_cast<double2 *>(base + o1);
    K.h2 = reinterpret_cast<double2 *>(base + o2);
    K.scal = reinterpret_cast<double *>(base + osc);
    K.kact = reinterpret_cast<int *>(base + ok);
    w->rr = reinterpret_cast<double2 *>(base + orr);
    w->tmp = reinterpret_cast<double2 *>(base + otm);
    w->x32 = reinterpret_cast<float2 *>(base + ox);
    w->y32 = reinterpret_cast<float2 *>(base + oy);
    if (cudaMemset(K.ticket, 0, sizeof(unsigned) * 3 * R) != cudaSuccess) {
        bk_free(w);
        return H2_ERR_CUDA;
    }
    h->bkrylov = w;
    *out = w;
    return H2_OK;
}

#define BKC(call)                                                                     \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

static h2_status bk_read(BKWork *w, cudaStream_t st)
{
    BKC(cudaMemcpyAsync(w->h_scal, w->K.scal, 4 * sizeof(double) * w->R, cudaMemcpyDeviceToHost, st));
    BKC(cudaStreamSynchronize(st));
    return H2_OK;
}

// rr = b - A x for all right-hand sides; |rr| -> scal
static h2_status bk_true_residual(h2_handle *h, BKWork *w, const double2 *b, int64_t ldb, const double2 *x,
                                  int64_t ldx, bool refine, h2_prec prec, cudaStream_t st)
{
    const int n = h->n, R = w->R;
    dim3 vg(std::min(1024, (n + 255) / 256), R);
    if (refine) {
        for (int r = 0; r < R; ++r) {
            h2_status s = h2_matvec(h, x + (size_t)r * ldx, w->tmp + (size_t)r * n, 1, n, H2_PREC_FP64ACC, st);
            if (s != H2_OK) return s;
        }
    } else {
        bk_to_c64<<<vg, 256, 0, st>>>(x, ldx, w->x32, n);
        h2_status s = h2_matvec(h, w->x32, w->y32, R, n, prec, st);
        if (s != H2_OK) return s;
        bk_to_c128<<<vg, 256, 0, st>>>(w->y32, w->tmp, n);
    }
    bk_residual<<<dim3(w->K.nblk, R), BT, 0, st>>>(w->K, b, ldb, w->tmp, w->rr);
    BKC(cudaGetLastError());
    return H2_OK;
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
    if (opts->precond) return (set_error("h2_gmres_batched: no preconditioner in the batched solver"), H2_ERR_ARG);
    BKC(cudaSetDevice(h->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BKWork *w = nullptr;
    h2_status s = bk_get(h, m, nrhs, &w);
    if (s != H2_OK) return s;
    BK &K = w->K;
    const int n = h->n, R = nrhs;
    const double2 *b = reinterpret_cast<const double2 *>(b_);
    double2 *x = reinterpret_cast<double2 *>(x_);
    const dim3 vg(std::min(1024, (n + 255) / 256), R);
    const dim3 bg(K.nblk, R);
    const size_t smem_dot = sizeof(double2) * (K.rows + (BT / 32) * (m + 2));
    const size_t smem_upd = smem_dot + sizeof(double2) * (m + 1);
    BKC(cudaFuncSetAttribute(bk_dot1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));
    BKC(cudaFuncSetAttribute(bk_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));
    BKC(cudaFuncSetAttribute(bk_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));

    // |b|
    bk_residual<<<bg, BT, 0, st>>>(K, b, ld, nullptr, w->rr);
    BKC(cudaGetLastError());
    if ((s = bk_read(w, st)) != H2_OK) return s;
    std::vector<double> bnorm(R), beta(R);
    std::vector<h2_solve_info> inf(R);
    for (int r = 0; r < R; ++r) bnorm[r] = w->h_scal[4 * r];
    if (!opts->x0_given)
        for (int r = 0; r < R; ++r) BKC(cudaMemsetAsync(x + (size_t)r * ld, 0, sizeof(double2) * n, st));
    if ((s = bk_true_residual(h, w, b, ld, x, ld, opts->refine != 0, prec, st)) != H2_OK) return s;
    if ((s = bk_read(w, st)) != H2_OK) return s;
    std::vector<char> active(R);
    auto update_active = [&]() {
        int na = 0;
        for (int r = 0; r < R; ++r) {
            beta[r] = w->h_scal[4 * r];
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
    while (update_active() > 0 && it < opts->maxit) {
        bk_start<<<vg, 256, 0, st>>>(K, w->rr, w->x32);
        BKC(cudaGetLastError());
        std::fill(conv.begin(), conv.end(), -1);
        int j = 0, k = 0;
        for (j = 0; j < m && it < opts->maxit; ++j) {
            if ((s = h2_matvec(h, w->x32, w->y32, R, n, prec, st)) != H2_OK) return s;
            bk_dot1<<<bg, BT, smem_dot, st>>>(K, w->y32, j);
            bk_update<false><<<bg, BT, smem_upd, st>>>(K, j);
            bk_update<true><<<bg, BT, smem_upd, st>>>(K, j);
            BKC(cudaGetLastError());
            ++it;
            k = j + 1;
            if ((s = bk_read(w, st)) != H2_OK) return s;
            bool all = true;
            for (int r = 0; r < R; ++r) {
                if (!active[r] || conv[r] >= 0) continue;
                const double est = w->h_scal[4 * r + 1];
                const bool lucky = w->h_scal[4 * r] <= 1e-14 * bnorm[r];
                if (w->h_scal[4 * r + 2] != 0.0 || est <= 0.5 * opts->tol * bnorm[r] || lucky) conv[r] = k;
                else all = false;
            }
            if (all) break;
            if (j + 1 < m) {
                bk_normalize<<<vg, 256, 0, st>>>(K, j + 1, w->x32);
                BKC(cudaGetLastError());
            }
        }
        for (int r = 0; r < R; ++r) {
            w->h_kact[r] = active[r] ? (conv[r] >= 0 ? conv[r] : k) : 0;
            if (active[r]) {
                inf[r].iterations += w->h_kact[r];
                ++inf[r].restarts;
            }
        }
        BKC(cudaMemcpyAsync(K.kact, w->h_kact, sizeof(int) * R, cudaMemcpyHostToDevice, st));
        bk_backsolve<<<(R + 127) / 128, 128, 0, st>>>(K);
        bk_xupdate<<<vg, 256, sizeof(double2) * (m + 1), st>>>(K, x, ld);
        BKC(cudaGetLastError());
        if ((s = bk_true_residual(h, w, b, ld, x, ld, opts->refine != 0, prec, st)) != H2_OK) return s;
        if ((s = bk_read(w, st)) != H2_OK) return s;
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
