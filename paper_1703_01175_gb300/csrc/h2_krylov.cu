// Restarted GMRES(m) around the H^2 product, on the device.
//
// The paper solves with BiCGStab (Sec. V); here the Krylov solver is restarted
// GMRES (Saad & Schultz 1986): Arnoldi with classical Gram-Schmidt applied
// twice (CGS2) in FP64 on complex128 vectors, Givens rotations of the
// Hessenberg matrix and its least-squares solve on the device, and the H^2
// product in FP32 (c64) inside the Arnoldi steps. With `refine` every restart
// residual r = b - A x is formed with the FP64-accumulated product, so that the
// outer loop is an iterative refinement of the FP32 inner solves.
//
// Each Arnoldi step is three kernels after the product:
//   dot1   : w <- c128(A v_j); h1 = V_j^H w            (partial sums per block)
//   upd1   : w -= V_j h1; h2 = V_j^H w
//   upd2   : w -= V_j h2; |w|^2; Hessenberg column, Givens, residual estimate
// and the next basis vector v_{j+1} = w / |w| is written (with its c64 copy
// for the next product) by `normalize`. The partial sums of a reduction are
// combined by the last block to finish (a ticket counter), so no kernel waits
// for another inside a launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "h2_internal.h"

namespace h2 {

static constexpr int KT = 256;     // threads per block of the vector kernels

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconj_mul(double2 a, double2 b)  // conj(a) * b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ double2 warp_sum(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

struct KrylovDev {
    double2 *V;        // n x (m+1) basis, column-major, leading dimension n
    double2 *w;        // n
    double2 *part;     // nblk x (m+2) partial sums
    unsigned *ticket;  // 3 counters
    double2 *H;        // (m+1) x m, column-major
    double *cs;        // m
    double2 *sn;       // m
    double2 *g;        // m+1
    double2 *h1;       // m+1 (first Gram-Schmidt coefficients)
    double2 *h2;       // m+1
    double *scal;      // [0] beta (|w|), [1] residual estimate |g_{j+1}|, [2] flags (nonfinite)
    int n, m, nblk, rows;  // rows per block
};

// Block-level: partial[l] = sum over this block's rows of conj(V[i,l]) * w[i],
// for l < ncols, written to part[blockIdx.x * (m+2) + l].
__device__ void block_dots(const KrylovDev &K, const double2 *ws, int r0, int nr, int ncols, double2 *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = KT / 32;
    for (int l = 0; l < ncols; ++l) {
        const double2 *Vl = K.V + (size_t)l * K.n + r0;
        double2 acc = make_double2(0, 0);
        for (int i = threadIdx.x; i < nr; i += KT) acc = cadd(acc, cconj_mul(Vl[i], ws[i]));
        acc = warp_sum(acc);
        if (lane == 0) red[warp * (K.m + 2) + l] = acc;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < ncols; l += KT) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < NW; ++q) s = cadd(s, red[q * (K.m + 2) + l]);
        K.part[(size_t)blockIdx.x * (K.m + 2) + l] = s;
    }
}

// last block to arrive sums the partial sums over blocks into out[0..ncols)
__device__ bool last_block_reduce(const KrylovDev &K, unsigned *ticket, int ncols, double2 *out)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int l = threadIdx.x; l < ncols; l += KT) {
        double2 s = make_double2(0, 0);
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const volatile double2 *p = K.part + (size_t)b * (K.m + 2) + l;
            s.x += p->x;
            s.y += p->y;
        }
        out[l] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// w <- c128(y32); h1 = V[:, 0..j]^H w
__global__ void __launch_bounds__(KT) k_dot1(KrylovDev K, const float2 *__restrict__ y32, int j)
{
    extern __shared__ double2 sm[];
    double2 *ws = sm;                 // rows of this block
    double2 *red = sm + K.rows;       // NW x (m+2)
    const int r0 = blockIdx.x * K.rows;
    const int nr = max(0, min(K.rows, K.n - r0));
    for (int i = threadIdx.x; i < nr; i += KT) {
        const float2 v = y32[r0 + i];
        const double2 d = make_double2(v.x, v.y);
        ws[i] = d;
        K.w[r0 + i] = d;
    }
    __syncthreads();
    block_dots(K, ws, r0, nr, j + 1, red);
    last_block_reduce(K, K.ticket + 0, j + 1, K.h1);
}

// w -= V h ; then (second pass) partial dots of the updated w, or |w|^2
template <bool SECOND>
__global__ void __launch_bounds__(KT) k_update(KrylovDev K, int j)
{
    extern __shared__ double2 sm[];
    double2 *ws = sm;
    double2 *red = sm + K.rows;
    double2 *hs = red + (KT / 32) * (K.m + 2);
    const double2 *h = SECOND ? K.h2 : K.h1;
    for (int l = threadIdx.x; l <= j; l += KT) hs[l] = h[l];
    __syncthreads();
    const int r0 = blockIdx.x * K.rows;
    const int nr = max(0, min(K.rows, K.n - r0));
    double nrm = 0.0;
    for (int i = threadIdx.x; i < nr; i += KT) {
        double2 acc = K.w[r0 + i];
        for (int l = 0; l <= j; ++l) acc = csub(acc, cmul(K.V[(size_t)l * K.n + r0 + i], hs[l]));
        K.w[r0 + i] = acc;
        ws[i] = acc;
        nrm += acc.x * acc.x + acc.y * acc.y;
    }
    __syncthreads();
    if (!SECOND) {
        block_dots(K, ws, r0, nr, j + 1, red);
        last_block_reduce(K, K.ticket + 1, j + 1, K.h2);
        return;
    }
    // |w|^2 partial
    double2 v = warp_sum(make_double2(nrm, 0.0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < KT / 32; ++q) s += red[q].x;
        K.part[(size_t)blockIdx.x * (K.m + 2)] = make_double2(s, 0.0);
    }
    __shared__ double2 tot;
    if (!last_block_reduce(K, K.ticket + 2, 1, &tot)) return;
    __syncthreads();
    if (threadIdx.x != 0) return;
    // Hessenberg column j: h = h1 + h2, h_{j+1,j} = |w|
    const int m = K.m;
    double2 *Hj = K.H + (size_t)j * (m + 1);
    for (int l = 0; l <= j; ++l) Hj[l] = cadd(K.h1[l], K.h2[l]);
    const double beta = sqrt(tot.x);
    Hj[j + 1] = make_double2(beta, 0.0);
    K.scal[0] = beta;
    // previous rotations: [c s; -conj(s) c]
    for (int l = 0; l < j; ++l) {
        const double c = K.cs[l];
        const double2 s = K.sn[l];
        const double2 a = Hj[l], b = Hj[l + 1];
        Hj[l] = cadd(make_double2(c * a.x, c * a.y), cmul(s, b));
        Hj[l + 1] = csub(make_double2(c * b.x, c * b.y), cconj_mul(s, a));
    }
    // new rotation zeroing H[j+1, j]
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
        // s = (a / |a|) * conj(b) / nr, b = beta real
        s = make_double2(a.x / na * beta / nr2, a.y / na * beta / nr2);
    }
    K.cs[j] = c;
    K.sn[j] = s;
    Hj[j] = cadd(make_double2(c * a.x, c * a.y), make_double2(s.x * beta, s.y * beta));
    Hj[j + 1] = make_double2(0, 0);
    const double2 gj = K.g[j];
    K.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
    K.g[j] = make_double2(c * gj.x, c * gj.y);
    K.scal[1] = hypot(K.g[j + 1].x, K.g[j + 1].y);
    bool bad = !isfinite(beta) || !isfinite(K.scal[1]);
    K.scal[2] = bad ? 1.0 : 0.0;
}

// v_{j+1} = w / beta (c128 into V, c64 into x32)
__global__ void k_normalize(KrylovDev K, int jn, float2 *__restrict__ x32)
{
    const double beta = K.scal[0];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    double2 *Vn = K.V + (size_t)jn * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 v = K.w[i];
        const double2 q = make_double2(v.x * inv, v.y * inv);
        Vn[i] = q;
        x32[i] = make_float2((float)q.x, (float)q.y);
    }
}

// r = b - y (y may be NULL: r = b); partial |r|^2 -> scal[0] via last block
__global__ void __launch_bounds__(KT) k_residual(KrylovDev K, const double2 *__restrict__ b, const double2 *__restrict__ y,
                                                 double2 *__restrict__ r)
{
    __shared__ double2 red[KT / 32];
    double nrm = 0;
    for (int i = blockIdx.x * KT + threadIdx.x; i < K.n; i += gridDim.x * KT) {
        double2 v = b[i];
        if (y) v = csub(v, y[i]);
        r[i] = v;
        nrm += v.x * v.x + v.y * v.y;
    }
    double2 s = warp_sum(make_double2(nrm, 0));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < KT / 32; ++q) t += red[q].x;
        K.part[(size_t)blockIdx.x * (K.m + 2)] = make_double2(t, 0);
    }
    __shared__ double2 tot;
    if (!last_block_reduce(K, K.ticket + 2, 1, &tot)) return;
    __syncthreads();
    if (threadIdx.x == 0) K.scal[0] = sqrt(tot.x);
}

// start a cycle: V0 = r / beta, x32 = c64(V0), g = [beta, 0 ...]
__global__ void k_start(KrylovDev K, const double2 *__restrict__ r, float2 *__restrict__ x32)
{
    const double beta = K.scal[0];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 v = r[i];
        const double2 q = make_double2(v.x * inv, v.y * inv);
        K.V[i] = q;
        x32[i] = make_float2((float)q.x, (float)q.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int l = 0; l <= K.m; ++l) K.g[l] = make_double2(0, 0);
        K.g[0] = make_double2(beta, 0);
    }
}

// y = H(1:k,1:k)^{-1} g(1:k) by back substitution (stored in h1)
__global__ void k_backsolve(KrylovDev K, int k)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = K.m;
    for (int i = k - 1; i >= 0; --i) {
        double2 s = K.g[i];
        for (int l = i + 1; l < k; ++l) s = csub(s, cmul(K.H[(size_t)l * (m + 1) + i], K.h1[l]));
        const double2 d = K.H[(size_t)i * (m + 1) + i];
        const double den = d.x * d.x + d.y * d.y;
        K.h1[i] = den > 0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                          : make_double2(0, 0);
    }
}

// x += B(:, 0..k) y with B = V (GMRES) or Z (flexible GMRES)
__global__ void k_xupdate(KrylovDev K, const double2 *__restrict__ basis, int k, double2 *__restrict__ x)
{
    extern __shared__ double2 ys[];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = K.h1[l];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        double2 acc = x[i];
        for (int l = 0; l < k; ++l) acc = cadd(acc, cmul(basis[(size_t)l * K.n + i], ys[l]));
        x[i] = acc;
    }
}

__global__ void k_c128_to_c64(const double2 *__restrict__ a, float2 *__restrict__ b, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_c64_to_c128(const float2 *__restrict__ a, double2 *__restrict__ b, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b[i] = make_double2(a[i].x, a[i].y);
}

}  // namespace h2

using namespace h2;

struct KrylovWork {
    int n = 0, m = 0;
    bool flexible = false;
    double2 *Z = nullptr;      // preconditioned directions (flexible GMRES)
    KrylovDev K{};
    double2 *r = nullptr, *tmp = nullptr;
    float2 *x32 = nullptr, *y32 = nullptr;
    double *h_scal = nullptr;  // pinned host copy of scal[0..2]
    void *block = nullptr;     // one device allocation for everything
};

static void free_work(KrylovWork *w)
{
    if (!w) return;
    cudaFree(w->block);
    cudaFreeHost(w->h_scal);
    delete w;
}

static h2_status get_work(h2_handle *h, int m, bool flexible, KrylovWork **out)
{
    KrylovWork *w = reinterpret_cast<KrylovWork *>(h->krylov);
    if (w && w->m == m && w->flexible == flexible) {
        *out = w;
        return H2_OK;
    }
    free_work(w);
    h->krylov = nullptr;
    w = new KrylovWork();
    const int n = h->n;
    w->n = n;
    w->m = m;
    w->flexible = flexible;
    // rows per block: enough blocks to fill the GPU, at most 2048 rows each
    int nblk = std::max(1, std::min((n + KT - 1) / KT, 2 * 152 * 2));
    int rows = (n + nblk - 1) / nblk;
    if (rows > 2048) {
        rows = 2048;
        nblk = (n + rows - 1) / rows;
    }
    rows = (rows + 31) / 32 * 32;
    nblk = (n + rows - 1) / rows;
    KrylovDev &K = w->K;
    K.n = n;
    K.m = m;
    K.nblk = nblk;
    K.rows = rows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oV = take(sizeof(double2) * (size_t)n * (m + 1));
    const size_t ow = take(sizeof(double2) * n);
    const size_t op = take(sizeof(double2) * (size_t)nblk * (m + 2));
    const size_t ot = take(sizeof(unsigned) * 4);
    const size_t oH = take(sizeof(double2) * (size_t)(m + 1) * m);
    const size_t oc = take(sizeof(double) * m);
    const size_t os = take(sizeof(double2) * m);
    const size_t og = take(sizeof(double2) * (m + 1));
    const size_t oh1 = take(sizeof(double2) * (m + 1));
    const size_t oh2 = take(sizeof(double2) * (m + 1));
    const size_t osc = take(sizeof(double) * 4);
    const size_t orr = take(sizeof(double2) * n);
    const size_t otm = take(sizeof(double2) * n);
    const size_t ox = take(sizeof(float2) * n);
    const size_t oy = take(sizeof(float2) * n);
    const size_t oz = flexible ? take(sizeof(double2) * (size_t)n * m) : 0;
    if (cudaMalloc(&w->block, off) != cudaSuccess || cudaMallocHost(&w->h_scal, 4 * sizeof(double)) != cudaSuccess) {
        free_work(w);
        set_error("h2_gmres: workspace allocation failed");
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
    K.h1 = reinterpret_cast<double2 *>(base + oh1);
    K.h2 = reinterpret_cast<double2 *>(base + oh2);
    K.scal = reinterpret_cast<double *>(base + osc);
    w->r = reinterpret_cast<double2 *>(base + orr);
    w->tmp = reinterpret_cast<double2 *>(base + otm);
    w->x32 = reinterpret_cast<float2 *>(base + ox);
    w->y32 = reinterpret_cast<float2 *>(base + oy);
    w->Z = flexible ? reinterpret_cast<double2 *>(base + oz) : nullptr;
    if (cudaMemset(K.ticket, 0, 4 * sizeof(unsigned)) != cudaSuccess) {
        free_work(w);
        return H2_ERR_CUDA;
    }
    h->krylov = w;
    *out = w;
    return H2_OK;
}

void h2_free_krylov(h2_handle *h)
{
    free_work(reinterpret_cast<KrylovWork *>(h->krylov));
    h->krylov = nullptr;
}

#define KCUDA(call)                                                                   \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

static h2_status read_scal(KrylovWork *w, cudaStream_t st)
{
    KCUDA(cudaMemcpyAsync(w->h_scal, w->K.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KCUDA(cudaStreamSynchronize(st));
    return H2_OK;
}

// r = b - A x (x, b: c128); FP64-accumulated product when `refine`, else the FP32 product.
static h2_status true_residual(h2_handle *h, KrylovWork *w, const double2 *b, const double2 *x, bool x_zero,
                               bool refine, cudaStream_t st)
{
    const int n = h->n;
    const int vb = std::min(1024, (n + 255) / 256);
    if (x_zero) {
        k_residual<<<w->K.nblk, KT, 0, st>>>(w->K, b, nullptr, w->r);
        KCUDA(cudaGetLastError());
        return H2_OK;
    }
    if (refine) {
        h2_status s = h2_matvec(h, x, w->tmp, 1, n, H2_PREC_FP64ACC, st);
        if (s != H2_OK) return s;
    } else {
        k_c128_to_c64<<<vb, 256, 0, st>>>(x, w->x32, n);
        h2_status s = h2_matvec(h, w->x32, w->y32, 1, n, H2_PREC_FP32, st);
        if (s != H2_OK) return s;
        k_c64_to_c128<<<vb, 256, 0, st>>>(w->y32, w->tmp, n);
    }
    k_residual<<<w->K.nblk, KT, 0, st>>>(w->K, b, w->tmp, w->r);
    KCUDA(cudaGetLastError());
    return H2_OK;
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
    KCUDA(cudaSetDevice(h->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    KrylovWork *w = nullptr;
    h2_status s = get_work(h, m, flexible, &w);
    if (s != H2_OK) return s;
    KrylovDev &K = w->K;
    const int n = h->n;
    const int vb = std::min(1024, (n + 255) / 256);
    const size_t smem_dot = sizeof(double2) * (K.rows + (KT / 32) * (m + 2));
    const size_t smem_upd = smem_dot + sizeof(double2) * (m + 1);
    KCUDA(cudaFuncSetAttribute(k_dot1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));
    KCUDA(cudaFuncSetAttribute(k_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));
    KCUDA(cudaFuncSetAttribute(k_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd));
    h2_status worst = H2_OK;
    for (int32_t c = 0; c < nrhs; ++c) {
        const double2 *b = reinterpret_cast<const double2 *>(b_) + (int64_t)c * ld;
        double2 *x = reinterpret_cast<double2 *>(x_) + (int64_t)c * ld;
        h2_solve_info inf{};
        // ||b||
        k_residual<<<K.nblk, KT, 0, st>>>(K, b, nullptr, w->r);
        KCUDA(cudaGetLastError());
        if ((s = read_scal(w, st)) != H2_OK) return s;
        const double bnorm = w->h_scal[0];
        if (!opts->x0_given) KCUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
        if (bnorm == 0.0) {
            KCUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
            inf.rel_res = 0.0;
            inf.status = H2_OK;
            if (info) info[c] = inf;
            continue;
        }
        bool x_zero = !opts->x0_given;
        if ((s = true_residual(h, w, b, x, x_zero, opts->refine != 0, st)) != H2_OK) return s;
        if ((s = read_scal(w, st)) != H2_OK) return s;
        double beta = w->h_scal[0];
        int it = 0;
        h2_status rs = H2_OK;
        bool pc = flexible;  // preconditioned cycles until one stagnates, then plain GMRES
        while (beta / bnorm > opts->tol && it < opts->maxit) {
            const double beta_start = beta;
            k_start<<<vb, 256, 0, st>>>(K, w->r, w->x32);
            KCUDA(cudaGetLastError());
            if (pc && (s = h2_apply_precond(h, K.V, w->Z, w->x32, st)) != H2_OK) return s;
            int j = 0, k = 0;
            for (j = 0; j < m && it < opts->maxit; ++j) {
                if ((s = h2_matvec(h, w->x32, w->y32, 1, n, H2_PREC_FP32, st)) != H2_OK) return s;
                k_dot1<<<K.nblk, KT, smem_dot, st>>>(K, w->y32, j);
                k_update<false><<<K.nblk, KT, smem_upd, st>>>(K, j);
                k_update<true><<<K.nblk, KT, smem_upd, st>>>(K, j);
                KCUDA(cudaGetLastError());
                ++it;
                k = j + 1;
                if ((s = read_scal(w, st)) != H2_OK) return s;
                if (w->h_scal[2] != 0.0) {
                    rs = H2_ERR_BREAKDOWN;
                    break;
                }
                const double est = w->h_scal[1];
                const bool lucky = w->h_scal[0] <= 1e-14 * bnorm;
                if (est <= 0.5 * opts->tol * bnorm || lucky) break;
                if (j + 1 < m) {
                    k_normalize<<<vb, 256, 0, st>>>(K, j + 1, w->x32);
                    KCUDA(cudaGetLastError());
                    if (pc && (s = h2_apply_precond(h, K.V + (size_t)(j + 1) * n, w->Z + (size_t)(j + 1) * n,
                                                    w->x32, st)) != H2_OK)
                        return s;
                }
            }
            if (rs != H2_OK) break;
            k_backsolve<<<1, 32, 0, st>>>(K, k);
            k_xupdate<<<vb, 256, sizeof(double2) * (m + 1), st>>>(K, pc ? w->Z : K.V, k, x);
            KCUDA(cudaGetLastError());
            ++inf.restarts;
            if (pc) ++inf.precond_cycles;
            if ((s = true_residual(h, w, b, x, false, opts->refine != 0, st)) != H2_OK) return s;
            if ((s = read_scal(w, st)) != H2_OK) return s;
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
