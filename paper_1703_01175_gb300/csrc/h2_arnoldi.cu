// FP64 Arnoldi process of restarted GMRES for R right-hand sides at once
// (R = 1 for the single-RHS solver). Each right-hand side owns its Krylov
// basis, Hessenberg matrix and Givens rotations; every kernel is batched over
// the right-hand sides with blockIdx.y = right-hand side.
//
// Orthogonalisation is classical Gram-Schmidt with selective
// reorthogonalisation (Daniel, Gragg, Kaufman & Stewart 1976): after one
// projection w' = w - V (V^H w), a second projection runs only when
// |w'| < eta |w| (eta = 1/sqrt(2) by default), i.e. when cancellation may have
// cost orthogonality: one projection leaves w' orthogonal to V to about
// u |w| / |w'| <= u / eta (u the unit roundoff).
// With no reorthogonalisation the step reads the basis twice (one dot pass,
// one update pass) instead of the four reads of CGS applied twice.
//
// Dot pass V^H w: one block per (basis column, row segment), so each block
// streams a long contiguous run of one column and reduces inside the block;
// only (columns x segments) partial sums remain, and the segment count shrinks
// as the basis grows (one segment per column once the grid is full). Update
// pass w - V h: blocks over rows, each thread sweeps the basis for its rows.
// Cross-block sums are combined in a fixed order by the last block to finish
// (a ticket counter), so results are bitwise reproducible.
//
// The small dense part of GMRES (Hessenberg column, Givens rotations,
// residual estimate, back-substitution) runs in FP64 on the host: each step
// already synchronises to test convergence, the coefficients of a step are a
// few kilobytes, and a sequential rotation sweep on one GPU thread would sit
// on GB300's narrow FP64 pipe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <string>

#include "h2_df.cuh"
#include "h2_reduce.cuh"
#include "h2_internal.h"

namespace h2 {
namespace {

constexpr int AT = 256;       // threads per block
constexpr int NW = AT / 32;
constexpr int TARGET = 4 * 152;       // blocks that fill the GPU (dot pass)
constexpr int TARGET_ROWS = 16 * 152; // blocks of the row-parallel passes (several resident per SM)

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 wsum(double2 v) { return warp_sum2(v); }
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }

__device__ __forceinline__ double2 block_sum(double2 v) { return block_sum2<AT>(v); }
__device__ __forceinline__ bool last_of_rhs(unsigned *ticket) { return last_block(ticket); }

__device__ __forceinline__ double2 vload(const volatile double2 *p)
{
    return make_double2(p->x, p->y);
}

// out[c] = sum_{s < S} part[c * S + s] for c < ncols (fixed order)
__device__ void reduce_columns(const double2 *part, int ncols, int S, double2 *out)
{
    const volatile double2 *p = part;
    if (S >= 8) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int c = warp; c < ncols; c += NW) {
            double2 a = make_double2(0, 0);
            for (int s = lane; s < S; s += 32) a = zadd(a, vload(p + (size_t)c * S + s));
            a = wsum(a);
            if (lane == 0) out[c] = a;
        }
    } else {
        for (int c = threadIdx.x; c < ncols; c += AT) {
            double2 a = make_double2(0, 0);
            for (int s = 0; s < S; ++s) a = zadd(a, vload(p + (size_t)c * S + s));
            out[c] = a;
        }
    }
    __syncthreads();
}

// conj(v) * w accumulated with four FMAs
__device__ __forceinline__ void cmac_conj(double2 &acc, double2 v, double2 w)
{
    acc.x = fma(v.x, w.x, acc.x);
    acc.x = fma(v.y, w.y, acc.x);
    acc.y = fma(v.x, w.y, acc.y);
    acc.y = fma(-v.y, w.x, acc.y);
}

// acc -= v * h with four FMAs
__device__ __forceinline__ void cmsub(double2 &acc, double2 v, double2 h)
{
    acc.x = fma(-v.x, h.x, acc.x);
    acc.x = fma(v.y, h.y, acc.x);
    acc.y = fma(-v.x, h.y, acc.y);
    acc.y = fma(-v.y, h.x, acc.y);
}

// w = c128(y32) (the product of the step, widened once)
__global__ void arn_widen(ArnDev K, const float2 *__restrict__ y32)
{
    const int r = blockIdx.y;
    const float2 *y = y32 + (size_t)r * K.n;
    double2 *w = K.w + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x)
        w[i] = make_double2(y[i].x, y[i].y);
}

// Dot pass: coefficients V^H w for columns 0..j. FIRST also forms |w|^2
// (pseudo-column j+1) into h1[j+1]; SECOND runs only for right-hand sides
// flagged for reorthogonalisation and writes h2.
template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_dot(ArnDev K, int j, int S, int seg)
{
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const int l = blockIdx.x / S, s = blockIdx.x - l * S;
    const int i0 = s * seg, i1 = min(K.n, i0 + seg);
    const double2 *w = K.w + (size_t)r * K.n;
    double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
    if (l <= j) {
        const double2 *Vl = K.V + ((size_t)l * K.R + r) * K.n;
        int i = i0 + threadIdx.x;
        for (; i + AT < i1; i += 2 * AT) {
            cmac_conj(acc0, ld_stream(Vl + i), w[i]);
            cmac_conj(acc1, ld_stream(Vl + i + AT), w[i + AT]);
        }
        if (i < i1) cmac_conj(acc0, ld_stream(Vl + i), w[i]);
    } else {  // FIRST only: |w|^2 over the segment
        for (int i = i0 + threadIdx.x; i < i1; i += AT) {
            const double2 v = w[i];
            acc0.x = fma(v.x, v.x, acc0.x);
            acc0.x = fma(v.y, v.y, acc0.x);
        }
    }
    const double2 tot = block_sum(zadd(acc0, acc1));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 2 : 0))) return;
    const int ncols = SECOND ? j + 1 : j + 2;
    reduce_columns(part, ncols, S, (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2));
}

// Update pass w -= V h (h = h1, or h2 in the second pass). The last block
// forms |w|^2; the first pass decides whether the right-hand side needs the
// second projection (flag scal[3]); the pass that ends the step stores
// beta = |w| in scal[0]. Dynamic shared memory: m + 2 complex entries.
template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_update(ArnDev K, int j, int rows)
{
    extern __shared__ double2 hs[];
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const double2 *h = (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2);
    for (int l = threadIdx.x; l <= j; l += AT) hs[l] = h[l];
    __syncthreads();
    const int i0 = blockIdx.x * rows, i1 = min(K.n, i0 + rows);
    double2 *w = K.w + (size_t)r * K.n;
    const double2 *V = K.V + (size_t)r * K.n;
    const size_t ldv = (size_t)K.R * K.n;
    double nrm = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += AT) {
        double2 acc = w[i];
        int l = 0;
        for (; l + 1 <= j; l += 2) {
            const double2 a = ld_stream(V + (size_t)l * ldv + i), b = ld_stream(V + (size_t)(l + 1) * ldv + i);
            cmsub(acc, a, hs[l]);
            cmsub(acc, b, hs[l + 1]);
        }
        if (l <= j) cmsub(acc, ld_stream(V + (size_t)l * ldv + i), hs[l]);
        w[i] = acc;
        nrm = fma(acc.x, acc.x, nrm);
        nrm = fma(acc.y, acc.y, nrm);
    }
    const double2 tot = block_sum(make_double2(nrm, 0.0));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 3 : 1))) return;
    double s = 0.0;
    const volatile double2 *p = part;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += AT) s += p[b].x;
    const double nw2 = block_sum(make_double2(s, 0.0)).x;
    if (threadIdx.x != 0) return;
    if (!SECOND) {
        const double rho = K.h1[(size_t)r * (K.m + 2) + j + 1].x;  // |w|^2 before the projection
        const bool again = !(nw2 >= K.eta2 * rho);
        K.scal[8 * r + 3] = again ? 1.0 : 0.0;
        if (again) return;
    }
    K.scal[8 * r] = sqrt(nw2);
}

// v_{jn} = w / beta (c128 into the basis, c64 into x32 for the next product)
__global__ void arn_normalize(ArnDev K, int jn, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    double2 *Vn = K.V + ((size_t)jn * K.R + r) * K.n;
    const double2 *w = K.w + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 v = w[i];
        const double2 q = make_double2(v.x * inv, v.y * inv);
        Vn[i] = q;
        x[i] = make_float2((float)q.x, (float)q.y);
    }
}

// rr = b - y (y may be NULL); |rr| -> scal[8 r]
__global__ void __launch_bounds__(AT) arn_residual(ArnDev K, const double2 *__restrict__ b, int64_t ldb,
                                                   const double2 *__restrict__ y, double2 *__restrict__ rr, int rows)
{
    const int r = blockIdx.y;
    const int i0 = blockIdx.x * rows, i1 = min(K.n, i0 + rows);
    double nrm = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += AT) {
        double2 v = b[(size_t)r * ldb + i];
        if (y) v = zsub(v, y[(size_t)r * K.n + i]);
        rr[(size_t)r * K.n + i] = v;
        nrm += v.x * v.x + v.y * v.y;
    }
    const double2 tot = block_sum(make_double2(nrm, 0.0));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + 4)) return;
    double s = 0.0;
    const volatile double2 *p = part;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += AT) s += p[q].x;
    const double t = block_sum(make_double2(s, 0.0)).x;
    if (threadIdx.x == 0) K.scal[8 * r] = sqrt(t);
}

// start a cycle: v_0 = rr / beta, x32 = c64(v_0)
__global__ void arn_start(ArnDev K, const double2 *__restrict__ rr, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    double2 *V0 = K.V + (size_t)r * K.n;
    const double2 *v = rr + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double2 q = make_double2(v[i].x * inv, v[i].y * inv);
        V0[i] = q;
        x[i] = make_float2((float)q.x, (float)q.y);
    }
}

// x += B y with B = V (GMRES) or Z (flexible GMRES), B laid out like V; y in h1
__global__ void arn_xupdate(ArnDev K, const double2 *__restrict__ basis, double2 *__restrict__ x, int64_t ldx)
{
    extern __shared__ double2 ys[];
    const int r = blockIdx.y;
    const int k = K.kact[r];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = K.h1[(size_t)r * (K.m + 2) + l];
    __syncthreads();
    if (k == 0) return;
    const size_t ldb = (size_t)K.R * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        double2 acc = x[(size_t)r * ldx + i];
        for (int l = 0; l < k; ++l) acc = zadd(acc, zmul(basis[(size_t)l * ldb + (size_t)r * K.n + i], ys[l]));
        x[(size_t)r * ldx + i] = acc;
    }
}

// basis column j of every right-hand side as c128 ([R][n]), whatever the
// basis arithmetic: FP64 copy, c64 widened, double-float hi + lo
__global__ void arn_basis_c128_kernel(ArnDev K, int mode, int j, double2 *__restrict__ out)
{
    const int r = blockIdx.y;
    const size_t col = ((size_t)j * K.R + r) * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        double2 v;
        if (mode == ARN_F32) {
            const float2 a = reinterpret_cast<const float2 *>(K.V)[col + i];
            v = make_double2(a.x, a.y);
        } else if (mode == ARN_DF) {
            const float4 q = reinterpret_cast<const float4 *>(K.V)[col + i];
            v = make_double2((double)q.x + (double)q.z, (double)q.y + (double)q.w);
        } else {
            v = K.V[col + i];
        }
        out[(size_t)r * K.n + i] = v;
    }
}

__global__ void arn_to_c64(const double2 *__restrict__ a, int64_t lda, float2 *__restrict__ b, int n)
{
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 v = a[(size_t)r * lda + i];
        b[(size_t)r * n + i] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void arn_to_c128(const float2 *__restrict__ a, double2 *__restrict__ b, int n)
{
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 v = a[(size_t)r * n + i];
        b[(size_t)r * n + i] = make_double2(v.x, v.y);
    }
}

// ---------------------------------------------------------------------------
// Double-float variant. GB300's FP64 pipe issues about 1/58 of the FP32 rate,
// so the O(j n) passes can instead carry every value as an unevaluated sum
// hi + lo of two floats (a 48-bit significand) and run on the FP32 pipes:
// products are split exactly (TwoProd with an FMA), running sums keep their
// rounding error in a second float (TwoSum, Knuth), i.e. the compensated dot
// product of Ogita, Rump & Oishi (2005). Per-thread results are converted to
// FP64 before any cross-thread reduction, so reductions, norms and the
// least-squares solve stay in FP64. Basis and work vectors are stored as
// float4 (re hi, im hi, re lo, im lo): the same 16 bytes per entry as c128.
// All df arithmetic uses the _rn intrinsics, which are never contracted.

__device__ __forceinline__ float4 df_pack(double2 v)
{
    const float2 a = d_to_df(v.x), b = d_to_df(v.y);
    return make_float4(a.x, b.x, a.y, b.y);
}

__device__ __forceinline__ float4 ldcs4(const float4 *p) { return __ldcs(p); }

// conj(v) w into (sr, cr) + i (si, ci)
__device__ __forceinline__ void df_cmac_conj(float *a, float4 v, float4 w)
{
    df_mac(a[0], a[1], v.x, v.z, w.x, w.z);
    df_mac(a[0], a[1], v.y, v.w, w.y, w.w);
    df_mac(a[2], a[3], v.x, v.z, w.y, w.w);
    df_mac(a[2], a[3], -v.y, -v.w, w.x, w.z);
}

// acc -= v h
__device__ __forceinline__ void df_cmsub(float *a, float4 v, float4 h)
{
    df_mac(a[0], a[1], -v.x, -v.z, h.x, h.z);
    df_mac(a[0], a[1], v.y, v.w, h.y, h.w);
    df_mac(a[2], a[3], -v.x, -v.z, h.y, h.w);
    df_mac(a[2], a[3], -v.y, -v.w, h.x, h.z);
}

// w = y32 (exact in double-float)
__global__ void arn_widen_df(ArnDev K, const float2 *__restrict__ y32)
{
    const int r = blockIdx.y;
    const float2 *y = y32 + (size_t)r * K.n;
    float4 *w = reinterpret_cast<float4 *>(K.w) + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x)
        w[i] = make_float4(y[i].x, y[i].y, 0.f, 0.f);
}

// Dot pass in double-float: one block per (basis column, row segment); FIRST
// adds the pseudo-column |w|^2. (Pairing two columns per block, or four
// entries per thread in flight, measured slower on the 32^3 cube.)
template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_dot_df(ArnDev K, int j, int S, int seg)
{
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const int l = blockIdx.x / S, s = blockIdx.x - l * S;
    const int i0 = s * seg, i1 = min(K.n, i0 + seg);
    const float4 *w = reinterpret_cast<const float4 *>(K.w) + (size_t)r * K.n;
    float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
    if (l <= j) {
        const float4 *Vl = reinterpret_cast<const float4 *>(K.V) + ((size_t)l * K.R + r) * K.n;
        int i = i0 + threadIdx.x;
        for (; i + AT < i1; i += 2 * AT) {
            df_cmac_conj(a0, ldcs4(Vl + i), w[i]);
            df_cmac_conj(a1, ldcs4(Vl + i + AT), w[i + AT]);
        }
        if (i < i1) df_cmac_conj(a0, ldcs4(Vl + i), w[i]);
    } else {  // FIRST only: |w|^2 over the segment
        for (int i = i0 + threadIdx.x; i < i1; i += AT) {
            const float4 v = w[i];
            df_mac(a0[0], a0[1], v.x, v.z, v.x, v.z);
            df_mac(a0[0], a0[1], v.y, v.w, v.y, v.w);
        }
    }
    const double2 mine = make_double2(df_to_d(a0[0], a0[1]) + df_to_d(a1[0], a1[1]),
                                      df_to_d(a0[2], a0[3]) + df_to_d(a1[2], a1[3]));
    const double2 tot = block_sum(mine);
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 2 : 0))) return;
    const int ncols = SECOND ? j + 1 : j + 2;
    reduce_columns(part, ncols, S, (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2));
}

// Dynamic shared memory: m + 2 float4 entries.
template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_update_df(ArnDev K, int j, int rows)
{
    extern __shared__ float4 hsf[];
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const double2 *h = (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2);
    for (int l = threadIdx.x; l <= j; l += AT) hsf[l] = df_pack(h[l]);
    __syncthreads();
    const int i0 = blockIdx.x * rows, i1 = min(K.n, i0 + rows);
    float4 *w = reinterpret_cast<float4 *>(K.w) + (size_t)r * K.n;
    const float4 *V = reinterpret_cast<const float4 *>(K.V) + (size_t)r * K.n;
    const size_t ldv = (size_t)K.R * K.n;
    double nrm = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += AT) {
        const float4 w0 = w[i];
        float a[4] = {w0.x, w0.z, w0.y, w0.w};
        int l = 0;
        for (; l + 3 <= j; l += 4) {  // four basis loads in flight
            const float4 va = ldcs4(V + (size_t)l * ldv + i), vb = ldcs4(V + (size_t)(l + 1) * ldv + i);
            const float4 vc = ldcs4(V + (size_t)(l + 2) * ldv + i), vd = ldcs4(V + (size_t)(l + 3) * ldv + i);
            df_cmsub(a, va, hsf[l]);
            df_cmsub(a, vb, hsf[l + 1]);
            df_cmsub(a, vc, hsf[l + 2]);
            df_cmsub(a, vd, hsf[l + 3]);
        }
        for (; l <= j; ++l) df_cmsub(a, ldcs4(V + (size_t)l * ldv + i), hsf[l]);
        const float2 re = df_norm(a[0], a[1]), im = df_norm(a[2], a[3]);
        w[i] = make_float4(re.x, im.x, re.y, im.y);
        const double dr = df_to_d(re.x, re.y), di = df_to_d(im.x, im.y);
        nrm = fma(dr, dr, nrm);
        nrm = fma(di, di, nrm);
    }
    const double2 tot = block_sum(make_double2(nrm, 0.0));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 3 : 1))) return;
    double s = 0.0;
    const volatile double2 *p = part;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += AT) s += p[b].x;
    const double nw2 = block_sum(make_double2(s, 0.0)).x;
    if (threadIdx.x != 0) return;
    if (!SECOND) {
        const double rho = K.h1[(size_t)r * (K.m + 2) + j + 1].x;
        const bool again = !(nw2 >= K.eta2 * rho);
        K.scal[8 * r + 3] = again ? 1.0 : 0.0;
        if (again) return;
    }
    K.scal[8 * r] = sqrt(nw2);
}

// v_{jn} = w / beta in double-float; x32 = its high part
__global__ void arn_normalize_df(ArnDev K, int jn, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const float2 inv = d_to_df(beta > 0.0 ? 1.0 / beta : 0.0);
    float4 *Vn = reinterpret_cast<float4 *>(K.V) + ((size_t)jn * K.R + r) * K.n;
    const float4 *w = reinterpret_cast<const float4 *>(K.w) + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const float4 v = w[i];
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        df_mac(sr, cr, v.x, v.z, inv.x, inv.y);
        df_mac(si, ci, v.y, v.w, inv.x, inv.y);
        const float2 re = df_norm(sr, cr), im = df_norm(si, ci);
        Vn[i] = make_float4(re.x, im.x, re.y, im.y);
        x[i] = make_float2(re.x, im.x);
    }
}

// v_0 = rr / beta
__global__ void arn_start_df(ArnDev K, const double2 *__restrict__ rr, float2 *__restrict__ x32)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    float4 *V0 = reinterpret_cast<float4 *>(K.V) + (size_t)r * K.n;
    const double2 *v = rr + (size_t)r * K.n;
    float2 *x = x32 + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const float4 q = df_pack(make_double2(v[i].x * inv, v[i].y * inv));
        V0[i] = q;
        x[i] = make_float2(q.x, q.y);
    }
}

// x += V y (c128 x; df basis); dynamic shared memory: m + 2 float4 entries
__global__ void arn_xupdate_df(ArnDev K, double2 *__restrict__ x, int64_t ldx)
{
    extern __shared__ float4 ysf[];
    const int r = blockIdx.y;
    const int k = K.kact[r];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ysf[l] = df_pack(K.h1[(size_t)r * (K.m + 2) + l]);
    __syncthreads();
    if (k == 0) return;
    const size_t ldb = (size_t)K.R * K.n;
    const float4 *V = reinterpret_cast<const float4 *>(K.V) + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const float4 x0 = df_pack(x[(size_t)r * ldx + i]);
        float a[4] = {x0.x, x0.z, x0.y, x0.w};
        for (int l = 0; l < k; ++l) {
            const float4 v = V[(size_t)l * ldb + i], y = ysf[l];
            df_mac(a[0], a[1], v.x, v.z, y.x, y.z);
            df_mac(a[0], a[1], -v.y, -v.w, y.y, y.w);
            df_mac(a[2], a[3], v.x, v.z, y.y, y.w);
            df_mac(a[2], a[3], v.y, v.w, y.x, y.z);
        }
        x[(size_t)r * ldx + i] = make_double2(df_to_d(a[0], a[1]), df_to_d(a[2], a[3]));
    }
}

// ---------------------------------------------------------------------------
// Single-precision basis. Basis and work vector are stored as c64: 8 bytes
// per entry, half the traffic of the FP64 and double-float modes in both
// O(j n) passes. Products are FP32; each thread sums them in groups of four
// (plain FMAs) and adds every group into a compensated running sum (TwoSum),
// so its error stays a few units of FP32 rounding however long the sum is.
// Per-thread sums are converted to FP64 before any cross-thread reduction, so
// coefficients, norms and the least squares stay FP64, as in the other modes.
// The stored vectors carry FP32 rounding (2^-24 relative), which bounds the
// accuracy of the Arnoldi relation near 1e-7: the mode is for tolerances far
// above that (split-bf16 products are themselves accurate to about 1e-5).

__device__ __forceinline__ float2 ldcs2(const float2 *p) { return __ldcs(p); }

// (s, c) += t, compensated
__device__ __forceinline__ void csum(float &s, float &c, float t)
{
    float u, q;
    two_sum(s, t, u, q);
    s = u;
    c = __fadd_rn(c, q);
}

// Dot pass with a c64 basis: one block per (basis column, row segment), four
// entries per thread in flight; FIRST adds the pseudo-column |w|^2.
template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_dot_f32(ArnDev K, int j, int S, int seg)
{
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const int l = blockIdx.x / S, s = blockIdx.x - l * S;
    const int i0 = s * seg, i1 = min(K.n, i0 + seg);
    const float2 *w = reinterpret_cast<const float2 *>(K.w) + (size_t)r * K.n;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    if (l <= j) {
        const float2 *Vl = reinterpret_cast<const float2 *>(K.V) + ((size_t)l * K.R + r) * K.n;
        int i = i0 + threadIdx.x;
        for (; i + 3 * AT < i1; i += 4 * AT) {
            const float2 v0 = ldcs2(Vl + i), v1 = ldcs2(Vl + i + AT), v2 = ldcs2(Vl + i + 2 * AT),
                         v3 = ldcs2(Vl + i + 3 * AT);
            const float2 w0 = w[i], w1 = w[i + AT], w2 = w[i + 2 * AT], w3 = w[i + 3 * AT];
            float tr = v0.x * w0.x;   // conj(v) w, four entries
            tr = fmaf(v0.y, w0.y, tr);
            tr = fmaf(v1.x, w1.x, tr);
            tr = fmaf(v1.y, w1.y, tr);
            tr = fmaf(v2.x, w2.x, tr);
            tr = fmaf(v2.y, w2.y, tr);
            tr = fmaf(v3.x, w3.x, tr);
            tr = fmaf(v3.y, w3.y, tr);
            float ti = v0.x * w0.y;
            ti = fmaf(-v0.y, w0.x, ti);
            ti = fmaf(v1.x, w1.y, ti);
            ti = fmaf(-v1.y, w1.x, ti);
            ti = fmaf(v2.x, w2.y, ti);
            ti = fmaf(-v2.y, w2.x, ti);
            ti = fmaf(v3.x, w3.y, ti);
            ti = fmaf(-v3.y, w3.x, ti);
            csum(sr, cr, tr);
            csum(si, ci, ti);
        }
        for (; i < i1; i += AT) {
            const float2 v = ldcs2(Vl + i), x = w[i];
            csum(sr, cr, fmaf(v.y, x.y, v.x * x.x));
            csum(si, ci, fmaf(-v.y, x.x, v.x * x.y));
        }
    } else {  // FIRST only: |w|^2 over the segment
        for (int i = i0 + threadIdx.x; i < i1; i += AT) {
            const float2 x = w[i];
            csum(sr, cr, fmaf(x.y, x.y, x.x * x.x));
        }
    }
    const double2 tot = block_sum(make_double2(df_to_d(sr, cr), df_to_d(si, ci)));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 2 : 0))) return;
    const int ncols = SECOND ? j + 1 : j + 2;
    reduce_columns(part, ncols, S, (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2));
}

// w -= V h with a c64 basis: each thread owns two rows (adjacent ones as one
// float4 when n is even, else i and i + AT) and sweeps the basis four columns
// at a time (h shared by both rows), plain FMAs within a group, groups added
// compensated; |w'|^2 in FP64.
// Dynamic shared memory: m + 2 float2 entries.
__device__ __forceinline__ void f32_group(float &sr, float &cr, float &si, float &ci, float2 va, float2 vb, float2 vc,
                                          float2 vd, float2 ha, float2 hb, float2 hc, float2 hd)
{
    float tr = va.y * ha.y;   // -Re(v h), four columns
    tr = fmaf(-va.x, ha.x, tr);
    tr = fmaf(-vb.x, hb.x, tr);
    tr = fmaf(vb.y, hb.y, tr);
    tr = fmaf(-vc.x, hc.x, tr);
    tr = fmaf(vc.y, hc.y, tr);
    tr = fmaf(-vd.x, hd.x, tr);
    tr = fmaf(vd.y, hd.y, tr);
    float ti = -va.x * ha.y;  // -Im(v h)
    ti = fmaf(-va.y, ha.x, ti);
    ti = fmaf(-vb.x, hb.y, ti);
    ti = fmaf(-vb.y, hb.x, ti);
    ti = fmaf(-vc.x, hc.y, ti);
    ti = fmaf(-vc.y, hc.x, ti);
    ti = fmaf(-vd.x, hd.y, ti);
    ti = fmaf(-vd.y, hd.x, ti);
    csum(sr, cr, tr);
    csum(si, ci, ti);
}

template <bool SECOND>
__global__ void __launch_bounds__(AT) arn_update_f32(ArnDev K, int j, int rows)
{
    extern __shared__ float2 hs32[];
    const int r = blockIdx.y;
    if (SECOND && K.scal[8 * r + 3] == 0.0) return;
    const double2 *h = (SECOND ? K.h2 : K.h1) + (size_t)r * (K.m + 2);
    for (int l = threadIdx.x; l <= j; l += AT) hs32[l] = make_float2((float)h[l].x, (float)h[l].y);
    __syncthreads();
    const int i0 = blockIdx.x * rows, i1 = min(K.n, i0 + rows);
    float2 *w = reinterpret_cast<float2 *>(K.w) + (size_t)r * K.n;
    const float2 *V = reinterpret_cast<const float2 *>(K.V) + (size_t)r * K.n;
    const size_t ldv = (size_t)K.R * K.n;
    double nrm = 0.0;
    if ((K.n & 1) == 0) {
        // even n: every column starts on 16 bytes and row blocks on even rows, so
        // a thread takes rows 2p, 2p + 1 as one float4 (512 contiguous bytes per
        // column per warp)
        const float4 *V4 = reinterpret_cast<const float4 *>(V);
        const size_t ldv4 = ldv / 2;
        float4 *w4 = reinterpret_cast<float4 *>(w);
        for (int q = i0 / 2 + threadIdx.x; q < i1 / 2; q += AT) {
            const float4 w0 = w4[q];
            float sr0 = w0.x, cr0 = 0.f, si0 = w0.y, ci0 = 0.f;
            float sr1 = w0.z, cr1 = 0.f, si1 = w0.w, ci1 = 0.f;
            int l = 0;
            for (; l + 3 <= j; l += 4) {
                const float4 *c0 = V4 + (size_t)l * ldv4 + q;
                const float4 a = ldcs4(c0), b = ldcs4(c0 + ldv4), e = ldcs4(c0 + 2 * ldv4), d = ldcs4(c0 + 3 * ldv4);
                const float2 ha = hs32[l], hb = hs32[l + 1], hc = hs32[l + 2], hd = hs32[l + 3];
                f32_group(sr0, cr0, si0, ci0, make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(e.x, e.y),
                          make_float2(d.x, d.y), ha, hb, hc, hd);
                f32_group(sr1, cr1, si1, ci1, make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(e.z, e.w),
                          make_float2(d.z, d.w), ha, hb, hc, hd);
            }
            for (; l <= j; ++l) {
                const float4 v = ldcs4(V4 + (size_t)l * ldv4 + q);
                const float2 hh = hs32[l];
                csum(sr0, cr0, fmaf(v.y, hh.y, -v.x * hh.x));
                csum(si0, ci0, fmaf(-v.y, hh.x, -v.x * hh.y));
                csum(sr1, cr1, fmaf(v.w, hh.y, -v.z * hh.x));
                csum(si1, ci1, fmaf(-v.w, hh.x, -v.z * hh.y));
            }
            const float4 o = make_float4(__fadd_rn(sr0, cr0), __fadd_rn(si0, ci0), __fadd_rn(sr1, cr1),
                                         __fadd_rn(si1, ci1));
            w4[q] = o;
            nrm = fma((double)o.x, (double)o.x, nrm);
            nrm = fma((double)o.y, (double)o.y, nrm);
            nrm = fma((double)o.z, (double)o.z, nrm);
            nrm = fma((double)o.w, (double)o.w, nrm);
        }
    } else
    for (int i = i0 + threadIdx.x; i < i1; i += 2 * AT) {
        const bool two = i + AT < i1;
        const int k = two ? i + AT : i;   // without a second row, row i twice (result dropped)
        const float2 w0 = w[i], w1 = w[k];
        float sr0 = w0.x, cr0 = 0.f, si0 = w0.y, ci0 = 0.f;
        float sr1 = w1.x, cr1 = 0.f, si1 = w1.y, ci1 = 0.f;
        int l = 0;
        for (; l + 3 <= j; l += 4) {
            const float2 *c0 = V + (size_t)l * ldv, *c1 = c0 + ldv, *c2 = c1 + ldv, *c3 = c2 + ldv;
            const float2 a0 = ldcs2(c0 + i), b0 = ldcs2(c1 + i), e0 = ldcs2(c2 + i), d0 = ldcs2(c3 + i);
            const float2 a1 = ldcs2(c0 + k), b1 = ldcs2(c1 + k), e1 = ldcs2(c2 + k), d1 = ldcs2(c3 + k);
            const float2 ha = hs32[l], hb = hs32[l + 1], hc = hs32[l + 2], hd = hs32[l + 3];
            f32_group(sr0, cr0, si0, ci0, a0, b0, e0, d0, ha, hb, hc, hd);
            f32_group(sr1, cr1, si1, ci1, a1, b1, e1, d1, ha, hb, hc, hd);
        }
        for (; l <= j; ++l) {
            const float2 v0 = ldcs2(V + (size_t)l * ldv + i), v1 = ldcs2(V + (size_t)l * ldv + k), hh = hs32[l];
            csum(sr0, cr0, fmaf(v0.y, hh.y, -v0.x * hh.x));
            csum(si0, ci0, fmaf(-v0.y, hh.x, -v0.x * hh.y));
            csum(sr1, cr1, fmaf(v1.y, hh.y, -v1.x * hh.x));
            csum(si1, ci1, fmaf(-v1.y, hh.x, -v1.x * hh.y));
        }
        const float2 o0 = make_float2(__fadd_rn(sr0, cr0), __fadd_rn(si0, ci0));
        w[i] = o0;
        nrm = fma((double)o0.x, (double)o0.x, nrm);
        nrm = fma((double)o0.y, (double)o0.y, nrm);
        if (two) {
            const float2 o1 = make_float2(__fadd_rn(sr1, cr1), __fadd_rn(si1, ci1));
            w[k] = o1;
            nrm = fma((double)o1.x, (double)o1.x, nrm);
            nrm = fma((double)o1.y, (double)o1.y, nrm);
        }
    }
    const double2 tot = block_sum(make_double2(nrm, 0.0));
    double2 *part = K.part + (size_t)r * K.np;
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (!last_of_rhs(K.ticket + 8 * r + (SECOND ? 3 : 1))) return;
    double sum = 0.0;
    const volatile double2 *p = part;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += AT) sum += p[b].x;
    const double nw2 = block_sum(make_double2(sum, 0.0)).x;
    if (threadIdx.x != 0) return;
    if (!SECOND) {
        const double rho = K.h1[(size_t)r * (K.m + 2) + j + 1].x;
        const bool again = !(nw2 >= K.eta2 * rho);
        K.scal[8 * r + 3] = again ? 1.0 : 0.0;
        if (again) return;
    }
    K.scal[8 * r] = sqrt(nw2);
}

// v_{jn} = w / beta (c64), four entries per thread in flight; the product of
// the next step reads v_{jn} in place
__global__ void arn_normalize_f32(ArnDev K, int jn)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const float inv = (float)(beta > 0.0 ? 1.0 / beta : 0.0);
    float2 *Vn = reinterpret_cast<float2 *>(K.V) + ((size_t)jn * K.R + r) * K.n;
    const float2 *w = reinterpret_cast<const float2 *>(K.w) + (size_t)r * K.n;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < K.n; i += 4 * stride) {
        const float2 a = w[i], b = w[i + stride], c = w[i + 2 * stride], d = w[i + 3 * stride];
        Vn[i] = make_float2(a.x * inv, a.y * inv);
        Vn[i + stride] = make_float2(b.x * inv, b.y * inv);
        Vn[i + 2 * stride] = make_float2(c.x * inv, c.y * inv);
        Vn[i + 3 * stride] = make_float2(d.x * inv, d.y * inv);
    }
    for (; i < K.n; i += stride) {
        const float2 a = w[i];
        Vn[i] = make_float2(a.x * inv, a.y * inv);
    }
}

// v_0 = rr / beta (c64), read in place by the first product
__global__ void arn_start_f32(ArnDev K, const double2 *__restrict__ rr)
{
    const int r = blockIdx.y;
    const double beta = K.scal[8 * r];
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    float2 *V0 = reinterpret_cast<float2 *>(K.V) + (size_t)r * K.n;
    const double2 *v = rr + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x)
        V0[i] = make_float2((float)(v[i].x * inv), (float)(v[i].y * inv));
}

// x += V y (c128 x, c64 basis, FP64 FMAs: once per restart cycle)
__global__ void arn_xupdate_f32(ArnDev K, double2 *__restrict__ x, int64_t ldx)
{
    extern __shared__ double2 ys64[];
    const int r = blockIdx.y;
    const int k = K.kact[r];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys64[l] = K.h1[(size_t)r * (K.m + 2) + l];
    __syncthreads();
    if (k == 0) return;
    const size_t ldb = (size_t)K.R * K.n;
    const float2 *V = reinterpret_cast<const float2 *>(K.V) + (size_t)r * K.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        double2 a = x[(size_t)r * ldx + i];
        for (int l = 0; l < k; ++l) {
            const float2 v = V[(size_t)l * ldb + i];
            const double2 y = ys64[l];
            a.x = fma((double)v.x, y.x, a.x);
            a.x = fma(-(double)v.y, y.y, a.x);
            a.y = fma((double)v.x, y.y, a.y);
            a.y = fma((double)v.y, y.x, a.y);
        }
        x[(size_t)r * ldx + i] = a;
    }
}

// segments of the dot pass at step j: enough blocks to fill the GPU
void dot_split(int n, int R, int j, int *S, int *seg)
{
    const int cols = j + 2;
    int s = (TARGET + cols * R - 1) / (cols * R);
    s = std::max(1, std::min(s, std::max(1, n / 1024)));
    int sg = (n + s - 1) / s;
    sg = (sg + 31) / 32 * 32;
    *seg = std::max(32, sg);
    *S = (n + *seg - 1) / *seg;
}

}  // namespace

#define ARNC(call)                                                                    \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

void arn_free(ArnWork *w)
{
    if (!w) return;
    cudaFree(w->block);
    cudaFreeHost(w->h_scal);
    cudaFreeHost(w->h_kact);
    cudaFreeHost(w->h_hh);
    delete w;
}

h2_status arn_get(ArnWork **slot, int n, int m, int R, int extra_cols, int mode)
{
    ArnWork *w = *slot;
    if (w && w->n == n && w->m == m && w->R == R && w->extra_cols == extra_cols && w->mode == mode) return H2_OK;
    arn_free(w);
    *slot = nullptr;
    if (mode != ARN_FP64 && mode != ARN_DF && mode != ARN_F32) return (set_error("GMRES: unknown Arnoldi arithmetic"), H2_ERR_ARG);
    w = new ArnWork();
    w->n = n;
    w->m = m;
    w->R = R;
    w->extra_cols = extra_cols;
    w->mode = mode;
    // update / residual grid: rows per block, multiple of 32
    int nb = std::max(1, std::min((n + AT - 1) / AT, (TARGET_ROWS + R - 1) / R));
    int rows = (n + nb - 1) / nb;
    rows = (rows + 31) / 32 * 32;
    w->rows = rows;
    w->nbu = (n + rows - 1) / rows;
    int np = w->nbu;
    for (int j = 0; j < m; ++j) {
        int S, seg;
        dot_split(n, R, j, &S, &seg);
        np = std::max(np, (j + 2) * S);
    }
    ArnDev &K = w->K;
    K.n = n;
    K.m = m;
    K.R = R;
    K.np = np;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t hh = (size_t)2 * R * (m + 2);  // h1 rows, then h2 rows
    const size_t ventry = mode == ARN_F32 ? sizeof(float2) : sizeof(double2);   // bytes per basis entry
    const size_t oV = take(ventry * (size_t)n * (m + 1) * R);
    const size_t oZ = extra_cols ? take(sizeof(double2) * (size_t)n * extra_cols * R) : 0;
    const size_t ow = take(ventry * (size_t)n * R);
    const size_t op = take(sizeof(double2) * (size_t)np * R);
    const size_t ot = take(sizeof(unsigned) * 8 * R);
    const size_t oh = take(sizeof(double2) * hh);
    const size_t osc = take(sizeof(double) * 8 * R);
    const size_t ok = take(sizeof(int) * R);
    const size_t orr = take(sizeof(double2) * (size_t)n * R);
    const size_t otm = take(sizeof(double2) * (size_t)n * R);
    const size_t ox = take(sizeof(float2) * (size_t)n * R);
    const size_t oy = take(sizeof(float2) * (size_t)n * R);
    if (cudaMalloc(&w->block, off) != cudaSuccess || cudaMallocHost(&w->h_scal, 8 * sizeof(double) * R) != cudaSuccess ||
        cudaMallocHost(&w->h_kact, sizeof(int) * R) != cudaSuccess ||
        cudaMallocHost(&w->h_hh, sizeof(double2) * hh) != cudaSuccess) {
        cudaGetLastError();  // an out-of-memory result must not stay behind as the last error
        arn_free(w);
        set_error("GMRES workspace allocation failed (" + std::to_string(off >> 20) + " MiB)");
        return H2_ERR_ALLOC;
    }
    char *base = reinterpret_cast<char *>(w->block);
    K.V = reinterpret_cast<double2 *>(base + oV);
    w->Z = extra_cols ? reinterpret_cast<double2 *>(base + oZ) : nullptr;
    K.w = reinterpret_cast<double2 *>(base + ow);
    K.part = reinterpret_cast<double2 *>(base + op);
    K.ticket = reinterpret_cast<unsigned *>(base + ot);
    K.h1 = reinterpret_cast<double2 *>(base + oh);
    K.h2 = K.h1 + (size_t)R * (m + 2);
    K.scal = reinterpret_cast<double *>(base + osc);
    K.kact = reinterpret_cast<int *>(base + ok);
    w->rr = reinterpret_cast<double2 *>(base + orr);
    w->tmp = reinterpret_cast<double2 *>(base + otm);
    w->x32 = reinterpret_cast<float2 *>(base + ox);
    w->y32 = reinterpret_cast<float2 *>(base + oy);
    if (cudaMemset(K.ticket, 0, sizeof(unsigned) * 8 * R) != cudaSuccess ||
        cudaMemset(K.scal, 0, sizeof(double) * 8 * R) != cudaSuccess) {
        arn_free(w);
        return H2_ERR_CUDA;
    }
    // dynamic shared memory of the update kernels: (m + 2) x 16 bytes <= 16.4 KB, under the default limit
    w->H.assign((size_t)R * m * (m + 1), 0.0);
    w->g.assign((size_t)R * (m + 1), 0.0);
    w->sn.assign((size_t)R * m, 0.0);
    w->cs.assign((size_t)R * m, 0.0);
    w->est.assign(R, 0.0);
    w->beta.assign(R, 0.0);
    w->bad.assign(R, 0);
    w->reorth.assign(R, 0);
    *slot = w;
    return H2_OK;
}

h2_status arn_set_eta(ArnWork *w, double eta)
{
    if (!(eta >= 0.0 && eta <= 1.0)) return (set_error("GMRES: reorthogonalisation threshold must lie in [0, 1]"), H2_ERR_ARG);
    const double e = eta == 0.0 ? std::sqrt(0.5) : eta;
    w->K.eta2 = e * e;
    return H2_OK;
}

static dim3 vec_grid(const ArnWork *w)
{
    return dim3(std::max(1, std::min((w->n + 255) / 256, (TARGET_ROWS + w->R - 1) / w->R)), w->R);
}

h2_status arn_residual(ArnWork *w, const double2 *b, int64_t ldb, const double2 *y, cudaStream_t st)
{
    arn_residual<<<dim3(w->nbu, w->R), AT, 0, st>>>(w->K, b, ldb, y, w->rr, w->rows);
    ARNC(cudaGetLastError());
    return H2_OK;
}

h2_status arn_start(ArnWork *w, cudaStream_t st)
{
    if (w->mode == ARN_DF)
        arn_start_df<<<vec_grid(w), 256, 0, st>>>(w->K, w->rr, w->x32);
    else if (w->mode == ARN_F32)
        arn_start_f32<<<vec_grid(w), 256, 0, st>>>(w->K, w->rr);
    else
        arn_start<<<vec_grid(w), 256, 0, st>>>(w->K, w->rr, w->x32);
    ARNC(cudaGetLastError());
    const int m = w->m;
    for (int r = 0; r < w->R; ++r) {
        std::complex<double> *g = w->g.data() + (size_t)r * (m + 1);
        std::fill(g, g + m + 1, 0.0);
        g[0] = w->h_scal[8 * r];
    }
    return H2_OK;
}

// Hessenberg column j of right-hand side r on the host: coefficients of the
// projection(s), subdiagonal beta, previous rotations, new rotation, rotated
// right-hand side and residual estimate |g_{j+1}|.
static void host_column(ArnWork *w, int r, int j)
{
    using C = std::complex<double>;
    const int m = w->m, R = w->R;
    const double2 *h1 = w->h_hh + (size_t)r * (m + 2);
    const double2 *h2 = w->h_hh + (size_t)(R + r) * (m + 2);
    const double *sc = w->h_scal + 8 * r;
    const bool again = sc[3] != 0.0;
    const double beta = sc[0];
    C *Hj = w->H.data() + ((size_t)r * m + j) * (m + 1);
    double *cs = w->cs.data() + (size_t)r * m;
    C *sn = w->sn.data() + (size_t)r * m;
    C *g = w->g.data() + (size_t)r * (m + 1);
    for (int l = 0; l <= j; ++l) {
        Hj[l] = C(h1[l].x, h1[l].y);
        if (again) Hj[l] += C(h2[l].x, h2[l].y);
    }
    for (int l = 0; l < j; ++l) {  // rotation l: [c s; -conj(s) c]
        const C a = Hj[l], b = Hj[l + 1];
        Hj[l] = cs[l] * a + sn[l] * b;
        Hj[l + 1] = cs[l] * b - std::conj(sn[l]) * a;
    }
    const C a = Hj[j];
    const double na = std::abs(a);
    double c;
    C s;
    if (beta == 0.0) {
        c = 1.0;
        s = 0.0;
    } else if (na == 0.0) {
        c = 0.0;
        s = 1.0;
    } else {
        const double nr = std::hypot(na, beta);
        c = na / nr;
        s = a / na * (beta / nr);
    }
    cs[j] = c;
    sn[j] = s;
    Hj[j] = c * a + s * beta;
    Hj[j + 1] = 0.0;
    g[j + 1] = -std::conj(s) * g[j];
    g[j] = c * g[j];
    w->beta[r] = beta;
    w->est[r] = std::abs(g[j + 1]);
    w->reorth[r] = again;
    w->bad[r] = !std::isfinite(beta) || !std::isfinite(w->est[r]);
}

h2_status arn_step(ArnWork *w, int j, cudaStream_t st)
{
    const ArnDev &K = w->K;
    int S, seg;
    dot_split(w->n, w->R, j, &S, &seg);
    const size_t smem = sizeof(double2) * (w->m + 2);
    const dim3 g1((j + 2) * S, w->R), g2((j + 1) * S, w->R), gu(w->nbu, w->R);
    if (w->mode == ARN_DF) {
        arn_widen_df<<<vec_grid(w), 256, 0, st>>>(K, w->y32);
        arn_dot_df<false><<<g1, AT, 0, st>>>(K, j, S, seg);
        arn_update_df<false><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_dot_df<true><<<g2, AT, 0, st>>>(K, j, S, seg);
        arn_update_df<true><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_normalize_df<<<vec_grid(w), 256, 0, st>>>(K, j + 1, w->x32);
    } else if (w->mode == ARN_F32) {
        ARNC(cudaMemcpyAsync(K.w, w->y32, sizeof(float2) * (size_t)w->n * w->R, cudaMemcpyDeviceToDevice, st));
        arn_dot_f32<false><<<g1, AT, 0, st>>>(K, j, S, seg);
        arn_update_f32<false><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_dot_f32<true><<<g2, AT, 0, st>>>(K, j, S, seg);
        arn_update_f32<true><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_normalize_f32<<<vec_grid(w), 256, 0, st>>>(K, j + 1);
    } else {
        arn_widen<<<vec_grid(w), 256, 0, st>>>(K, w->y32);
        arn_dot<false><<<g1, AT, 0, st>>>(K, j, S, seg);
        arn_update<false><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_dot<true><<<g2, AT, 0, st>>>(K, j, S, seg);
        arn_update<true><<<gu, AT, smem, st>>>(K, j, w->rows);
        arn_normalize<<<vec_grid(w), 256, 0, st>>>(K, j + 1, w->x32);
    }
    ARNC(cudaGetLastError());
    ARNC(cudaMemcpyAsync(w->h_hh, K.h1, sizeof(double2) * 2 * w->R * (w->m + 2), cudaMemcpyDeviceToHost, st));
    ARNC(cudaMemcpyAsync(w->h_scal, K.scal, 8 * sizeof(double) * w->R, cudaMemcpyDeviceToHost, st));
    ARNC(cudaStreamSynchronize(st));
    for (int r = 0; r < w->R; ++r) host_column(w, r, j);
    return H2_OK;
}

const float2 *arn_input(const ArnWork *w, int j)
{
    if (w->mode == ARN_F32) return reinterpret_cast<const float2 *>(w->K.V) + (size_t)j * w->R * w->n;
    return w->x32;
}

h2_status arn_read(ArnWork *w, cudaStream_t st)
{
    ARNC(cudaMemcpyAsync(w->h_scal, w->K.scal, 8 * sizeof(double) * w->R, cudaMemcpyDeviceToHost, st));
    ARNC(cudaStreamSynchronize(st));
    return H2_OK;
}

h2_status arn_finish(ArnWork *w, const double2 *basis, double2 *x, int64_t ldx, cudaStream_t st)
{
    using C = std::complex<double>;
    const int m = w->m;
    for (int r = 0; r < w->R; ++r) {  // y = H(1:k,1:k)^{-1} g(1:k) by back substitution
        const int k = w->h_kact[r];
        const C *H = w->H.data() + (size_t)r * m * (m + 1), *g = w->g.data() + (size_t)r * (m + 1);
        double2 *y = w->h_hh + (size_t)r * (m + 2);
        std::vector<C> yc(std::max(k, 1));
        for (int i = k - 1; i >= 0; --i) {
            C s = g[i];
            for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * yc[l];
            const C d = H[(size_t)i * (m + 1) + i];
            yc[i] = std::norm(d) > 0.0 ? s / d : C(0.0);
            y[i] = make_double2(yc[i].real(), yc[i].imag());
        }
    }
    ARNC(cudaMemcpyAsync(w->K.h1, w->h_hh, sizeof(double2) * w->R * (m + 2), cudaMemcpyHostToDevice, st));
    ARNC(cudaMemcpyAsync(w->K.kact, w->h_kact, sizeof(int) * w->R, cudaMemcpyHostToDevice, st));
    if (basis != w->K.V)   // flexible variant: the c128 preconditioned directions, every arithmetic
        arn_xupdate<<<vec_grid(w), 256, sizeof(double2) * (m + 2), st>>>(w->K, basis, x, ldx);
    else if (w->mode == ARN_DF)
        arn_xupdate_df<<<vec_grid(w), 256, sizeof(double2) * (m + 2), st>>>(w->K, x, ldx);
    else if (w->mode == ARN_F32)
        arn_xupdate_f32<<<vec_grid(w), 256, sizeof(double2) * (m + 2), st>>>(w->K, x, ldx);
    else
        arn_xupdate<<<vec_grid(w), 256, sizeof(double2) * (m + 2), st>>>(w->K, basis, x, ldx);
    ARNC(cudaGetLastError());
    return H2_OK;
}

h2_status arn_basis_c128(ArnWork *w, int j, double2 *out, cudaStream_t st)
{
    arn_basis_c128_kernel<<<vec_grid(w), 256, 0, st>>>(w->K, w->mode, j, out);
    ARNC(cudaGetLastError());
    return H2_OK;
}

h2_status arn_c128_to_c64(ArnWork *w, const double2 *a, int64_t lda, float2 *b, cudaStream_t st)
{
    arn_to_c64<<<vec_grid(w), 256, 0, st>>>(a, lda, b, w->n);
    ARNC(cudaGetLastError());
    return H2_OK;
}

h2_status arn_c64_to_c128(ArnWork *w, const float2 *a, double2 *b, cudaStream_t st)
{
    arn_to_c128<<<vec_grid(w), 256, 0, st>>>(a, b, w->n);
    ARNC(cudaGetLastError());
    return H2_OK;
}

}  // namespace h2
