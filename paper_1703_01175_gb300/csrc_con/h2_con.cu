// GPU kernels of the H^2 constructor (include/h2con.h): VIE kernel entries,
// near-field blocks, Stage I adaptive cross approximation (Sec. III.B, Eq. 6),
// grouped complex GEMMs for the Stage I recompression and the Stage II Gram
// and projection products (Sec. III.C, Eqs. 10-16), and the coupling products
// of Eq. 18 with the kernel entries generated inside the product.
//
// Precision: geometry, distance and the phase k r reduced modulo 2 pi are
// FP64 (k r reaches 1e4 on the longest geometries, where FP32 would lose the
// phase); everything after the reduction, the cross approximation and the
// products are FP32 complex, except the grouped GEMM's FP64-accumulating form.
#include <cuda_runtime.h>

#include <cstdint>

#include "h2con.h"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

struct Vie {
    double k, dv;
    double pref;      // dv k^2 / (4 pi)
    float self_re, self_im;
};

__host__ Vie make_vie(const h2c_vie &v)
{
    Vie o;
    o.k = v.k;
    o.dv = v.dv;
    o.pref = v.dv * v.k * v.k / (2.0 * kTwoPi);
    o.self_re = (float)v.self_re;
    o.self_im = (float)v.self_im;
    return o;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cfms(float2 acc, float2 a, float2 b)  // acc - a b
{
    acc.x -= a.x * b.x - a.y * b.y;
    acc.y -= a.x * b.y + a.y * b.x;
    return acc;
}
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// The dyad of voxels p, q: K_ab = cb h_a h_b + ca delta_ab, or the self term
// when p and q coincide (self = true, K = s I).
struct Dyad {
    float2 ca, cb;
    float h[3];
    bool self;
};

__device__ __forceinline__ Dyad dyad(const double *__restrict__ c, int64_t p, int64_t q, const Vie &P)
{
    Dyad d;
    const double dx = c[3 * p] - c[3 * q], dy = c[3 * p + 1] - c[3 * q + 1], dz = c[3 * p + 2] - c[3 * q + 2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) {
        d.self = true;
        d.ca = make_float2(P.self_re, P.self_im);
        d.cb = make_float2(0.f, 0.f);
        d.h[0] = d.h[1] = d.h[2] = 0.f;
        return d;
    }
    d.self = false;
    const double r = sqrt(r2);
    const double rinv = 1.0 / r;
    const double kr = P.k * r;
    const double nw = rint(kr * (1.0 / kTwoPi));
    const float red = (float)fma(-nw, kTwoPi, kr);   // k r modulo 2 pi, in [-pi, pi]
    float sn, cs;
    sincosf(red, &sn, &cs);
    const float sc = (float)(P.pref * rinv);        // dv k^2 / (4 pi r)
    const float inv = (float)(rinv / P.k);          // 1 / (k r)
    const float2 g = make_float2(sc * cs, -sc * sn); // dv k^2 e^{-jkr} / (4 pi r)
    d.ca = cmul(g, make_float2(1.f - inv * inv, -inv));
    d.cb = cmul(g, make_float2(-1.f + 3.f * inv * inv, 3.f * inv));
    d.h[0] = (float)(dx * rinv);
    d.h[1] = (float)(dy * rinv);
    d.h[2] = (float)(dz * rinv);
    return d;
}

__device__ __forceinline__ float2 dyad_entry(const Dyad &d, int a, int b)
{
    if (d.self) return a == b ? d.ca : make_float2(0.f, 0.f);
    const float w = d.h[a] * d.h[b];
    float2 v = make_float2(d.cb.x * w, d.cb.y * w);
    if (a == b) {
        v.x += d.ca.x;
        v.y += d.ca.y;
    }
    return v;
}

// ---------------------------------------------------------------------------
// near-field blocks
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) near_kernel(const double *__restrict__ cen, Vie P, const float2 *__restrict__ chi,
                                                   const h2c_near_desc *__restrict__ desc, float2 *__restrict__ Z)
{
    const h2c_near_desc D = desc[blockIdx.x];
    const int64_t ld = 3 * (int64_t)D.row_nv;
    float2 *out = Z + D.out_off;
    const int npair = D.row_nv * D.col_nv;
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        const int pr = e % D.row_nv, pc = e / D.row_nv;   // consecutive threads along rows
        const int64_t p = D.row_v0 + pr, q = D.col_v0 + pc;
        const Dyad d = dyad(cen, p, q, P);
        const float2 x = chi[q];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float2 *col = out + (3 * (int64_t)pc + b) * ld + 3 * pr;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float2 v = cmul(dyad_entry(d, a, b), x);
                v.x = -v.x;
                v.y = -v.y;
                if (D.diag && pr == pc && a == b) v.x += 1.f;
                col[a] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------

constexpr int ACA_THREADS = 512;
constexpr int ACA_WARPS = ACA_THREADS / 32;
constexpr int ACA_KMAX = 4096;   // largest rank of one cross approximation (32 KB of shared memory)

struct ArgMax {
    float v;
    int i;
};

// larger value wins; equal values: smaller index (first maximum)
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b)
{
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
    return a;
}

__device__ ArgMax block_argmax(ArgMax x, ArgMax *sh)
{
    for (int o = 16; o > 0; o >>= 1) {
        ArgMax y;
        y.v = __shfl_xor_sync(0xffffffffu, x.v, o);
        y.i = __shfl_xor_sync(0xffffffffu, x.i, o);
        x = better(x, y);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        x = l < ACA_WARPS ? sh[l] : ArgMax{-2.f, 0x7fffffff};
        for (int o = 16; o > 0; o >>= 1) {
            ArgMax y;
            y.v = __shfl_xor_sync(0xffffffffu, x.v, o);
            y.i = __shfl_xor_sync(0xffffffffu, x.i, o);
            x = better(x, y);
        }
        if (l == 0) sh[0] = x;
    }
    __syncthreads();
    return sh[0];
}

__device__ double block_sum(double x, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        x = l < ACA_WARPS ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) sh[0] = x;
    }
    __syncthreads();
    return sh[0];
}

// ---------------------------------------------------------------------------
// Stage I: adaptive cross approximation, one thread block per job
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(ACA_THREADS) aca_kernel(const double *__restrict__ cen, Vie P,
                                                          const int32_t *__restrict__ colvox,
                                                          const h2c_aca_job *__restrict__ jobs, float eps,
                                                          float2 *__restrict__ U, float2 *__restrict__ V,
                                                          uint8_t *__restrict__ used, int32_t *__restrict__ piv_row,
                                                          float2 *__restrict__ piv_val, int32_t *__restrict__ k_out,
                                                          int32_t *__restrict__ status)
{
    extern __shared__ float2 vec[];   // [kmax]: U[i, :k] in the row pass, V[jp, :k] in the column pass
    __shared__ ArgMax sh_arg[ACA_WARPS];
    __shared__ double sh_sum[ACA_WARPS];
    const h2c_aca_job J = jobs[blockIdx.x];
    const int tid = threadIdx.x;
    const int64_t m = 3 * (int64_t)J.row_nv, n = 3 * (int64_t)J.col_nv;
    const int kmax = min(J.kmax, ACA_KMAX);
    float2 *Uj = U + J.u_off;
    float2 *Vj = V + J.v_off;
    uint8_t *uj = used + J.used_off;
    const int32_t *cv = colvox + J.col_off;
    for (int64_t q = tid; q < m; q += ACA_THREADS) uj[q] = 0;
    __syncthreads();

    int i = 0, k = 0, small = 0, st = 0;
    double norm2 = 0.0;
    bool done = false;
    while (k < kmax && !done) {
        for (int l = tid; l < k; l += ACA_THREADS) vec[l] = Uj[(int64_t)l * m + i];
        __syncthreads();
        // residual row i against every column, written as candidate column k of V
        const int64_t pi = J.row_v0 + i / 3;
        const int a = i % 3;
        ArgMax best{-1.f, 0x7fffffff};
        for (int64_t c = tid; c < J.col_nv; c += ACA_THREADS) {
            const Dyad d = dyad(cen, pi, cv[c], P);
            float2 r[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) r[b] = dyad_entry(d, a, b);
            for (int l = 0; l < k; ++l) {
                const float2 u = vec[l];
                const float2 *vl = Vj + (int64_t)l * n + 3 * c;
#pragma unroll
                for (int b = 0; b < 3; ++b) r[b] = cfms(r[b], u, vl[b]);
            }
            float2 *vk = Vj + (int64_t)k * n + 3 * c;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                vk[b] = r[b];
                best = better(best, ArgMax{cabs2(r[b]), (int)(3 * c + b)});
            }
        }
        best = block_argmax(best, sh_arg);
        if (tid == 0) uj[i] = 1;
        if (!(best.v > 0.f)) {
            // zero residual row: continue from the first row not used yet
            ArgMax f{-1.f, 0x7fffffff};
            __syncthreads();
            for (int64_t q = tid; q < m; q += ACA_THREADS)
                if (!uj[q]) {
                    f = better(f, ArgMax{0.f, (int)q});
                    break;
                }
            f = block_argmax(f, sh_arg);
            if (f.v < 0.f) {
                done = true;   // every row used: the approximation is complete
                break;
            }
            i = f.i;
            continue;
        }
        const int jp = best.i;
        const float2 piv = Vj[(int64_t)k * n + jp];
        const float den = cabs2(piv);
        const float2 inv = make_float2(piv.x / den, -piv.y / den);
        double nv2 = 0.0;
        for (int64_t j = tid; j < n; j += ACA_THREADS) {
            float2 *p = Vj + (int64_t)k * n + j;
            const float2 v = cmul(*p, inv);
            *p = v;
            nv2 += (double)cabs2(v);
        }
        nv2 = block_sum(nv2, sh_sum);
        for (int l = tid; l < k; l += ACA_THREADS) vec[l] = Vj[(int64_t)l * n + jp];
        __syncthreads();
        // residual column jp against every row, written as column k of U
        const int64_t qv = cv[jp / 3];
        const int b = jp % 3;
        double nu2 = 0.0;
        ArgMax nxt{-1.f, 0x7fffffff};
        for (int64_t p = tid; p < J.row_nv; p += ACA_THREADS) {
            const Dyad d = dyad(cen, J.row_v0 + p, qv, P);
            float2 u[3];
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) u[aa] = dyad_entry(d, aa, b);
            for (int l = 0; l < k; ++l) {
                const float2 v = vec[l];
                const float2 *ul = Uj + (int64_t)l * m + 3 * p;
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) u[aa] = cfms(u[aa], ul[aa], v);
            }
            float2 *uk = Uj + (int64_t)k * m + 3 * p;
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                uk[aa] = u[aa];
                const float w = cabs2(u[aa]);
                nu2 += (double)w;
                if (!uj[3 * p + aa]) nxt = better(nxt, ArgMax{w, (int)(3 * p + aa)});
            }
        }
        nu2 = block_sum(nu2, sh_sum);
        nxt = block_argmax(nxt, sh_arg);
        if (tid == 0) {
            piv_row[J.piv_off + k] = i;
            piv_val[J.piv_off + k] = piv;
        }
        ++k;
        norm2 += nu2 * nv2;
        if (sqrt(nu2 * nv2) <= (double)eps * sqrt(norm2)) {
            if (++small >= 2) done = true;
        } else {
            small = 0;
        }
        if (nxt.v < 0.f) done = true;   // every row used
        i = nxt.i;
        __syncthreads();
    }
    if (!done && k >= kmax) st = (kmax >= (int)min(m, n)) ? 0 : 1;
    if (tid == 0) {
        k_out[blockIdx.x] = k;
        status[blockIdx.x] = st;
    }
}

// ---------------------------------------------------------------------------
// grouped complex GEMM: 64 x 64 output tiles, K steps of 16, 256 threads
// ---------------------------------------------------------------------------

constexpr int GT = 64, GK = 16, GTHREADS = 256;

template <class Acc>
struct AccOps;
template <>
struct AccOps<float2> {
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static void mac(float2 &c, float2 a, float2 b)
    {
        c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
        c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
    }
};
template <>
struct AccOps<double2> {
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static void mac(double2 &c, float2 a, float2 b)
    {
        const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
        c.x = fma(ax, bx, fma(-ay, by, c.x));
        c.y = fma(ax, by, fma(ay, bx, c.y));
    }
};

__device__ __forceinline__ float2 load_op(const float2 *__restrict__ M, int64_t ld, int op, int64_t r, int64_t c)
{
    // element (r, c) of op(M)
    float2 v;
    if (op == H2C_N || op == H2C_R) v = M[r + c * ld];
    else v = M[c + r * ld];
    if (op == H2C_C || op == H2C_R) v.y = -v.y;
    return v;
}

template <class Acc>
__global__ void __launch_bounds__(GTHREADS) gemm_kernel(const h2c_gemm *__restrict__ desc,
                                                        const int32_t *__restrict__ tile_prob,
                                                        const int32_t *__restrict__ tile_idx)
{
    __shared__ float2 As[GK][GT + 1];
    __shared__ float2 Bs[GK][GT + 1];
    const h2c_gemm D = desc[tile_prob[blockIdx.x]];
    const int tmc = (D.m + GT - 1) / GT;
    const int ti = tile_idx[blockIdx.x];
    const int m0 = (ti % tmc) * GT, n0 = (ti / tmc) * GT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float2 *A = reinterpret_cast<const float2 *>(D.A);
    const float2 *B = reinterpret_cast<const float2 *>(D.B);
    Acc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = AccOps<Acc>::zero();
    const bool a_rows = (D.opa == H2C_N || D.opa == H2C_R);   // consecutive elements along op(A)'s rows
    const bool b_rows = (D.opb == H2C_N || D.opb == H2C_R);
    for (int k0 = 0; k0 < D.k; k0 += GK) {
#pragma unroll
        for (int q = 0; q < (GT * GK) / GTHREADS; ++q) {
            const int e = tid + q * GTHREADS;
            int ii, kk;
            if (a_rows) {
                ii = e % GT;
                kk = e / GT;
            } else {
                kk = e % GK;
                ii = e / GK;
            }
            const int r = m0 + ii, c = k0 + kk;
            As[kk][ii] = (r < D.m && c < D.k) ? load_op(A, D.lda, D.opa, r, c) : make_float2(0.f, 0.f);
            int jj, kb;
            if (b_rows) {
                kb = e % GK;
                jj = e / GK;
            } else {
                jj = e % GT;
                kb = e / GT;
            }
            const int rb = k0 + kb, cb = n0 + jj;
            Bs[kb][jj] = (rb < D.k && cb < D.n) ? load_op(B, D.ldb, D.opb, rb, cb) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) AccOps<Acc>::mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + tx + 16 * i, c = n0 + ty + 16 * j;
            if (r >= D.m || c >= D.n) continue;
            const Acc v = acc[i][j];
            if constexpr (sizeof(Acc) == sizeof(float2)) {
                float2 *C = reinterpret_cast<float2 *>(D.C) + r + (int64_t)c * D.ldc;
                float2 o = make_float2(D.alpha_re * v.x - D.alpha_im * v.y, D.alpha_re * v.y + D.alpha_im * v.x);
                if (D.beta) {
                    o.x += C->x;
                    o.y += C->y;
                }
                *C = o;
            } else {
                double2 *C = reinterpret_cast<double2 *>(D.C) + r + (int64_t)c * D.ldc;
                const double ar = D.alpha_re, ai = D.alpha_im;
                double2 o = make_double2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
                if (D.beta) {
                    o.x += C->x;
                    o.y += C->y;
                }
                *C = o;
            }
        }
}

// ---------------------------------------------------------------------------
// coupling products Q = V^{sH} K[s, I_t], entries generated per K step of
// 8 voxels (24 unknowns)
// ---------------------------------------------------------------------------

constexpr int CV = 8, CK = 3 * CV;

__global__ void __launch_bounds__(GTHREADS) couple_kernel(const double *__restrict__ cen, Vie P,
                                                          const h2c_couple *__restrict__ desc,
                                                          const int32_t *__restrict__ tile_prob,
                                                          const int32_t *__restrict__ tile_idx)
{
    __shared__ float2 As[CK][GT + 1];   // conj(Vs) rows of this K step
    __shared__ float2 Bs[CK][GT + 1];   // K[rows of this K step, pivots]
    const h2c_couple D = desc[tile_prob[blockIdx.x]];
    const int tmc = (D.ks + GT - 1) / GT;
    const int ti = tile_idx[blockIdx.x];
    const int m0 = (ti % tmc) * GT, n0 = (ti / tmc) * GT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float2 *Vs = reinterpret_cast<const float2 *>(D.Vs);
    const int ns = 3 * D.s_nv;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int v0 = 0; v0 < D.s_nv; v0 += CV) {
        const int r0 = 3 * v0;
        // A: (row kk of the step, basis column ii) -> conj(Vs[r0 + kk, m0 + ii])
        for (int e = tid; e < CK * GT; e += GTHREADS) {
            const int kk = e % CK, ii = e / CK;
            const int r = r0 + kk, c = m0 + ii;
            float2 v = make_float2(0.f, 0.f);
            if (r < ns && c < D.ks) {
                v = Vs[r + (int64_t)c * D.ldv];
                v.y = -v.y;
            }
            As[kk][ii] = v;
        }
        // B: one dyad per (voxel, pivot) pair gives the three rows of that voxel
        for (int e = tid; e < CV * GT; e += GTHREADS) {
            const int pv = e % CV, jj = e / CV;
            const int vox = v0 + pv, col = n0 + jj;
            if (vox < D.s_nv && col < D.kp) {
                const int pu = D.piv[col];
                const Dyad d = dyad(cen, D.s_v0 + vox, pu / 3, P);
                const int b = pu % 3;
#pragma unroll
                for (int a = 0; a < 3; ++a) Bs[3 * pv + a][jj] = dyad_entry(d, a, b);
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) Bs[3 * pv + a][jj] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < CK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) AccOps<float2>::mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    float2 *Q = reinterpret_cast<float2 *>(D.Q);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + tx + 16 * i, c = n0 + ty + 16 * j;
            if (r < D.ks && c < D.kp) Q[r + (int64_t)c * D.ldq] = acc[i][j];
        }
}

// ---------------------------------------------------------------------------
// coupling symmetrisation
// ---------------------------------------------------------------------------

__global__ void sym_average_kernel(float2 *__restrict__ S, const int64_t *__restrict__ off_ts,
                                   const int64_t *__restrict__ off_st, const int32_t *__restrict__ kt,
                                   const int32_t *__restrict__ ks)
{
    const int p = blockIdx.x;
    const int a_n = kt[p], b_n = ks[p];
    float2 *Sts = S + off_ts[p], *Sst = S + off_st[p];
    for (int e = threadIdx.x; e < a_n * b_n; e += blockDim.x) {
        const int a = e % a_n, b = e / a_n;
        const float2 x = Sts[a + (int64_t)b * a_n], y = Sst[b + (int64_t)a * b_n];
        const float2 mval = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y + y.y));
        Sts[a + (int64_t)b * a_n] = mval;
        Sst[b + (int64_t)a * b_n] = mval;
    }
}

}  // namespace

extern "C" {

int h2c_near_blocks(const double *centres, h2c_vie vie, const float *chi, const h2c_near_desc *desc, int64_t ndesc,
                    float *Z, void *stream)
{
    if (ndesc < 0 || ndesc > 0x7fffffff || (ndesc > 0 && (!centres || !chi || !desc || !Z))) return -1;
    if (ndesc == 0) return 0;
    near_kernel<<<(unsigned)ndesc, 256, 0, (cudaStream_t)stream>>>(centres, make_vie(vie),
                                                                    reinterpret_cast<const float2 *>(chi), desc,
                                                                    reinterpret_cast<float2 *>(Z));
    return (int)cudaGetLastError();
}

int h2c_aca(const double *centres, h2c_vie vie, const int32_t *colvox, const h2c_aca_job *jobs, int32_t njobs,
            float eps, float *U, float *V, uint8_t *used, int32_t *piv_row, float *piv_val, int32_t *k_out,
            int32_t *status, void *stream)
{
    if (njobs < 0 || (njobs > 0 && (!centres || !colvox || !jobs || !U || !V || !used || !piv_row || !piv_val ||
                                    !k_out || !status)))
        return -1;
    if (njobs == 0) return 0;
    // the shared vector holds ACA_KMAX entries; a job's kmax is clamped to it
    const size_t smem = ACA_KMAX * sizeof(float2);
    aca_kernel<<<njobs, ACA_THREADS, smem, (cudaStream_t)stream>>>(
        centres, make_vie(vie), colvox, jobs, eps, reinterpret_cast<float2 *>(U), reinterpret_cast<float2 *>(V),
        used, piv_row, reinterpret_cast<float2 *>(piv_val), k_out, status);
    return (int)cudaGetLastError();
}

int h2c_gemm_grouped(const h2c_gemm *desc, const int32_t *tile_prob, const int32_t *tile_idx, int64_t ntiles,
                     int32_t out_f64, void *stream)
{
    if (ntiles < 0 || ntiles > 0x7fffffff || (ntiles > 0 && (!desc || !tile_prob || !tile_idx))) return -1;
    if (ntiles == 0) return 0;
    if (out_f64)
        gemm_kernel<double2><<<(unsigned)ntiles, GTHREADS, 0, (cudaStream_t)stream>>>(desc, tile_prob, tile_idx);
    else
        gemm_kernel<float2><<<(unsigned)ntiles, GTHREADS, 0, (cudaStream_t)stream>>>(desc, tile_prob, tile_idx);
    return (int)cudaGetLastError();
}

int h2c_couple_grouped(const double *centres, h2c_vie vie, const h2c_couple *desc, const int32_t *tile_prob,
                       const int32_t *tile_idx, int64_t ntiles, void *stream)
{
    if (ntiles < 0 || ntiles > 0x7fffffff || (ntiles > 0 && (!centres || !desc || !tile_prob || !tile_idx))) return -1;
    if (ntiles == 0) return 0;
    couple_kernel<<<(unsigned)ntiles, GTHREADS, 0, (cudaStream_t)stream>>>(centres, make_vie(vie), desc, tile_prob,
                                                                           tile_idx);
    return (int)cudaGetLastError();
}

int h2c_sym_average(float *S, const int64_t *off_ts, const int64_t *off_st, const int32_t *kt, const int32_t *ks,
                    int64_t npairs, void *stream)
{
    if (npairs < 0 || npairs > 0x7fffffff || (npairs > 0 && (!S || !off_ts || !off_st || !kt || !ks))) return -1;
    if (npairs == 0) return 0;
    sym_average_kernel<<<(unsigned)npairs, 128, 0, (cudaStream_t)stream>>>(reinterpret_cast<float2 *>(S), off_ts,
                                                                          off_st, kt, ks);
    return (int)cudaGetLastError();
}

}  // extern "C"
