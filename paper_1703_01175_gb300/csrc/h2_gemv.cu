// Level-batched, variable-size complex block-row GEMV kernels.
//
// Every stage of the single-RHS H^2 product (Sec. IV.B) is a set of
// independent "tasks": one output segment (a cluster's coefficient vector or a
// leaf's rows of y) accumulating the product of one column-major complex matrix
// with a gathered input vector:
//
//   forward (leaf)   xh^t = W^{tT} x|_t
//   upward           xh^t = T^{t1 T} xh^{t1} + T^{t2 T} xh^{t2}           (Eq. 9)
//   coupling + down  yh^t = sum_{s in R^t} S^{t,s} xh^s + T^t yh^{parent}
//   backward (leaf)  y|_t += U^t yh^t
//   near field       y|_t  = sum_{s in N(t)} Z^{t,s} x|_s
//
// The loader concatenates each task's blocks into ONE contiguous column-major
// matrix (rows padded to an even count), so a task is a dense m x ncol GEMV.
// One CTA owns one task (no atomics, deterministic): its input entries are
// staged in shared memory, each thread owns a row pair (16-byte streaming loads
// of two interleaved complex entries) and a residue class of columns, and the
// column groups are reduced in shared memory at the end.
#include <cuda_runtime.h>

#include "h2_df.cuh"
#include "h2_internal.h"

namespace h2 {

template <typename VT> struct VT_ {};
template <> struct VT_<float2> {
    using S = float;
    static constexpr int CHUNK = 4096;  // staged input columns per pass (32 KB)
    __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct VT_<double2> {
    using S = double;
    static constexpr int CHUNK = 2048;  // 32 KB
    __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};

template <int THREADS, typename VT>
__global__ void __launch_bounds__(THREADS)
rowgemv_kernel(const Task *__restrict__ tasks, const Seg *__restrict__ segs,
               const float2 *__restrict__ mat, const VT *__restrict__ in0,
               const VT *__restrict__ in1, VT *__restrict__ out, int beta_one)
{
    using S = typename VT_<VT>::S;
    constexpr int CHUNK = VT_<VT>::CHUNK;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *xs = reinterpret_cast<VT *>(smem_raw);

    const Task tk = tasks[blockIdx.x];
    const int tid = threadIdx.x;
    const int P = tk.mpad >> 1;          // row pairs, 1 <= P <= THREADS
    const int G = THREADS / P;           // column groups
    const int r = tid % P;
    const int g = tid / P;
    const bool active = g < G;

    S a0r = 0, a0i = 0, a1r = 0, a1i = 0;
    const float4 *A = reinterpret_cast<const float4 *>(mat + tk.mat_off) + r;

    for (int c0 = 0; c0 < tk.ncol; c0 += CHUNK) {
        const int cn = min(CHUNK, tk.ncol - c0);
        __syncthreads();
        // gather input columns [c0, c0 + cn) from the task's segments
        int cpos = 0;
        for (int s = tk.seg_begin; s < tk.seg_end && cpos < c0 + cn; ++s) {
            const Seg sg = segs[s];
            const int lo = max(cpos, c0), hi = min(cpos + sg.n, c0 + cn);
            if (lo < hi) {
                const VT *src = sg.in_off >= 0 ? in0 + sg.in_off : in1 + (-(int64_t)sg.in_off - 1);
                for (int c = lo + tid; c < hi; c += THREADS) xs[c - c0] = src[c - cpos];
            }
            cpos += sg.n;
        }
        __syncthreads();
        if (active) {
            const float4 *Ac = A + (size_t)c0 * P;
            int c = g;
            for (; c + 3 * G < cn; c += 4 * G) {
                const float4 m0 = __ldcs(Ac + (size_t)c * P);
                const float4 m1 = __ldcs(Ac + (size_t)(c + G) * P);
                const float4 m2 = __ldcs(Ac + (size_t)(c + 2 * G) * P);
                const float4 m3 = __ldcs(Ac + (size_t)(c + 3 * G) * P);
                const VT x0 = xs[c], x1 = xs[c + G], x2 = xs[c + 2 * G], x3 = xs[c + 3 * G];
#define H2_CMAC(mm, xx)                                               \
    a0r = fma((S)mm.x, xx.x, a0r);                                    \
    a0r = fma(-(S)mm.y, xx.y, a0r);                                   \
    a0i = fma((S)mm.x, xx.y, a0i);                                    \
    a0i = fma((S)mm.y, xx.x, a0i);                                    \
    a1r = fma((S)mm.z, xx.x, a1r);                                    \
    a1r = fma(-(S)mm.w, xx.y, a1r);                                   \
    a1i = fma((S)mm.z, xx.y, a1i);                                    \
    a1i = fma((S)mm.w, xx.x, a1i);
                H2_CMAC(m0, x0)
                H2_CMAC(m1, x1)
                H2_CMAC(m2, x2)
                H2_CMAC(m3, x3)
            }
            for (; c < cn; c += G) {
                const float4 m0 = __ldcs(Ac + (size_t)c * P);
                const VT x0 = xs[c];
                H2_CMAC(m0, x0)
            }
#undef H2_CMAC
        }
    }
    __syncthreads();
    VT *red = xs;  // G * mpad <= 2 * THREADS entries
    if (active) {
        red[g * tk.mpad + 2 * r] = VT_<VT>::make(a0r, a0i);
        red[g * tk.mpad + 2 * r + 1] = VT_<VT>::make(a1r, a1i);
    }
    __syncthreads();
    for (int i = tid; i < tk.m; i += THREADS) {
        S sr = 0, si = 0;
        for (int gg = 0; gg < G; ++gg) {
            const VT v = red[gg * tk.mpad + i];
            sr += v.x;
            si += v.y;
        }
        VT *o = out + tk.out_off + i;
        if (beta_one) {
            const VT p = *o;
            sr += p.x;
            si += p.y;
        }
        *o = VT_<VT>::make(sr, si);
    }
}

// Same task structure with c128 inputs and outputs, accumulated in
// double-float on the FP32 pipes: inputs are split into hi + lo floats when
// staged, every product of a (float) matrix entry with an input is split
// exactly, and each thread's partial sums are compensated; the column-group
// reduction and the output are FP64. About 44 FP32 operations per complex
// entry instead of 6 FP64 ones, which GB300 issues at 1/58 of the FP32 rate.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
rowgemv_df_kernel(const Task *__restrict__ tasks, const Seg *__restrict__ segs, const float2 *__restrict__ mat,
                  const double2 *__restrict__ in0, const double2 *__restrict__ in1, double2 *__restrict__ out,
                  int beta_one)
{
    constexpr int CHUNK = 2048;  // staged input columns per pass (32 KB of float4)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *xs = reinterpret_cast<float4 *>(smem_raw);

    const Task tk = tasks[blockIdx.x];
    const int tid = threadIdx.x;
    const int P = tk.mpad >> 1;
    const int G = THREADS / P;
    const int r = tid % P;
    const int g = tid / P;
    const bool active = g < G;

    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // (s, c) of row 0 re, im; row 1 re, im
    const float4 *A = reinterpret_cast<const float4 *>(mat + tk.mat_off) + r;

    for (int c0 = 0; c0 < tk.ncol; c0 += CHUNK) {
        const int cn = min(CHUNK, tk.ncol - c0);
        __syncthreads();
        int cpos = 0;
        for (int s = tk.seg_begin; s < tk.seg_end && cpos < c0 + cn; ++s) {
            const Seg sg = segs[s];
            const int lo = max(cpos, c0), hi = min(cpos + sg.n, c0 + cn);
            if (lo < hi) {
                const double2 *src = sg.in_off >= 0 ? in0 + sg.in_off : in1 + (-(int64_t)sg.in_off - 1);
                for (int c = lo + tid; c < hi; c += THREADS) {
                    const double2 v = src[c - cpos];
                    const float2 re = d_to_df(v.x), im = d_to_df(v.y);
                    xs[c - c0] = make_float4(re.x, im.x, re.y, im.y);
                }
            }
            cpos += sg.n;
        }
        __syncthreads();
        if (active) {
            const float4 *Ac = A + (size_t)c0 * P;
#define H2_CMAC_DF(mm, xx)                                  \
    df_macf(a[0], a[1], mm.x, xx.x, xx.z);                  \
    df_macf(a[0], a[1], -mm.y, xx.y, xx.w);                 \
    df_macf(a[2], a[3], mm.x, xx.y, xx.w);                  \
    df_macf(a[2], a[3], mm.y, xx.x, xx.z);                  \
    df_macf(a[4], a[5], mm.z, xx.x, xx.z);                  \
    df_macf(a[4], a[5], -mm.w, xx.y, xx.w);                 \
    df_macf(a[6], a[7], mm.z, xx.y, xx.w);                  \
    df_macf(a[6], a[7], mm.w, xx.x, xx.z);
            int c = g;
            for (; c + G < cn; c += 2 * G) {
                const float4 m0 = __ldcs(Ac + (size_t)c * P);
                const float4 m1 = __ldcs(Ac + (size_t)(c + G) * P);
                const float4 x0 = xs[c], x1 = xs[c + G];
                H2_CMAC_DF(m0, x0)
                H2_CMAC_DF(m1, x1)
            }
            for (; c < cn; c += G) {
                const float4 m0 = __ldcs(Ac + (size_t)c * P);
                const float4 x0 = xs[c];
                H2_CMAC_DF(m0, x0)
            }
#undef H2_CMAC_DF
        }
    }
    __syncthreads();
    double2 *red = reinterpret_cast<double2 *>(smem_raw);  // G * mpad <= 2 * THREADS entries
    if (active) {
        red[g * tk.mpad + 2 * r] = make_double2(df_to_d(a[0], a[1]), df_to_d(a[2], a[3]));
        red[g * tk.mpad + 2 * r + 1] = make_double2(df_to_d(a[4], a[5]), df_to_d(a[6], a[7]));
    }
    __syncthreads();
    for (int i = tid; i < tk.m; i += THREADS) {
        double sr = 0, si = 0;
        for (int gg = 0; gg < G; ++gg) {
            const double2 v = red[gg * tk.mpad + i];
            sr += v.x;
            si += v.y;
        }
        double2 *o = out + tk.out_off + i;
        if (beta_one) {
            const double2 p = *o;
            sr += p.x;
            si += p.y;
        }
        *o = make_double2(sr, si);
    }
}

template <int THREADS>
static cudaError_t launch_df_t(const Phase &ph, const float2 *mat, const Seg *segs, const double2 *in0,
                               const double2 *in1, double2 *out, int beta_one, cudaStream_t st)
{
    const size_t smem = (size_t)(2048 > 2 * THREADS ? 2048 : 2 * THREADS) * sizeof(float4);
    rowgemv_df_kernel<THREADS><<<ph.ntask(), THREADS, smem, st>>>(ph.d_tasks, segs, mat, in0, in1, out, beta_one);
    return cudaGetLastError();
}

template <int THREADS, typename VT>
static cudaError_t launch_t(const Phase &ph, const float2 *mat, const Seg *segs, const VT *in0,
                            const VT *in1, VT *out, int beta_one, cudaStream_t st)
{
    constexpr int CHUNK = VT_<VT>::CHUNK;
    const size_t smem = (size_t)(CHUNK > 2 * THREADS ? CHUNK : 2 * THREADS) * sizeof(VT);
    rowgemv_kernel<THREADS, VT><<<ph.ntask(), THREADS, smem, st>>>(ph.d_tasks, segs, mat, in0, in1,
                                                                    out, beta_one);
    return cudaGetLastError();
}

template <typename VT>
static cudaError_t launch_any(const Phase &ph, const float2 *mat, const Seg *segs, const VT *in0,
                             const VT *in1, VT *out, int beta_one, cudaStream_t st)
{
    if (ph.ntask() == 0) return cudaSuccess;
    switch (ph.threads) {
        case 128: return launch_t<128, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 192: return launch_t<192, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 256: return launch_t<256, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 384: return launch_t<384, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 512: return launch_t<512, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 768: return launch_t<768, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 1024: return launch_t<1024, VT>(ph, mat, segs, in0, in1, out, beta_one, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t launch_phase_f32(const Phase &ph, const float2 *mat, const Seg *segs, const float2 *in0,
                             const float2 *in1, float2 *out, int beta_one, cudaStream_t st)
{
    return launch_any<float2>(ph, mat, segs, in0, in1, out, beta_one, st);
}

cudaError_t launch_phase_f64(const Phase &ph, const float2 *mat, const Seg *segs, const double2 *in0,
                             const double2 *in1, double2 *out, int beta_one, cudaStream_t st)
{
    return launch_any<double2>(ph, mat, segs, in0, in1, out, beta_one, st);
}

cudaError_t launch_phase_df(const Phase &ph, const float2 *mat, const Seg *segs, const double2 *in0,
                            const double2 *in1, double2 *out, int beta_one, cudaStream_t st)
{
    if (ph.ntask() == 0) return cudaSuccess;
    switch (ph.threads) {
        case 128: return launch_df_t<128>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 192: return launch_df_t<192>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 256: return launch_df_t<256>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 384: return launch_df_t<384>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 512: return launch_df_t<512>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 768: return launch_df_t<768>(ph, mat, segs, in0, in1, out, beta_one, st);
        case 1024: return launch_df_t<1024>(ph, mat, segs, in0, in1, out, beta_one, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace h2
