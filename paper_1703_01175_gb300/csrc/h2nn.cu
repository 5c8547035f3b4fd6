// Kernels of the learned preconditioner (include/h2nn.h): 3x3x3 convolutions
// as implicit GEMMs on the tensor cores (bf16 in, FP32 accumulate), their
// gradients, ReLU backward, a relative mean-square loss, Adam, and the
// mapping between tree-order residual vectors and channel-last voxel grids.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "h2_internal.h"
#include "h2nn.h"

namespace h2 {
namespace {

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ bool neighbour(int v, int tap, int Dx, int Dy, int Dz, int &nv)
{
    const int x = v % Dx, y = (v / Dx) % Dy, z = v / (Dx * Dy);
    const int nx = x + tap % 3 - 1, ny = y + (tap / 3) % 3 - 1, nz = z + tap / 9 - 1;
    if (nx < 0 || ny < 0 || nz < 0 || nx >= Dx || ny >= Dy || nz >= Dz) return false;
    nv = nx + Dx * (ny + Dy * nz);
    return true;
}

// Implicit-GEMM convolution: a CTA owns 64 voxels of one sample and all Cout
// channels; each of its 4 warps computes a 16-voxel x Cout block with
// m16n8k16 bf16 tensor-core MMAs over K = 27 Cin in steps of 16.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_fwd_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f,
                int Dx, int Dy, int Dz, int relu)
{
    constexpr int K = 27 * CIN;
    constexpr int KS = (K + 15) / 16;
    constexpr int NT = COUT / 8;
    __shared__ __align__(16) __nv_bfloat16 As[64][24];
    __shared__ __align__(16) __nv_bfloat16 Bs[COUT][24];
    const int V = Dx * Dy * Dz;
    const int b = blockIdx.y;
    const int v0 = blockIdx.x * 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, c = lane & 3;
    const int arow = tid >> 1, achunk = tid & 1;
    const int va = v0 + arow;
    const __nv_bfloat16 *inb = in + (size_t)b * V * CIN;
    float acc[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;

    for (int ks = 0; ks < KS; ++ks) {
        {
            const int k = ks * 16 + achunk * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            int nv;
            if (va < V && k < K && neighbour(va, k / CIN, Dx, Dy, Dz, nv))
                val = *reinterpret_cast<const uint4 *>(inb + (size_t)nv * CIN + (k % CIN));
            *reinterpret_cast<uint4 *>(&As[arow][achunk * 8]) = val;
        }
        if (tid < COUT * 2) {
            const int co = tid >> 1, ch = tid & 1;
            const int kb = ks * 16 + ch * 8;
            uint4 wv = make_uint4(0, 0, 0, 0);
            if (kb < K) wv = *reinterpret_cast<const uint4 *>(w + (size_t)co * K + kb);
            *reinterpret_cast<uint4 *>(&Bs[co][ch * 8]) = wv;
        }
        __syncthreads();
        uint32_t a[4];
        const int r = warp * 16 + g;
        a[0] = *reinterpret_cast<const uint32_t *>(&As[r][2 * c]);
        a[1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * c]);
        a[2] = *reinterpret_cast<const uint32_t *>(&As[r][2 * c + 8]);
        a[3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * c + 8]);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Bs[t * 8 + g][2 * c]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Bs[t * 8 + g][2 * c + 8]);
            mma_bf16_16816(acc[t], a, b0, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int co = t * 8 + 2 * c;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = v0 + warp * 16 + g + 8 * h;
            if (v >= V) continue;
            float x0 = acc[t][2 * h] + b0, x1 = acc[t][2 * h + 1] + b1;
            if (relu) {
                x0 = fmaxf(x0, 0.f);
                x1 = fmaxf(x1, 0.f);
            }
            const size_t o = ((size_t)b * V + v) * COUT + co;
            if (out_bf) *reinterpret_cast<__nv_bfloat162 *>(out_bf + o) = __floats2bfloat162_rn(x0, x1);
            if (out_f) *reinterpret_cast<float2 *>(out_f + o) = make_float2(x0, x1);
        }
    }
}

__global__ void flip_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt, int Cin, int Cout)
{
    const int n = Cout * 27 * Cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, t = (i / Cin) % 27, co = i / (27 * Cin);
        wt[((size_t)ci * 27 + (26 - t)) * Cout + co] = w[i];
    }
}

// dw[co][t][ci] += sum dz[b][v][co] in[b][v + off(t)][ci]: one CTA per (tap,
// voxel chunk); the CTA loops over samples and 64-voxel tiles.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
conv_bwdw_kernel(const float *__restrict__ dz, const __nv_bfloat16 *__restrict__ in, float *__restrict__ dw,
                 int B, int Dx, int Dy, int Dz, int vchunk)
{
    constexpr int TV = 64;
    constexpr int NP = (CIN * COUT + 255) / 256;
    __shared__ float dzs[TV][COUT];
    __shared__ float ins[TV][CIN + 1];
    const int V = Dx * Dy * Dz;
    const int tap = blockIdx.x;
    const int vbeg = blockIdx.y * vchunk, vend = min(V, vbeg + vchunk);
    float acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = 0.f;
    for (int b = 0; b < B; ++b) {
        for (int t0 = vbeg; t0 < vend; t0 += TV) {
            for (int e = threadIdx.x; e < TV * COUT; e += 256) {
                const int tv = e / COUT, co = e % COUT, v = t0 + tv;
                dzs[tv][co] = v < vend ? dz[((size_t)b * V + v) * COUT + co] : 0.f;
            }
            for (int e = threadIdx.x; e < TV * CIN; e += 256) {
                const int tv = e / CIN, ci = e % CIN, v = t0 + tv;
                int nv;
                float val = 0.f;
                if (v < vend && neighbour(v, tap, Dx, Dy, Dz, nv))
                    val = __bfloat162float(in[((size_t)b * V + nv) * CIN + ci]);
                ins[tv][ci] = val;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int p = threadIdx.x + 256 * q;
                if (p < CIN * COUT) {
                    const int co = p / CIN, ci = p % CIN;
                    float s = 0.f;
#pragma unroll 8
                    for (int tv = 0; tv < TV; ++tv) s += dzs[tv][co] * ins[tv][ci];
                    acc[q] += s;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int p = threadIdx.x + 256 * q;
        if (p < CIN * COUT) {
            const int co = p / CIN, ci = p % CIN;
            atomicAdd(&dw[((size_t)co * 27 + tap) * CIN + ci], acc[q]);
        }
    }
}

__global__ void bias_grad_kernel(const float *__restrict__ dz, float *__restrict__ db, int64_t rows, int C)
{
    // one block per channel chunk: blockIdx.y = channel
    const int co = blockIdx.y;
    float s = 0.f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        s += dz[r * C + co];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(&db[co], t);
    }
}

__global__ void relu_bwd_kernel(const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ y, float *dz,
                                int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : 0.f;
}

__global__ void f2bf_kernel(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// per-sample sums: parts[b] = sum (out - t)^2, parts[B + b] = sum t^2 (channels < Cu)
__global__ void mse_sums_kernel(const float *__restrict__ out, const float *__restrict__ tg, float *parts,
                                int B, int64_t V, int C, int Cu)
{
    const int b = blockIdx.y;
    float se = 0.f, st = 0.f;
    const int64_t n = V * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if ((int)(i % C) >= Cu) continue;
        const float o = out[(size_t)b * n + i], t = tg[(size_t)b * n + i];
        se += (o - t) * (o - t);
        st += t * t;
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&parts[b], se);
        atomicAdd(&parts[B + b], st);
    }
}

__global__ void mse_grad_kernel(const float *__restrict__ out, const float *__restrict__ tg, float *__restrict__ grad,
                                float *parts, int B, int64_t V, int C, int Cu)
{
    const int b = blockIdx.y;
    const int64_t n = V * C;
    const float den = fmaxf(parts[B + b], 1e-30f);
    const float sc = 2.f / (den * B);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const size_t k = (size_t)b * n + i;
        grad[k] = (int)(i % C) < Cu ? sc * (out[k] - tg[k]) : 0.f;
    }
}

__global__ void mse_finish_kernel(float *parts, int B)
{
    const int b = threadIdx.x;
    if (b < B) parts[b] = parts[b] / fmaxf(parts[B + b], 1e-30f);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void pack_kernel(const double2 *__restrict__ vec, int64_t ldv, const int32_t *__restrict__ grid_of,
                            const float *__restrict__ aux, const double *__restrict__ scale,
                            __nv_bfloat16 *__restrict__ chan, int nv, int64_t V)
{
    const int b = blockIdx.y;
    const double s = scale ? scale[b] : 1.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nv; p += gridDim.x * blockDim.x) {
        const int64_t v = grid_of[p];
        const double2 *q = vec + (int64_t)b * ldv + 3 * (int64_t)p;
        __nv_bfloat16 *o = chan + ((int64_t)b * V + v) * 8;
        __align__(16) __nv_bfloat16 t[8];
        for (int c = 0; c < 3; ++c) {
            t[2 * c] = __float2bfloat16_rn((float)(s * q[c].x));
            t[2 * c + 1] = __float2bfloat16_rn((float)(s * q[c].y));
        }
        t[6] = __float2bfloat16_rn(aux ? aux[v] : 0.f);
        t[7] = __float2bfloat16_rn(0.f);
        *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(t);
    }
}

__global__ void unpack_kernel(const float *__restrict__ chan, int C, const int32_t *__restrict__ grid_of,
                              const double *__restrict__ scale, double2 *__restrict__ vec, int64_t ldv, int nv,
                              int64_t V)
{
    const int b = blockIdx.y;
    const double s = scale ? scale[b] : 1.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nv; p += gridDim.x * blockDim.x) {
        const int64_t v = grid_of[p];
        const float *i = chan + ((int64_t)b * V + v) * C;
        double2 *q = vec + (int64_t)b * ldv + 3 * (int64_t)p;
        for (int c = 0; c < 3; ++c) q[c] = make_double2(s * i[2 * c], s * i[2 * c + 1]);
    }
}

inline int gridsz(int64_t n, int bs = 256) { return (int)std::min<int64_t>(4096, (n + bs - 1) / bs); }

}  // namespace

template <int CIN, int COUT>
static cudaError_t launch_fwd(const void *in, const void *w, const float *bias, void *ob, float *of, int B, int Dx,
                              int Dy, int Dz, int relu, cudaStream_t st)
{
    const int V = Dx * Dy * Dz;
    dim3 grid((V + 63) / 64, B);
    conv_fwd_kernel<CIN, COUT><<<grid, 128, 0, st>>>(
        reinterpret_cast<const __nv_bfloat16 *>(in), reinterpret_cast<const __nv_bfloat16 *>(w), bias,
        reinterpret_cast<__nv_bfloat16 *>(ob), of, Dx, Dy, Dz, relu);
    return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t launch_bwdw(const float *dz, const void *in, float *dw, int B, int Dx, int Dy, int Dz,
                               cudaStream_t st)
{
    const int V = Dx * Dy * Dz;
    const int vchunk = 2048;
    dim3 grid(27, (V + vchunk - 1) / vchunk);
    conv_bwdw_kernel<CIN, COUT><<<grid, 256, 0, st>>>(dz, reinterpret_cast<const __nv_bfloat16 *>(in), dw, B, Dx, Dy,
                                                      Dz, vchunk);
    return cudaGetLastError();
}

}  // namespace h2

using namespace h2;

static h2_status nn_err(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return H2_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return H2_ERR_CUDA;
}

static bool chan_ok(int c) { return c == 8 || c == 16 || c == 32; }

extern "C" {

h2_status h2nn_conv3d_fwd(const void *in, const void *w, const float *bias, void *out_bf16, float *out_f32,
                          int32_t B, int32_t Dx, int32_t Dy, int32_t Dz, int32_t Cin, int32_t Cout, int32_t relu,
                          void *stream)
{
    if (!in || !w || (!out_bf16 && !out_f32) || B < 1 || Dx < 1 || Dy < 1 || Dz < 1 || !chan_ok(Cin) ||
        !chan_ok(Cout) || (int64_t)Dx * Dy * Dz > (1LL << 30)) {
        set_error("h2nn_conv3d_fwd: bad argument");
        return H2_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaErrorInvalidValue;
#define H2NN_FWD(ci, co)                                                                          \
    if (Cin == ci && Cout == co) e = launch_fwd<ci, co>(in, w, bias, out_bf16, out_f32, B, Dx, Dy, Dz, relu, st);
    H2NN_FWD(8, 8) H2NN_FWD(8, 16) H2NN_FWD(8, 32) H2NN_FWD(16, 8) H2NN_FWD(16, 16) H2NN_FWD(16, 32)
    H2NN_FWD(32, 8) H2NN_FWD(32, 16) H2NN_FWD(32, 32)
#undef H2NN_FWD
    return nn_err(e, "h2nn_conv3d_fwd");
}

h2_status h2nn_flip_weights(const void *w, void *wt, int32_t Cin, int32_t Cout, void *stream)
{
    if (!w || !wt || Cin < 1 || Cout < 1) {
        set_error("h2nn_flip_weights: bad argument");
        return H2_ERR_ARG;
    }
    flip_kernel<<<gridsz((int64_t)Cout * 27 * Cin), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const __nv_bfloat16 *>(w), reinterpret_cast<__nv_bfloat16 *>(wt), Cin, Cout);
    return nn_err(cudaGetLastError(), "h2nn_flip_weights");
}

h2_status h2nn_conv3d_bwd_weight(const float *dz, const void *in, float *dw, float *db, int32_t B, int32_t Dx,
                                 int32_t Dy, int32_t Dz, int32_t Cin, int32_t Cout, int32_t accumulate,
                                 void *stream)
{
    if (!dz || !in || !dw || B < 1 || Dx < 1 || Dy < 1 || Dz < 1 || !chan_ok(Cin) || !chan_ok(Cout)) {
        set_error("h2nn_conv3d_bwd_weight: bad argument");
        return H2_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!accumulate) {
        if ((e = cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)Cout * 27 * Cin, st)) != cudaSuccess)
            return nn_err(e, "h2nn_conv3d_bwd_weight");
        if (db && (e = cudaMemsetAsync(db, 0, sizeof(float) * Cout, st)) != cudaSuccess)
            return nn_err(e, "h2nn_conv3d_bwd_weight");
    }
    e = cudaErrorInvalidValue;
#define H2NN_BW(ci, co) \
    if (Cin == ci && Cout == co) e = launch_bwdw<ci, co>(dz, in, dw, B, Dx, Dy, Dz, st);
    H2NN_BW(8, 8) H2NN_BW(8, 16) H2NN_BW(8, 32) H2NN_BW(16, 8) H2NN_BW(16, 16) H2NN_BW(16, 32)
    H2NN_BW(32, 8) H2NN_BW(32, 16) H2NN_BW(32, 32)
#undef H2NN_BW
    if (e != cudaSuccess) return nn_err(e, "h2nn_conv3d_bwd_weight");
    if (db) {
        const int64_t rows = (int64_t)B * Dx * Dy * Dz;
        dim3 grid((unsigned)std::min<int64_t>(256, (rows + 255) / 256), Cout);
        bias_grad_kernel<<<grid, 256, 0, st>>>(dz, db, rows, Cout);
        e = cudaGetLastError();
    }
    return nn_err(e, "h2nn_conv3d_bwd_weight");
}

h2_status h2nn_relu_bwd(const float *dy, const void *y, float *dz, int64_t count, void *stream)
{
    if (!dy || !y || !dz || count < 0) {
        set_error("h2nn_relu_bwd: bad argument");
        return H2_ERR_ARG;
    }
    if (count == 0) return H2_OK;
    relu_bwd_kernel<<<gridsz(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        dy, reinterpret_cast<const __nv_bfloat16 *>(y), dz, count);
    return nn_err(cudaGetLastError(), "h2nn_relu_bwd");
}

h2_status h2nn_f32_to_bf16(const float *in, void *out, int64_t count, void *stream)
{
    if (!in || !out || count < 0) {
        set_error("h2nn_f32_to_bf16: bad argument");
        return H2_ERR_ARG;
    }
    if (count == 0) return H2_OK;
    f2bf_kernel<<<gridsz(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        in, reinterpret_cast<__nv_bfloat16 *>(out), count);
    return nn_err(cudaGetLastError(), "h2nn_f32_to_bf16");
}

h2_status h2nn_mse(const float *out, const float *target, float *grad, float *loss_parts, int32_t B, int64_t V,
                   int32_t C, int32_t Cu, void *stream)
{
    if (!out || !target || !grad || !loss_parts || B < 1 || V < 1 || C < 1 || Cu < 1 || Cu > C || B > 65535) {
        set_error("h2nn_mse: bad argument");
        return H2_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(loss_parts, 0, sizeof(float) * 2 * B, st);
    if (e != cudaSuccess) return nn_err(e, "h2nn_mse");
    dim3 grid((unsigned)std::min<int64_t>(1024, (V * C + 255) / 256), B);
    mse_sums_kernel<<<grid, 256, 0, st>>>(out, target, loss_parts, B, V, C, Cu);
    mse_grad_kernel<<<grid, 256, 0, st>>>(out, target, grad, loss_parts, B, V, C, Cu);
    mse_finish_kernel<<<1, 1024, 0, st>>>(loss_parts, B);
    return nn_err(cudaGetLastError(), "h2nn_mse");
}

h2_status h2nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, int64_t count, float lr, float beta1,
                    float beta2, float eps, int32_t step, void *stream)
{
    if (!p || !g || !m || !v || count < 0 || step < 1) {
        set_error("h2nn_adam: bad argument");
        return H2_ERR_ARG;
    }
    if (count == 0) return H2_OK;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<gridsz(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        p, g, m, v, reinterpret_cast<__nv_bfloat16 *>(p_bf16), count, lr, beta1, beta2, eps, c1, c2);
    return nn_err(cudaGetLastError(), "h2nn_adam");
}

h2_status h2nn_pack(const void *vec, int64_t ldv, const int32_t *grid_of, const float *aux, const double *scale,
                    void *chan, int32_t B, int32_t nv, int64_t V, void *stream)
{
    if (!vec || !grid_of || !chan || B < 1 || nv < 1 || V < nv || ldv < 3LL * nv || B > 65535) {
        set_error("h2nn_pack: bad argument");
        return H2_ERR_ARG;
    }
    dim3 grid((unsigned)std::min(1024, (nv + 255) / 256), B);
    pack_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const double2 *>(vec), ldv, grid_of, aux, scale, reinterpret_cast<__nv_bfloat16 *>(chan),
        nv, V);
    return nn_err(cudaGetLastError(), "h2nn_pack");
}

h2_status h2nn_unpack(const float *chan, int32_t C, const int32_t *grid_of, const double *scale, void *vec,
                      int64_t ldv, int32_t B, int32_t nv, int64_t V, void *stream)
{
    if (!chan || !grid_of || !vec || C < 6 || B < 1 || nv < 1 || V < nv || ldv < 3LL * nv || B > 65535) {
        set_error("h2nn_unpack: bad argument");
        return H2_ERR_ARG;
    }
    dim3 grid((unsigned)std::min(1024, (nv + 255) / 256), B);
    unpack_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        chan, C, grid_of, scale, reinterpret_cast<double2 *>(vec), ldv, nv, V);
    return nn_err(cudaGetLastError(), "h2nn_unpack");
}

}  // extern "C"
