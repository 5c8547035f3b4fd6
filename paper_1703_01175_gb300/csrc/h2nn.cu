// Kernels of the learned preconditioner (include/h2nn.h): the entry points of
// the 3x3x3 convolutions (tcgen05 implicit GEMMs in h2nn_tc.cu), bias
// gradients, ReLU backward, a relative mean-square loss, Adam, and the
// mapping between tree-order residual vectors and channel-last voxel grids.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "h2_internal.h"
#include "h2nn.h"

namespace h2 {

template <int CIN, int COUT>
cudaError_t launch_fwd_tc(const void *in, const void *w, const float *bias, void *out_bf16, float *out_f32, int B,
                          int Dx, int Dy, int Dz, int relu, cudaStream_t st);
template <int CIN, int COUT>
cudaError_t launch_bwdw_tc(const float *dz, const void *in, float *dw, int B, int Dx, int Dy, int Dz, cudaStream_t st);
int nn_tc_take_error();

namespace {

__global__ void flip_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt, int Cin, int Cout)
{
    const int n = Cout * 27 * Cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, t = (i / Cin) % 27, co = i / (27 * Cin);
        wt[((size_t)ci * 27 + (26 - t)) * Cout + co] = w[i];
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
    if (Cin == ci && Cout == co) e = launch_fwd_tc<ci, co>(in, w, bias, out_bf16, out_f32, B, Dx, Dy, Dz, relu, st);
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
    if (Cin == ci && Cout == co) e = launch_bwdw_tc<ci, co>(dz, in, dw, B, Dx, Dy, Dz, st);
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

h2_status h2nn_device_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        set_error("h2nn_device_status: device synchronisation failed");
        return H2_ERR_CUDA;
    }
    const int f = nn_tc_take_error();
    if (f < 0) {
        set_error("h2nn_device_status: reading the error flag failed");
        return H2_ERR_CUDA;
    }
    return f ? H2_ERR_TIMEOUT : H2_OK;
}

}  // extern "C"
