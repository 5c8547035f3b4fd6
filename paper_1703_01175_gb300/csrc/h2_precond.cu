// The learned preconditioner held by a handle: a 3-D convolutional network
// on the voxel grid (weights and grid map copied from the caller), applied
// to one vector inside flexible GMRES (h2_krylov.cu), or to the R vectors of
// a batched solve in one pass of the network over R grids (h2_bkrylov.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "h2_internal.h"
#include "h2nn.h"

namespace {

struct Layer {
    int ci, co, relu;
    __nv_bfloat16 *w = nullptr;
    float *b = nullptr;
};

struct PrecondState {
    int Dx = 0, Dy = 0, Dz = 0;
    int64_t V = 0;
    int nv = 0;
    int32_t *grid_of = nullptr;
    float *aux = nullptr;
    std::vector<Layer> layers;
    __nv_bfloat16 *act[2] = {nullptr, nullptr};
    float *out = nullptr;
    double *scale = nullptr;  // [0] = sqrt(3 nv) / |v|, [1] = its inverse (set per application)
    int cmax = 8;
    // batched application: activations and outputs of bcap grids, scales [2][bcap]
    int bcap = 0;
    __nv_bfloat16 *bact[2] = {nullptr, nullptr};
    float *bout = nullptr;
    double *bscale = nullptr;
};

// scale[r] = sqrt(n) / |v_r|, scale[R + r] = its inverse: one block per vector
__global__ void set_scale_batched_kernel(const double2 *__restrict__ v, int64_t ldv, int n, int R, double *scale)
{
    const int r = blockIdx.x;
    const double2 *x = v + (size_t)r * ldv;
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i].x * x[i].x + x[i].y * x[i].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        const double nrm = sqrt(t);
        const double sc = nrm > 0 ? sqrt((double)n) / nrm : 1.0;
        scale[r] = sc;
        scale[R + r] = 1.0 / sc;
    }
}

// z_r += v_r, and z32_r = c64(z_r) when z32 is not NULL
__global__ void add_batched_kernel(double2 *__restrict__ z, int64_t ldz, const double2 *__restrict__ v, int64_t ldv,
                                   float2 *__restrict__ z32, int n)
{
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 a = z[(size_t)r * ldz + i];
        const double2 b = v[(size_t)r * ldv + i];
        a.x += b.x;
        a.y += b.y;
        z[(size_t)r * ldz + i] = a;
        if (z32) z32[(size_t)r * n + i] = make_float2((float)a.x, (float)a.y);
    }
}

__global__ void set_scale_kernel(const double2 *__restrict__ v, int n, double *scale)
{
    // one block: |v| by a block reduction
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i].x * v[i].x + v[i].y * v[i].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        const double nrm = sqrt(t);
        const double sc = nrm > 0 ? sqrt((double)n) / nrm : 1.0;
        scale[0] = sc;
        scale[1] = 1.0 / sc;
    }
}

// z += v (the network models the correction beyond the identity)
__global__ void add_c128_kernel(double2 *__restrict__ z, const double2 *__restrict__ v, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        z[i].x += v[i].x;
        z[i].y += v[i].y;
    }
}

__global__ void c128_to_c64_kernel(const double2 *__restrict__ a, float2 *__restrict__ b, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

void free_state(PrecondState *P)
{
    if (!P) return;
    cudaFree(P->grid_of);
    cudaFree(P->aux);
    for (auto &L : P->layers) {
        cudaFree(L.w);
        cudaFree(L.b);
    }
    cudaFree(P->act[0]);
    cudaFree(P->act[1]);
    cudaFree(P->out);
    cudaFree(P->scale);
    cudaFree(P->bact[0]);
    cudaFree(P->bact[1]);
    cudaFree(P->bout);
    cudaFree(P->bscale);
    delete P;
}

}  // namespace

void h2_free_precond(h2_handle *h)
{
    free_state(reinterpret_cast<PrecondState *>(h->precond));
    h->precond = nullptr;
}

h2_status h2_apply_precond(h2_handle *h, const double2 *v, double2 *z, float2 *z32, cudaStream_t st)
{
    PrecondState *P = reinterpret_cast<PrecondState *>(h->precond);
    if (!P) return H2_ERR_STATE;
    const int n = 3 * P->nv;
    set_scale_kernel<<<1, 1024, 0, st>>>(v, n, P->scale);
    if (P->nv < P->V) {  // grid voxels that are not unknowns read as zero
        if (cudaMemsetAsync(P->act[0], 0, (size_t)P->V * 8 * 2, st) != cudaSuccess) return H2_ERR_CUDA;
    }
    h2_status s = h2nn_pack(v, n, P->grid_of, P->aux, P->scale, P->act[0], 1, P->nv, P->V, st);
    if (s != H2_OK) return s;
    int cur = 0;
    for (size_t li = 0; li < P->layers.size(); ++li) {
        const Layer &L = P->layers[li];
        const bool last = li + 1 == P->layers.size();
        s = h2nn_conv3d_fwd(P->act[cur], L.w, L.b, last ? nullptr : P->act[1 - cur], last ? P->out : nullptr, 1,
                            P->Dx, P->Dy, P->Dz, L.ci, L.co, L.relu, st);
        if (s != H2_OK) return s;
        cur = 1 - cur;
    }
    s = h2nn_unpack(P->out, P->layers.back().co, P->grid_of, P->scale + 1, z, n, 1, P->nv, P->V, st);
    if (s != H2_OK) return s;
    add_c128_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(z, v, n);
    if (z32) {
        c128_to_c64_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(z, z32, n);
        if (cudaGetLastError() != cudaSuccess) return H2_ERR_CUDA;
    }
    return H2_OK;
}

h2_status h2_apply_precond_batched(h2_handle *h, const double2 *v, int64_t ldv, int R, double2 *z, int64_t ldz,
                                   float2 *z32, cudaStream_t st)
{
    PrecondState *P = reinterpret_cast<PrecondState *>(h->precond);
    if (!P) return H2_ERR_STATE;
    if (R < 1) return H2_ERR_ARG;
    if (R > P->bcap) {
        cudaFree(P->bact[0]);
        cudaFree(P->bact[1]);
        cudaFree(P->bout);
        cudaFree(P->bscale);
        P->bact[0] = P->bact[1] = nullptr;
        P->bout = nullptr;
        P->bscale = nullptr;
        P->bcap = 0;
        const size_t act = (size_t)R * P->V * P->cmax * 2;
        if (cudaMalloc(&P->bact[0], act) != cudaSuccess || cudaMalloc(&P->bact[1], act) != cudaSuccess ||
            cudaMalloc(&P->bout, (size_t)R * P->V * 8 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&P->bscale, 2 * (size_t)R * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            h2::set_error("learned preconditioner: allocation of the batched activations failed");
            return H2_ERR_ALLOC;
        }
        // grid voxels that are not unknowns read as zero input
        if (cudaMemset(P->bact[0], 0, act) != cudaSuccess) return H2_ERR_CUDA;
        P->bcap = R;
    }
    const int n = 3 * P->nv;
    set_scale_batched_kernel<<<R, 1024, 0, st>>>(v, ldv, n, R, P->bscale);
    if (P->nv < P->V) {  // grid voxels that are not unknowns read as zero (the layers reuse the buffer)
        if (cudaMemsetAsync(P->bact[0], 0, (size_t)R * P->V * 8 * 2, st) != cudaSuccess) return H2_ERR_CUDA;
    }
    h2_status s = h2nn_pack(v, ldv, P->grid_of, P->aux, P->bscale, P->bact[0], R, P->nv, P->V, st);
    if (s != H2_OK) return s;
    int cur = 0;
    for (size_t li = 0; li < P->layers.size(); ++li) {
        const Layer &L = P->layers[li];
        const bool last = li + 1 == P->layers.size();
        s = h2nn_conv3d_fwd(P->bact[cur], L.w, L.b, last ? nullptr : P->bact[1 - cur], last ? P->bout : nullptr, R,
                            P->Dx, P->Dy, P->Dz, L.ci, L.co, L.relu, st);
        if (s != H2_OK) return s;
        cur = 1 - cur;
    }
    s = h2nn_unpack(P->bout, P->layers.back().co, P->grid_of, P->bscale + R, z, ldz, R, P->nv, P->V, st);
    if (s != H2_OK) return s;
    dim3 g(std::min(1024, (n + 255) / 256), R);
    add_batched_kernel<<<g, 256, 0, st>>>(z, ldz, v, ldv, z32, n);
    return cudaGetLastError() == cudaSuccess ? H2_OK : H2_ERR_CUDA;
}

extern "C" h2_status h2_set_preconditioner(h2_handle *h, int32_t Dx, int32_t Dy, int32_t Dz,
                                           const int32_t *grid_of, const float *aux, int32_t n_layers,
                                           const int32_t *layer_spec, const void *weights, const float *biases)
{
    if (!h) {
        h2::set_error("h2_set_preconditioner: NULL handle");
        return H2_ERR_ARG;
    }
    if (n_layers == 0) {  // remove
        h2_free_precond(h);
        return H2_OK;
    }
    const int64_t V = (int64_t)Dx * Dy * Dz;
    if (Dx < 1 || Dy < 1 || Dz < 1 || n_layers < 1 || !grid_of || !layer_spec || !weights || !biases ||
        h->n % 3 != 0 || V < h->n / 3) {
        h2::set_error("h2_set_preconditioner: bad argument");
        return H2_ERR_ARG;
    }
    const int nv = h->n / 3;
    for (int p = 0; p < nv; ++p)
        if (grid_of[p] < 0 || grid_of[p] >= V) {
            h2::set_error("h2_set_preconditioner: grid index out of range");
            return H2_ERR_ARG;
        }
    int prev = 8;
    for (int l = 0; l < n_layers; ++l) {
        const int ci = layer_spec[3 * l], co = layer_spec[3 * l + 1];
        const bool ok = (ci == 8 || ci == 16 || ci == 32) && (co == 8 || co == 16 || co == 32) && ci == prev;
        if (!ok) {
            h2::set_error("h2_set_preconditioner: layer channels must chain 8 -> ... -> 8 in {8, 16, 32}");
            return H2_ERR_ARG;
        }
        prev = co;
    }
    if (prev != 8) {
        h2::set_error("h2_set_preconditioner: the last layer must have 8 output channels");
        return H2_ERR_ARG;
    }
    h2::DeviceGuard dev_guard(h->device);
    if (dev_guard.err != cudaSuccess) return H2_ERR_CUDA;
    h2_free_precond(h);
    auto *P = new PrecondState();
    P->Dx = Dx;
    P->Dy = Dy;
    P->Dz = Dz;
    P->V = V;
    P->nv = nv;
    P->bcap = 0;
    auto fail = [&](const char *what) {
        cudaGetLastError();  // clear an out-of-memory result
        h2::set_error(std::string("h2_set_preconditioner: ") + what);
        free_state(P);
        return H2_ERR_ALLOC;
    };
    int cmax = 8;
    const uint16_t *wsrc = reinterpret_cast<const uint16_t *>(weights);
    const float *bsrc = biases;
    for (int l = 0; l < n_layers; ++l) {
        Layer L;
        L.ci = layer_spec[3 * l];
        L.co = layer_spec[3 * l + 1];
        L.relu = layer_spec[3 * l + 2];
        cmax = std::max(cmax, std::max(L.ci, L.co));
        P->cmax = cmax;
        const size_t nw = (size_t)L.co * 27 * L.ci;
        if (cudaMalloc(&L.w, nw * 2) != cudaSuccess || cudaMalloc(&L.b, L.co * sizeof(float)) != cudaSuccess) {
            P->layers.push_back(L);
            return fail("allocation failed");
        }
        cudaMemcpy(L.w, wsrc, nw * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(L.b, bsrc, L.co * sizeof(float), cudaMemcpyHostToDevice);
        wsrc += nw;
        bsrc += L.co;
        P->layers.push_back(L);
    }
    if (cudaMalloc(&P->grid_of, nv * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&P->aux, V * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P->act[0], V * cmax * 2) != cudaSuccess || cudaMalloc(&P->act[1], V * cmax * 2) != cudaSuccess ||
        cudaMalloc(&P->out, V * 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P->scale, 2 * sizeof(double)) != cudaSuccess)
        return fail("allocation failed");
    cudaMemcpy(P->grid_of, grid_of, nv * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (aux)
        cudaMemcpy(P->aux, aux, V * sizeof(float), cudaMemcpyHostToDevice);
    else
        cudaMemset(P->aux, 0, V * sizeof(float));
    // grid voxels that are not unknowns must read as zero input
    cudaMemset(P->act[0], 0, V * cmax * 2);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_state(P);
        h2::set_error("h2_set_preconditioner: upload failed");
        return H2_ERR_CUDA;
    }
    h->precond = P;
    return H2_OK;
}
