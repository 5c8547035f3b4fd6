// Multi-RHS H^2 product in FP32 (CUDA cores): every stage of the single-RHS
// product (Sec. IV.B; block-row tasks built by h2_load) becomes a small complex
// GEMM, out (m x R) (+)= M (m x ncol) X (ncol x R), for R right-hand sides at
// once (Sec. IV.D applies the same H^2 structure to a block of vectors).
//
// One CTA owns (task, chunk of RC = 32 right-hand sides, tile of 64 rows):
// the task's matrix columns and the gathered input rows are staged in shared
// memory 16 columns at a time, and each thread accumulates a 4-row x 2-RHS
// block of complex outputs in registers. Vectors are column-major with a
// leading dimension per buffer (x: ld0, coefficients: ld1, y: ldo).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "h2_internal.h"

namespace h2 {

namespace {
constexpr int MT = 256;   // threads
constexpr int RT = 64;    // rows per tile
constexpr int RC = 32;    // right-hand sides per CTA
constexpr int KB = 16;    // columns per stage
constexpr int IDXCAP = 4096;

__global__ void __launch_bounds__(MT)
rowgemm_f32_kernel(const Task *__restrict__ tasks, const Seg *__restrict__ segs, const float2 *__restrict__ mat,
                   const float2 *__restrict__ in0, int64_t ld0, const float2 *__restrict__ in1, int64_t ld1,
                   float2 *__restrict__ out, int64_t ldo, int nrhs, int beta_one)
{
    __shared__ float2 As[KB][RT];
    __shared__ float2 Xs[KB][RC];
    __shared__ int cidx[IDXCAP];          // encoded input index of each column of the current chunk

    const Task tk = tasks[blockIdx.x];
    const int r0 = blockIdx.y * RC;       // first right-hand side of this CTA
    const int row0 = blockIdx.z * RT;     // first row of this tile
    if (row0 >= tk.m) return;
    const int tid = threadIdx.x;
    const int rg = tid >> 4;              // 16 row groups of 4 rows
    const int cg = tid & 15;              // 16 rhs groups of 2 rhs
    float acc[4][2][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = 0.f;

    for (int c0 = 0; c0 < tk.ncol; c0 += IDXCAP) {
        const int cn = min(IDXCAP, tk.ncol - c0);
        __syncthreads();
        int cpos = 0;
        for (int s = tk.seg_begin; s < tk.seg_end && cpos < c0 + cn; ++s) {
            const Seg sg = segs[s];
            const int lo = max(cpos, c0), hi = min(cpos + sg.n, c0 + cn);
            for (int c = lo + tid; c < hi; c += MT) {
                const int j = c - cpos;
                cidx[c - c0] = sg.in_off >= 0 ? sg.in_off + j : sg.in_off - j;  // keeps the sign encoding
            }
            cpos += sg.n;
        }
        __syncthreads();
        for (int k0 = 0; k0 < cn; k0 += KB) {
            // A tile: KB columns x RT rows (column-major source, rows contiguous)
            for (int e = tid; e < KB * RT; e += MT) {
                const int j = e / RT, i = e % RT;
                const int col = k0 + j, row = row0 + i;
                float2 v = make_float2(0.f, 0.f);
                if (col < cn && row < tk.m) v = mat[tk.mat_off + (int64_t)(c0 + col) * tk.mpad + row];
                As[j][i] = v;
            }
            // X tile: KB columns x RC right-hand sides (columns fastest: contiguous within a segment)
            for (int e = tid; e < KB * RC; e += MT) {
                const int j = e % KB, r = e / KB;
                const int col = k0 + j, rr = r0 + r;
                float2 v = make_float2(0.f, 0.f);
                if (col < cn && rr < nrhs) {
                    const int ix = cidx[col];
                    v = ix >= 0 ? in0[(int64_t)rr * ld0 + ix] : in1[(int64_t)rr * ld1 + (-(int64_t)ix - 1)];
                }
                Xs[j][r] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                float2 a[4], x[2];
#pragma unroll
                for (int q = 0; q < 4; ++q) a[q] = As[j][rg * 4 + q];
#pragma unroll
                for (int q = 0; q < 2; ++q) x[q] = Xs[j][cg * 2 + q];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        acc[p][q][0] += a[p].x * x[q].x - a[p].y * x[q].y;
                        acc[p][q][1] += a[p].x * x[q].y + a[p].y * x[q].x;
                    }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int row = row0 + rg * 4 + p;
        if (row >= tk.m) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int rr = r0 + cg * 2 + q;
            if (rr >= nrhs) continue;
            float2 *o = out + (int64_t)rr * ldo + tk.out_off + row;
            float2 v = make_float2(acc[p][q][0], acc[p][q][1]);
            if (beta_one) {
                const float2 pv = *o;
                v.x += pv.x;
                v.y += pv.y;
            }
            *o = v;
        }
    }
}
}  // namespace

cudaError_t launch_phase_mrhs_f32(const Phase &ph, const float2 *mat, const Seg *segs, const float2 *in0,
                                  int64_t ld0, const float2 *in1, int64_t ld1, float2 *out, int64_t ldo, int nrhs,
                                  int beta_one, cudaStream_t st)
{
    if (ph.ntask() == 0) return cudaSuccess;
    const int rowtiles = (ph.max_mpad + RT - 1) / RT;
    dim3 grid(ph.ntask(), (nrhs + RC - 1) / RC, rowtiles);
    rowgemm_f32_kernel<<<grid, MT, 0, st>>>(ph.d_tasks, segs, mat, in0, ld0, in1, ld1, out, ldo, nrhs, beta_one);
    return cudaGetLastError();
}

}  // namespace h2

using namespace h2;

#define MR_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

h2_status h2_ensure_coefm(h2_handle *h, int nrhs)
{
    const int64_t ldc = std::max<int64_t>(2, 2 * h->ktot);
    const int64_t bytes = ldc * nrhs * (int64_t)sizeof(float2);
    if (bytes <= h->coefm_bytes) return H2_OK;
    cudaFree(h->d_coefm);
    h->d_coefm = nullptr;
    h->coefm_bytes = 0;
    if (cudaMalloc(&h->d_coefm, bytes) != cudaSuccess) {
        set_error("h2_matvec: multi-RHS coefficient allocation failed");
        return H2_ERR_ALLOC;
    }
    h->coefm_bytes = bytes;
    return H2_OK;
}

h2_status h2_run_multi_f32(h2_handle *h, const float2 *x, int64_t ldx, float2 *y, int64_t ldy, int nrhs,
                           cudaStream_t st)
{
    h2_status s = h2_ensure_coefm(h, nrhs);
    if (s != H2_OK) return s;
    const int64_t ldc = std::max<int64_t>(2, 2 * h->ktot);
    float2 *coef = reinterpret_cast<float2 *>(h->d_coefm);
    const float2 *mat = h->d_mat;
    const Seg *segs = h->d_segs;
    MR_CUDA(cudaMemsetAsync(coef, 0, sizeof(float2) * ldc * nrhs, st));
    MR_CUDA(cudaEventRecord(h->ev_fork, st));
    MR_CUDA(cudaStreamWaitEvent(h->s_aux, h->ev_fork, 0));
    MR_CUDA(launch_phase_mrhs_f32(h->near, mat, segs, x, ldx, coef, ldc, y, ldy, nrhs, 0, h->s_aux));
    MR_CUDA(cudaEventRecord(h->ev_near, h->s_aux));
    MR_CUDA(launch_phase_mrhs_f32(h->upleaf, mat, segs, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    for (int l = h->nlev - 1; l >= 0; --l)
        MR_CUDA(launch_phase_mrhs_f32(h->up[l], mat, segs, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    MR_CUDA(launch_phase_mrhs_f32(h->couple, mat, segs, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    for (int l = 0; l < h->nlev; ++l)
        MR_CUDA(launch_phase_mrhs_f32(h->down[l], mat, segs, x, ldx, coef, ldc, coef, ldc, nrhs, 1, st));
    MR_CUDA(cudaStreamWaitEvent(st, h->ev_near, 0));
    MR_CUDA(launch_phase_mrhs_f32(h->leafexp, mat, segs, x, ldx, coef, ldc, y, ldy, nrhs, 1, st));
    return H2_OK;
}
