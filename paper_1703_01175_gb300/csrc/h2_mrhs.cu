// Multi-RHS H^2 product in FP32 (CUDA cores): every stage of the single-RHS
// product (Sec. IV.B; block-row tasks built by h2_load) becomes a small complex
// GEMM, out (m x R) (+)= M (m x ncol) X (ncol x R), for R right-hand sides at
// once (Sec. IV.D applies the same H^2 structure to a block of vectors).
//
// One CTA owns (task, tile of MR = 32 rows, chunk of NR = 32 RPT right-hand
// sides): with NR = 128 a task's matrix is read from memory once for all
// right-hand sides. KB = 16 matrix columns and the matching gathered input
// rows are staged in shared memory per stage by asynchronous copies, NSTG
// stages in flight. Warp w owns rows 4w..4w+3 of the tile and lane l the
// right-hand sides l, l+32, ..., so a thread accumulates 4 x RPT complex
// outputs; the finished tile is transposed in shared memory so that the
// stores (and the reads of beta = 1) are 256-byte runs. The input index
// of every task column comes from a table built once (h2_ensure_colidx).
// Vectors are column-major with a leading dimension per buffer (x: ld0,
// coefficients: ld1, y: ldo).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "h2_internal.h"

namespace h2 {

namespace {
constexpr int GT = 256;   // threads
constexpr int MR = 32;    // rows per tile
constexpr int KB = 16;    // columns per stage
constexpr int NSTG = 3;   // stages in flight

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr size_t gemm_smem_bytes(int rpt)
{
    const size_t pipe = sizeof(float2) * NSTG * KB * (MR + 32 * rpt + 1);
    const size_t tile = sizeof(float2) * 32 * rpt * (MR + 1);
    return pipe > tile ? pipe : tile;
}

template <int RPT>
__global__ void __launch_bounds__(GT, 2)
rowgemm_f32_kernel(const Task *__restrict__ tasks, const int32_t *__restrict__ coloff,
                   const int32_t *__restrict__ colidx, const float2 *__restrict__ mat, const float2 *__restrict__ in0,
                   int64_t ld0, const float2 *__restrict__ in1, int64_t ld1, float2 *__restrict__ out, int64_t ldo,
                   int nrhs, int beta_one)
{
    constexpr int NR = 32 * RPT;
    constexpr int XS = NR + 1;  // odd row length of the X tile: conflict-free gathers
    extern __shared__ __align__(16) float2 gsm[];
    float2 *As = gsm;                     // [NSTG][KB][MR]
    float2 *Xs = gsm + NSTG * KB * MR;    // [NSTG][KB][XS]
    const Task tk = tasks[blockIdx.x];
    const int row0 = blockIdx.z * MR;
    if (row0 >= tk.m) return;
    const int r0 = blockIdx.y * NR;
    const int tid = threadIdx.x, lane = tid & 31, rg = tid >> 5;
    const int32_t *cix = colidx + coloff[blockIdx.x];
    const int nst = (tk.ncol + KB - 1) / KB;

    // Thread tid copies input column tid % KB of every stage (KB divides GT), so
    // it needs one column index per stage; the index of the next stage to be
    // issued is loaded one iteration ahead, off the critical path.
    const int xc = tid % KB, xr = tid / KB;
    auto col_index = [&](int stage) {
        const int col = stage * KB + xc;
        return col < tk.ncol ? cix[col] : 0;
    };
    auto load_stage = [&](int stage, int buf, int ix) {
        const int k0 = stage * KB;
        {  // matrix: KB columns x MR rows, two rows (16 bytes) per thread
            const int c = tid >> 4, rp = tid & 15;
            const int col = k0 + c, row = row0 + 2 * rp;
            const bool ok = col < tk.ncol && row < tk.mpad;
            const float2 *src = ok ? mat + tk.mat_off + (int64_t)col * tk.mpad + row : mat;
            cp_async16(As + (buf * KB + c) * MR + 2 * rp, src, ok);
        }
        const bool colok = k0 + xc < tk.ncol;
        const float2 *base = ix >= 0 ? in0 + ix : in1 + (-(int64_t)ix - 1);
        const int64_t ld = ix >= 0 ? ld0 : ld1;
#pragma unroll
        for (int q = 0; q < KB * NR / GT; ++q) {  // inputs: column xc, right-hand sides xr + (GT / KB) q
            const int r = xr + q * (GT / KB), rr = r0 + r;
            const bool ok = colok && rr < nrhs;
            cp_async8(Xs + (buf * KB + xc) * XS + r, ok ? base + (int64_t)rr * ld : in0, ok);
        }
    };

    float acc[4][RPT][2];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[p][q][0] = acc[p][q][1] = 0.f;

#pragma unroll
    for (int s = 0; s < NSTG - 1; ++s) {
        if (s < nst) load_stage(s, s, col_index(s));
        cp_async_commit();
    }
    int ix_next = col_index(NSTG - 1);
    for (int stage = 0; stage < nst; ++stage) {
        cp_async_wait<NSTG - 2>();
        __syncthreads();  // stage ready for all; buffer of stage - 1 free
        {
            const int ns = stage + NSTG - 1;
            if (ns < nst) load_stage(ns, ns % NSTG, ix_next);
            cp_async_commit();
            ix_next = col_index(ns + 1);
        }
        const int buf = stage % NSTG;
        const float2 *A = As + buf * KB * MR + rg * 4;
        const float2 *X = Xs + buf * KB * XS + lane;
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            const float4 a01 = *reinterpret_cast<const float4 *>(A + c * MR);
            const float4 a23 = *reinterpret_cast<const float4 *>(A + c * MR + 2);
            const float ar[4] = {a01.x, a01.z, a23.x, a23.z}, ai[4] = {a01.y, a01.w, a23.y, a23.w};
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const float2 x = X[c * XS + 32 * q];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    acc[p][q][0] = fmaf(ar[p], x.x, acc[p][q][0]);
                    acc[p][q][0] = fmaf(-ai[p], x.y, acc[p][q][0]);
                    acc[p][q][1] = fmaf(ar[p], x.y, acc[p][q][1]);
                    acc[p][q][1] = fmaf(ai[p], x.x, acc[p][q][1]);
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    // Epilogue through shared memory: the tile is transposed so that each warp
    // writes (and, with beta_one, reads) 32 consecutive rows of one right-hand
    // side, i.e. 256 contiguous bytes, instead of one scattered 32-byte run
    // per lane.
    constexpr int TS = MR + 1;  // odd stride: conflict-free transposition
    float2 *T = gsm;            // [NR][TS], fits in the pipeline buffers
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) T[(lane + 32 * q) * TS + rg * 4 + p] = make_float2(acc[p][q][0], acc[p][q][1]);
    __syncthreads();
    const int row = row0 + lane;
    if (row < tk.m) {
        for (int rl = rg; rl < NR; rl += GT / 32) {
            const int rr = r0 + rl;
            if (rr >= nrhs) break;
            float2 *o = out + (int64_t)rr * ldo + tk.out_off + row;
            float2 v = T[rl * TS + lane];
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

cudaError_t launch_phase_mrhs_f32(const Phase &ph, const float2 *mat, const float2 *in0, int64_t ld0,
                                  const float2 *in1, int64_t ld1, float2 *out, int64_t ldo, int nrhs, int beta_one,
                                  cudaStream_t st)
{
    if (ph.ntask() == 0) return cudaSuccess;
    const int rowtiles = (ph.max_mpad + MR - 1) / MR;
    const int rpt = nrhs > 64 ? 4 : nrhs > 32 ? 2 : 1;
    dim3 grid(ph.ntask(), (nrhs + 32 * rpt - 1) / (32 * rpt), rowtiles);
    const int32_t *ci = ph.d_colidx;
    switch (rpt) {
    case 4:
        rowgemm_f32_kernel<4><<<grid, GT, gemm_smem_bytes(4), st>>>(ph.d_tasks, ph.d_coloff, ci, mat, in0, ld0, in1,
                                                                     ld1, out, ldo, nrhs, beta_one);
        break;
    case 2:
        rowgemm_f32_kernel<2><<<grid, GT, gemm_smem_bytes(2), st>>>(ph.d_tasks, ph.d_coloff, ci, mat, in0, ld0, in1,
                                                                     ld1, out, ldo, nrhs, beta_one);
        break;
    default:
        rowgemm_f32_kernel<1><<<grid, GT, gemm_smem_bytes(1), st>>>(ph.d_tasks, ph.d_coloff, ci, mat, in0, ld0, in1,
                                                                     ld1, out, ldo, nrhs, beta_one);
        break;
    }
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
        cudaGetLastError();  // clear the out-of-memory result
        set_error("h2_matvec: multi-RHS coefficient allocation failed");
        return H2_ERR_ALLOC;
    }
    h->coefm_bytes = bytes;
    return H2_OK;
}

h2_status h2_ensure_colidx(h2_handle *h)
{
    if (h->d_colidx) return H2_OK;
    std::vector<Phase *> phases = {&h->near, &h->upleaf, &h->couple, &h->leafexp};
    for (auto &p : h->up) phases.push_back(&p);
    for (auto &p : h->down) phases.push_back(&p);
    std::vector<int32_t> idx;                       // column index tables, then the per-task offsets
    std::vector<std::vector<int32_t>> offs(phases.size());
    for (size_t k = 0; k < phases.size(); ++k) {
        for (const Task &t : phases[k]->tasks) {
            if (idx.size() > (size_t)INT_MAX) return (set_error("multi-RHS column table exceeds 2^31 entries"), H2_ERR_ARG);
            offs[k].push_back((int32_t)idx.size());
            for (int si = t.seg_begin; si < t.seg_end; ++si) {
                const Seg &sg = h->segs_host[si];
                for (int j = 0; j < sg.n; ++j) idx.push_back(sg.in_off >= 0 ? sg.in_off + j : sg.in_off - j);
            }
        }
    }
    const size_t nidx = idx.size();
    for (auto &o : offs) idx.insert(idx.end(), o.begin(), o.end());
    int32_t *d = nullptr;
    MR_CUDA(cudaMalloc(&d, std::max<size_t>(1, idx.size()) * sizeof(int32_t)));
    if (!idx.empty()) {
        cudaError_t e = cudaMemcpy(d, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            set_error(std::string("multi-RHS column table: ") + cudaGetErrorString(e));
            return H2_ERR_CUDA;
        }
    }
    size_t pos = nidx;
    for (size_t k = 0; k < phases.size(); ++k) {
        phases[k]->d_colidx = d;
        phases[k]->d_coloff = d + pos;
        pos += offs[k].size();
    }
    h->d_colidx = d;
    MR_CUDA(cudaFuncSetAttribute(rowgemm_f32_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_smem_bytes(4)));
    MR_CUDA(cudaFuncSetAttribute(rowgemm_f32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_smem_bytes(2)));
    MR_CUDA(cudaFuncSetAttribute(rowgemm_f32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_smem_bytes(1)));
    return H2_OK;
}

h2_status h2_run_multi_f32(h2_handle *h, const float2 *x, int64_t ldx, float2 *y, int64_t ldy, int nrhs,
                           cudaStream_t st)
{
    h2_status s = h2_ensure_coefm(h, nrhs);
    if (s != H2_OK) return s;
    if ((s = h2_ensure_colidx(h)) != H2_OK) return s;
    const int64_t ldc = std::max<int64_t>(2, 2 * h->ktot);
    float2 *coef = reinterpret_cast<float2 *>(h->d_coefm);
    const float2 *mat = h->d_mat;
    MR_CUDA(cudaMemsetAsync(coef, 0, sizeof(float2) * ldc * nrhs, st));
    MR_CUDA(cudaEventRecord(h->ev_fork, st));
    MR_CUDA(cudaStreamWaitEvent(h->s_aux, h->ev_fork, 0));
    MR_CUDA(launch_phase_mrhs_f32(h->near, mat, x, ldx, coef, ldc, y, ldy, nrhs, 0, h->s_aux));
    MR_CUDA(cudaEventRecord(h->ev_near, h->s_aux));
    MR_CUDA(launch_phase_mrhs_f32(h->upleaf, mat, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    for (int l = h->nlev - 1; l >= 0; --l)
        MR_CUDA(launch_phase_mrhs_f32(h->up[l], mat, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    MR_CUDA(launch_phase_mrhs_f32(h->couple, mat, x, ldx, coef, ldc, coef, ldc, nrhs, 0, st));
    for (int l = 0; l < h->nlev; ++l)
        MR_CUDA(launch_phase_mrhs_f32(h->down[l], mat, x, ldx, coef, ldc, coef, ldc, nrhs, 1, st));
    MR_CUDA(cudaStreamWaitEvent(st, h->ev_near, 0));
    MR_CUDA(launch_phase_mrhs_f32(h->leafexp, mat, x, ldx, coef, ldc, y, ldy, nrhs, 1, st));
    return H2_OK;
}
