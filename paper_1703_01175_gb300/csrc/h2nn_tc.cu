// 3x3x3 convolutions of the learned preconditioner on the 5th-generation
// tensor cores (tcgen05): the forward (and, with flipped weights, data-
// gradient) implicit GEMM and the weight-gradient GEMM, bf16 operands with
// FP32 accumulation in tensor memory (include/h2nn.h).
//
// Forward: a CTA owns 128 consecutive voxels of one sample (M = 128, one TMEM
// lane each) and all output channels (N = Cout, at least 16). The 27 taps are
// the K stages: per tap every thread gathers its voxel's neighbour row (Cin
// bf16 = Cin / 8 chunks of 16 bytes, zero outside the grid) into a shared-
// memory tile in the canonical no-swizzle K-major layout (chunk-major: a chunk
// is 16 bytes of all 128 rows), double buffered; one thread issues the MMAs of
// the tap against the weights, which stay in shared memory for all 27 taps, and
// commits them to the buffer's mbarrier. The epilogue reads the accumulator
// (thread = voxel), adds the bias, applies ReLU and stores bf16 and/or FP32.
//
// Weight gradient: dw[co][t][ci] = sum over samples and voxels of
// dz[v][co] in[v + off(t)][ci]. M = 128 rows = (tap, ci) pairs of 128 / Cin
// taps, N = Cout, K = voxels in stages of 64; the activations are bf16 already
// (exact operand), dz (FP32) is split into bf16 hi + lo and both products are
// accumulated, so the result keeps about 16 significant bits per term. Each
// CTA covers one M tile and one range of voxels and adds its tile into dw
// atomically.
//
// Every mbarrier wait is bounded; a wait that runs out sets a device flag
// (h2nn_device_status), lets the issued MMAs drain and skips the output.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "h2_internal.h"
#include "h2_tc.cuh"

namespace h2 {
namespace {

using namespace tc;

__device__ int g_h2nn_tc_error = 0;
constexpr uint32_t kConvWaitLimit = 1u << 24;

__device__ __forceinline__ bool neighbour_of(int x, int y, int z, int tap, int Dx, int Dy, int Dz, int &nv)
{
    const int nx = x + tap % 3 - 1, ny = y + (tap / 3) % 3 - 1, nz = z + tap / 9 - 1;
    if (nx < 0 || ny < 0 || nz < 0 || nx >= Dx || ny >= Dy || nz >= Dz) return false;
    nv = nx + Dx * (ny + Dy * nz);
    return true;
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[N])
{
    static_assert(N == 16 || N == 32, "16 or 32 accumulator columns");
#pragma unroll
    for (int h = 0; h < N / 16; ++h) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + (uint32_t)(16 * h)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) v[16 * h + q] = __uint_as_float(r[q]);
    }
}

template <int CIN, int COUT>
struct ConvShape {
    static constexpr int CP = CIN < 16 ? 16 : CIN;     // K per tap, padded to the MMA's K of 16
    static constexpr int NCH = CP / 8;                 // 16-byte chunks per operand row
    static constexpr int N = COUT < 16 ? 16 : COUT;    // MMA N
    static constexpr int ABYTES = NCH * 128 * 16;      // one tap's activation tile
    static constexpr int WTAP = NCH * N * 16;          // one tap's weights
    static constexpr size_t SMEM = 1024 + 2 * ABYTES + 27 * WTAP + 64;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_fwd_tc_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                   const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f,
                   int Dx, int Dy, int Dz, int relu)
{
    using S = ConvShape<CIN, COUT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *As = base;                                  // 2 x ABYTES
    uint8_t *Ws = base + 2 * S::ABYTES;                  // 27 x WTAP
    uint64_t *empty = reinterpret_cast<uint64_t *>(Ws + 27 * S::WTAP);   // 2 mbarriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty + 2);
    __shared__ int abort_flag;
    __shared__ int committed;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int V = Dx * Dy * Dz;
    const int b = blockIdx.y;
    const int v = blockIdx.x * 128 + tid;
    const bool vok = v < V;
    const int x = v % Dx, y = (v / Dx) % Dy, z = v / (Dx * Dy);
    const __nv_bfloat16 *inb = in + (size_t)b * V * CIN;

    // weights of all taps in the K-major layout: tap t, chunk c, row co
    for (int e = tid; e < 27 * S::N * S::NCH; e += 128) {
        const int c = e % S::NCH, co = (e / S::NCH) % S::N, t = e / (S::NCH * S::N);
        uint4 val = make_uint4(0, 0, 0, 0);
        if (co < COUT && 8 * c < CIN) val = *reinterpret_cast<const uint4 *>(w + ((size_t)co * 27 + t) * CIN + 8 * c);
        *reinterpret_cast<uint4 *>(Ws + t * S::WTAP + c * (16 * S::N) + co * 16) = val;
    }
    if (tid == 0) {
        abort_flag = 0;
        committed = 0;
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = idesc_bf16(S::N);

    for (int t = 0; t < 27; ++t) {
        const int buf = t & 1;
        if (t >= 2 && tid == 0 && !mbar_wait(&empty[buf], ((t - 2) >> 1) & 1, kConvWaitLimit)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        uint8_t *A = As + buf * S::ABYTES;
        int nv = 0;
        const bool ok = vok && neighbour_of(x, y, z, t, Dx, Dy, Dz, nv);
#pragma unroll
        for (int c = 0; c < S::NCH; ++c) {
            uint4 val = make_uint4(0, 0, 0, 0);
            if (ok && 8 * c < CIN) val = *reinterpret_cast<const uint4 *>(inb + (size_t)nv * CIN + 8 * c);
            *reinterpret_cast<uint4 *>(A + c * 2048 + tid * 16) = val;
        }
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aa = smem_u32(A), wa = smem_u32(Ws + t * S::WTAP);
#pragma unroll
            for (int q = 0; q < S::NCH / 2; ++q)
                umma(tmem, kdesc(aa + q * 4096, 2048), bdesc(wa + q * 2 * 16 * S::N, S::N), idesc,
                     (t > 0 || q > 0) ? 1u : 0u);
            umma_commit(&empty[buf]);
            committed = t + 1;
        }
    }
    __syncthreads();
    if (tid == 0 && committed > 0) {
        // the last commit covers every MMA issued before it
        const int last = committed - 1;
        if (!mbar_wait(&empty[last & 1], (last >> 1) & 1, kConvWaitLimit)) abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(&g_h2nn_tc_error, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag) {
        float acc[S::N];
        tmem_load_row<S::N>(tmem + ((uint32_t)(warp * 32) << 16), acc);
        if (vok) {
            const size_t o = ((size_t)b * V + v) * COUT;
#pragma unroll
            for (int co = 0; co < COUT; co += 2) {
                float a0 = acc[co] + (bias ? bias[co] : 0.f), a1 = acc[co + 1] + (bias ? bias[co + 1] : 0.f);
                if (relu) {
                    a0 = fmaxf(a0, 0.f);
                    a1 = fmaxf(a1, 0.f);
                }
                if (out_bf) *reinterpret_cast<__nv_bfloat162 *>(out_bf + o + co) = __floats2bfloat162_rn(a0, a1);
                if (out_f) *reinterpret_cast<float2 *>(out_f + o + co) = make_float2(a0, a1);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

template <int CIN, int COUT>
struct BwdShape {
    static constexpr int TPT = 128 / CIN;              // taps per M tile
    static constexpr int MT = (27 + TPT - 1) / TPT;    // M tiles
    static constexpr int N = COUT < 16 ? 16 : COUT;
    static constexpr int KV = 64;                      // voxels per K stage
    static constexpr int NCH = KV / 8;                 // 16-byte chunks along K
    static constexpr int ABYTES = NCH * 128 * 16;      // activation tile
    static constexpr int BBYTES = NCH * N * 16;        // one dz plane (hi or lo)
    static constexpr int STAGE = ABYTES + 2 * BBYTES;
    static constexpr size_t SMEM = 1024 + 2 * STAGE + 64;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_bwdw_tc_kernel(const float *__restrict__ dz, const __nv_bfloat16 *__restrict__ in, float *__restrict__ dw,
                    int B, int Dx, int Dy, int Dz, int vchunk)
{
    using S = BwdShape<CIN, COUT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *empty = reinterpret_cast<uint64_t *>(base + 2 * S::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty + 2);
    __shared__ int abort_flag;
    __shared__ int committed;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int V = Dx * Dy * Dz;
    const int64_t total = (int64_t)B * V;
    const int tap0 = blockIdx.x * S::TPT;
    const int64_t k0 = (int64_t)blockIdx.y * vchunk, k1 = k0 + vchunk < total ? k0 + vchunk : total;
    const int nst = (int)((k1 - k0 + S::KV - 1) / S::KV);

    if (tid == 0) {
        abort_flag = 0;
        committed = 0;
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = idesc_bf16(S::N);

    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        if (s >= 2 && tid == 0 && !mbar_wait(&empty[buf], ((s - 2) >> 1) & 1, kConvWaitLimit)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        uint8_t *A = base + buf * S::STAGE;
        uint8_t *Bh = A + S::ABYTES, *Bl = Bh + S::BBYTES;
        const int64_t kb = k0 + (int64_t)s * S::KV;
        // activations: row (tap tt, channel ci) = tt * CIN + ci, column k (voxel kb + k); one 16-byte
        // load of 8 channels per (k, tt, chunk), scattered into 8 rows
        for (int e = tid; e < S::KV * S::TPT * (CIN / 8); e += 128) {
            const int k = e % S::KV, rest = e / S::KV, tt = rest % S::TPT, ch = rest / S::TPT;
            const int64_t kv = kb + k;
            const int tap = tap0 + tt;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (kv < k1 && tap < 27) {
                const int bb = (int)(kv / V), vv = (int)(kv % V);
                const int x = vv % Dx, y = (vv / Dx) % Dy, z = vv / (Dx * Dy);
                int nv;
                if (neighbour_of(x, y, z, tap, Dx, Dy, Dz, nv))
                    val = *reinterpret_cast<const uint4 *>(in + ((size_t)bb * V + nv) * CIN + 8 * ch);
            }
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&val);
            uint8_t *col = A + (k >> 3) * 2048 + (k & 7) * 2;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<__nv_bfloat16 *>(col + (tt * CIN + 8 * ch + q) * 16) = h[q];
        }
        // dz split into bf16 hi and lo: row co, column k
        for (int e = tid; e < S::KV * (S::N / 4); e += 128) {
            const int k = e % S::KV, c4 = e / S::KV;
            const int64_t kv = kb + k;
            float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kv < k1 && 4 * c4 < COUT) d = *reinterpret_cast<const float4 *>(dz + (size_t)kv * COUT + 4 * c4);
            const float dv[4] = {d.x, d.y, d.z, d.w};
            const int off = (k >> 3) * (16 * S::N) + (k & 7) * 2;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat16 hi = __float2bfloat16_rn(dv[q]);
                const __nv_bfloat16 lo = __float2bfloat16_rn(dv[q] - __bfloat162float(hi));
                *reinterpret_cast<__nv_bfloat16 *>(Bh + off + (4 * c4 + q) * 16) = hi;
                *reinterpret_cast<__nv_bfloat16 *>(Bl + off + (4 * c4 + q) * 16) = lo;
            }
        }
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aa = smem_u32(A), ha = smem_u32(Bh), la = smem_u32(Bl);
#pragma unroll
            for (int q = 0; q < S::NCH / 2; ++q) {
                const uint64_t ad = kdesc(aa + q * 4096, 2048);
                umma(tmem, ad, bdesc(ha + q * 2 * 16 * S::N, S::N), idesc, (s > 0 || q > 0) ? 1u : 0u);
                umma(tmem, ad, bdesc(la + q * 2 * 16 * S::N, S::N), idesc, 1u);
            }
            umma_commit(&empty[buf]);
            committed = s + 1;
        }
    }
    __syncthreads();
    if (tid == 0 && committed > 0) {
        const int last = committed - 1;
        if (!mbar_wait(&empty[last & 1], (last >> 1) & 1, kConvWaitLimit)) abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(&g_h2nn_tc_error, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag && committed > 0) {
        float acc[S::N];
        tmem_load_row<S::N>(tmem + ((uint32_t)(warp * 32) << 16), acc);
        const int tt = tid / CIN, ci = tid % CIN, tap = tap0 + tt;
        if (tap < 27) {
#pragma unroll
            for (int co = 0; co < COUT; ++co) atomicAdd(&dw[((size_t)co * 27 + tap) * CIN + ci], acc[co]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

}  // namespace

template <int CIN, int COUT>
cudaError_t launch_fwd_tc(const void *in, const void *w, const float *bias, void *out_bf16, float *out_f32, int B,
                          int Dx, int Dy, int Dz, int relu, cudaStream_t st)
{
    using S = ConvShape<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(conv_fwd_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t V = (int64_t)Dx * Dy * Dz;
    dim3 grid((unsigned)((V + 127) / 128), (unsigned)B);
    conv_fwd_tc_kernel<CIN, COUT><<<grid, 128, S::SMEM, st>>>(
        reinterpret_cast<const __nv_bfloat16 *>(in), reinterpret_cast<const __nv_bfloat16 *>(w), bias,
        reinterpret_cast<__nv_bfloat16 *>(out_bf16), out_f32, Dx, Dy, Dz, relu);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_bwdw_tc(const float *dz, const void *in, float *dw, int B, int Dx, int Dy, int Dz, cudaStream_t st)
{
    using S = BwdShape<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(conv_bwdw_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)B * Dx * Dy * Dz;
    // about four CTAs per SM of 152 over the M tiles and voxel ranges, each range a whole number of stages
    int64_t chunks = std::max<int64_t>(1, (4 * 152 + S::MT - 1) / S::MT);
    int64_t vchunk = (total + chunks - 1) / chunks;
    vchunk = std::max<int64_t>(S::KV, (vchunk + S::KV - 1) / S::KV * S::KV);
    chunks = (total + vchunk - 1) / vchunk;
    dim3 grid((unsigned)S::MT, (unsigned)chunks);
    conv_bwdw_tc_kernel<CIN, COUT><<<grid, 128, S::SMEM, st>>>(dz, reinterpret_cast<const __nv_bfloat16 *>(in), dw,
                                                              B, Dx, Dy, Dz, (int)vchunk);
    return cudaGetLastError();
}

#define H2NN_TC_INST(ci, co)                                                                                      \
    template cudaError_t launch_fwd_tc<ci, co>(const void *, const void *, const float *, void *, float *, int, int, \
                                               int, int, int, cudaStream_t);                                       \
    template cudaError_t launch_bwdw_tc<ci, co>(const float *, const void *, float *, int, int, int, int, cudaStream_t);
H2NN_TC_INST(8, 8)
H2NN_TC_INST(8, 16)
H2NN_TC_INST(8, 32)
H2NN_TC_INST(16, 8)
H2NN_TC_INST(16, 16)
H2NN_TC_INST(16, 32)
H2NN_TC_INST(32, 8)
H2NN_TC_INST(32, 16)
H2NN_TC_INST(32, 32)
#undef H2NN_TC_INST

int nn_tc_take_error()
{
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_h2nn_tc_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (flag) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_h2nn_tc_error, &zero, sizeof(int));
    }
    return flag;
}

}  // namespace h2
