// Multi-RHS H2 product on the 5th-generation tensor cores (tcgen05), with
// operands split into two bf16 terms and FP32 accumulation in tensor memory.
//
// For R right-hand sides a task out (m x R) = M (m x ncol) X (ncol x R) is the
// real GEMM  D (R x 2m) = Xr (R x 2 ncol) . A2 (2m x 2 ncol)^T  with
//   Xr[r][2c + 0/1] = Re/Im x_r(c)  and, per complex entry a = M[i][c],
//   A2[2i][2c] = Re a, A2[2i][2c+1] = -Im a, A2[2i+1][2c] = Im a, A2[2i+1][2c+1] = Re a,
// so that D[r][2i], D[r][2i+1] are the real and imaginary parts of y_r(i).
// Each operand is split as v = hi + lo (bf16) and D accumulates hi.hi, hi.lo and
// lo.hi (the lo.lo term is below the FP32 rounding of the result).
//
// Tiles: M = 128 right-hand sides (one tile of TMEM lanes), N = 2 m rounded up
// to 16 (<= 256), K staged 32 bf16 (16 complex columns) at a time in the
// no-swizzle K-major shared-memory layout. The matrix operand is pre-packed
// once on the device into that exact shared-memory image and fetched with one
// bulk asynchronous copy per stage. The right-hand-side operand lives in one
// pair of bf16 planes (hi, lo) stored chunk-major: a chunk is 4 complex
// entries (16 bytes) of all 128 right-hand sides of a tile, 2 KB contiguous,
// and every input segment starts on a chunk boundary, so a stage's operand is
// 4 bulk copies per plane. The planes hold x, the coefficients xh of the
// upward pass and yh of the downward pass; every transform writes its output
// split straight into them (thread = right-hand side = one 16-byte chunk row),
// so the tree passes never round-trip through FP32 buffers. The couplings of
// a cluster and its downward transfer share one tile (their columns
// concatenated along K), as do the near field and the leaf expansion of a leaf.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <unordered_map>
#include <vector>

#include "h2_internal.h"

namespace h2 {

namespace {

constexpr int UT = 128;               // threads per CTA (4 warps)
constexpr int KST = 32;               // bf16 K elements per stage
constexpr int CPS = KST / 2;          // complex columns per stage
constexpr int NCH = KST / 8;          // 16-byte K chunks per stage
constexpr int MT = 128;               // right-hand sides per tile (TMEM lanes)
constexpr int XPLANE = NCH * MT * 16; // bytes of one X plane image per stage
constexpr uint32_t kDrainLimit = 1u << 22;  // waits for copies and MMAs in flight after an abort

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for the phase with the given parity; false when `limit` polls ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor of the matrix operand: K-major, no swizzle,
// N rows of 16-byte chunks: 8-row core matrices 128 B apart, chunks 16 N B apart
__device__ __forceinline__ uint64_t bdesc(uint32_t saddr, int n)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)((16 * n) >> 4) << 16;             // leading byte offset: next chunk along K
    d |= (uint64_t)(128 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // layout type 0: no swizzle
}

// shared-memory matrix descriptor: K-major, no swizzle, 128 rows of 16-byte
// chunks: 8-row core matrices 128 B apart (stride), chunks 2 KB apart (leading)
__device__ __forceinline__ uint64_t xdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)(2048 >> 4) << 16;                 // leading byte offset: next chunk along K
    d |= (uint64_t)(128 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // layout type 0: no swizzle
}

// byte offset of chunk c (4 complex entries) of right-hand-side tile t in a
// chunk-major plane with nchp chunks per tile (the last one all zero)
__device__ __forceinline__ int64_t plane_chunk(int t, int64_t nchp, int c) { return ((int64_t)t * nchp + c) * (MT * 16); }

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

}  // namespace

// One tile of a split-bf16 task (see h2_internal.h: UTask), NS-stage pipelined. Thread 0
// produces: for each K stage it waits until the buffer is free (tcgen05.commit
// of the MMAs that read it) and issues the bulk copies of the matrix image and
// of the 16 right-hand-side chunks, which complete on the stage's `full`
// barrier (expect_tx); a missing chunk reads the plane's zero chunk. Lane 0 of
// warp 3 issues the MMAs of a stage once it is full and commits them to the
// stage's `empty` barrier. All four warps then read the accumulator out of
// tensor memory. Both operands use the no-swizzle K-major layout: right-hand
// sides as whole 2 KB chunks, the matrix image as NCH chunks of N rows.
template <int NS>
__global__ void __launch_bounds__(UT, 1)
umma_ws_kernel(const UTask *__restrict__ tasks, const int32_t *__restrict__ chunks,
               const uint8_t *__restrict__ images, __nv_bfloat16 *phi, __nv_bfloat16 *plo, int64_t nchp,
               int nrhs, float2 *__restrict__ out, int64_t ldo, int nmax, uint32_t tcols, int *__restrict__ err,
               uint32_t wait_limit)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const UTask tk = tasks[blockIdx.x];
    const int N = tk.n;
    const uint32_t abytes = (uint32_t)N * 16u * NCH;       // one plane of the matrix image per stage
    const uint32_t astride = 2u * (uint32_t)nmax * 16u * NCH;
    uint8_t *sxb = base;                                   // NS x (hi, lo) X planes
    uint8_t *sab = base + NS * 2 * XPLANE;                 // NS x (hi, lo) matrix planes
    uint64_t *bars = reinterpret_cast<uint64_t *>(sab + NS * astride);
    uint64_t *full = bars;
    uint64_t *empty = bars + NS;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS);
    __shared__ int abort_flag, issued, consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.y * MT;
    if (tid == 0) {
        abort_flag = 0;
        issued = consumed = 0;
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        // producer: per stage one bulk copy of the matrix image and 2 NCH bulk
        // copies of right-hand-side chunks (NCH per plane), all completing on
        // the stage's `full` barrier; chunk indices are read a stage ahead
        const uint8_t *ph = reinterpret_cast<const uint8_t *>(phi), *pl = reinterpret_cast<const uint8_t *>(plo);
        static_assert(NCH == 4, "one int4 of chunk indices per stage");
        const int4 *cq = reinterpret_cast<const int4 *>(chunks + tk.chunk_off);
        int4 c0 = tk.nst > 0 ? cq[0] : make_int4(-1, -1, -1, -1);
        for (int s = 0; s < tk.nst; ++s) {
            const int b = s % NS;
            const int ci[NCH] = {c0.x, c0.y, c0.z, c0.w};
            if (s + 1 < tk.nst) c0 = cq[s + 1];
            if (s >= NS && !mbar_wait(&empty[b], ((s / NS) - 1) & 1, wait_limit)) {
                abort_flag = 1;
                break;
            }
            issued = s + 1;
            uint8_t *sx = sxb + b * 2 * XPLANE;
            uint8_t *sa = sab + b * astride;
            mbar_expect_tx(&full[b], 2 * abytes + 2 * XPLANE);
            bulk_g2s(sa, images + tk.img_off + (int64_t)s * 2 * abytes, 2 * abytes, &full[b]);
#pragma unroll
            for (int q = 0; q < NCH; ++q) {
                const int64_t off = plane_chunk(blockIdx.y, nchp, ci[q] >= 0 ? ci[q] >> 2 : (int)nchp - 1);
                bulk_g2s(sx + q * 2048, ph + off, 2048, &full[b]);
                bulk_g2s(sx + XPLANE + q * 2048, pl + off, 2048, &full[b]);
            }
        }
    } else if (warp == 3 && lane == 0) {
        const uint32_t idesc = idesc_bf16(N);
        for (int s = 0; s < tk.nst; ++s) {
            const int b = s % NS;
            if (!mbar_wait(&full[b], (s / NS) & 1, wait_limit)) {
                abort_flag = 1;
                break;
            }
            consumed = s + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t xa = smem_u32(sxb + b * 2 * XPLANE), xb = xa + XPLANE;
            const uint32_t aa = smem_u32(sab + b * astride), ab = aa + abytes;
#pragma unroll
            for (int k = 0; k < KST / 16; ++k) {
                const uint32_t xo = k * 2 * 2048, bo = k * 2 * 16 * (uint32_t)N;   // two chunks per K step
                const uint32_t first = (s == 0 && k == 0) ? 0u : 1u;
                umma(tmem, xdesc(xa + xo), bdesc(aa + bo, N), idesc, first);   // hi . hi
                umma(tmem, xdesc(xa + xo), bdesc(ab + bo, N), idesc, 1u);      // hi . lo
                umma(tmem, xdesc(xb + xo), bdesc(aa + bo, N), idesc, 1u);      // lo . hi
            }
            umma_commit(&empty[b]);
        }
    }
    __syncthreads();
    if (!abort_flag && tk.nst > 0) {
        const int last = tk.nst - 1;
        if (tid == 0 && !mbar_wait(&empty[last % NS], (last / NS) & 1, wait_limit)) abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag && tid == 0) {
        // a wait ran out: before the CTA releases its shared and tensor memory,
        // let the copies of issued stages land and the committed MMAs finish
        for (int st = consumed; st < issued; ++st) mbar_wait(&full[st % NS], (st / NS) & 1, kDrainLimit);
        if (consumed > 0) mbar_wait(&empty[(consumed - 1) % NS], ((consumed - 1) / NS) & 1, kDrainLimit);
        atomicExch(err, 1);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag && tk.nst > 0) {
        // thread = right-hand side r (TMEM lane); accumulator columns 2i, 2i + 1
        // = Re, Im of output row i
        const int rr = warp * 32 + lane, r = r0 + rr;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j0 = 0; j0 < N; j0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tl + (uint32_t)j0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < nrhs) {
                const int i0 = j0 >> 1;
                if (out) {
                    float2 *o = out + (int64_t)r * ldo + tk.out_off;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (i0 + q < tk.m) o[i0 + q] = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
                } else {
                    // split into the plane: two chunks of 4 complex entries (a chunk
                    // that starts below m may hold padding rows, whose sums are 0)
#pragma unroll
                    for (int hc = 0; hc < 2; ++hc) {
                        const int ib = i0 + 4 * hc;
                        if (ib < tk.m) {
                            __align__(16) __nv_bfloat16 hv[8];
                            __align__(16) __nv_bfloat16 lv[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float f = __uint_as_float(v[8 * hc + e]);
                                hv[e] = __float2bfloat16_rn(f);
                                lv[e] = __float2bfloat16_rn(f - __bfloat162float(hv[e]));
                            }
                            const int64_t off =
                                (((int64_t)blockIdx.y * nchp + ((tk.out_off + ib) >> 2)) * MT + rr) * 8;
                            *reinterpret_cast<uint4 *>(phi + off) = *reinterpret_cast<const uint4 *>(hv);
                            *reinterpret_cast<uint4 *>(plo + off) = *reinterpret_cast<const uint4 *>(lv);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

size_t umma_ws_smem_bytes(int ns, int nmax) { return (size_t)ns * (2 * XPLANE + 2 * (size_t)nmax * 16 * NCH) + 1024 + 128; }

// Pack the real-expanded, bf16-split matrix images of every tile/stage; column
// pc of a task starts at element colmap[colmap_off + pc] of mat (-1: padding).
__global__ void umma_pack_kernel(const UTask *__restrict__ tasks, const UPackInfo *__restrict__ info,
                                 const int64_t *__restrict__ colmap, const float2 *__restrict__ mat,
                                 uint8_t *__restrict__ images)
{
    const UTask tk = tasks[blockIdx.x];
    const UPackInfo pi = info[blockIdx.x];
    const int N = tk.n;
    const int s = blockIdx.y;
    if (s >= tk.nst) return;
    uint8_t *img = images + tk.img_off + (int64_t)s * 2 * N * 16 * NCH;
    for (int e = threadIdx.x; e < N * KST; e += blockDim.x) {
        const int nr = e / KST, kk = e % KST;
        const int i = pi.row0 + (nr >> 1);                 // complex row in the task matrix
        const int pc = s * CPS + (kk >> 1);                // padded complex column
        const int64_t c = pc < pi.npc ? colmap[pi.colmap_off + pc] : -1;   // column start in mat
        float v = 0.f;
        if (c >= 0 && (nr >> 1) < tk.m) {
            const float2 a = mat[c + i];
            const int part = nr & 1, comp = kk & 1;
            v = part == 0 ? (comp == 0 ? a.x : -a.y) : (comp == 0 ? a.y : a.x);
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const int byte = (kk >> 3) * (16 * N) + nr * 16 + (kk & 7) * 2;   // chunk, row, element
        *reinterpret_cast<__nv_bfloat16 *>(img + byte) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(img + N * 16 * NCH + byte) = lo;
    }
}

// Fill plane positions [p0, pend) of chunk-major bf16 hi/lo planes: position
// d of right-hand side r holds src[r * lds + pos[d]] (zero where pos[d] < 0),
// stored in chunk d / 4 of tile r / 128, row r % 128, bytes 4 (d % 4) .. + 4
// (Re, Im); nchp chunks per tile; p0 is a multiple of 4. A block transposes
// 32 positions x 32 right-hand sides through shared memory, so that reads run
// along positions and each warp writes 32 consecutive 16-byte chunk rows.
__global__ void __launch_bounds__(256)
split_scatter_kernel(const float2 *__restrict__ src, int64_t lds, const int32_t *__restrict__ pos, int p0, int pend,
                     int nrhs, __nv_bfloat16 *__restrict__ phi, __nv_bfloat16 *__restrict__ plo, int64_t nchp)
{
    __shared__ float2 tile[32][33];
    const int d0 = p0 + blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int pd = d0 + tx < pend ? pos[d0 + tx] : -1;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr;
        tile[rr][tx] = (pd >= 0 && r < nrhs) ? src[(int64_t)r * lds + pd] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int r = r0 + tx, c = (d0 >> 2) + ty;
    if (r >= nrhs || 4 * c >= pend) return;
    __align__(16) __nv_bfloat16 hv[8];
    __align__(16) __nv_bfloat16 lv[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 v = tile[tx][4 * ty + k];
        hv[2 * k] = __float2bfloat16_rn(v.x);
        hv[2 * k + 1] = __float2bfloat16_rn(v.y);
        lv[2 * k] = __float2bfloat16_rn(v.x - __bfloat162float(hv[2 * k]));
        lv[2 * k + 1] = __float2bfloat16_rn(v.y - __bfloat162float(hv[2 * k + 1]));
    }
    const int64_t off = (((int64_t)(r / MT) * nchp + c) * MT + (r % MT)) * 8;
    *reinterpret_cast<uint4 *>(phi + off) = *reinterpret_cast<const uint4 *>(hv);
    *reinterpret_cast<uint4 *>(plo + off) = *reinterpret_cast<const uint4 *>(lv);
}


}  // namespace h2

using namespace h2;

#define UM_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));           \
            return H2_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

// A task of the tensor-core path: one output block and the handle's tasks
// that write it, concatenated along K (their columns follow one another).
struct MTask {
    int32_t out_off;                 // y offset or plane position of the first output row
    int32_t m;                       // output rows (every part has m rows)
    std::vector<const Task *> parts;
};

// Host side: build tiles, chunk tables and packed images of one phase. seg_pos
// gives the plane position of a segment's first entry.
template <class SegPos>
static h2_status build_uphase(h2_handle *h, std::vector<MTask> mts, const std::vector<Seg> &hsegs, SegPos seg_pos,
                              UPhase &U)
{
    // largest tasks first, as the handle orders its own phases
    auto work = [](const MTask &t) {
        int64_t c = 0;
        for (const Task *p : t.parts) c += p->ncol;
        return (int64_t)t.m * c;
    };
    std::stable_sort(mts.begin(), mts.end(), [&](const MTask &a, const MTask &b) { return work(a) > work(b); });
    std::vector<UTask> tiles;
    std::vector<UPackInfo> infos;
    std::vector<int32_t> chunks;
    std::vector<int64_t> colmap;
    int64_t img = 0;
    for (const MTask &t : mts) {
        // padded columns: each segment rounded up to a multiple of 4 complex entries
        std::vector<int64_t> cm;        // padded column -> element offset of the column in mat (-1 pad)
        std::vector<int32_t> chunk_src; // per 4-column chunk: plane position of its first entry
        for (const Task *pt : t.parts) {
            int orig = 0;
            for (int si = pt->seg_begin; si < pt->seg_end; ++si) {
                const Seg &sg = hsegs[si];
                const int32_t pbase = seg_pos(sg);
                const int np = (sg.n + 3) / 4 * 4;
                for (int j = 0; j < np; ++j) cm.push_back(j < sg.n ? pt->mat_off + (int64_t)(orig + j) * pt->mpad : -1);
                for (int j = 0; j < np; j += 4) chunk_src.push_back(pbase + j);
                orig += sg.n;
            }
        }
        const int npc = (int)cm.size();
        const int nst = (npc + CPS - 1) / CPS;
        while ((int)chunk_src.size() < nst * (CPS / 4)) chunk_src.push_back(-1);
        const int64_t colmap_off = (int64_t)colmap.size();
        colmap.insert(colmap.end(), cm.begin(), cm.end());
        const int chunk_off = (int)chunks.size();
        chunks.insert(chunks.end(), chunk_src.begin(), chunk_src.end());
        for (int row0 = 0; row0 < t.m; row0 += 128) {
            const int mt = std::min(128, t.m - row0);
            UTask u{};
            u.out_off = t.out_off + row0;
            u.m = mt;
            u.n = 2 * ((mt + 7) / 8 * 8);
            u.nst = nst;
            u.img_off = img;
            u.chunk_off = chunk_off;
            img += (int64_t)nst * 2 * u.n * 16 * NCH;
            tiles.push_back(u);
            UPackInfo pi{};
            pi.row0 = row0;
            pi.npc = npc;
            pi.colmap_off = colmap_off;
            infos.push_back(pi);
        }
    }
    U.ntile = (int)tiles.size();
    U.image_bytes = img;
    U.nmax = 16;
    U.maxnst = 0;
    for (auto &u : tiles) {
        U.nmax = std::max(U.nmax, u.n);
        U.maxnst = std::max(U.maxnst, u.nst);
    }
    if (U.ntile == 0) return H2_OK;
    UTask *d_tiles = nullptr;
    UPackInfo *d_info = nullptr;
    int64_t *d_colmap = nullptr;
    UM_CUDA(cudaMalloc(&d_tiles, tiles.size() * sizeof(UTask)));
    UM_CUDA(cudaMalloc(&d_info, infos.size() * sizeof(UPackInfo)));
    UM_CUDA(cudaMalloc(&d_colmap, std::max<size_t>(1, colmap.size()) * sizeof(int64_t)));
    UM_CUDA(cudaMalloc(&U.d_chunks, std::max<size_t>(1, chunks.size()) * sizeof(int32_t)));
    UM_CUDA(cudaMalloc(&U.d_images, std::max<int64_t>(16, img)));
    UM_CUDA(cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(UTask), cudaMemcpyHostToDevice));
    UM_CUDA(cudaMemcpy(d_info, infos.data(), infos.size() * sizeof(UPackInfo), cudaMemcpyHostToDevice));
    if (!colmap.empty())
        UM_CUDA(cudaMemcpy(d_colmap, colmap.data(), colmap.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (!chunks.empty())
        UM_CUDA(cudaMemcpy(U.d_chunks, chunks.data(), chunks.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    int maxst = 0;
    for (auto &u : tiles) maxst = std::max(maxst, u.nst);
    dim3 grid(U.ntile, maxst);
    umma_pack_kernel<<<grid, 256>>>(d_tiles, d_info, d_colmap, h->d_mat, U.d_images);
    UM_CUDA(cudaGetLastError());
    UM_CUDA(cudaDeviceSynchronize());
    U.d_tasks = d_tiles;
    cudaFree(d_info);
    cudaFree(d_colmap);
    return H2_OK;
}

static h2_status split_init(h2_handle *h)
{
    if (h->split) return H2_OK;
    auto *S = new SplitState();
    h->split = S;
    S->pipeline = h->tc_pipeline;
    S->wait_limit = h->wait_limit;
    // plane layout: leaves in tree order (x), then the coefficient blocks of
    // the clusters (xh, then yh), each block padded to 4 complex entries
    std::vector<int32_t> leaf_pbase(h->nc, -1), coef_pbase(h->nc, -1);
    int64_t p = 0;
    std::vector<int32_t> xs, xd;
    for (int t = 0; t < h->nc; ++t) {
        if (h->child[2 * t] >= 0) continue;
        leaf_pbase[t] = (int32_t)p;
        for (int i = 0; i < h->size[t]; ++i) {
            xs.push_back(h->begin[t] + i);
            xd.push_back((int32_t)(p + i));
        }
        p += (h->size[t] + 3) / 4 * 4;
    }
    S->np_x = std::max<int64_t>(8, (p + 3) / 4 * 4);
    int64_t q = 0;
    for (int t = 0; t < h->nc; ++t) {
        if (h->rank[t] == 0) continue;
        coef_pbase[t] = (int32_t)q;
        q += (h->rank[t] + 3) / 4 * 4;
    }
    S->np_c = std::max<int64_t>(8, (q + 3) / 4 * 4);
    S->nch = (S->np_x + 2 * S->np_c) / 4 + 1;
    if ((S->nch - 1) * 4 > INT32_MAX) {
        set_error("split-bf16: plane positions exceed 32 bits");
        return H2_ERR_STATE;
    }
    const int32_t xh0 = (int32_t)S->np_x, yh0 = (int32_t)(S->np_x + S->np_c);
    std::vector<int32_t> xpos(S->np_x, -1);
    for (size_t k = 0; k < xs.size(); ++k) xpos[xd[k]] = xs[k];
    UM_CUDA(cudaMalloc(&S->d_xpos, xpos.size() * sizeof(int32_t)));
    UM_CUDA(cudaMemcpy(S->d_xpos, xpos.data(), xpos.size() * sizeof(int32_t), cudaMemcpyHostToDevice));

    // plane position of a segment: x entries of a leaf, or a cluster's xh / yh
    const std::vector<Seg> &hsegs = h->segs_host;
    std::unordered_map<int32_t, int32_t> leaf_of_begin, cluster_of_xo;
    for (int t = 0; t < h->nc; ++t) {
        if (h->child[2 * t] < 0) leaf_of_begin[h->begin[t]] = t;
        if (h->rank[t] > 0) cluster_of_xo[h->xo[t]] = t;
    }
    auto seg_pos = [&](const Seg &sg) -> int32_t {
        if (sg.in_off >= 0) return leaf_pbase[leaf_of_begin.at(sg.in_off)];   // whole leaves
        const int64_t off = -(int64_t)sg.in_off - 1;
        if (off >= h->ktot) return yh0 + coef_pbase[cluster_of_xo.at((int32_t)(off - h->ktot))];
        return xh0 + coef_pbase[cluster_of_xo.at((int32_t)off)];
    };
    // the handle's tasks by output offset (y rows, xh or yh of a cluster)
    auto by_out = [](const Phase &ph) {
        std::unordered_map<int32_t, const Task *> m;
        for (const Task &t : ph.tasks) m[t.out_off] = &t;
        return m;
    };
    auto find = [](const std::unordered_map<int32_t, const Task *> &m, int32_t k) -> const Task * {
        auto it = m.find(k);
        return it == m.end() ? nullptr : it->second;
    };
    const auto near = by_out(h->near), leafexp = by_out(h->leafexp), upleaf = by_out(h->upleaf),
               couple = by_out(h->couple);
    std::vector<std::unordered_map<int32_t, const Task *>> up(h->nlev), down(h->nlev);
    for (int l = 0; l < h->nlev; ++l) {
        up[l] = by_out(h->up[l]);
        down[l] = by_out(h->down[l]);
    }
    std::vector<MTask> leaf_t, upleaf_t;
    std::vector<std::vector<MTask>> up_t(h->nlev), level_t(h->nlev);
    for (int t = 0; t < h->nc; ++t) {
        const int l = h->level[t];
        const bool is_leaf = h->child[2 * t] < 0;
        if (is_leaf) {
            MTask m{h->begin[t], h->size[t], {}};
            if (const Task *a = find(near, h->begin[t])) m.parts.push_back(a);
            if (const Task *a = find(leafexp, h->begin[t])) m.parts.push_back(a);
            if (m.parts.empty()) S->zero_y = true;
            else leaf_t.push_back(m);
        }
        if (h->rank[t] == 0) continue;
        const int32_t xo = (int32_t)h->xo[t], yo = (int32_t)(h->ktot + h->xo[t]);
        if (is_leaf) {
            if (const Task *a = find(upleaf, xo)) upleaf_t.push_back({xh0 + coef_pbase[t], h->rank[t], {a}});
        } else if (const Task *a = find(up[l], xo)) {
            up_t[l].push_back({xh0 + coef_pbase[t], h->rank[t], {a}});
        }
        MTask m{yh0 + coef_pbase[t], h->rank[t], {}};
        if (const Task *a = find(couple, yo)) m.parts.push_back(a);
        if (const Task *a = find(down[l], yo)) m.parts.push_back(a);
        if (!m.parts.empty()) level_t[l].push_back(m);
    }
    h2_status st;
    if ((st = build_uphase(h, leaf_t, hsegs, seg_pos, S->leaf)) != H2_OK) return st;
    if ((st = build_uphase(h, upleaf_t, hsegs, seg_pos, S->upleaf)) != H2_OK) return st;
    S->up.resize(h->nlev);
    S->level.resize(h->nlev);
    for (int l = 0; l < h->nlev; ++l) {
        if ((st = build_uphase(h, up_t[l], hsegs, seg_pos, S->up[l])) != H2_OK) return st;
        if ((st = build_uphase(h, level_t[l], hsegs, seg_pos, S->level[l])) != H2_OK) return st;
    }
    int nmax = std::max(S->leaf.nmax, S->upleaf.nmax);
    for (int l = 0; l < h->nlev; ++l) nmax = std::max(nmax, std::max(S->up[l].nmax, S->level[l].nmax));
    {
        // dynamic shared memory limit = opt-in per-block maximum minus the kernels' static shared memory
        int optin = 0;
        UM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
        cudaFuncAttributes fa{};
        UM_CUDA(cudaFuncGetAttributes(&fa, umma_ws_kernel<2>));
        S->dyn_smem_limit = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (umma_ws_smem_bytes(2, nmax) > S->dyn_smem_limit) {
            set_error("split-bf16: two pipeline stages of the widest tile exceed shared memory");
            return H2_ERR_STATE;
        }
        const int lim = (int)S->dyn_smem_limit;
        UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    }
    UM_CUDA(cudaMalloc(&S->d_err, sizeof(int)));
    UM_CUDA(cudaMemset(S->d_err, 0, sizeof(int)));
    return H2_OK;
}

static h2_status ensure_planes(h2_handle *h, int rpad)
{
    SplitState *S = h->split;
    if (rpad <= S->rcap) return H2_OK;
    cudaFree(S->phi);
    cudaFree(S->plo);
    S->phi = S->plo = nullptr;
    S->rcap = 0;
    // chunk-major: per tile of 128 right-hand sides, nch chunks of 2 KB
    const size_t bytes = (size_t)rpad * S->nch * 16;
    if (cudaMalloc(&S->phi, bytes) != cudaSuccess || cudaMalloc(&S->plo, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("split-bf16 plane allocation failed");
        return H2_ERR_ALLOC;
    }
    // entries that no kernel writes stay zero: the zero chunk, padding between
    // blocks, and the xh / yh of clusters that no task writes
    UM_CUDA(cudaMemset(S->phi, 0, bytes));
    UM_CUDA(cudaMemset(S->plo, 0, bytes));
    S->rcap = rpad;
    return H2_OK;
}

// Deepest pipeline that fits in shared memory and that the phase's longest
// tile can use (two stages when the pipeline option is off); tensor memory
// columns: the power of two that holds the widest accumulator.
static cudaError_t launch_umma(const UPhase &U, const SplitState *S, int nrhs, float2 *out, int64_t ldo,
                               cudaStream_t st)
{
    if (U.ntile == 0) return cudaSuccess;
    dim3 grid(U.ntile, (nrhs + MT - 1) / MT);
    int ns = 2;
    if (S->pipeline)
        for (int c = std::min(6, std::max(2, U.maxnst)); c > 2; --c)
            if (umma_ws_smem_bytes(c, U.nmax) <= S->dyn_smem_limit) {
                ns = c;
                break;
            }
    uint32_t tcols = 32;
    while ((int)tcols < U.nmax) tcols <<= 1;
    const size_t sm = umma_ws_smem_bytes(ns, U.nmax);
    __nv_bfloat16 *phi = reinterpret_cast<__nv_bfloat16 *>(S->phi), *plo = reinterpret_cast<__nv_bfloat16 *>(S->plo);
#define H2_UMMA_LAUNCH(NSV)                                                                                  \
    umma_ws_kernel<NSV><<<grid, UT, sm, st>>>(U.d_tasks, U.d_chunks, U.d_images, phi, plo, S->nch, nrhs, out, \
                                              ldo, U.nmax, tcols, S->d_err, S->wait_limit)
    switch (ns) {
        case 6: H2_UMMA_LAUNCH(6); break;
        case 5: H2_UMMA_LAUNCH(5); break;
        case 4: H2_UMMA_LAUNCH(4); break;
        case 3: H2_UMMA_LAUNCH(3); break;
        default: H2_UMMA_LAUNCH(2); break;
    }
#undef H2_UMMA_LAUNCH
    return cudaGetLastError();
}

void h2_free_split(h2_handle *h)
{
    SplitState *S = h->split;
    if (!S) return;
    std::vector<UPhase *> all = {&S->leaf, &S->upleaf};
    for (UPhase &U : S->up) all.push_back(&U);
    for (UPhase &U : S->level) all.push_back(&U);
    for (UPhase *U : all) {
        cudaFree(U->d_tasks);
        cudaFree(U->d_chunks);
        cudaFree(U->d_images);
    }
    cudaFree(S->d_xpos);
    cudaFree(S->phi);
    cudaFree(S->plo);
    cudaFree(S->d_err);
    delete S;
    h->split = nullptr;
}

// Product for R right-hand sides: x is split into the plane once; every
// transform writes its output coefficients into the plane, split, where the
// next level's tiles read them; only the leaf phase writes FP32 (y).
h2_status h2_run_multi_split(h2_handle *h, const float2 *x, int64_t ldx, float2 *y, int64_t ldy, int nrhs,
                             cudaStream_t st)
{
    h2_status s = split_init(h);
    if (s != H2_OK) return s;
    SplitState *S = h->split;
    const int rpad = (nrhs + MT - 1) / MT * MT;
    if ((s = ensure_planes(h, rpad)) != H2_OK) return s;
    dim3 g((unsigned)((S->np_x + 31) / 32), (nrhs + 31) / 32);
    split_scatter_kernel<<<g, 256, 0, st>>>(x, ldx, S->d_xpos, 0, (int)S->np_x, nrhs,
                                            reinterpret_cast<__nv_bfloat16 *>(S->phi),
                                            reinterpret_cast<__nv_bfloat16 *>(S->plo), S->nch);
    UM_CUDA(cudaGetLastError());
    // upward pass: forward transforms of the leaves, then level by level
    UM_CUDA(launch_umma(S->upleaf, S, nrhs, nullptr, 0, st));
    for (int l = h->nlev - 1; l >= 0; --l) UM_CUDA(launch_umma(S->up[l], S, nrhs, nullptr, 0, st));
    // couplings with the downward transfer from the parent, root to leaves
    for (int l = 0; l < h->nlev; ++l) UM_CUDA(launch_umma(S->level[l], S, nrhs, nullptr, 0, st));
    if (S->zero_y) UM_CUDA(cudaMemset2DAsync(y, sizeof(float2) * ldy, 0, sizeof(float2) * h->n, nrhs, st));
    UM_CUDA(launch_umma(S->leaf, S, nrhs, y, ldy, st));
    return H2_OK;
}

h2_status h2_split_error_flag(h2_handle *h, int *flag)
{
    *flag = 0;
    if (!h->split) return H2_OK;
    UM_CUDA(cudaMemcpy(flag, h->split->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return H2_OK;
}

h2_status h2_split_set_pipeline(h2_handle *h, int on)
{
    h2_status s = split_init(h);
    if (s != H2_OK) return s;
    h->split->pipeline = on != 0;
    return H2_OK;
}
