// Multi-RHS H2 product on the 5th-generation tensor cores (tcgen05), with
// operands split into two bf16 terms and FP32 accumulation in tensor memory.
//
// For R right-hand sides a task out (m x R) = M (m x ncol) X (ncol x R) is
// formed from two real GEMMs that share one matrix operand:
//   P (R x 2m) = Xre (R x ncol) . B (2m x ncol)^T,
//   Q (R x 2m) = Xim (R x ncol) . B (2m x ncol)^T,
// where B holds each complex entry a = M[i][c] once: row "re i" = Re a, row
// "im i" = Im a, in groups of 8 output rows (8 re rows, then the 8 im rows).
// Then y_r(i) = (P[r][re i] - Q[r][im i]) + j (P[r][im i] + Q[r][re i]):
// the complex product needs no real expansion of the matrix, which is stored
// and streamed at 8 bytes per complex entry (hi and lo bf16 of Re and Im).
// Each operand is split as v = hi + lo (bf16); P and Q accumulate hi.hi,
// hi.lo and lo.hi (the lo.lo term is below the FP32 rounding of the result).
//
// Tiles: M = 128 right-hand sides (one tile of TMEM lanes), N = 2 m rounded
// up to 16 (<= 256), K staged 16 complex columns (one MMA K step) at a time
// in the no-swizzle K-major shared-memory layout. The matrix operand is
// pre-packed once on the device into that exact shared-memory image and
// fetched with one bulk asynchronous copy per stage. The right-hand-side
// operand lives in one pair of bf16 planes (hi, lo) stored group-major: a
// group is 8 complex entries of all 128 right-hand sides of a tile, as a
// 2 KB chunk of their real parts followed by a 2 KB chunk of their imaginary
// parts, and every input segment starts on a group boundary, so a stage's
// operand is one or two bulk copies per plane. The planes hold x, the
// coefficients xh of the upward pass and yh of the downward pass; every
// transform writes its output split straight into them (thread = right-hand
// side = one 16-byte chunk row per part), so the tree passes never
// round-trip through FP32 buffers. The couplings of a cluster and its
// downward transfer share one tile (their columns concatenated along K), as
// do the near field and the leaf expansion of a leaf.
//
// At most 64 right-hand sides use a packed plane layout: a group is one 2 KB
// chunk whose rows 0-63 hold the real parts and rows 64-127 the imaginary
// parts, so one 128-row operand carries both and a single accumulator D holds
// P in TMEM lanes 0-63 and Q in lanes 64-127 (three MMAs per stage instead of
// six, half the right-hand-side bytes, so deeper pipelines fit); the epilogue
// exchanges the two lane halves through shared memory. The layout is a
// template parameter of the kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <unordered_map>
#include <vector>

#include "h2_internal.h"
#include "h2_tc.cuh"

namespace h2 {

namespace {

using namespace tc;

constexpr int UT = 128;               // threads per CTA (4 warps)
constexpr int CPS = 16;               // complex columns per stage (one MMA K step of 16)
constexpr int GRP = 8;                // complex entries per plane group (one 16-byte chunk row per part)
constexpr int MT = 128;               // right-hand sides per tile (TMEM lanes)
constexpr int CHUNK = MT * 16;        // bytes of one chunk (16 bytes of each of 128 right-hand sides)
constexpr int GBYTES = 2 * CHUNK;     // bytes of one group of one plane: Re chunk, then Im chunk
constexpr int XPLANE = (CPS / GRP) * GBYTES;  // bytes of one plane's right-hand-side operand per stage
constexpr int NSMAX = 8;              // deepest pipeline (16 NSMAX + 4 bytes of barriers fit the 256 reserved)

// shared-memory matrix descriptor of the right-hand-side operand: K-major, no
// swizzle, 128 rows of 16-byte chunks: 8-row core matrices 128 B apart
// (stride), consecutive K chunks one plane group (4 KB) apart (leading)
__device__ __forceinline__ uint64_t xdesc(uint32_t saddr, uint32_t lbo = GBYTES)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;       // leading byte offset: next chunk along K
    d |= (uint64_t)(128 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // layout type 0: no swizzle
}

// byte offset of group g (8 complex entries) of right-hand-side tile t in a
// group-major plane with ngrp groups per tile (the last one all zero); gbytes
// is GBYTES, or CHUNK in the packed layout of at most 64 right-hand sides (one
// 2 KB chunk per group: rows 0-63 the real parts, rows 64-127 the imaginary
// parts of right-hand sides 0-63)
__device__ __forceinline__ int64_t plane_group(int t, int64_t ngrp, int64_t g, uint32_t gbytes = GBYTES)
{
    return ((int64_t)t * ngrp + g) * gbytes;
}

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes (one
// per thread); the caller waits (tcgen05.wait::ld) before using them
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(u[e]);
}

__device__ __forceinline__ void split_bf16x8(const float *v, __nv_bfloat16 *hv, __nv_bfloat16 *lv)
{
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        hv[e] = __float2bfloat16_rn(v[e]);
        lv[e] = __float2bfloat16_rn(v[e] - __bfloat162float(hv[e]));
    }
}

}  // namespace

// One tile of a split-bf16 task (see h2_internal.h: UTask), NS-stage pipelined. Thread 0
// produces: for each K stage it waits until the buffer is free (tcgen05.commit
// of the MMAs that read it) and issues the bulk copies of the matrix image and
// of the stage's two right-hand-side groups (merged into one copy per plane
// when they are adjacent), which complete on the stage's `full` barrier
// (expect_tx); a missing group reads the plane's zero group. Lane 0 of warp 3
// issues the MMAs of a stage once it is full (three split products into P from
// the real parts, three into Q from the imaginary parts) and commits them to
// the stage's `empty` barrier. All four warps then read both accumulators out
// of tensor memory and combine them.
template <int NS, bool packed>
__global__ void __launch_bounds__(UT, 1)
umma_ws_kernel(const UTask *__restrict__ tasks, const int32_t *__restrict__ groups,
               const uint8_t *__restrict__ images, __nv_bfloat16 *phi, __nv_bfloat16 *plo, int64_t ngrp,
               int nrhs, float2 *__restrict__ out, int64_t ldo, int nmax, uint32_t tcols, int *__restrict__ err,
               uint32_t wait_limit)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const UTask tk = tasks[blockIdx.x];
    const int N = tk.n;
    const uint32_t abytes = (uint32_t)N * 16u * (CPS / 8);  // half of a stage's matrix image (hi or lo rows)
    const uint32_t astride = 2u * (uint32_t)nmax * 16u * (CPS / 8);
    const uint32_t qcol = tcols >> 1;                      // Q accumulator: second half of the columns
    // when P and Q fit 2N columns each in the launch's allocation (sized for
    // N columns each of the widest tile), the hi and lo rows of the image form
    // one 2N-row operand: four MMAs per stage instead of six (the
    // right-hand-side operand, re-read from shared memory by every MMA, is
    // read four times), the lo half added in the epilogue
    // packed (at most 64 right-hand sides): the real parts of x in TMEM lanes
    // 0-63 and the imaginary parts in lanes 64-127 of one accumulator D (P in
    // the first half, Q in the second), three MMAs per stage (two fused)
    const bool fused = packed ? (N <= 128 && 2u * (uint32_t)N <= tcols) : 2u * (uint32_t)N <= qcol;
    constexpr uint32_t gbytes = packed ? (uint32_t)CHUNK : (uint32_t)GBYTES;   // bytes of one plane group
    // per stage: the hi and lo right-hand-side operands (XST bytes; the packed
    // layout needs half), then the matrix image
    constexpr uint32_t XST = packed ? XPLANE : 2 * XPLANE, XLO = XST / 2;
    uint8_t *sxb = base;                                   // NS x (hi, lo) X planes
    uint8_t *sab = base + NS * XST;                        // NS x (hi, lo) matrix planes
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
        // producer: per stage one bulk copy of the matrix image and one or two
        // bulk copies per plane of right-hand-side groups, all completing on
        // the stage's `full` barrier; group indices are read a stage ahead
        const uint8_t *ph = reinterpret_cast<const uint8_t *>(phi), *pl = reinterpret_cast<const uint8_t *>(plo);
        static_assert(CPS / GRP == 2, "one int2 of group positions per stage");
        const int2 *gq = reinterpret_cast<const int2 *>(groups + tk.chunk_off);
        int2 g0 = tk.nst > 0 ? gq[0] : make_int2(-1, -1);
        for (int s = 0; s < tk.nst; ++s) {
            const int b = s % NS;
            const int64_t ga = g0.x >= 0 ? g0.x / GRP : ngrp - 1, gb = g0.y >= 0 ? g0.y / GRP : ngrp - 1;
            if (s + 1 < tk.nst) g0 = gq[s + 1];
            if (s >= NS && !mbar_wait(&empty[b], ((s / NS) - 1) & 1, wait_limit)) {
                abort_flag = 1;
                break;
            }
            issued = s + 1;
            uint8_t *sx = sxb + b * XST;
            uint8_t *sa = sab + b * astride;
            mbar_expect_tx(&full[b], 2 * abytes + 4 * gbytes);
            bulk_g2s(sa, images + tk.img_off + (int64_t)s * 2 * abytes, 2 * abytes, &full[b]);
            const int64_t oa = plane_group(blockIdx.y, ngrp, ga, gbytes), ob = plane_group(blockIdx.y, ngrp, gb, gbytes);
            if (gb == ga + 1) {
                bulk_g2s(sx, ph + oa, 2 * gbytes, &full[b]);
                bulk_g2s(sx + XLO, pl + oa, 2 * gbytes, &full[b]);
            } else {
                bulk_g2s(sx, ph + oa, gbytes, &full[b]);
                bulk_g2s(sx + gbytes, ph + ob, gbytes, &full[b]);
                bulk_g2s(sx + XLO, pl + oa, gbytes, &full[b]);
                bulk_g2s(sx + XLO + gbytes, pl + ob, gbytes, &full[b]);
            }
        }
    } else if (warp == 3 && lane == 0) {
        const uint32_t idesc = idesc_bf16(N);
        const uint32_t idesc2 = fused ? idesc_bf16(2 * N) : idesc;
        const uint32_t tq = tmem + qcol;
        for (int s = 0; s < tk.nst; ++s) {
            const int b = s % NS;
            if (!mbar_wait(&full[b], (s / NS) & 1, wait_limit)) {
                abort_flag = 1;
                break;
            }
            consumed = s + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t xa = smem_u32(sxb + b * XST), xb = xa + XLO;   // hi, lo planes (wide: Re at +0, Im at +2 KB)
            // image of the stage: per K chunk, N hi rows then N lo rows (16 B each)
            const uint32_t aa = smem_u32(sab + b * astride), ab = aa + 16u * (uint32_t)N;
            const uint64_t bh = kdesc(aa, 32u * (uint32_t)N), bl = kdesc(ab, 32u * (uint32_t)N);
            const uint32_t first = s == 0 ? 0u : 1u;
            if constexpr (packed) {
                // A = [Re x; Im x] of 64 right-hand sides, K chunks one 2 KB group apart
                if (fused) {
                    umma(tmem, xdesc(xa, CHUNK), bh, idesc2, first);           // D: x hi . [hi; lo]
                    umma(tmem, xdesc(xb, CHUNK), bh, idesc, 1u);               // D: x lo . hi
                } else {
                    umma(tmem, xdesc(xa, CHUNK), bh, idesc, first);            // D: x hi . hi
                    umma(tmem, xdesc(xa, CHUNK), bl, idesc, 1u);               // D: x hi . lo
                    umma(tmem, xdesc(xb, CHUNK), bh, idesc, 1u);               // D: x lo . hi
                }
            } else if (fused) {
                // [hi; lo] as one operand of 2N rows: columns [0, N) take hi, [N, 2N) lo
                umma(tmem, xdesc(xa), bh, idesc2, first);                      // P: Re hi . [hi; lo]
                umma(tmem, xdesc(xb), bh, idesc, 1u);                          // P: Re lo . hi
                umma(tq, xdesc(xa + CHUNK), bh, idesc2, first);                // Q: Im hi . [hi; lo]
                umma(tq, xdesc(xb + CHUNK), bh, idesc, 1u);                    // Q: Im lo . hi
            } else {
                umma(tmem, xdesc(xa), bh, idesc, first);                       // P: Re hi . hi
                umma(tmem, xdesc(xa), bl, idesc, 1u);                          // P: Re hi . lo
                umma(tmem, xdesc(xb), bh, idesc, 1u);                          // P: Re lo . hi
                umma(tq, xdesc(xa + CHUNK), bh, idesc, first);                 // Q: Im hi . hi
                umma(tq, xdesc(xa + CHUNK), bl, idesc, 1u);                    // Q: Im hi . lo
                umma(tq, xdesc(xb + CHUNK), bh, idesc, 1u);                    // Q: Im lo . hi
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
    if (packed && !abort_flag && tk.nst > 0) {
        // lanes 0-63 hold P of right-hand side r = lane, lanes 64-127 its Q;
        // per group of 8 output rows the Q half goes through shared memory (the
        // stage buffers are free: every copy landed and every MMA completed)
        float *xch = reinterpret_cast<float *>(base);     // [64][17]
        const int rr = warp * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int g = 0; g < N / 16; ++g) {
            float pv[16];
            tmem_ld16(tl + (uint32_t)(16 * g), pv);
            if (fused) {
                float pl[16];
                tmem_ld16(tl + (uint32_t)(N + 16 * g), pl);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) pv[e] += pl[e];
            } else {
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            if (rr >= 64) {
#pragma unroll
                for (int e = 0; e < 16; ++e) xch[(rr - 64) * 17 + e] = pv[e];
            }
            __syncthreads();
            if (rr < 64 && rr < nrhs) {
                float yre[8], yim[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    yre[e] = pv[e] - xch[rr * 17 + 8 + e];
                    yim[e] = pv[8 + e] + xch[rr * 17 + e];
                }
                const int i0 = 8 * g;
                if (out) {
                    float2 *o = out + (int64_t)rr * ldo + tk.out_off;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (i0 + e < tk.m) o[i0 + e] = make_float2(yre[e], yim[e]);
                } else if (i0 < tk.m) {
                    // the group's Re row rr and Im row 64 + rr, hi and lo planes
                    __align__(16) __nv_bfloat16 hv[8];
                    __align__(16) __nv_bfloat16 lv[8];
                    const int64_t goff = plane_group(0, ngrp, (tk.out_off + i0) / GRP, CHUNK) + rr * 16;
                    uint8_t *bh = reinterpret_cast<uint8_t *>(phi) + goff, *bl = reinterpret_cast<uint8_t *>(plo) + goff;
                    split_bf16x8(yre, hv, lv);
                    *reinterpret_cast<uint4 *>(bh) = *reinterpret_cast<const uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(bl) = *reinterpret_cast<const uint4 *>(lv);
                    split_bf16x8(yim, hv, lv);
                    *reinterpret_cast<uint4 *>(bh + 64 * 16) = *reinterpret_cast<const uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(bl + 64 * 16) = *reinterpret_cast<const uint4 *>(lv);
                }
            }
            __syncthreads();
        }
    } else if (!packed && !abort_flag && tk.nst > 0) {
        // thread = right-hand side r (TMEM lane); per group of 8 output rows,
        // accumulator columns 16 g + e hold the Re rows and 16 g + 8 + e the Im
        // rows of B, in P (real parts of x) and Q (imaginary parts of x)
        const int rr = warp * 32 + lane, r = r0 + rr;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int g = 0; g < N / 16; ++g) {
            float pv[16], qv[16];
            tmem_ld16(tl + (uint32_t)(16 * g), pv);
            tmem_ld16(tl + qcol + (uint32_t)(16 * g), qv);
            if (fused) {
                // the hi . lo halves, N columns further on
                float pl[16], ql[16];
                tmem_ld16(tl + (uint32_t)(N + 16 * g), pl);
                tmem_ld16(tl + qcol + (uint32_t)(N + 16 * g), ql);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    pv[e] += pl[e];
                    qv[e] += ql[e];
                }
            } else {
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            if (r < nrhs) {
                float yre[8], yim[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    yre[e] = pv[e] - qv[8 + e];
                    yim[e] = pv[8 + e] + qv[e];
                }
                const int i0 = 8 * g;
                if (out) {
                    float2 *o = out + (int64_t)r * ldo + tk.out_off;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (i0 + e < tk.m) o[i0 + e] = make_float2(yre[e], yim[e]);
                } else if (i0 < tk.m) {
                    // split into the plane: the group's Re and Im chunk rows (rows
                    // of the group at or beyond m are padding, whose sums are 0)
                    __align__(16) __nv_bfloat16 hv[8];
                    __align__(16) __nv_bfloat16 lv[8];
                    const int64_t goff = plane_group(blockIdx.y, ngrp, (tk.out_off + i0) / GRP) + rr * 16;
                    uint8_t *bh = reinterpret_cast<uint8_t *>(phi) + goff, *bl = reinterpret_cast<uint8_t *>(plo) + goff;
                    split_bf16x8(yre, hv, lv);
                    *reinterpret_cast<uint4 *>(bh) = *reinterpret_cast<const uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(bl) = *reinterpret_cast<const uint4 *>(lv);
                    split_bf16x8(yim, hv, lv);
                    *reinterpret_cast<uint4 *>(bh + CHUNK) = *reinterpret_cast<const uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(bl + CHUNK) = *reinterpret_cast<const uint4 *>(lv);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

size_t umma_ws_smem_bytes(int ns, int nmax, bool packed = false)
{
    // + alignment of the base to 1 KB, + the barriers (2 NS x 8 B) and the TMEM address slot
    return (size_t)ns * ((packed ? 1 : 2) * XPLANE + 2 * (size_t)nmax * 16 * (CPS / 8)) + 1024 + 256;
}

// Pack the bf16-split matrix images of every tile/stage: per stage two K
// chunks (8 complex columns each), each N hi rows then N lo rows of 16 bytes;
// row 16 q + e is Re of task row row0 + 8 q + e and row 16 q + 8 + e its Im
// (e < 8). Column pc
// of a task starts at element colmap[colmap_off + pc] of mat (-1: padding).
__global__ void umma_pack_kernel(const UTask *__restrict__ tasks, const UPackInfo *__restrict__ info,
                                 const int64_t *__restrict__ colmap, const float2 *__restrict__ mat,
                                 uint8_t *__restrict__ images)
{
    const UTask tk = tasks[blockIdx.x];
    const UPackInfo pi = info[blockIdx.x];
    const int N = tk.n;
    const int s = blockIdx.y;
    if (s >= tk.nst) return;
    const int abytes = N * 16 * (CPS / 8);
    uint8_t *img = images + tk.img_off + (int64_t)s * 2 * abytes;
    for (int e = threadIdx.x; e < N * CPS; e += blockDim.x) {
        const int nr = e / CPS, kk = e % CPS;
        const int li = 8 * (nr >> 4) + (nr & 7);           // row of the tile
        const int part = (nr >> 3) & 1;                    // 0: Re, 1: Im
        const int pc = s * CPS + kk;                       // padded complex column
        const int64_t c = pc < pi.npc ? colmap[pi.colmap_off + pc] : -1;   // column start in mat
        float v = 0.f;
        if (c >= 0 && li < tk.m) {
            const float2 a = mat[c + pi.row0 + li];
            v = part == 0 ? a.x : a.y;
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const int byte = (kk >> 3) * (32 * N) + nr * 16 + (kk & 7) * 2;   // chunk, row, element
        *reinterpret_cast<__nv_bfloat16 *>(img + byte) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(img + 16 * N + byte) = lo;
    }
}

// Fill plane positions [p0, pend) of group-major bf16 hi/lo planes: position
// d of right-hand side r holds src[r * lds + pos[d]] (zero where pos[d] < 0);
// its real part sits in the Re chunk of group d / 8 of tile r / 128, row
// r % 128, bytes 2 (d % 8) .. + 2, its imaginary part in the Im chunk; ngrp
// groups per tile; p0 is a multiple of 8. A block transposes 32 positions x 32
// right-hand sides through shared memory, so that reads run along positions
// and each thread writes one 16-byte chunk row (8 Re or 8 Im values) per plane.
__global__ void __launch_bounds__(256)
split_scatter_kernel(const float2 *__restrict__ src, int64_t lds, const int32_t *__restrict__ pos, int p0, int pend,
                     int nrhs, __nv_bfloat16 *__restrict__ phi, __nv_bfloat16 *__restrict__ plo, int64_t ngrp,
                     int packed)
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
    const int r = r0 + tx, gi = ty >> 1, part = ty & 1;   // 4 groups of 8 positions, Re or Im
    const int64_t g = (d0 >> 3) + gi;
    if (r >= nrhs || 8 * g >= pend) return;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float2 c = tile[tx][8 * gi + e];
        v[e] = part ? c.y : c.x;
    }
    __align__(16) __nv_bfloat16 hv[8];
    __align__(16) __nv_bfloat16 lv[8];
    split_bf16x8(v, hv, lv);
    // packed (nrhs <= 64): row part * 64 + r of the group's one chunk
    const int64_t off = packed ? plane_group(0, ngrp, g, CHUNK) + (part * 64 + r) * 16
                               : plane_group(r / MT, ngrp, g) + part * CHUNK + (r % MT) * 16;
    *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(phi) + off) = *reinterpret_cast<const uint4 *>(hv);
    *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(plo) + off) = *reinterpret_cast<const uint4 *>(lv);
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
        // padded columns: each segment rounded up to a whole plane group (8 complex entries)
        std::vector<int64_t> cm;        // padded column -> element offset of the column in mat (-1 pad)
        std::vector<int32_t> chunk_src; // per 8-column group: plane position of its first entry
        for (const Task *pt : t.parts) {
            int orig = 0;
            for (int si = pt->seg_begin; si < pt->seg_end; ++si) {
                const Seg &sg = hsegs[si];
                const int32_t pbase = seg_pos(sg);
                const int np = (sg.n + GRP - 1) / GRP * GRP;
                for (int j = 0; j < np; ++j) cm.push_back(j < sg.n ? pt->mat_off + (int64_t)(orig + j) * pt->mpad : -1);
                for (int j = 0; j < np; j += GRP) chunk_src.push_back(pbase + j);
                orig += sg.n;
            }
        }
        const int npc = (int)cm.size();
        const int nst = (npc + CPS - 1) / CPS;
        while ((int)chunk_src.size() < nst * (CPS / GRP)) chunk_src.push_back(-1);
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
            img += (int64_t)nst * 2 * u.n * 16 * (CPS / 8);
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
    // the clusters (xh, then yh), each block padded to a whole group of 8
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
        p += (h->size[t] + GRP - 1) / GRP * GRP;
    }
    S->np_x = std::max<int64_t>(GRP, p);
    int64_t q = 0;
    for (int t = 0; t < h->nc; ++t) {
        if (h->rank[t] == 0) continue;
        coef_pbase[t] = (int32_t)q;
        q += (h->rank[t] + GRP - 1) / GRP * GRP;
    }
    S->np_c = std::max<int64_t>(GRP, q);
    S->nch = (S->np_x + 2 * S->np_c) / GRP + 1;   // groups per tile, the last one all zero
    if ((S->nch - 1) * GRP > INT32_MAX) {
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
        cudaFuncAttributes fa{}, fp{};
        UM_CUDA(cudaFuncGetAttributes(&fa, umma_ws_kernel<2, false>));
        UM_CUDA(cudaFuncGetAttributes(&fp, umma_ws_kernel<2, true>));
        const int stat = (int)std::max(fa.sharedSizeBytes, fp.sharedSizeBytes);
        S->dyn_smem_limit = optin > stat ? (size_t)optin - stat : 0;
        if (umma_ws_smem_bytes(2, nmax) > S->dyn_smem_limit) {
            set_error("split-bf16: two pipeline stages of the widest tile exceed shared memory");
            return H2_ERR_STATE;
        }
        const int lim = (int)S->dyn_smem_limit;
#define H2_UMMA_ATTR(NSV)                                                                                   \
    UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<NSV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)); \
    UM_CUDA(cudaFuncSetAttribute(umma_ws_kernel<NSV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))
        H2_UMMA_ATTR(2);
        H2_UMMA_ATTR(3);
        H2_UMMA_ATTR(4);
        H2_UMMA_ATTR(5);
        H2_UMMA_ATTR(6);
        H2_UMMA_ATTR(7);
        H2_UMMA_ATTR(8);
#undef H2_UMMA_ATTR
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
    // group-major: per tile of 128 right-hand sides, nch groups of 4 KB (Re and Im chunks)
    const size_t bytes = (size_t)(rpad / MT) * S->nch * GBYTES;
    if (cudaMalloc(&S->phi, bytes) != cudaSuccess || cudaMalloc(&S->plo, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("split-bf16 plane allocation failed");
        return H2_ERR_ALLOC;
    }
    // entries that no kernel writes stay zero: the zero group, padding between
    // blocks, and the xh / yh of clusters that no task writes
    UM_CUDA(cudaMemset(S->phi, 0, bytes));
    UM_CUDA(cudaMemset(S->plo, 0, bytes));
    S->rcap = rpad;
    return H2_OK;
}

// Deepest pipeline that fits in shared memory and that the phase's longest
// tile can use (two stages when the pipeline option is off); tensor memory
// columns: the power of two that holds both accumulators of the widest tile.
static cudaError_t launch_umma(const UPhase &U, const SplitState *S, int nrhs, float2 *out, int64_t ldo,
                               cudaStream_t st)
{
    if (U.ntile == 0) return cudaSuccess;
    const int packed = nrhs <= MT / 2;   // at most 64 right-hand sides: Re and Im in one 128-lane tile
    dim3 grid(U.ntile, (nrhs + MT - 1) / MT);
    int ns = 2;
    if (S->pipeline) {
        const int want = U.ns > 0 ? std::min(NSMAX, U.ns) : std::min(NSMAX, std::max(2, U.maxnst));
        for (int c = want; c > 2; --c)
            if (umma_ws_smem_bytes(c, U.nmax, packed) <= S->dyn_smem_limit) {
                ns = c;
                break;
            }
    }
    // P and Q: N columns each for the widest tile (2N for the tiles that fit
    // them, which then fuse their hi and lo operands); a larger allocation
    // would keep two CTAs from sharing an SM's tensor memory
    uint32_t tcols = 32;
    while ((int)tcols < 2 * U.nmax) tcols <<= 1;
    const size_t sm = umma_ws_smem_bytes(ns, U.nmax, packed);
    __nv_bfloat16 *phi = reinterpret_cast<__nv_bfloat16 *>(S->phi), *plo = reinterpret_cast<__nv_bfloat16 *>(S->plo);
#define H2_UMMA_LAUNCH(NSV)                                                                                  \
    umma_ws_kernel<NSV, PK><<<grid, UT, sm, st>>>(U.d_tasks, U.d_chunks, U.d_images, phi, plo, S->nch, nrhs, \
                                                  out, ldo, U.nmax, tcols, S->d_err, S->wait_limit)
#define H2_UMMA_SWITCH                     \
    switch (ns) {                          \
        case 8: H2_UMMA_LAUNCH(8); break;  \
        case 7: H2_UMMA_LAUNCH(7); break;  \
        case 6: H2_UMMA_LAUNCH(6); break;  \
        case 5: H2_UMMA_LAUNCH(5); break;  \
        case 4: H2_UMMA_LAUNCH(4); break;  \
        case 3: H2_UMMA_LAUNCH(3); break;  \
        default: H2_UMMA_LAUNCH(2); break; \
    }
    if (packed) {
        constexpr bool PK = true;
        H2_UMMA_SWITCH
    } else {
        constexpr bool PK = false;
        H2_UMMA_SWITCH
    }
#undef H2_UMMA_SWITCH
#undef H2_UMMA_LAUNCH
    return cudaGetLastError();
}

void h2_free_split(h2_handle *h)
{
    h2_drop_split_graphs(h);
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
    const int packed = nrhs <= MT / 2;
    if (packed) {
        // the packed layout's zero group lies where the 128-wide layout keeps data
        UM_CUDA(cudaMemsetAsync(static_cast<uint8_t *>(S->phi) + (S->nch - 1) * (int64_t)CHUNK, 0, CHUNK, st));
        UM_CUDA(cudaMemsetAsync(static_cast<uint8_t *>(S->plo) + (S->nch - 1) * (int64_t)CHUNK, 0, CHUNK, st));
    }
    dim3 g((unsigned)((S->np_x + 31) / 32), (nrhs + 31) / 32);
    split_scatter_kernel<<<g, 256, 0, st>>>(x, ldx, S->d_xpos, 0, (int)S->np_x, nrhs,
                                            reinterpret_cast<__nv_bfloat16 *>(S->phi),
                                            reinterpret_cast<__nv_bfloat16 *>(S->plo), S->nch, packed);
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

h2_status h2_split_prepare(h2_handle *h, int nrhs, int *realloc)
{
    h2_status s = split_init(h);
    if (s != H2_OK) return s;
    const int before = h->split->rcap;
    s = ensure_planes(h, (nrhs + MT - 1) / MT * MT);
    if (realloc) *realloc = h->split->rcap != before;
    return s;
}

// the tensor-core phases with their report names
static std::vector<std::pair<std::string, UPhase *>> split_phases(SplitState *S)
{
    std::vector<std::pair<std::string, UPhase *>> v = {{"tc_leaf", &S->leaf}, {"tc_upleaf", &S->upleaf}};
    for (size_t l = 0; l < S->up.size(); ++l) v.push_back({"tc_up" + std::to_string(l), &S->up[l]});
    for (size_t l = 0; l < S->level.size(); ++l) v.push_back({"tc_level" + std::to_string(l), &S->level[l]});
    return v;
}

bool h2_split_set_ns(h2_handle *h, const std::string &name, int ns)
{
    if (!h->split) return false;
    for (auto &pu : split_phases(h->split))
        if (pu.first == name) {
            pu.second->ns = ns;
            return true;
        }
    return false;
}

h2_status h2_split_autotune(h2_handle *h, int nrhs, std::string &js, bool &first)
{
    h2_status s = h2_split_prepare(h, nrhs, nullptr);
    if (s != H2_OK) return s;
    SplitState *S = h->split;
    float2 *yb = nullptr;
    if (cudaMalloc(&yb, sizeof(float2) * (size_t)h->n * nrhs) != cudaSuccess) {
        cudaGetLastError();
        set_error("h2_autotune_tc: allocation failed");
        return H2_ERR_ALLOC;
    }
    cudaStream_t st = h->s_aux;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const bool pipeline = S->pipeline;
    S->pipeline = true;
    for (auto &pu : split_phases(S)) {
        UPhase &U = *pu.second;
        if (e != cudaSuccess || U.ntile == 0) continue;
        int best = 0;
        float best_us = 1e30f;
        std::string tried;
        const int old_ns = U.ns;
        for (int c = 2; c <= NSMAX && e == cudaSuccess; ++c) {
            if (umma_ws_smem_bytes(c, U.nmax, nrhs <= MT / 2) > S->dyn_smem_limit) break;
            if (c > 2 && c > U.maxnst) break;   // deeper than the longest tile's stages buys nothing
            U.ns = c;
            float ts[3] = {0, 0, 0};
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, st);
                if (e == cudaSuccess) e = launch_umma(U, S, nrhs, &U == &S->leaf ? yb : nullptr, h->n, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ts[rep - 1] = ms;
            }
            std::sort(ts, ts + 3);
            const float us = ts[1] * 1e3f;
            tried += (tried.empty() ? "" : ", ") + std::string("\"") + std::to_string(c) + "\": " + std::to_string(us);
            if (us < best_us) {
                best_us = us;
                best = c;
            }
        }
        U.ns = best > 0 ? best : old_ns;
        js += (first ? "" : ", ") + std::string("\"") + pu.first + "\": {\"ns\": " + std::to_string(U.ns) +
              ", \"us\": " + std::to_string(best_us) + ", \"tiles\": " + std::to_string(U.ntile) +
              ", \"tried\": {" + tried + "}}";
        first = false;
    }
    S->pipeline = pipeline;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(yb);
    h2_drop_split_graphs(h);
    if (e != cudaSuccess) {
        set_error(std::string("h2_autotune_tc: ") + cudaGetErrorString(e));
        return H2_ERR_CUDA;
    }
    // the timing runs overwrote the planes' coefficient blocks, which every product rewrites before reading
    return H2_OK;
}

void h2_drop_split_graphs(h2_handle *h)
{
    for (auto &g : h->split_graphs) cudaGraphExecDestroy(g.exec);
    h->split_graphs.clear();
}

h2_status h2_split_set_pipeline(h2_handle *h, int on)
{
    h2_status s = split_init(h);
    if (s != H2_OK) return s;
    h->split->pipeline = on != 0;
    return H2_OK;
}
