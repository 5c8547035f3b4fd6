// Symmetric storage of the couplings for the single-RHS FP32 product.
//
// The couplings come from the H^2 form of the complex-symmetric kernel with
// one basis per cluster (Eq. 8), so S^{s,t} = (S^{t,s})^T for every admissible
// pair. This path keeps only the blocks with s > t (cluster index) and makes
// one pass over them:
//
//   direct      yh^t += S^{t,s} xh^s          (the task's own output)
//   transposed  c_{s<-t} = (S^{t,s})^T xh^t   (one entry per stored column)
//
// so every stored entry is read from HBM once and serves both products. The
// transposed contributions go to a scratch vector (one entry per stored
// column); a second launch adds, for every cluster s, the contributions of all
// t < s in a fixed order. No atomics: the product stays deterministic.
//
// The stored columns reach shared memory through a bulk-copy pipeline: one
// producer thread streams each task's column-major matrix (contiguous, a
// whole number of 16-byte row pairs per column) into a ring of stages with
// cp.async.bulk, each completing on the stage's `full` mbarrier; the consumer
// warps compute from the ring and release a stage on its `empty` mbarrier.
// The bytes in flight per CTA are set by the ring, not by registers. Every
// wait is bounded: when one runs out the CTA lets its copies land, sets the
// handle's error flag and writes nothing. The inputs of a chunk of stored
// columns are gathered into shared memory through a per-column source table.
//
// Thread mapping of the consumers: a warp covers CS = 32 / Pp columns at a
// time, Pp lanes per column (a power of two, 8 to 32); lane rl holds row pair
// rl of a column (rows 2 rl, 2 rl + 1, one 16-byte shared-memory load) and,
// for tasks with more than 16 row pairs, row pair rl + Pp as well. The direct
// sums stay in registers; the transposed sums of a slot's four columns of a
// stage are one butterfly reduction over its Pp lanes. A stage holds exactly
// four columns per slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "h2_internal.h"
#include "h2_tc.cuh"

namespace h2 {
namespace {

using tc::kDrainLimit;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::named_sync;

constexpr int SYM_UNROLL = 4;                    // columns per slot and stage
constexpr int SYM_GATHER = 8;                    // input entries per thread in flight while staging
constexpr int SYM_MAXST = 8;                     // stages at most

// Launch shapes of the dual kernel: CW consumer warps and one producer warp;
// 8 warps with a 96 KB ring (two CTAs per SM) or 4 warps with a 48 KB ring
// (three CTAs per SM); 2048 staged input columns. Either ring holds at least
// three stages.
template <int CW> struct SymCfg {
    static constexpr int CONS = 32 * CW;                         // consumer threads
    static constexpr int THREADS = CONS + 32;
    static constexpr int CHUNK = 2048;
    static constexpr uint32_t RING = CW == 8 ? 96u * 1024u : 48u * 1024u;
    static constexpr int MINB = CW == 8 ? 2 : 3;                // CTAs per SM
    static constexpr size_t SMEM = RING + CHUNK * sizeof(float2) + 2 * SYM_MAXST * sizeof(uint64_t);
};

__device__ __forceinline__ void cmac_pair(float &ar, float &ai, float &br, float &bi, float4 m, float2 x)
{
    ar = fmaf(m.x, x.x, ar);
    ar = fmaf(-m.y, x.y, ar);
    ai = fmaf(m.x, x.y, ai);
    ai = fmaf(m.y, x.x, ai);
    br = fmaf(m.z, x.x, br);
    br = fmaf(-m.w, x.y, br);
    bi = fmaf(m.z, x.y, bi);
    bi = fmaf(m.w, x.x, bi);
}

// (S^{t,s})^T xh^t restricted to this lane's rows: sum of m[row] * xt[row]
__device__ __forceinline__ void tdot(float &tr, float &ti, float4 m, float2 u, float2 v)
{
    tr = fmaf(m.x, u.x, tr);
    tr = fmaf(-m.y, u.y, tr);
    ti = fmaf(m.x, u.y, ti);
    ti = fmaf(m.y, u.x, ti);
    tr = fmaf(m.z, v.x, tr);
    tr = fmaf(-m.w, v.y, tr);
    ti = fmaf(m.z, v.y, ti);
    ti = fmaf(m.w, v.x, ti);
}

// Reduce v[0..7] (Re, Im of four columns) over the Pp lanes of a column slot
// (8 <= Pp <= 32, a power of two): three halving steps leave each lane one of
// the eight partial sums (index 4 b16 + 2 b8 + b4 from its lane bits
// Pp/2, Pp/4, Pp/8), the remaining steps add across the rest of the slot;
// 9 shuffles for Pp = 32 instead of 40 separate reductions.
__device__ __forceinline__ float slot_reduce8(float v[8], int Pp, int rl, int &idx)
{
    int o = Pp >> 1;
    idx = 0;
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) {   // halving steps: 8 -> 4 -> 2 -> 1 values
        const bool up = (rl & o) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = up ? v[k] : v[k + h];
            const float keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        idx += up ? h : 0;
        o >>= 1;
    }
    float r = v[0];
    for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// Stage geometry of a task: P row pairs, Pp lanes per column (each holding
// one row pair, or two when P > 16), C columns and SB bytes per stage, NS
// stages in the ring.
struct SymGeom {
    int P, Pp, CS, nslot, C, NS;
    uint32_t SB;
};

template <int CW>
__device__ __forceinline__ SymGeom sym_geom(int mpad)
{
    SymGeom g;
    g.P = mpad >> 1;
    // one row pair per lane up to P = 16, else two (rl and rl + Pp)
    const int need = g.P <= 16 ? g.P : (g.P + 1) >> 1;
    g.Pp = 8;
    while (g.Pp < need) g.Pp <<= 1;                    // 8, 16 or 32
    g.CS = 32 / g.Pp;
    g.nslot = CW * g.CS;
    g.C = SYM_UNROLL * g.nslot;                        // 128 CW / Pp: divides CHUNK
    g.SB = (uint32_t)g.C * (uint32_t)mpad * 8u;        // 2 KB x CW x P / Pp <= 4 KB x CW
    g.NS = min(SYM_MAXST, (int)(SymCfg<CW>::RING / g.SB));   // >= 3
    return g;
}

// Consumer warps of one task: stored column c takes its input from
// xin[xsrc[c]] when xsrc[c] >= 0, else from coef[-xsrc[c] - 1]; xt is
// the task's own-row vector of the transposed products; the direct sums go to
// out[out_off ...].
template <int CW, bool TWO>
__device__ __forceinline__ void sym_consume(const Task &tk, const SymGeom &g, int64_t col0,
                                            const int32_t *__restrict__ xsrc, const float2 *coef, const float2 *xin,
                                            const float2 *xt, float2 *out, float2 *__restrict__ scratch, float2 *xs,
                                            const float4 *ring, uint64_t *full, uint64_t *empty,
                                            volatile int *abort_flag, uint32_t wait_limit)
{
    const int P = g.P, Pp = g.Pp, nslot = g.nslot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = lane / Pp, rl = lane % Pp;
    const int r1 = rl + Pp;   // second row pair (TWO)
    const bool has0 = rl < P, has1 = TWO && r1 < P;
    const int slot = warp * g.CS + sl;

    const float2 z2 = make_float2(0.f, 0.f);
    const float2 u0 = has0 && 2 * rl < tk.m ? xt[2 * rl] : z2;
    const float2 v0 = has0 && 2 * rl + 1 < tk.m ? xt[2 * rl + 1] : z2;
    const float2 u1 = has1 && 2 * r1 < tk.m ? xt[2 * r1] : z2;
    const float2 v1 = has1 && 2 * r1 + 1 < tk.m ? xt[2 * r1 + 1] : z2;

    float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f, b0r = 0.f, b0i = 0.f, b1r = 0.f, b1i = 0.f;
    float *sc = reinterpret_cast<float *>(scratch + col0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int sbf4 = (int)(g.SB >> 4);

    int b = 0;          // ring slot of the current stage
    uint32_t ph = 0;    // parity of its `full` phase
    for (int c0 = 0; c0 < tk.ncol; c0 += SymCfg<CW>::CHUNK) {
        const int cn = min(SymCfg<CW>::CHUNK, tk.ncol - c0);
        named_sync(1, SymCfg<CW>::CONS);
        // gather the chunk's inputs through the per-column source table: all
        // index loads, then all value loads, then the stores
        const int32_t *ci = xsrc + col0 + c0;
        for (int cb = threadIdx.x; cb < cn; cb += SymCfg<CW>::CONS * SYM_GATHER) {
            int32_t id[SYM_GATHER];
            float2 xv[SYM_GATHER];
#pragma unroll
            for (int u = 0; u < SYM_GATHER; ++u) {
                const int c = cb + u * SymCfg<CW>::CONS;
                id[u] = c < cn ? ci[c] : 0;
            }
#pragma unroll
            for (int u = 0; u < SYM_GATHER; ++u) {
                const int c = cb + u * SymCfg<CW>::CONS;
                xv[u] = c >= cn ? z2 : id[u] >= 0 ? xin[id[u]] : coef[-(int64_t)id[u] - 1];
            }
#pragma unroll
            for (int u = 0; u < SYM_GATHER; ++u) {
                const int c = cb + u * SymCfg<CW>::CONS;
                if (c < cn) xs[c] = xv[u];
            }
        }
        named_sync(1, SymCfg<CW>::CONS);
        // stages never straddle a chunk: C divides SymCfg<CW>::CHUNK
        for (int j0 = 0; j0 < cn; j0 += g.C) {
            int ok = 0;
            if (lane == 0) ok = !*abort_flag && mbar_wait(&full[b], ph, wait_limit);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) {
                const float4 *As = ring + b * sbf4;
                float v[8];
#pragma unroll
                for (int q = 0; q < SYM_UNROLL; ++q) {
                    const int lc = slot + q * nslot, c = j0 + lc;
                    const bool in = c < cn;
                    const float4 m0 = in && has0 ? As[lc * P + rl] : z4;
                    const float2 x = in ? xs[c] : z2;
                    float tr = 0.f, ti = 0.f;
                    cmac_pair(a0r, a0i, a1r, a1i, m0, x);
                    tdot(tr, ti, m0, u0, v0);
                    if (TWO) {
                        const float4 m1 = in && has1 ? As[lc * P + r1] : z4;
                        cmac_pair(b0r, b0i, b1r, b1i, m1, x);
                        tdot(tr, ti, m1, u1, v1);
                    }
                    v[2 * q] = tr;
                    v[2 * q + 1] = ti;
                }
                int idx;
                const float r = slot_reduce8(v, Pp, rl, idx);
                // every lane holds the full sum of value idx (column idx / 2, Re or Im);
                // the lanes whose bits below Pp / 8 are zero write the eight of them
                const int c = j0 + slot + (idx >> 1) * nslot;
                if ((rl & ((Pp >> 3) - 1)) == 0 && c < cn) sc[2 * (c0 + c) + (idx & 1)] = r;
            } else if (lane == 0) {
                *abort_flag = 1;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
            if (++b == g.NS) {
                b = 0;
                ph ^= 1u;
            }
        }
    }
    // direct sums: one partial per (slot, row), summed over the slots in a fixed order
    named_sync(1, SymCfg<CW>::CONS);
    float2 *red = xs;   // nslot * mpad <= 1024 entries
    if (has0) {
        red[slot * tk.mpad + 2 * rl] = make_float2(a0r, a0i);
        red[slot * tk.mpad + 2 * rl + 1] = make_float2(a1r, a1i);
    }
    if (has1) {
        red[slot * tk.mpad + 2 * r1] = make_float2(b0r, b0i);
        red[slot * tk.mpad + 2 * r1 + 1] = make_float2(b1r, b1i);
    }
    named_sync(1, SymCfg<CW>::CONS);
    if (*abort_flag) return;
    for (int i = threadIdx.x; i < tk.m; i += SymCfg<CW>::CONS) {
        float sr = 0.f, si = 0.f;
        for (int q = 0; q < nslot; ++q) {
            const float2 v = red[q * tk.mpad + i];
            sr += v.x;
            si += v.y;
        }
        out[tk.out_off + i] = make_float2(sr, si);
    }
}

// One block per task (tasks sorted by stored work, both row-pair layouts in
// one launch so that small tasks fill in behind large ones); warps 0 .. CW-1
// consume, warp CW produces.
// (couplings: xt = coef + out_off - ktot, out = coef; near field: xt = chi x
// + out_off, out = y)
template <int CW>
__global__ void __launch_bounds__(SymCfg<CW>::THREADS, SymCfg<CW>::MINB)
symcouple_kernel(const Task *__restrict__ tasks, const int32_t *__restrict__ xsrc, const float2 *__restrict__ mat,
                 const int64_t *__restrict__ col0, const float2 *coef, const float2 *xin, const float2 *xtv,
                 int64_t xt_shift, float2 *out, float2 *__restrict__ scratch, int *__restrict__ err,
                 uint32_t wait_limit)
{
    extern __shared__ __align__(128) unsigned char sym_smem[];
    float4 *ring = reinterpret_cast<float4 *>(sym_smem);
    float2 *xs = reinterpret_cast<float2 *>(sym_smem + SymCfg<CW>::RING);
    uint64_t *full = reinterpret_cast<uint64_t *>(sym_smem + SymCfg<CW>::RING + SymCfg<CW>::CHUNK * sizeof(float2));
    uint64_t *empty = full + SYM_MAXST;
    __shared__ volatile int abort_flag;
    __shared__ int issued;

    const Task tk = tasks[blockIdx.x];
    const SymGeom g = sym_geom<CW>(tk.mpad);
    const int nst = (tk.ncol + g.C - 1) / g.C;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        issued = 0;
        for (int i = 0; i < g.NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], CW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x >= SymCfg<CW>::CONS) {
        if (threadIdx.x == SymCfg<CW>::CONS) {
            // producer: stage s holds columns [s C, s C + C) of the task's matrix
            const unsigned char *src = reinterpret_cast<const unsigned char *>(mat + tk.mat_off);
            unsigned char *dst = reinterpret_cast<unsigned char *>(ring);
            int b = 0;
            uint32_t ph = 1u;   // parity of the `empty` phase that frees slot b (none in the first round)
            for (int s = 0; s < nst; ++s) {
                if (s >= g.NS && !mbar_wait(&empty[b], ph, wait_limit)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                const uint32_t bytes = (uint32_t)min(g.C, tk.ncol - s * g.C) * (uint32_t)tk.mpad * 8u;
                mbar_expect_tx(&full[b], bytes);
                tc::bulk_g2s(dst + (size_t)b * g.SB, src + (size_t)s * g.SB, bytes, &full[b]);
                issued = s + 1;
                if (++b == g.NS) {
                    b = 0;
                    ph ^= 1u;
                }
            }
        }
    } else {
        const float2 *xt = xtv + (tk.out_off + xt_shift);
        if (tk.mpad > 32)
            sym_consume<CW, true>(tk, g, col0[blockIdx.x], xsrc, coef, xin, xt, out, scratch, xs, ring, full, empty,
                              &abort_flag, wait_limit);
        else
            sym_consume<CW, false>(tk, g, col0[blockIdx.x], xsrc, coef, xin, xt, out, scratch, xs, ring, full, empty,
                               &abort_flag, wait_limit);
    }
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        // copies of the last stage issued into each slot land before the CTA
        // releases its shared memory
        for (int st = max(0, issued - g.NS); st < issued; ++st)
            mbar_wait(&full[st % g.NS], (uint32_t)(st / g.NS) & 1u, kDrainLimit);
        atomicExch(err, 1);
    }
}

// out_s += rs_s * (sum over t < s of c_{s<-t}), in a fixed order (one block
// per target s; rs NULL: no scale, else one complex factor per output entry).
// The block stages its list of scratch columns in shared memory; each thread
// issues GATHER_U scratch loads before adding them in list order.
constexpr int GATHER_LIST = 512;
constexpr int GATHER_U = 8;

__global__ void __launch_bounds__(128)
symgather_kernel(const int32_t *__restrict__ gptr, const int64_t *__restrict__ gcol, const int32_t *__restrict__ gout,
                 const int32_t *__restrict__ gk, const float2 *__restrict__ scratch, const float2 *__restrict__ rs,
                 float2 *__restrict__ out)
{
    __shared__ int64_t cols[GATHER_LIST];
    const int tg = blockIdx.x;
    const int k = gk[tg], e0 = gptr[tg], e1 = gptr[tg + 1];
    float2 *o = out + gout[tg];
    float sr[2] = {0.f, 0.f}, si[2] = {0.f, 0.f};   // rows threadIdx.x and threadIdx.x + 128 (k <= 128)
    for (int l0 = e0; l0 < e1; l0 += GATHER_LIST) {
        const int ln = min(GATHER_LIST, e1 - l0);
        __syncthreads();
        for (int e = threadIdx.x; e < ln; e += blockDim.x) cols[e] = gcol[l0 + e];
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = threadIdx.x + h * 128;
            if (i >= k) continue;
            for (int e = 0; e < ln; e += GATHER_U) {
                float2 v[GATHER_U];
#pragma unroll
                for (int u = 0; u < GATHER_U; ++u) v[u] = e + u < ln ? scratch[cols[e + u] + i] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < GATHER_U; ++u) {
                    sr[h] += v[u].x;
                    si[h] += v[u].y;
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = threadIdx.x + h * 128;
        if (i >= k) continue;
        float a = sr[h], b = si[h];
        if (rs) {
            const float2 f = rs[gout[tg] + i];
            const float t = a * f.x - b * f.y;
            b = a * f.y + b * f.x;
            a = t;
        }
        o[i] = make_float2(o[i].x + a, o[i].y + b);
    }
}

// xs = chi x (near field: the transposed products use the scaled input)
__global__ void symscale_kernel(const float2 *__restrict__ chi, const float2 *__restrict__ x, float2 *__restrict__ xs,
                                int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 c = chi[i], v = x[i];
        xs[i] = make_float2(c.x * v.x - c.y * v.y, c.x * v.y + c.y * v.x);
    }
}

// copy the kept columns into the symmetric matrix: one block per task
__global__ void symcopy_kernel(const Task *__restrict__ tasks, const int64_t *__restrict__ col0,
                               const int64_t *__restrict__ matsrc, const float2 *__restrict__ src,
                               float2 *__restrict__ dst)
{
    const Task tk = tasks[blockIdx.x];
    const int64_t base = col0[blockIdx.x];
    const int64_t total = (int64_t)tk.ncol * tk.mpad;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int64_t j = e / tk.mpad, i = e - j * tk.mpad;
        dst[tk.mat_off + e] = src[matsrc[base + j] + i];
    }
}

// per stored block: max |S^{t,s} - (S^{s,t})^T| / max |S^{t,s}|, maximum over
// blocks in *worst (non-negative floats order like their bit patterns)
struct SymPair {
    int64_t a, b;      // offsets of S^{t,s} (rows k_t, stride mpa) and S^{s,t} (rows k_s, stride mpb)
    int32_t mpa, mpb, kt, ks;
    int32_t ra, cs;    // near field: unknown index of row 0 of t and of column 0 of s
};

// chi NULL: B^{s,t} against (B^{t,s})^T; else against diag(1/chi_s) (B^{t,s})^T diag(chi_t)
__global__ void symcheck_kernel(const SymPair *__restrict__ pairs, const float2 *__restrict__ mat,
                                const float2 *__restrict__ chi, unsigned *__restrict__ worst)
{
    const SymPair p = pairs[blockIdx.x];
    float d = 0.f, g = 0.f;
    for (int e = threadIdx.x; e < p.kt * p.ks; e += blockDim.x) {
        const int j = e / p.kt, i = e - j * p.kt;   // row i of t, column j of s
        float2 a = mat[p.a + (int64_t)j * p.mpa + i];
        const float2 b = mat[p.b + (int64_t)i * p.mpb + j];
        if (chi) {
            const float2 ct = chi[p.ra + i], cs = chi[p.cs + j];
            const float2 u = make_float2(a.x * ct.x - a.y * ct.y, a.x * ct.y + a.y * ct.x);
            const float den = cs.x * cs.x + cs.y * cs.y;
            a = make_float2((u.x * cs.x + u.y * cs.y) / den, (u.y * cs.x - u.x * cs.y) / den);
        }
        d = fmaxf(d, hypotf(a.x - b.x, a.y - b.y));
        g = fmaxf(g, hypotf(a.x, a.y));
    }
    __shared__ float sd[256], sg[256];
    sd[threadIdx.x] = d;
    sg[threadIdx.x] = g;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sd[threadIdx.x] = fmaxf(sd[threadIdx.x], sd[threadIdx.x + o]);
            sg[threadIdx.x] = fmaxf(sg[threadIdx.x], sg[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float r = sd[0] > 0.f ? sd[0] / fmaxf(sg[0], 1e-30f) : 0.f;
        atomicMax(worst, __float_as_uint(r));
    }
}

}  // namespace

namespace {

void free_state(SymState *S)
{
    if (!S) return;
    for (void *p : {(void *)S->d_tasks, (void *)S->d_xsrc, (void *)S->d_mat, (void *)S->d_col0,
                    (void *)S->d_scratch, (void *)S->d_gptr, (void *)S->d_gcol, (void *)S->d_gout, (void *)S->d_gk,
                    (void *)S->d_chi, (void *)S->d_rs, (void *)S->d_xs, (void *)S->d_err})
        cudaFree(p);
    delete S;
}

// Build the once-per-pair structure of the couplings (near = false: ids are
// clusters found by coefficient offset, kept blocks s > t) or of the near
// field (near = true: ids are leaves found by their first unknown, kept
// blocks s >= t, the diagonal block only for the direct product; chi has one
// entry per unknown in tree order). The kept columns are copied on the
// device and every pair is checked there against its stored partner.
h2_status build_sym(h2_handle *h, bool near, const std::vector<float2> *chi, SymState **out)
{
    const Phase &C = near ? h->near : h->couple;
    const std::string what = near ? "symmetric near field: " : "symmetric couplings: ";
    const std::vector<Seg> &hsegs = h->segs_host;
    std::unordered_map<int32_t, int32_t> id;
    for (int t = 0; t < h->nc; ++t) {
        if (near && h->child[2 * t] < 0) id[h->begin[t]] = t;
        if (!near && h->rank[t] > 0) id[h->xo[t]] = t;
    }
    auto out_id = [&](const Task &tk) -> int32_t {
        const auto it = id.find((int32_t)(near ? tk.out_off : tk.out_off - h->ktot));
        return it == id.end() ? -1 : it->second;
    };
    auto seg_id = [&](const Seg &sg) -> int32_t {
        if (near != (sg.in_off >= 0)) return -1;
        const auto it = id.find((int32_t)(near ? sg.in_off : -(int64_t)sg.in_off - 1));
        if (it == id.end() || (near ? h->size[it->second] : h->rank[it->second]) != sg.n) return -1;
        return it->second;
    };
    struct Blk {
        int64_t off;
        int32_t mpad, kt, ks;
    };
    std::unordered_map<int64_t, Blk> blocks;   // key t * nc + s
    for (const Task &tk : C.tasks) {
        const int32_t t = out_id(tk);
        if (t < 0) return (set_error(what + "unknown output block"), H2_ERR_STATE);
        int col = 0;
        for (int si = tk.seg_begin; si < tk.seg_end; ++si) {
            const int32_t s = seg_id(hsegs[si]);
            if (s < 0) return (set_error(what + "an input segment is not a whole cluster block"), H2_ERR_STATE);
            blocks[(int64_t)t * h->nc + s] = {tk.mat_off + (int64_t)col * tk.mpad, tk.mpad, tk.m, hsegs[si].n};
            col += hsegs[si].n;
        }
    }
    // kept blocks per task, in the handle's task order
    std::vector<Task> tasks;
    std::vector<int64_t> col0, matsrc;   // per stored column: its first entry in the loaded matrix
    std::vector<int32_t> xsrc;           // per stored column: its input (>= 0: x[.], else coef[-. - 1])
    std::vector<SymPair> pairs;
    std::vector<std::vector<int64_t>> lower(h->nc);   // per id s: first scratch column of each (t, s), t < s
    int64_t mat_elems = 0, ncols = 0, stored = 0;
    for (const Task &tk : C.tasks) {
        if (tk.mpad > 128) return (set_error(what + "blocks with more than 128 rows are not supported"), H2_ERR_STATE);
        const int32_t t = out_id(tk);
        Task u = tk;
        u.ncol = 0;
        u.mat_off = mat_elems;
        u.seg_begin = u.seg_end = 0;   // the kernel reads its inputs through xsrc
        const int64_t c0 = ncols;
        for (int si = tk.seg_begin; si < tk.seg_end; ++si) {
            const Seg &sg = hsegs[si];
            const int32_t s = seg_id(sg);
            if (s < t || (s == t && !near)) continue;
            const Blk &f = blocks.at((int64_t)t * h->nc + s);
            if (s > t) {
                const auto back = blocks.find((int64_t)s * h->nc + t);
                if (back == blocks.end()) return (set_error(what + "a block pair without its transpose"), H2_ERR_STATE);
                lower[s].push_back(c0 + u.ncol);
                SymPair pr{f.off, back->second.off, f.mpad, back->second.mpad, f.kt, f.ks, 0, 0};
                if (near) {
                    pr.ra = h->begin[t];
                    pr.cs = h->begin[s];
                }
                pairs.push_back(pr);
            }
            for (int j = 0; j < sg.n; ++j) {
                matsrc.push_back(f.off + (int64_t)j * f.mpad);
                xsrc.push_back(sg.in_off >= 0 ? sg.in_off + j : sg.in_off - j);
            }
            u.ncol += sg.n;
            stored += (int64_t)f.kt * f.ks;
        }
        if (u.ncol == 0) continue;
        tasks.push_back(u);
        col0.push_back(c0);
        ncols += u.ncol;
        mat_elems += ((int64_t)u.mpad * u.ncol + 31) / 32 * 32;
    }
    // largest stored work first
    {
        std::vector<size_t> ord(tasks.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t i, size_t j) {
            return (int64_t)tasks[i].mpad * tasks[i].ncol > (int64_t)tasks[j].mpad * tasks[j].ncol;
        });
        std::vector<Task> t2;
        std::vector<int64_t> c2;
        for (size_t i : ord) {
            t2.push_back(tasks[i]);
            c2.push_back(col0[i]);
        }
        tasks.swap(t2);
        col0.swap(c2);
    }
    std::vector<int32_t> gptr(1, 0), gout, gk;
    std::vector<int64_t> gcol;
    for (int s = 0; s < h->nc; ++s) {
        if (lower[s].empty()) continue;
        gcol.insert(gcol.end(), lower[s].begin(), lower[s].end());
        gptr.push_back((int32_t)gcol.size());
        gout.push_back((int32_t)(near ? h->begin[s] : h->ktot + h->xo[s]));
        gk.push_back(near ? h->size[s] : h->rank[s]);
    }

    auto *S = new SymState();
    S->ntask = (int)tasks.size();
    S->ntarget = (int)gout.size();
    S->wait_limit = h->wait_limit;
    S->warps = h->sym_warps[near ? 1 : 0];
    S->stored_elems = stored;
    S->scratch_entries = ncols;
    auto up = [&](auto &vec, auto **dptr) -> cudaError_t {
        using T = typename std::remove_reference<decltype(vec)>::type::value_type;
        cudaError_t e = cudaMalloc(dptr, std::max<size_t>(1, vec.size()) * sizeof(T));
        if (e == cudaSuccess && !vec.empty()) e = cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
        return e;
    };
    int64_t *d_matsrc = nullptr;
    SymPair *d_pairs = nullptr;
    unsigned *d_worst = nullptr;
    auto tmp_free = [&]() {
        cudaFree(d_matsrc);
        cudaFree(d_pairs);
        cudaFree(d_worst);
    };
    std::vector<float2> rs;
    if (near) {
        rs.resize(chi->size());
        for (size_t i = 0; i < rs.size(); ++i) {   // 1 / chi
            const double cr = (*chi)[i].x, ci = (*chi)[i].y, d = cr * cr + ci * ci;
            rs[i] = make_float2((float)(cr / d), (float)(-ci / d));
        }
    }
    cudaError_t e = cudaSuccess;
    if ((e = up(tasks, &S->d_tasks)) != cudaSuccess || (e = up(xsrc, &S->d_xsrc)) != cudaSuccess ||
        (e = up(col0, &S->d_col0)) != cudaSuccess || (e = up(gptr, &S->d_gptr)) != cudaSuccess ||
        (e = up(gcol, &S->d_gcol)) != cudaSuccess || (e = up(gout, &S->d_gout)) != cudaSuccess ||
        (e = up(gk, &S->d_gk)) != cudaSuccess || (e = up(matsrc, &d_matsrc)) != cudaSuccess ||
        (e = up(pairs, &d_pairs)) != cudaSuccess ||
        (near && ((e = up(*chi, &S->d_chi)) != cudaSuccess || (e = up(rs, &S->d_rs)) != cudaSuccess ||
                  (e = cudaMalloc(&S->d_xs, std::max<size_t>(1, chi->size()) * sizeof(float2))) != cudaSuccess)) ||
        (e = cudaMalloc(&S->d_mat, std::max<int64_t>(32, mat_elems) * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_scratch, std::max<int64_t>(1, ncols) * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(S->d_err, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(symcouple_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SymCfg<8>::SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(symcouple_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SymCfg<4>::SMEM)) != cudaSuccess ||
        (e = cudaMalloc(&d_worst, sizeof(unsigned))) != cudaSuccess || (e = cudaMemset(d_worst, 0, sizeof(unsigned))) != cudaSuccess) {
        cudaGetLastError();
        tmp_free();
        free_state(S);
        set_error(what + "device allocation failed: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? H2_ERR_ALLOC : H2_ERR_CUDA;
    }
    if (S->ntask > 0) symcopy_kernel<<<S->ntask, 256>>>(S->d_tasks, S->d_col0, d_matsrc, h->d_mat, S->d_mat);
    if (!pairs.empty()) symcheck_kernel<<<(unsigned)pairs.size(), 256>>>(d_pairs, h->d_mat, S->d_chi, d_worst);
    unsigned worst = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&worst, d_worst, sizeof(unsigned), cudaMemcpyDeviceToHost);
    tmp_free();
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_state(S);
        set_error(what + cudaGetErrorString(e));
        return H2_ERR_CUDA;
    }
    float w;
    memcpy(&w, &worst, sizeof(w));
    S->max_asym = w;
    if (!(w <= 1e-5f)) {
        free_state(S);
        set_error(what + "a block differs from its stored partner by " + std::to_string(w) + " relative (limit 1e-5)");
        return H2_ERR_STATE;
    }
    *out = S;
    return H2_OK;
}

}  // namespace

void h2_free_sym(h2_handle *h)
{
    free_state(h->sym);
    h->sym = nullptr;
    free_state(h->symnear);
    h->symnear = nullptr;
}

void symnear_free(h2_handle *h)
{
    free_state(h->symnear);
    h->symnear = nullptr;
}

// host tables are built with std containers: an allocation failure becomes
// H2_ERR_ALLOC instead of an exception crossing the C boundary
static h2_status build_sym_safe(h2_handle *h, bool near, const std::vector<float2> *chi, SymState **out)
{
    try {
        return build_sym(h, near, chi, out);
    } catch (const std::bad_alloc &) {
        set_error(near ? "symmetric near field: host allocation failed" : "symmetric couplings: host allocation failed");
        return H2_ERR_ALLOC;
    }
}

h2_status h2_sym_init(h2_handle *h)
{
    if (h->sym) return H2_OK;
    return build_sym_safe(h, false, nullptr, &h->sym);
}

h2_status symnear_init(h2_handle *h, const std::vector<float2> &chi)
{
    symnear_free(h);
    return build_sym_safe(h, true, &chi, &h->symnear);
}

// error flags of the symmetric-storage kernels (1: a bounded wait ran out)
h2_status h2_sym_error_flag(h2_handle *h, int *flag)
{
    *flag = 0;
    for (const SymState *S : {h->sym, h->symnear}) {
        if (!S) continue;
        int f = 0;
        const cudaError_t e = cudaMemcpy(&f, S->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("symmetric storage: reading the error flag failed: ") + cudaGetErrorString(e));
            return H2_ERR_CUDA;
        }
        *flag |= f;
    }
    return H2_OK;
}

// one launch of the dual kernel with the state's launch shape
template <int CW>
static void launch_dual_cw(const SymState *S, const float2 *coef, const float2 *xin, const float2 *xtv,
                           int64_t xt_shift, float2 *out, cudaStream_t st)
{
    symcouple_kernel<CW><<<S->ntask, SymCfg<CW>::THREADS, SymCfg<CW>::SMEM, st>>>(
        S->d_tasks, S->d_xsrc, S->d_mat, S->d_col0, coef, xin, xtv, xt_shift, out, S->d_scratch, S->d_err,
        S->wait_limit);
}

static void launch_dual(const SymState *S, const float2 *coef, const float2 *xin, const float2 *xtv,
                        int64_t xt_shift, float2 *out, cudaStream_t st)
{
    if (S->ntask == 0) return;
    if (S->warps == 4)
        launch_dual_cw<4>(S, coef, xin, xtv, xt_shift, out, st);
    else
        launch_dual_cw<8>(S, coef, xin, xtv, xt_shift, out, st);
}

bool sym_set_warps(h2_handle *h, bool near, int warps)
{
    if (warps != 4 && warps != 8) return false;
    h->sym_warps[near ? 1 : 0] = warps;
    SymState *S = near ? h->symnear : h->sym;
    if (S) S->warps = warps;
    return true;
}

// couplings of all levels with the symmetric storage: yh = S xh (FP32)
cudaError_t h2_sym_couple(h2_handle *h, float2 *coef, cudaStream_t st)
{
    const SymState *S = h->sym;
    launch_dual(S, coef, nullptr, coef, -h->ktot, coef, st);
    if (S->ntarget > 0)
        symgather_kernel<<<S->ntarget, 128, 0, st>>>(S->d_gptr, S->d_gcol, S->d_gout, S->d_gk, S->d_scratch, nullptr,
                                                     coef);
    return cudaGetLastError();
}

// near field with the symmetric storage: y = Z x (FP32), written, not added
cudaError_t symnear_run(h2_handle *h, const float2 *x, float2 *y, cudaStream_t st)
{
    const SymState *S = h->symnear;
    symscale_kernel<<<std::max(1, std::min(1024, (h->n + 255) / 256)), 256, 0, st>>>(S->d_chi, x, S->d_xs, h->n);
    launch_dual(S, x, x, S->d_xs, 0, y, st);
    if (S->ntarget > 0)
        symgather_kernel<<<S->ntarget, 128, 0, st>>>(S->d_gptr, S->d_gcol, S->d_gout, S->d_gk, S->d_scratch, S->d_rs,
                                                     y);
    return cudaGetLastError();
}

}  // namespace h2
