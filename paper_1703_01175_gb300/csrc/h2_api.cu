// libh2 C ABI: loading (validation + re-packing), products, statistics.
//
// h2_load turns the caller's tree, bases, transfers, couplings and near
// blocks (Sec. III.C, Sec. IV.A) into the task lists executed by the
// block-row GEMV kernels. The device layout is:
//   mat   one float2 array holding every task's column-major matrix,
//         each starting on a 256-byte boundary, rows padded to even;
//   coef  2 * sum(k_t) coefficients: xh^t at xo[t], yh^t at ktot + xo[t];
//   tasks/segs  the task and input-segment descriptors of every phase.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "h2_internal.h"

namespace h2 {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

#define H2_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e__ = (call);                                                         \
        if (e__ != cudaSuccess) {                                                         \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));               \
            return H2_ERR_CUDA;                                                           \
        }                                                                                 \
    } while (0)

static h2_status arg_error(const std::string &msg)
{
    set_error(msg);
    return H2_ERR_ARG;
}

// read complex element i of a c64 / c128 host array
struct CplxIn {
    const void *p;
    h2_dtype dt;
    inline float2 at(int64_t i) const
    {
        if (dt == H2_C64) return reinterpret_cast<const float2 *>(p)[i];
        const double2 v = reinterpret_cast<const double2 *>(p)[i];
        return make_float2((float)v.x, (float)v.y);
    }
};

static int choose_threads(const std::vector<Task> &tasks)
{
    static const int cand[] = {128, 192, 256, 384, 512, 768, 1024};
    int maxP = 1;
    double total = 0;
    for (const Task &t : tasks) {
        maxP = std::max(maxP, t.mpad / 2);
        total += (double)t.mpad * t.ncol;
    }
    int best = 1024;
    double best_score = -1e30;
    for (int T : cand) {
        if (T < maxP) continue;
        double eff = 0;
        for (const Task &t : tasks) {
            const int P = t.mpad / 2;
            eff += (double)t.mpad * t.ncol * (double)((T / P) * P) / T;
        }
        eff = total > 0 ? eff / total : 1.0;
        // prefer full thread utilisation, then 256-512 thread CTAs
        const double score = eff - 0.03 * std::fabs(std::log2((double)T / 384.0));
        if (score > best_score) {
            best_score = score;
            best = T;
        }
    }
    return best;
}

}  // namespace h2

using namespace h2;

static h2_status validate_tree(const h2_tree *tr, std::vector<int32_t> &parent,
                               std::vector<int32_t> &level)
{
    if (!tr) return arg_error("tree is NULL");
    const int32_t n = tr->n, nc = tr->n_clusters, nl = tr->n_levels;
    if (n <= 0 || nc <= 0 || nl <= 0) return arg_error("tree: n, n_clusters and n_levels must be > 0");
    if (!tr->level_ptr || !tr->child || !tr->begin || !tr->size || !tr->rank)
        return arg_error("tree: NULL array");
    if (tr->level_ptr[0] != 0 || tr->level_ptr[nl] != nc) return arg_error("tree: level_ptr must span [0, n_clusters]");
    if (tr->level_ptr[1] != 1) return arg_error("tree: level 0 must hold only the root");
    parent.assign(nc, -1);
    level.assign(nc, -1);
    for (int l = 0; l < nl; ++l) {
        if (tr->level_ptr[l + 1] < tr->level_ptr[l]) return arg_error("tree: level_ptr not monotone");
        for (int t = tr->level_ptr[l]; t < tr->level_ptr[l + 1]; ++t) level[t] = l;
    }
    if (tr->begin[0] != 0 || tr->size[0] != n) return arg_error("tree: root must cover [0, n)");
    for (int t = 0; t < nc; ++t) {
        if (tr->size[t] <= 0) return arg_error("tree: cluster sizes must be > 0");
        if (tr->rank[t] < 0) return arg_error("tree: negative rank");
        const int32_t c1 = tr->child[2 * t], c2 = tr->child[2 * t + 1];
        if ((c1 < 0) != (c2 < 0)) return arg_error("tree: a cluster must have 0 or 2 children");
        if (c1 < 0) {
            if (tr->rank[t] > tr->size[t]) return arg_error("tree: leaf rank exceeds leaf size");
            if (tr->size[t] > 2048) return arg_error("tree: leaf size above 2048");
            continue;
        }
        if (c1 >= nc || c2 >= nc || c1 == c2) return arg_error("tree: child index out of range");
        if (parent[c1] != -1 || parent[c2] != -1 || c1 == 0 || c2 == 0)
            return arg_error("tree: a cluster has two parents");
        parent[c1] = t;
        parent[c2] = t;
        if (level[c1] != level[t] + 1 || level[c2] != level[t] + 1)
            return arg_error("tree: children must be on the next level");
        if (tr->begin[c1] != tr->begin[t] || tr->begin[c2] != tr->begin[c1] + tr->size[c1] ||
            tr->size[c1] + tr->size[c2] != tr->size[t])
            return arg_error("tree: children must split the parent's range in order");
        if (tr->rank[t] > tr->rank[c1] + tr->rank[c2])
            return arg_error("tree: non-leaf rank exceeds the sum of its children's ranks");
    }
    for (int t = 1; t < nc; ++t)
        if (parent[t] < 0) return arg_error("tree: cluster without parent");
    for (int t = 0; t < nc; ++t)
        if (tr->rank[t] > 2048) return arg_error("tree: rank above 2048");
    return H2_OK;
}

static h2_status validate_data(const h2_tree *tr, const h2_data *d, const std::vector<int32_t> &parent)
{
    if (!d) return arg_error("data is NULL");
    if (d->dtype != H2_C64 && d->dtype != H2_C128) return arg_error("data: bad dtype");
    const int32_t nc = tr->n_clusters, n = tr->n;
    auto leaf = [&](int t) { return tr->child[2 * t] < 0; };
    bool any_rank = false;
    for (int t = 0; t < nc; ++t) any_rank |= tr->rank[t] > 0;
    if (any_rank && (!d->U || !d->U_off)) return arg_error("data: U missing");
    for (int t = 0; t < nc; ++t) {
        const int64_t k = tr->rank[t], nt = tr->size[t];
        if (leaf(t) && k > 0) {
            if (d->U_off[t] < 0 || d->U_off[t] + nt * k > d->U_len) return arg_error("data: U block out of range");
            if (d->W) {
                if (!d->W_off) return arg_error("data: W_off missing");
                if (d->W_off[t] < 0 || d->W_off[t] + nt * k > d->W_len) return arg_error("data: W block out of range");
            }
        }
        if (t > 0 && k > 0 && tr->rank[parent[t]] > 0) {
            if (!d->T || !d->T_off) return arg_error("data: T missing");
            const int64_t kp = tr->rank[parent[t]];
            if (d->T_off[t] < 0 || d->T_off[t] + k * kp > d->T_len) return arg_error("data: T block out of range");
        }
    }
    if (!d->adm_ptr || !d->near_ptr || !d->near_col || !d->Z || !d->Z_off)
        return arg_error("data: CSR arrays missing");
    if (d->adm_ptr[0] != 0 || d->near_ptr[0] != 0) return arg_error("data: CSR must start at 0");
    for (int t = 0; t < nc; ++t) {
        if (d->adm_ptr[t + 1] < d->adm_ptr[t] || d->near_ptr[t + 1] < d->near_ptr[t])
            return arg_error("data: CSR pointers not monotone");
        for (int j = d->adm_ptr[t]; j < d->adm_ptr[t + 1]; ++j) {
            const int s = d->adm_col[j];
            if (s < 0 || s >= nc) return arg_error("data: admissible column out of range");
            const int64_t kk = (int64_t)tr->rank[t] * tr->rank[s];
            if (kk > 0 && (!d->S || !d->S_off || d->S_off[j] < 0 || d->S_off[j] + kk > d->S_len))
                return arg_error("data: S block out of range");
        }
        if (d->near_ptr[t + 1] > d->near_ptr[t] && !leaf(t)) return arg_error("data: near block on a non-leaf row");
        for (int j = d->near_ptr[t]; j < d->near_ptr[t + 1]; ++j) {
            const int s = d->near_col[j];
            if (s < 0 || s >= nc || !leaf(s)) return arg_error("data: near column is not a leaf");
            const int64_t nn = (int64_t)tr->size[t] * tr->size[s];
            if (d->Z_off[j] < 0 || d->Z_off[j] + nn > d->Z_len) return arg_error("data: Z block out of range");
        }
    }
    // the blocks covering the rows of each leaf must tile [0, n) exactly once
    std::vector<std::pair<int32_t, int32_t>> iv;
    for (int t = 0; t < nc; ++t) {
        if (!leaf(t)) continue;
        iv.clear();
        for (int j = d->near_ptr[t]; j < d->near_ptr[t + 1]; ++j) {
            const int s = d->near_col[j];
            iv.emplace_back(tr->begin[s], tr->size[s]);
        }
        for (int a = t; a >= 0; a = parent[a])
            for (int j = d->adm_ptr[a]; j < d->adm_ptr[a + 1]; ++j) {
                const int s = d->adm_col[j];
                iv.emplace_back(tr->begin[s], tr->size[s]);
            }
        std::sort(iv.begin(), iv.end());
        int64_t pos = 0;
        for (auto &p : iv) {
            if (p.first != pos) return arg_error("data: blocks do not tile the matrix exactly once");
            pos += p.second;
        }
        if (pos != n) return arg_error("data: blocks do not tile the matrix exactly once");
    }
    return H2_OK;
}

extern "C" {

const char *h2_status_string(h2_status s)
{
    switch (s) {
        case H2_OK: return "ok";
        case H2_ERR_ARG: return "invalid argument";
        case H2_ERR_ALLOC: return "allocation failed";
        case H2_ERR_CUDA: return "CUDA error";
        case H2_ERR_NOT_CONVERGED: return "not converged";
        case H2_ERR_BREAKDOWN: return "breakdown";
        case H2_ERR_TIMEOUT: return "timeout";
        case H2_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char *h2_last_error(void) { return g_last_error.c_str(); }

void h2_free(h2_handle *h)
{
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->s_aux) cudaStreamSynchronize(h->s_aux);
    cudaDeviceSynchronize();
    h2_free_krylov(h);
    h2_free_split(h);
    h2::h2_free_sym(h);
    h2_free_precond(h);
    h2_free_bkrylov(h);
    h2_free_bicgstab(h);
    cudaFree(h->d_mat);
    cudaFree(h->d_segs);
    cudaFree(h->d_tasks);
    cudaFree(h->d_coef);
    cudaFree(h->d_coefm);
    cudaFree(h->d_colidx);
    cudaFree(h->d_xbuf);
    cudaFree(h->d_ybuf);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    h2_drop_split_graphs(h);
    if (h->s_cap) cudaStreamDestroy(h->s_cap);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_near) cudaEventDestroy(h->ev_near);
    if (h->s_aux) cudaStreamDestroy(h->s_aux);
    cudaSetDevice(cur);
    delete h;
}

// Upload the packed matrices, task and segment tables of a handle whose host
// fields (tree, ktot, mat_elems, statistics) are set, create its streams and
// events, and fill the phases from the task counts (order: near, leaf forward,
// leaf expansion, couplings, upward[l], downward[l]). Frees the handle and
// returns the status on failure.
static h2_status upload_and_finish(h2_handle *h, int device, const float2 *mat, std::vector<Task> htasks,
                                   std::vector<Seg> hsegs, const std::vector<int32_t> &counts)
{
    const int nl = h->nlev;
    auto fail = [&](h2_status s) {
        h2_free(h);
        return s;
    };
    if ((int)counts.size() != 4 + 2 * nl) {
        set_error("phase table does not match the tree depth");
        return fail(H2_ERR_ARG);
    }
    int64_t total = 0;
    for (int32_t c : counts) total += c;
    if (total != (int64_t)htasks.size()) {
        set_error("phase table does not match the task list");
        return fail(H2_ERR_ARG);
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("no CUDA device " + std::to_string(device));
        return fail(H2_ERR_CUDA);
    }
    DeviceGuard dev_guard(device);
    if (dev_guard.err != cudaSuccess) return fail(H2_ERR_CUDA);
#define H2_LOAD_CUDA(call)                                                         \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) {                                                  \
            cudaGetLastError();                                                    \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e__));        \
            return fail(e__ == cudaErrorMemoryAllocation ? H2_ERR_ALLOC : H2_ERR_CUDA); \
        }                                                                          \
    } while (0)
    const int64_t melems = std::max<int64_t>(h->mat_elems, 32);
    H2_LOAD_CUDA(cudaMalloc(&h->d_mat, (size_t)melems * sizeof(float2)));
    if (mat) H2_LOAD_CUDA(cudaMemcpy(h->d_mat, mat, (size_t)melems * sizeof(float2), cudaMemcpyHostToDevice));
    h->segs_host = hsegs;
    H2_LOAD_CUDA(cudaMalloc(&h->d_segs, std::max<size_t>(1, hsegs.size()) * sizeof(Seg)));
    if (!hsegs.empty())
        H2_LOAD_CUDA(cudaMemcpy(h->d_segs, hsegs.data(), hsegs.size() * sizeof(Seg), cudaMemcpyHostToDevice));
    H2_LOAD_CUDA(cudaMalloc(&h->d_tasks, std::max<size_t>(1, htasks.size()) * sizeof(Task)));
    if (!htasks.empty())
        H2_LOAD_CUDA(cudaMemcpy(h->d_tasks, htasks.data(), htasks.size() * sizeof(Task), cudaMemcpyHostToDevice));
    H2_LOAD_CUDA(cudaMalloc(&h->d_coef, std::max<int64_t>(1, 2 * h->ktot) * sizeof(double2)));
    H2_LOAD_CUDA(cudaStreamCreateWithFlags(&h->s_aux, cudaStreamNonBlocking));
    H2_LOAD_CUDA(cudaStreamCreateWithFlags(&h->s_cap, cudaStreamNonBlocking));
    H2_LOAD_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    H2_LOAD_CUDA(cudaEventCreateWithFlags(&h->ev_near, cudaEventDisableTiming));
#undef H2_LOAD_CUDA

    int64_t tpos = 0;
    size_t k = 0;
    auto fill = [&](Phase &P, const char *name) {
        const int32_t cnt = counts[k++];
        P.name = name;
        P.tasks.assign(htasks.begin() + tpos, htasks.begin() + tpos + cnt);
        P.max_mpad = P.max_ncol = 0;
        P.elems = 0;
        for (const Task &t : P.tasks) {
            P.max_mpad = std::max(P.max_mpad, t.mpad);
            P.max_ncol = std::max(P.max_ncol, t.ncol);
            P.elems += (int64_t)t.m * t.ncol;
        }
        P.d_tasks = h->d_tasks + tpos;
        tpos += cnt;
        P.threads = choose_threads(P.tasks);
    };
    fill(h->near, "near");
    fill(h->upleaf, "upleaf");
    fill(h->leafexp, "leafexp");
    fill(h->couple, "couple");
    h->up.resize(nl);
    h->down.resize(nl);
    for (int l = 0; l < nl; ++l) fill(h->up[l], "up");
    for (int l = 0; l < nl; ++l) fill(h->down[l], "down");

    h2_stats &S = h->stats;
    int nk = (h->near.ntask() > 0) + (h->upleaf.ntask() > 0) + (h->leafexp.ntask() > 0) + (h->couple.ntask() > 0);
    for (int l = 0; l < nl; ++l) nk += (h->up[l].ntask() > 0) + (h->down[l].ntask() > 0);
    S.kernels_per_matvec = nk;
    S.device_bytes = melems * 8 + (int64_t)hsegs.size() * sizeof(Seg) + (int64_t)htasks.size() * sizeof(Task) +
                     2 * h->ktot * 16;
    return H2_OK;
}

}  // extern "C"

// Device packing of h2_load_device: one piece of a task matrix copied from the
// caller's device block (column-major rows x cols, optionally transposed)
// into the task's column range of the packed matrix.
struct DevPiece {
    const float2 *src;
    int64_t dst;          // element offset of the piece's first column in the packed matrix
    int32_t rows, cols;   // source block shape
    int32_t mpad;         // leading dimension of the packed task matrix
    int32_t transpose;
};

__global__ void dev_pack_kernel(const DevPiece *__restrict__ pieces, float2 *__restrict__ mat, int *__restrict__ bad)
{
    const DevPiece P = pieces[blockIdx.x];
    const int orows = P.transpose ? P.cols : P.rows, ocols = P.transpose ? P.rows : P.cols;
    const int64_t total = (int64_t)orows * ocols;
    int nonfinite = 0;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = (int)(e % orows), j = (int)(e / orows);
        const float2 v = P.transpose ? P.src[(int64_t)r * P.rows + j] : P.src[(int64_t)j * P.rows + r];
        nonfinite |= !(isfinite(v.x) && isfinite(v.y));
        mat[P.dst + (int64_t)j * P.mpad + r] = v;
    }
    if (nonfinite) atomicExch(bad, 1);
}

static h2_status load_impl(const h2_tree *tree, const h2_data *data, const char *opts, h2_handle **out,
                           bool on_device)
{
    if (!out) return arg_error("out is NULL");
    *out = nullptr;
    std::vector<int32_t> parent, level;
    h2_status st = validate_tree(tree, parent, level);
    if (st != H2_OK) return st;
    st = validate_data(tree, data, parent);
    if (st != H2_OK) return st;
    if (on_device && data->dtype != H2_C64) return arg_error("h2_load_device: blocks must be complex64");

    int device = 0;
    bool use_graphs = true, tc_pipeline = true, sym_couple = false;
    uint32_t wait_limit = 1u << 24;
    if (opts) {
        const char *p = strstr(opts, "device=");
        if (p) device = atoi(p + 7);
        const char *g = strstr(opts, "graphs=");
        if (g) use_graphs = atoi(g + 7) != 0;
        const char *tp = strstr(opts, "tc_pipeline=");
        if (tp) tc_pipeline = atoi(tp + 12) != 0;
        const char *sc = strstr(opts, "sym_couple=");
        if (sc) sym_couple = atoi(sc + 11) != 0;
        const char *wl = strstr(opts, "wait_limit=");
        if (wl) {
            const long long v = atoll(wl + 11);
            if (v < 0 || v > 0xFFFFFFFFll) return arg_error("h2_load: wait_limit must lie in [0, 2^32)");
            wait_limit = (uint32_t)v;
        }
    }
    h2_handle *h = new (std::nothrow) h2_handle();
    if (!h) return H2_ERR_ALLOC;
    h->device = device;
    h->use_graphs = use_graphs;
    h->tc_pipeline = tc_pipeline;
    h->wait_limit = wait_limit;
    h->sym_couple = sym_couple;
    const int32_t n = tree->n, nc = tree->n_clusters, nl = tree->n_levels;
    h->n = n;
    h->nc = nc;
    h->nlev = nl;
    h->level_ptr.assign(tree->level_ptr, tree->level_ptr + nl + 1);
    h->child.assign(tree->child, tree->child + 2 * nc);
    h->begin.assign(tree->begin, tree->begin + nc);
    h->size.assign(tree->size, tree->size + nc);
    h->rank.assign(tree->rank, tree->rank + nc);
    h->parent = parent;
    h->level = level;
    h->xo.assign(nc, 0);
    int64_t ktot = 0;
    for (int t = 0; t < nc; ++t) {
        h->xo[t] = (int32_t)ktot;
        ktot += tree->rank[t];
    }
    h->ktot = ktot;
    if (2 * ktot + 2 * (int64_t)n > INT32_MAX) {
        delete h;
        return arg_error("problem too large for 32-bit offsets");
    }
    auto leaf = [&](int t) { return tree->child[2 * t] < 0; };
    auto enc1 = [](int64_t off) { return (int32_t)(-off - 1); };
    const int32_t *rk = tree->rank;

    // ---- build the task lists --------------------------------------------------
    struct Piece {
        int kind;  // 0 Z, 1 U, 2 W, 3 T, 4 S
        int64_t off;
        int32_t rows, cols;  // source block shape (column-major)
        bool transpose;
    };
    struct TaskBuild {
        Task t;
        std::vector<Seg> segs;
        std::vector<Piece> pieces;
    };
    std::vector<std::vector<TaskBuild>> phases(4 + 2 * nl);
    // index: 0 near, 1 upleaf, 2 leafexp, 3 couple (all levels), 4.. up[l], down[l]
    const int IDX_NEAR = 0, IDX_UPLEAF = 1, IDX_LEAFEXP = 2, IDX_COUPLE = 3;
    auto idx_up = [&](int l) { return 4 + l; };
    auto idx_down = [&](int l) { return 4 + nl + l; };
    phases.resize(4 + 2 * nl);

    auto new_task = [&](int32_t out_off, int32_t m) {
        TaskBuild tb;
        tb.t.out_off = out_off;
        tb.t.m = m;
        tb.t.mpad = m + (m & 1);
        tb.t.ncol = 0;
        tb.t.mat_off = 0;
        return tb;
    };
    int64_t near_elems = 0, coupling_elems = 0, transfer_elems = 0, leaf_elems = 0, nleaves = 0;
    int64_t near_blocks = 0, adm_blocks = 0;
    int32_t max_rank = 0;
    for (int t = 0; t < nc; ++t) max_rank = std::max(max_rank, rk[t]);

    for (int t = 0; t < nc; ++t) {
        const int32_t kt = rk[t];
        const int l = level[t];
        if (leaf(t)) {
            ++nleaves;
            // near field
            TaskBuild tb = new_task(tree->begin[t], tree->size[t]);
            for (int j = data->near_ptr[t]; j < data->near_ptr[t + 1]; ++j) {
                const int s = data->near_col[j];
                tb.segs.push_back({tree->begin[s], tree->size[s]});
                tb.pieces.push_back({0, data->Z_off[j], tree->size[t], tree->size[s], false});
                tb.t.ncol += tree->size[s];
                near_elems += (int64_t)tree->size[t] * tree->size[s];
                ++near_blocks;
            }
            if (tb.t.ncol > 0) phases[IDX_NEAR].push_back(std::move(tb));
            if (kt > 0) {
                leaf_elems += (int64_t)tree->size[t] * kt;
                TaskBuild f = new_task((int32_t)h->xo[t], kt);
                f.segs.push_back({tree->begin[t], tree->size[t]});
                f.pieces.push_back({data->W ? 2 : 1, data->W ? data->W_off[t] : data->U_off[t],
                                    tree->size[t], kt, true});
                f.t.ncol = tree->size[t];
                phases[IDX_UPLEAF].push_back(std::move(f));
                TaskBuild b = new_task(tree->begin[t], tree->size[t]);
                b.segs.push_back({enc1(ktot + h->xo[t]), kt});
                b.pieces.push_back({1, data->U_off[t], tree->size[t], kt, false});
                b.t.ncol = kt;
                phases[IDX_LEAFEXP].push_back(std::move(b));
            }
        } else if (kt > 0) {
            TaskBuild u = new_task((int32_t)h->xo[t], kt);
            for (int c = 0; c < 2; ++c) {
                const int ch = tree->child[2 * t + c];
                if (rk[ch] == 0) continue;
                u.segs.push_back({enc1(h->xo[ch]), rk[ch]});
                u.pieces.push_back({3, data->T_off[ch], rk[ch], kt, true});
                u.t.ncol += rk[ch];
            }
            if (u.t.ncol > 0) phases[idx_up(l)].push_back(std::move(u));
        }
        if (t > 0 && kt > 0 && rk[parent[t]] > 0) transfer_elems += (int64_t)kt * rk[parent[t]];
        // couplings (all levels in one phase) and the downward transfer (per level)
        if (kt > 0) {
            TaskBuild d = new_task((int32_t)(ktot + h->xo[t]), kt);
            for (int j = data->adm_ptr[t]; j < data->adm_ptr[t + 1]; ++j) {
                const int s = data->adm_col[j];
                ++adm_blocks;
                if (rk[s] == 0) continue;
                d.segs.push_back({enc1(h->xo[s]), rk[s]});
                d.pieces.push_back({4, data->S_off[j], kt, rk[s], false});
                d.t.ncol += rk[s];
                coupling_elems += (int64_t)kt * rk[s];
            }
            if (d.t.ncol > 0) phases[IDX_COUPLE].push_back(std::move(d));
            if (t > 0 && rk[parent[t]] > 0) {
                const int p = parent[t];
                TaskBuild e = new_task((int32_t)(ktot + h->xo[t]), kt);
                e.segs.push_back({enc1(ktot + h->xo[p]), rk[p]});
                e.pieces.push_back({3, data->T_off[t], kt, rk[p], false});
                e.t.ncol = rk[p];
                phases[idx_down(l)].push_back(std::move(e));
            }
        } else {
            adm_blocks += data->adm_ptr[t + 1] - data->adm_ptr[t];
        }
    }

    // ---- lay out matrices, sort tasks by decreasing work -------------------------------
    int64_t mat_elems = 0;
    int64_t nseg = 0, ntask = 0;
    for (auto &ph : phases) {
        std::stable_sort(ph.begin(), ph.end(), [](const TaskBuild &a, const TaskBuild &b) {
            return (int64_t)a.t.mpad * a.t.ncol > (int64_t)b.t.mpad * b.t.ncol;
        });
        for (auto &tb : ph) {
            tb.t.mat_off = mat_elems;
            mat_elems += ((int64_t)tb.t.mpad * tb.t.ncol + 31) / 32 * 32;
            tb.t.seg_begin = (int32_t)nseg;
            nseg += (int64_t)tb.segs.size();
            tb.t.seg_end = (int32_t)nseg;
            ++ntask;
        }
    }
    if (nseg > INT32_MAX) {
        delete h;
        return arg_error("too many blocks");
    }
    std::vector<float2> hmat;
    std::vector<DevPiece> dpieces;
    bool finite = true;
    if (on_device) {
        // the pieces are copied on the device after the upload step allocated the matrix
        for (auto &ph : phases)
            for (const TaskBuild &tb : ph) {
                int64_t col = 0;
                for (const Piece &pc : tb.pieces) {
                    const void *base = pc.kind == 0 ? data->Z : pc.kind == 1 ? data->U : pc.kind == 2 ? data->W
                                                                : pc.kind == 3 ? data->T : data->S;
                    DevPiece d;
                    d.src = reinterpret_cast<const float2 *>(base) + pc.off;
                    d.dst = tb.t.mat_off + col * tb.t.mpad;
                    d.rows = pc.rows;
                    d.cols = pc.cols;
                    d.mpad = tb.t.mpad;
                    d.transpose = pc.transpose ? 1 : 0;
                    if ((int64_t)pc.rows * pc.cols > 0) dpieces.push_back(d);
                    col += pc.transpose ? pc.rows : pc.cols;
                }
            }
    }
    if (!on_device) {
    try {
        hmat.assign((size_t)std::max<int64_t>(mat_elems, 32), make_float2(0.f, 0.f));
    } catch (...) {
        delete h;
        set_error("host allocation of the staging matrix failed");
        return H2_ERR_ALLOC;
    }
    }
    const CplxIn srcZ{data->Z, data->dtype}, srcU{data->U, data->dtype}, srcW{data->W, data->dtype},
        srcT{data->T, data->dtype}, srcS{data->S, data->dtype};
    if (!on_device)
    for (auto &ph : phases) {
        const int64_t np = (int64_t)ph.size();
#pragma omp parallel for schedule(dynamic, 4) reduction(&& : finite)
        for (int64_t i = 0; i < np; ++i) {
            const TaskBuild &tb = ph[i];
            float2 *dst = hmat.data() + tb.t.mat_off;
            int64_t col = 0;
            for (const Piece &pc : tb.pieces) {
                const CplxIn &src = pc.kind == 0 ? srcZ : pc.kind == 1 ? srcU : pc.kind == 2 ? srcW
                                                         : pc.kind == 3 ? srcT : srcS;
                const int32_t orows = pc.transpose ? pc.cols : pc.rows;  // rows placed
                const int32_t ocols = pc.transpose ? pc.rows : pc.cols;
                for (int32_t j = 0; j < ocols; ++j) {
                    float2 *dc = dst + (col + j) * tb.t.mpad;
                    for (int32_t r = 0; r < orows; ++r) {
                        const int64_t si = pc.transpose ? pc.off + (int64_t)r * pc.rows + j
                                                        : pc.off + (int64_t)j * pc.rows + r;
                        const float2 v = src.at(si);
                        finite = finite && std::isfinite(v.x) && std::isfinite(v.y);
                        dc[r] = v;
                    }
                }
                col += ocols;
            }
        }
    }
    if (!finite) {
        delete h;
        return arg_error("data: non-finite entry (or entry overflowing FP32)");
    }

    std::vector<Task> htasks;
    std::vector<Seg> hsegs;
    std::vector<int32_t> counts;
    htasks.reserve(ntask);
    hsegs.reserve(nseg);
    for (auto &ph : phases) {
        counts.push_back((int32_t)ph.size());
        for (auto &tb : ph) {
            htasks.push_back(tb.t);
            hsegs.insert(hsegs.end(), tb.segs.begin(), tb.segs.end());
        }
    }
    phases.clear();
    h2_stats &S = h->stats;
    S.n = n;
    S.n_clusters = nc;
    S.n_leaves = nleaves;
    S.n_levels = nl;
    S.near_blocks = near_blocks;
    S.adm_blocks = adm_blocks;
    S.near_elems = near_elems;
    S.coupling_elems = coupling_elems;
    S.transfer_elems = transfer_elems;
    S.leaf_elems = leaf_elems;
    S.max_rank = max_rank;
    h->mat_elems = mat_elems;
    st = upload_and_finish(h, device, on_device ? nullptr : hmat.data(), std::move(htasks), std::move(hsegs), counts);
    if (st != H2_OK) return st;
    if (on_device) {
        DeviceGuard dev_guard(device);
        DevPiece *d_pieces = nullptr;
        int *d_bad = nullptr;
        int bad = 0;
        cudaError_t e = dev_guard.err;
        const size_t npc = dpieces.size();
        if (e == cudaSuccess) e = cudaMemset(h->d_mat, 0, (size_t)std::max<int64_t>(h->mat_elems, 32) * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
        // pieces in chunks, so that the descriptor buffer stays small
        const size_t chunk = 1u << 20;
        if (e == cudaSuccess && npc) e = cudaMalloc(&d_pieces, std::min(npc, chunk) * sizeof(DevPiece));
        for (size_t p0 = 0; e == cudaSuccess && p0 < npc; p0 += chunk) {
            const size_t cnt = std::min(chunk, npc - p0);
            e = cudaMemcpy(d_pieces, dpieces.data() + p0, cnt * sizeof(DevPiece), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                dev_pack_kernel<<<(unsigned)cnt, 256>>>(d_pieces, h->d_mat, d_bad);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
        if (d_pieces) cudaFree(d_pieces);
        if (d_bad) cudaFree(d_bad);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("h2_load_device: packing failed: ") + cudaGetErrorString(e));
            h2_free(h);
            return e == cudaErrorMemoryAllocation ? H2_ERR_ALLOC : H2_ERR_CUDA;
        }
        if (bad) {
            h2_free(h);
            return arg_error("data: non-finite entry");
        }
    }
    *out = h;
    return H2_OK;
}

extern "C" {

h2_status h2_load(const h2_tree *tree, const h2_data *data, const char *opts, h2_handle **out)
{
    return load_impl(tree, data, opts, out, false);
}

h2_status h2_load_device(const h2_tree *tree, const h2_data *data, const char *opts, h2_handle **out)
{
    return load_impl(tree, data, opts, out, true);
}

h2_status h2_device_status(h2_handle *h)
{
    if (!h) return arg_error("h2_device_status: NULL handle");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    H2_CUDA(cudaDeviceSynchronize());
    int flag = 0;
    h2_status s = h2_split_error_flag(h, &flag);
    if (s != H2_OK) return s;
    int sflag = 0;
    s = h2::h2_sym_error_flag(h, &sflag);
    if (s != H2_OK) return s;
    if (sflag) {
        set_error("a bounded wait inside the symmetric-storage kernel ran out");
        return H2_ERR_TIMEOUT;
    }
    if (flag) {
        set_error("a bounded wait inside a tensor-core kernel ran out");
        return H2_ERR_TIMEOUT;
    }
    return H2_OK;
}

// ---- saving and reloading a loaded operator (.h2 files) -------------------------------
// Layout (little-endian): magic "H2PACKED", u32 version, i32 n, nc, nlev, i64 ktot,
// mat_elems, ntask, nseg, i32 task counts per phase [4 + 2 nlev], h2_stats,
// i32 arrays level_ptr [nlev + 1], child [2 nc], begin, size, rank, parent,
// level, xo [nc], Task [ntask], Seg [nseg], float2 matrices [max(mat_elems, 32)],
// u64 FNV-1a hash of everything before it.

namespace {
constexpr char kMagic[8] = {'H', '2', 'P', 'A', 'C', 'K', 'E', 'D'};
constexpr uint32_t kVersion = 1;

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

struct Writer {
    FILE *f;
    Fnv fnv;
    bool ok = true;
    void put(const void *p, size_t n)
    {
        if (!ok || n == 0) return;
        fnv.add(p, n);
        ok = fwrite(p, 1, n, f) == n;
    }
};

struct Reader {
    FILE *f;
    Fnv fnv;
    bool ok = true;
    void get(void *p, size_t n)
    {
        if (!ok || n == 0) return;
        ok = fread(p, 1, n, f) == n;
        if (ok) fnv.add(p, n);
    }
};
}  // namespace

h2_status h2_save(const h2_handle *h, const char *path)
{
    if (!h || !path) return arg_error("h2_save: NULL argument");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    FILE *f = fopen(path, "wb");
    if (!f) return arg_error(std::string("h2_save: cannot open ") + path);
    Writer w{f};
    const int32_t hdr[3] = {h->n, h->nc, h->nlev};
    std::vector<int32_t> counts;
    counts.push_back(h->near.ntask());
    counts.push_back(h->upleaf.ntask());
    counts.push_back(h->leafexp.ntask());
    counts.push_back(h->couple.ntask());
    for (const Phase &p : h->up) counts.push_back(p.ntask());
    for (const Phase &p : h->down) counts.push_back(p.ntask());
    std::vector<Task> tasks;
    auto add = [&](const Phase &p) { tasks.insert(tasks.end(), p.tasks.begin(), p.tasks.end()); };
    add(h->near);
    add(h->upleaf);
    add(h->leafexp);
    add(h->couple);
    for (const Phase &p : h->up) add(p);
    for (const Phase &p : h->down) add(p);
    const int64_t sizes[4] = {h->ktot, h->mat_elems, (int64_t)tasks.size(), (int64_t)h->segs_host.size()};
    w.put(kMagic, 8);
    w.put(&kVersion, 4);
    w.put(hdr, sizeof(hdr));
    w.put(sizes, sizeof(sizes));
    w.put(counts.data(), counts.size() * 4);
    w.put(&h->stats, sizeof(h2_stats));
    for (const std::vector<int32_t> *v : {&h->level_ptr, &h->child, &h->begin, &h->size, &h->rank, &h->parent,
                                          &h->level, &h->xo})
        w.put(v->data(), v->size() * 4);
    w.put(tasks.data(), tasks.size() * sizeof(Task));
    w.put(h->segs_host.data(), h->segs_host.size() * sizeof(Seg));
    // matrices, through a bounded host staging buffer
    const int64_t melems = std::max<int64_t>(h->mat_elems, 32);
    const int64_t chunk = (int64_t)1 << 25;  // 256 MB of float2
    std::vector<float2> buf((size_t)std::min(melems, chunk));
    for (int64_t o = 0; o < melems && w.ok; o += chunk) {
        const int64_t m = std::min(chunk, melems - o);
        if (cudaMemcpy(buf.data(), h->d_mat + o, (size_t)m * sizeof(float2), cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            set_error("h2_save: device read failed");
            return H2_ERR_CUDA;
        }
        w.put(buf.data(), (size_t)m * sizeof(float2));
    }
    const uint64_t hash = w.fnv.h;
    if (w.ok) w.ok = fwrite(&hash, 1, 8, f) == 8;
    const bool closed = fclose(f) == 0;
    if (!w.ok || !closed) return arg_error(std::string("h2_save: write failed: ") + path);
    return H2_OK;
}

h2_status h2_load_file(const char *path, const char *opts, h2_handle **out)
{
    if (!path || !out) return arg_error("h2_load_file: NULL argument");
    *out = nullptr;
    int device = 0;
    bool use_graphs = true, tc_pipeline = true, sym_couple = false;
    uint32_t wait_limit = 1u << 24;
    if (opts) {
        const char *p = strstr(opts, "device=");
        if (p) device = atoi(p + 7);
        const char *g = strstr(opts, "graphs=");
        if (g) use_graphs = atoi(g + 7) != 0;
        const char *tp = strstr(opts, "tc_pipeline=");
        if (tp) tc_pipeline = atoi(tp + 12) != 0;
        const char *sc = strstr(opts, "sym_couple=");
        if (sc) sym_couple = atoi(sc + 11) != 0;
        const char *wl = strstr(opts, "wait_limit=");
        if (wl) {
            const long long v = atoll(wl + 11);
            if (v < 0 || v > 0xFFFFFFFFll) return arg_error("h2_load_file: wait_limit must lie in [0, 2^32)");
            wait_limit = (uint32_t)v;
        }
    }
    FILE *f = fopen(path, "rb");
    if (!f) return arg_error(std::string("h2_load_file: cannot open ") + path);
    Reader r{f};
    char magic[8];
    uint32_t version = 0;
    int32_t hdr[3];
    int64_t sizes[4];
    r.get(magic, 8);
    r.get(&version, 4);
    r.get(hdr, sizeof(hdr));
    r.get(sizes, sizeof(sizes));
    auto bad = [&](const std::string &why) {
        fclose(f);
        return arg_error("h2_load_file: " + why + ": " + path);
    };
    if (!r.ok || memcmp(magic, kMagic, 8) != 0 || version != kVersion) return bad("not a version-1 .h2 file");
    const int32_t n = hdr[0], nc = hdr[1], nl = hdr[2];
    if (n < 1 || nc < 1 || nl < 1 || nl > 64 || sizes[0] < 0 || sizes[1] < 0 || sizes[2] < 0 || sizes[3] < 0 ||
        sizes[1] > ((int64_t)1 << 40) || sizes[2] > INT32_MAX || sizes[3] > INT32_MAX)
        return bad("header out of range");
    h2_handle *h = new (std::nothrow) h2_handle();
    if (!h) {
        fclose(f);
        return H2_ERR_ALLOC;
    }
    h->device = device;
    h->use_graphs = use_graphs;
    h->tc_pipeline = tc_pipeline;
    h->wait_limit = wait_limit;
    h->sym_couple = sym_couple;
    h->n = n;
    h->nc = nc;
    h->nlev = nl;
    h->ktot = sizes[0];
    h->mat_elems = sizes[1];
    std::vector<int32_t> counts(4 + 2 * nl);
    r.get(counts.data(), counts.size() * 4);
    r.get(&h->stats, sizeof(h2_stats));
    h->level_ptr.resize(nl + 1);
    h->child.resize(2 * (size_t)nc);
    for (std::vector<int32_t> *v : {&h->begin, &h->size, &h->rank, &h->parent, &h->level, &h->xo}) v->resize(nc);
    for (std::vector<int32_t> *v : {&h->level_ptr, &h->child, &h->begin, &h->size, &h->rank, &h->parent, &h->level,
                                    &h->xo})
        r.get(v->data(), v->size() * 4);
    std::vector<Task> tasks((size_t)sizes[2]);
    std::vector<Seg> segs((size_t)sizes[3]);
    r.get(tasks.data(), tasks.size() * sizeof(Task));
    r.get(segs.data(), segs.size() * sizeof(Seg));
    std::vector<float2> mat;
    try {
        mat.resize((size_t)std::max<int64_t>(sizes[1], 32));
    } catch (...) {
        delete h;
        fclose(f);
        set_error("h2_load_file: host allocation failed");
        return H2_ERR_ALLOC;
    }
    r.get(mat.data(), mat.size() * sizeof(float2));
    uint64_t hash = 0;
    const uint64_t expect = r.fnv.h;
    const bool ok = r.ok && fread(&hash, 1, 8, f) == 8 && hash == expect;
    fclose(f);
    if (!ok) {
        delete h;
        return arg_error(std::string("h2_load_file: truncated or corrupted file: ") + path);
    }
    // every task and segment must stay inside the matrices and vectors
    const int64_t melems = std::max<int64_t>(sizes[1], 32);
    for (const Task &t : tasks)
        if (t.m < 0 || t.mpad < t.m || t.ncol < 0 || t.mat_off < 0 || t.mat_off + (int64_t)t.mpad * t.ncol > melems ||
            t.seg_begin < 0 || t.seg_end < t.seg_begin || t.seg_end > (int64_t)segs.size()) {
            delete h;
            return arg_error("h2_load_file: task table out of range");
        }
    for (const Seg &g : segs) {
        const int64_t lo = g.in_off >= 0 ? g.in_off : -(int64_t)g.in_off - 1;
        const int64_t lim = g.in_off >= 0 ? n : 2 * h->ktot;
        if (g.n < 0 || lo + g.n > lim) {
            delete h;
            return arg_error("h2_load_file: segment table out of range");
        }
    }
    h2_status st = upload_and_finish(h, device, mat.data(), std::move(tasks), std::move(segs), counts);
    if (st != H2_OK) return st;
    *out = h;
    return H2_OK;
}

h2_status h2_get_stats(const h2_handle *h, h2_stats *out)
{
    if (!h || !out) return arg_error("NULL argument");
    *out = h->stats;
    return H2_OK;
}

h2_status h2_sym_stats(h2_handle *h, int64_t *stored_elems, int64_t *scratch_entries, double *max_asym)
{
    if (!h || !stored_elems || !scratch_entries || !max_asym) return arg_error("h2_sym_stats: NULL argument");
    if (!h->sym_couple) return (set_error("h2_sym_stats: the handle was loaded without sym_couple=1"), H2_ERR_STATE);
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    if (!h->sym) {
        const h2_status s = h2::h2_sym_init(h);
        if (s != H2_OK) return s;
    }
    *stored_elems = h->sym->stored_elems;
    *scratch_entries = h->sym->scratch_entries;
    *max_asym = h->sym->max_asym;
    return H2_OK;
}

}  // extern "C"

// ---- products -------------------------------------------------------------------------

// df: c128 product accumulated in double-float (H2_PREC_DFACC) instead of FP64
template <typename VT>
static h2_status run_single(h2_handle *h, const VT *x, VT *y, cudaStream_t st, bool df = false)
{
    VT *coef = reinterpret_cast<VT *>(h->d_coef);
    const float2 *mat = h->d_mat;
    const Seg *segs = h->d_segs;
    auto launch = [&](const Phase &ph, const VT *in0, VT *outp, int beta, cudaStream_t s) {
        if constexpr (std::is_same<VT, float2>::value)
            return launch_phase_f32(ph, mat, segs, in0, coef, outp, beta, s);
        else
            return df ? launch_phase_df(ph, mat, segs, in0, coef, outp, beta, s)
                      : launch_phase_f64(ph, mat, segs, in0, coef, outp, beta, s);
    };
    H2_CUDA(cudaMemsetAsync(coef, 0, sizeof(VT) * 2 * std::max<int64_t>(1, h->ktot), st));
    H2_CUDA(cudaEventRecord(h->ev_fork, st));
    H2_CUDA(cudaStreamWaitEvent(h->s_aux, h->ev_fork, 0));
    if constexpr (std::is_same<VT, float2>::value) {
        if (h->symnear) H2_CUDA(h2::symnear_run(h, x, y, h->s_aux));   // near blocks stored once per leaf pair
        else H2_CUDA(launch(h->near, x, y, 0, h->s_aux));
    } else {
        H2_CUDA(launch(h->near, x, y, 0, h->s_aux));
    }
    H2_CUDA(cudaEventRecord(h->ev_near, h->s_aux));
    H2_CUDA(launch(h->upleaf, x, coef, 0, st));
    for (int l = h->nlev - 1; l >= 0; --l) H2_CUDA(launch(h->up[l], x, coef, 0, st));
    if constexpr (std::is_same<VT, float2>::value) {
        if (h->sym) H2_CUDA(h2::h2_sym_couple(h, coef, st));   // couplings stored once per pair
        else H2_CUDA(launch(h->couple, x, coef, 0, st));
    } else {
        H2_CUDA(launch(h->couple, x, coef, 0, st));
    }
    for (int l = 0; l < h->nlev; ++l) H2_CUDA(launch(h->down[l], x, coef, 1, st));
    H2_CUDA(cudaStreamWaitEvent(st, h->ev_near, 0));
    H2_CUDA(launch(h->leafexp, x, y, 1, st));
    return H2_OK;
}

// The single-RHS FP32 product as one CUDA graph launch: captured once per
// (x, y) pair on an internal stream (the fork to the near-field stream and the
// join are captured as graph edges) and replayed on the caller's stream.
static h2_status run_single_graph(h2_handle *h, const float2 *x, float2 *y, cudaStream_t st)
{
    for (auto &g : h->graphs)
        if (g.x == x && g.y == y) {
            g.last_use = ++h->graph_clock;
            H2_CUDA(cudaGraphLaunch(g.exec, st));
            return H2_OK;
        }
    cudaGraph_t graph = nullptr;
    H2_CUDA(cudaStreamBeginCapture(h->s_cap, cudaStreamCaptureModeThreadLocal));
    h2_status s = run_single<float2>(h, x, y, h->s_cap);
    const cudaError_t ec = cudaStreamEndCapture(h->s_cap, &graph);
    if (s != H2_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        h->use_graphs = false;  // capture unsupported here: direct launches from now on
        return run_single<float2>(h, x, y, st);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        h->use_graphs = false;
        return run_single<float2>(h, x, y, st);
    }
    if (h->graphs.size() >= 8) {
        auto victim = std::min_element(h->graphs.begin(), h->graphs.end(),
                                       [](const auto &a, const auto &b) { return a.last_use < b.last_use; });
        cudaGraphExecDestroy(victim->exec);
        h->graphs.erase(victim);
    }
    h->graphs.push_back({x, y, exec, ++h->graph_clock});
    H2_CUDA(cudaGraphLaunch(exec, st));
    return H2_OK;
}

static void drop_graphs(h2_handle *h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    h2_drop_split_graphs(h);
}

// The split-bf16 product of nrhs columns captured into a CUDA graph per
// (x, y, ld, nrhs) on first use and replayed afterwards (at most 8 kept, least
// recently used out); the tensor-core state and planes are allocated before
// any capture, and graphs are dropped whenever the planes move.
static h2_status run_split_graph(h2_handle *h, const float2 *x, float2 *y, int64_t ld, int nrhs, cudaStream_t st)
{
    int moved = 0;
    h2_status s = h2_split_prepare(h, nrhs, &moved);
    if (s != H2_OK) return s;
    if (moved) h2_drop_split_graphs(h);
    for (auto &g : h->split_graphs)
        if (g.x == x && g.y == y && g.ld == ld && g.nrhs == nrhs) {
            g.last_use = ++h->graph_clock;
            H2_CUDA(cudaGraphLaunch(g.exec, st));
            return H2_OK;
        }
    cudaGraph_t graph = nullptr;
    H2_CUDA(cudaStreamBeginCapture(h->s_cap, cudaStreamCaptureModeThreadLocal));
    s = h2_run_multi_split(h, x, ld, y, ld, nrhs, h->s_cap);
    const cudaError_t ec = cudaStreamEndCapture(h->s_cap, &graph);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaErrorUnknown;
    if (s == H2_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        h->use_graphs = false;  // capture unsupported here: direct launches from now on
        return h2_run_multi_split(h, x, ld, y, ld, nrhs, st);
    }
    if (h->split_graphs.size() >= 8) {
        auto victim = std::min_element(h->split_graphs.begin(), h->split_graphs.end(),
                                       [](const auto &a, const auto &b) { return a.last_use < b.last_use; });
        cudaGraphExecDestroy(victim->exec);
        h->split_graphs.erase(victim);
    }
    h->split_graphs.push_back({x, y, ld, nrhs, exec, ++h->graph_clock});
    H2_CUDA(cudaGraphLaunch(exec, st));
    return H2_OK;
}

extern "C" {

h2_status h2_sym_near(h2_handle *h, const void *chi, h2_dtype dtype)
{
    if (!h) return arg_error("h2_sym_near: NULL handle");
    if (chi && dtype != H2_C64 && dtype != H2_C128) return arg_error("h2_sym_near: bad dtype");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    H2_CUDA(cudaDeviceSynchronize());
    drop_graphs(h);   // captured products use the previous near-field structure
    if (!chi) {
        h2::symnear_free(h);
        return H2_OK;
    }
    std::vector<float2> c(h->n);
    for (int32_t i = 0; i < h->n; ++i) {
        double re, im;
        if (dtype == H2_C128) {
            re = static_cast<const double *>(chi)[2 * i];
            im = static_cast<const double *>(chi)[2 * i + 1];
        } else {
            re = static_cast<const float *>(chi)[2 * i];
            im = static_cast<const float *>(chi)[2 * i + 1];
        }
        if (!std::isfinite(re) || !std::isfinite(im)) return arg_error("h2_sym_near: non-finite chi");
        c[i] = make_float2((float)re, (float)im);
        if (c[i].x == 0.f && c[i].y == 0.f) {
            h2::symnear_free(h);
            set_error("h2_sym_near: chi is zero at unknown " + std::to_string(i) +
                      " (a void voxel): its near-field columns do not determine their transposes");
            return H2_ERR_STATE;
        }
    }
    return h2::symnear_init(h, c);
}

h2_status h2_sym_near_stats(h2_handle *h, int64_t *stored_elems, int64_t *scratch_entries, double *max_asym)
{
    if (!h || !stored_elems || !scratch_entries || !max_asym) return arg_error("h2_sym_near_stats: NULL argument");
    if (!h->symnear) return (set_error("h2_sym_near_stats: no symmetric near field (call h2_sym_near)"), H2_ERR_STATE);
    *stored_elems = h->symnear->stored_elems;
    *scratch_entries = h->symnear->scratch_entries;
    *max_asym = h->symnear->max_asym;
    return H2_OK;
}


h2_status h2_matvec(h2_handle *h, const void *x, void *y, int32_t nrhs, int64_t ld, h2_prec prec,
                    void *stream)
{
    if (!h || !x || !y) return arg_error("h2_matvec: NULL argument");
    if (nrhs < 1) return arg_error("h2_matvec: nrhs must be >= 1");
    if (nrhs > 1 && ld < h->n) return arg_error("h2_matvec: ld < n");
    if (x == y) return arg_error("h2_matvec: x and y must not overlap");
    if (prec != H2_PREC_FP32 && prec != H2_PREC_FP64ACC && prec != H2_PREC_SPLITBF16 && prec != H2_PREC_DFACC)
        return arg_error("h2_matvec: bad precision");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (prec == H2_PREC_SPLITBF16) {
        const int64_t ldd = nrhs > 1 ? ld : h->n;
        if (h->use_graphs)
            return run_split_graph(h, reinterpret_cast<const float2 *>(x), reinterpret_cast<float2 *>(y), ldd, nrhs, st);
        return h2_run_multi_split(h, reinterpret_cast<const float2 *>(x), ldd, reinterpret_cast<float2 *>(y), ldd,
                                  nrhs, st);
    }
    if (nrhs > 1 && prec == H2_PREC_FP32)
        return h2_run_multi_f32(h, reinterpret_cast<const float2 *>(x), ld, reinterpret_cast<float2 *>(y), ld, nrhs, st);
    if (nrhs == 1 && prec == H2_PREC_FP32 && h->sym_couple && !h->sym) {
        const h2_status s = h2::h2_sym_init(h);   // before any graph capture
        if (s != H2_OK) return s;
    }
    if (nrhs == 1 && prec == H2_PREC_FP32 && h->use_graphs)
        return run_single_graph(h, reinterpret_cast<const float2 *>(x), reinterpret_cast<float2 *>(y), st);
    for (int32_t r = 0; r < nrhs; ++r) {
        h2_status s;
        if (prec == H2_PREC_FP32)
            s = run_single<float2>(h, reinterpret_cast<const float2 *>(x) + (int64_t)r * ld,
                                   reinterpret_cast<float2 *>(y) + (int64_t)r * ld, st);
        else
            s = run_single<double2>(h, reinterpret_cast<const double2 *>(x) + (int64_t)r * ld,
                                    reinterpret_cast<double2 *>(y) + (int64_t)r * ld, st, prec == H2_PREC_DFACC);
        if (s != H2_OK) return s;
    }
    return H2_OK;
}

h2_status h2_matvec_host(h2_handle *h, const void *x_host, void *y_host, int32_t nrhs, int64_t ld,
                         h2_prec prec)
{
    if (!h || !x_host || !y_host) return arg_error("h2_matvec_host: NULL argument");
    if (nrhs < 1) return arg_error("h2_matvec_host: nrhs must be >= 1");
    if (nrhs == 1) ld = h->n;
    if (ld < h->n) return arg_error("h2_matvec_host: ld < n");
    const size_t esz = (prec == H2_PREC_FP64ACC || prec == H2_PREC_DFACC) ? sizeof(double2) : sizeof(float2);
    const int64_t bytes = (int64_t)esz * ld * nrhs;
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    if (bytes > h->buf_bytes) {
        cudaFree(h->d_xbuf);
        cudaFree(h->d_ybuf);
        h->d_xbuf = h->d_ybuf = nullptr;
        h->buf_bytes = 0;
        if (cudaMalloc(&h->d_xbuf, bytes) != cudaSuccess || cudaMalloc(&h->d_ybuf, bytes) != cudaSuccess) {
            cudaGetLastError();  // clear the out-of-memory result
            set_error("h2_matvec_host: staging allocation failed");
            return H2_ERR_ALLOC;
        }
        h->buf_bytes = bytes;
    }
    cudaStream_t st = nullptr;  // legacy default stream
    H2_CUDA(cudaMemcpyAsync(h->d_xbuf, x_host, bytes, cudaMemcpyHostToDevice, st));
    h2_status s = h2_matvec(h, h->d_xbuf, h->d_ybuf, nrhs, ld, prec, st);
    if (s != H2_OK) return s;
    H2_CUDA(cudaMemcpyAsync(y_host, h->d_ybuf, bytes, cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaStreamSynchronize(st));
    return H2_OK;
}

h2_status h2_profile_matvec(h2_handle *h, const void *x, void *y, int32_t iters, double *ms, int32_t n_ms)
{
    if (!h || !x || !y || !ms || iters < 1 || n_ms < 1) return arg_error("h2_profile_matvec: bad argument");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    if (h->sym_couple && !h->sym) {
        const h2_status s = h2::h2_sym_init(h);
        if (s != H2_OK) return s;
    }
    cudaStream_t st = h->s_aux;
    const float2 *xx = reinterpret_cast<const float2 *>(x);
    float2 *yy = reinterpret_cast<float2 *>(y);
    float2 *coef = reinterpret_cast<float2 *>(h->d_coef);
    // the events are released on every return path
    struct Events {
        cudaEvent_t e[7] = {};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs;
    cudaEvent_t *ev = evs.e;
    for (int k = 0; k < 7; ++k) H2_CUDA(cudaEventCreate(&ev[k]));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int it = 0; it <= iters; ++it) {
        H2_CUDA(cudaMemsetAsync(coef, 0, sizeof(float2) * 2 * std::max<int64_t>(1, h->ktot), st));
        H2_CUDA(cudaEventRecord(ev[0], st));
        if (h->symnear) H2_CUDA(h2::symnear_run(h, xx, yy, st));
        else H2_CUDA(launch_phase_f32(h->near, h->d_mat, h->d_segs, xx, coef, yy, 0, st));
        H2_CUDA(cudaEventRecord(ev[1], st));
        H2_CUDA(launch_phase_f32(h->upleaf, h->d_mat, h->d_segs, xx, coef, coef, 0, st));
        H2_CUDA(cudaEventRecord(ev[2], st));
        for (int l = h->nlev - 1; l >= 0; --l)
            H2_CUDA(launch_phase_f32(h->up[l], h->d_mat, h->d_segs, xx, coef, coef, 0, st));
        H2_CUDA(cudaEventRecord(ev[3], st));
        if (h->sym) H2_CUDA(h2::h2_sym_couple(h, coef, st));
        else H2_CUDA(launch_phase_f32(h->couple, h->d_mat, h->d_segs, xx, coef, coef, 0, st));
        H2_CUDA(cudaEventRecord(ev[4], st));
        for (int l = 0; l < h->nlev; ++l)
            H2_CUDA(launch_phase_f32(h->down[l], h->d_mat, h->d_segs, xx, coef, coef, 1, st));
        H2_CUDA(cudaEventRecord(ev[5], st));
        H2_CUDA(launch_phase_f32(h->leafexp, h->d_mat, h->d_segs, xx, coef, yy, 1, st));
        H2_CUDA(cudaEventRecord(ev[6], st));
        H2_CUDA(cudaEventSynchronize(ev[6]));
        if (it == 0) continue;  // warm-up
        for (int k = 0; k < 6; ++k) {
            float f = 0;
            H2_CUDA(cudaEventElapsedTime(&f, ev[k], ev[k + 1]));
            acc[k] += f;
        }
    }
    // whole product on the concurrent path
    H2_CUDA(cudaEventRecord(ev[0], st));
    for (int it = 0; it < iters; ++it) {
        h2_status s = run_single<float2>(h, xx, yy, st);
        if (s != H2_OK) return s;
    }
    H2_CUDA(cudaEventRecord(ev[1], st));
    H2_CUDA(cudaEventSynchronize(ev[1]));
    float f = 0;
    H2_CUDA(cudaEventElapsedTime(&f, ev[0], ev[1]));
    acc[6] = f;
    for (int k = 0; k < n_ms && k < 7; ++k) ms[k] = acc[k] / iters;
    return H2_OK;
}

}  // extern "C"

// ---- autotuner -----------------------------------------------------------------------
// For every phase, time the block-row GEMV launch with each admissible CTA
// size (CUDA events, median of 3 after a warm-up) and keep the fastest. The
// report is a JSON object {phase: {"threads": T, "us": t, "tried": {T: t}}}.
extern "C" h2_status h2_autotune(h2_handle *h, char *report, int32_t report_len)
{
    if (!h) return arg_error("h2_autotune: NULL handle");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    cudaStream_t st = h->s_aux;
    float2 *xb = nullptr, *yb = nullptr;
    if (cudaMalloc(&xb, sizeof(float2) * h->n) != cudaSuccess || cudaMalloc(&yb, sizeof(float2) * h->n) != cudaSuccess) {
        cudaGetLastError();  // clear the out-of-memory result
        cudaFree(xb);
        set_error("h2_autotune: allocation failed");
        return H2_ERR_ALLOC;
    }
    H2_CUDA(cudaMemsetAsync(xb, 0, sizeof(float2) * h->n, st));
    float2 *coef = reinterpret_cast<float2 *>(h->d_coef);
    H2_CUDA(cudaMemsetAsync(coef, 0, sizeof(float2) * 2 * std::max<int64_t>(1, h->ktot), st));
    cudaEvent_t e0, e1;
    H2_CUDA(cudaEventCreate(&e0));
    H2_CUDA(cudaEventCreate(&e1));
    std::string js = "{";
    bool first = true;
    auto tune = [&](Phase &ph, const std::string &name, bool to_y) -> h2_status {
        if (ph.ntask() == 0) return H2_OK;
        int maxP = 1;
        for (const Task &t : ph.tasks) maxP = std::max(maxP, t.mpad / 2);
        static const int cand[] = {128, 192, 256, 384, 512, 768, 1024};
        int best = ph.threads;
        float best_us = 1e30f;
        std::string tried;
        for (int T : cand) {
            if (T < maxP) continue;
            ph.threads = T;
            float ts[3];
            for (int rep = 0; rep < 4; ++rep) {
                H2_CUDA(cudaEventRecord(e0, st));
                H2_CUDA(launch_phase_f32(ph, h->d_mat, h->d_segs, xb, coef, to_y ? yb : coef, 0, st));
                H2_CUDA(cudaEventRecord(e1, st));
                H2_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0) ts[rep - 1] = ms;
            }
            std::sort(ts, ts + 3);
            const float us = ts[1] * 1e3f;
            tried += (tried.empty() ? "" : ", ") + std::string("\"") + std::to_string(T) + "\": " + std::to_string(us);
            if (us < best_us) {
                best_us = us;
                best = T;
            }
        }
        ph.threads = best;
        js += (first ? "" : ", ") + std::string("\"") + name + "\": {\"threads\": " + std::to_string(best) +
              ", \"us\": " + std::to_string(best_us) + ", \"tried\": {" + tried + "}}";
        first = false;
        return H2_OK;
    };
    h2_status s = H2_OK;
    if ((s = tune(h->near, "near", true)) == H2_OK && (s = tune(h->couple, "couple", false)) == H2_OK &&
        (s = tune(h->upleaf, "upleaf", false)) == H2_OK && (s = tune(h->leafexp, "leafexp", true)) == H2_OK) {
        for (int l = 0; l < h->nlev && s == H2_OK; ++l) s = tune(h->up[l], "up" + std::to_string(l), false);
        for (int l = 0; l < h->nlev && s == H2_OK; ++l) s = tune(h->down[l], "down" + std::to_string(l), false);
    }
    // symmetric storage: consumer warps of the dual kernel (4: three CTAs per SM, 8: two)
    auto tune_sym = [&](bool near) -> h2_status {
        const std::string name = near ? "sym_near" : "sym_couple";
        int best = h->sym_warps[near ? 1 : 0];
        float best_us = 1e30f;
        std::string tried;
        for (int w : {4, 8}) {
            h2::sym_set_warps(h, near, w);
            float ts[3];
            for (int rep = 0; rep < 4; ++rep) {
                H2_CUDA(cudaEventRecord(e0, st));
                H2_CUDA(near ? h2::symnear_run(h, xb, yb, st) : h2::h2_sym_couple(h, coef, st));
                H2_CUDA(cudaEventRecord(e1, st));
                H2_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0) ts[rep - 1] = ms;
            }
            std::sort(ts, ts + 3);
            const float us = ts[1] * 1e3f;
            const int threads = 32 * (w + 1);
            tried += (tried.empty() ? "" : ", ") + std::string("\"") + std::to_string(threads) + "\": " +
                     std::to_string(us);
            if (us < best_us) {
                best_us = us;
                best = w;
            }
        }
        h2::sym_set_warps(h, near, best);
        js += (first ? "" : ", ") + std::string("\"") + name + "\": {\"threads\": " + std::to_string(32 * (best + 1)) +
              ", \"us\": " + std::to_string(best_us) + ", \"tried\": {" + tried + "}}";
        first = false;
        return H2_OK;
    };
    if (s == H2_OK && h->sym_couple) {
        if (!h->sym) s = h2::h2_sym_init(h);
        if (s == H2_OK) s = tune_sym(false);
    }
    if (s == H2_OK && h->symnear) s = tune_sym(true);
    js += "}";
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xb);
    cudaFree(yb);
    drop_graphs(h);  // launch shapes changed: re-capture
    if (report && report_len > 0) {
        strncpy(report, js.c_str(), (size_t)report_len - 1);
        report[report_len - 1] = 0;
    }
    return s;
}

extern "C" h2_status h2_autotune_tc(h2_handle *h, int32_t nrhs, char *report, int32_t report_len)
{
    if (!h) return arg_error("h2_autotune_tc: NULL handle");
    if (nrhs < 1) return arg_error("h2_autotune_tc: nrhs must be >= 1");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    std::string js = "{";
    bool first = true;
    const h2_status s = h2_split_autotune(h, nrhs, js, first);
    js += "}";
    if (report && report_len > 0) {
        strncpy(report, js.c_str(), (size_t)report_len - 1);
        report[report_len - 1] = 0;
    }
    return s;
}

// Entries of a tuning report: "<phase>": {"threads": N ...} (CTA size of an FP32
// phase) or "<phase>": {"ns": N ...} (pipeline depth of a tensor-core phase).
extern "C" h2_status h2_apply_tuning(h2_handle *h, const char *report)
{
    if (!h || !report) return arg_error("h2_apply_tuning: NULL argument");
    std::unordered_map<std::string, Phase *> fp;
    fp["near"] = &h->near;
    fp["couple"] = &h->couple;
    fp["upleaf"] = &h->upleaf;
    fp["leafexp"] = &h->leafexp;
    for (int l = 0; l < h->nlev; ++l) {
        fp["up" + std::to_string(l)] = &h->up[l];
        fp["down" + std::to_string(l)] = &h->down[l];
    }
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    const std::string r(report);
    bool tc_seen = false;
    for (const char *field : {"{\"threads\": ", "{\"ns\": "}) {
        size_t pos = 0;
        while ((pos = r.find(field, pos)) != std::string::npos) {
            const int val = atoi(r.c_str() + pos + strlen(field));
            // the key: the quoted name before the ": " that precedes this object
            const size_t q1 = r.rfind('"', pos >= 3 ? pos - 3 : 0);
            const size_t q0 = q1 == std::string::npos || q1 == 0 ? std::string::npos : r.rfind('"', q1 - 1);
            pos += strlen(field);
            if (q0 == std::string::npos) return arg_error("h2_apply_tuning: malformed report");
            const std::string key = r.substr(q0 + 1, q1 - q0 - 1);
            if (field[2] == 't' && (key == "sym_couple" || key == "sym_near")) {
                // symmetric storage: 32 (consumer warps + 1) threads
                if (val % 32 || !h2::sym_set_warps(h, key == "sym_near", val / 32 - 1))
                    return arg_error("h2_apply_tuning: bad CTA size for " + key);
            } else if (field[2] == 't') {
                auto it = fp.find(key);
                if (it == fp.end()) return arg_error("h2_apply_tuning: unknown phase " + key);
                int maxP = 1;
                for (const Task &t : it->second->tasks) maxP = std::max(maxP, t.mpad / 2);
                if (val < maxP || val > 1024 || val % 32) return arg_error("h2_apply_tuning: bad CTA size for " + key);
                it->second->threads = val;
            } else {
                if (!tc_seen) {
                    // the tensor-core state is built before the first depth is set
                    const h2_status s = h2_split_prepare(h, 1, nullptr);
                    if (s != H2_OK) return s;
                    tc_seen = true;
                }
                if (val < 0 || val > 8) return arg_error("h2_apply_tuning: bad pipeline depth for " + key);
                if (!h2_split_set_ns(h, key, val)) return arg_error("h2_apply_tuning: unknown phase " + key);
            }
        }
    }
    drop_graphs(h);
    return H2_OK;
}

extern "C" h2_status h2_configure(h2_handle *h, const char *opts)
{
    if (!h || !opts) return arg_error("h2_configure: NULL argument");
    DeviceGuard dev_guard(h->device);
    H2_CUDA(dev_guard.err);
    const char *g = strstr(opts, "graphs=");
    const char *tp = strstr(opts, "tc_pipeline=");
    if (!g && !tp) return arg_error("h2_configure: no known option");
    if (g) {
        h->use_graphs = atoi(g + 7) != 0;
        drop_graphs(h);
    }
    if (tp) {
        h->tc_pipeline = atoi(tp + 12) != 0;
        if (h->split) {
            const h2_status s = h2_split_set_pipeline(h, h->tc_pipeline ? 1 : 0);
            if (s != H2_OK) return s;
        }
        h2_drop_split_graphs(h);
    }
    return H2_OK;
}
