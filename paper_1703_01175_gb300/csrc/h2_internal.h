// Internal declarations of libh2 (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "h2.h"

namespace h2 {

// One output segment of a block-row product:
//   out[out_off + i] (+)= sum_c M[i, c] * in(c),   i < m, c < ncol
// M is the task's own column-major matrix of mpad x ncol complex entries
// stored at mat[mat_off] (mpad = m rounded up to even, zero padded), and the
// input column c is gathered from the task's segments (in order).
struct Task {
    int32_t out_off;
    int32_t m;
    int32_t mpad;
    int32_t ncol;
    int64_t mat_off;
    int32_t seg_begin;
    int32_t seg_end;
};

// A run of n consecutive input entries: in0[in_off ...] when in_off >= 0,
// else in1[-in_off - 1 ...].
struct Seg {
    int32_t in_off;
    int32_t n;
};

// A batch of independent tasks executed by one launch.
struct Phase {
    const char *name = "";
    std::vector<Task> tasks;       // host copy, sorted by decreasing work
    Task *d_tasks = nullptr;       // device copy (points into the handle's task pool)
    int32_t max_mpad = 0;
    int32_t max_ncol = 0;
    int64_t elems = 0;             // matrix entries streamed (sum of m * ncol)
    int threads = 256;
    int32_t *d_coloff = nullptr;   // multi-RHS path: first entry of each task in d_colidx
    const int32_t *d_colidx = nullptr;  // multi-RHS path: input index of every task column (handle's table)
    int ntask() const { return (int)tasks.size(); }
};

enum PhaseKind { PH_NEAR = 0, PH_UPLEAF, PH_UP, PH_DOWN, PH_LEAFEXP, PH_COUNT };

// One tile of the split-bf16 tensor-core path (h2_umma.cu): up to 128 output
// rows of a task (or of several tasks with the same output merged along K),
// its packed matrix images and its input group table.
struct UTask {
    int32_t out_off;    // first output row: complex offset in y, or position in the bf16 plane
    int32_t m;          // complex rows in this tile (<= 128)
    int32_t n;          // real MMA N = 2 * round_up(m, 8)
    int32_t nst;        // K stages of 16 complex columns
    int64_t img_off;    // byte offset of stage 0's image (per K chunk: N hi rows, then N lo rows)
    int32_t chunk_off;  // first entry in the group table (2 plane positions per stage)
    int32_t pad_;
};

struct UPackInfo {
    int32_t row0, npc;    // first task row of the tile; padded columns of the task
    int64_t colmap_off;   // first entry of the task's column table
};

struct UPhase {
    int ntile = 0;
    UTask *d_tasks = nullptr;
    int32_t *d_chunks = nullptr;  // plane position of every 8-column group of every tile
    uint8_t *d_images = nullptr;
    int64_t image_bytes = 0;
    int nmax = 16;                // largest MMA N of the phase's tiles
    int maxnst = 0;               // most K stages of a tile
    int ns = 0;                   // pipeline stages chosen by the autotuner (0: the deepest that fits)
};

struct SplitState {
    // leaf: near field and leaf expansion of every leaf (output y); upleaf and
    // up[l]: forward transforms and upward transfer (output xh); level[l]:
    // couplings and downward transfer of the clusters of level l (output yh)
    UPhase leaf, upleaf;
    std::vector<UPhase> up, level;
    // one bf16 plane: x at positions [0, np_x), xh at [np_x, np_x + np_c), yh
    // at [np_x + np_c, np_x + 2 np_c); nch groups of 8 positions per tile (a
    // Re chunk and an Im chunk each), the last one zero
    int64_t np_x = 0, np_c = 0, nch = 0;
    int32_t *d_xpos = nullptr;    // x plane position -> index into x (-1: padding)
    void *phi = nullptr, *plo = nullptr;
    bool zero_y = false;          // some leaf has no task: clear y first
    int rcap = 0;
    int *d_err = nullptr;         // set when a bounded wait ran out
    uint32_t wait_limit = 1u << 24;  // polls of a bounded mbarrier wait
    bool pipeline = true;         // deepest pipeline that fits (else two stages)
    size_t dyn_smem_limit = 0;    // dynamic shared memory a block may use
};

void set_error(const std::string &msg);

// Makes a device current for the lifetime of the guard and restores the
// caller's current device when it goes out of scope, so that no entry point
// changes the calling thread's device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            cudaGetLastError();
        }
        err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Couplings stored once per admissible pair (h2_sym.cu): tasks hold the blocks
// S^{t,s} with s > t; scratch holds (S^{t,s})^T xh^t, one entry per stored
// column; gather lists add those into yh^s.
struct SymState {
    int ntask = 0, ntarget = 0;
    Task *d_tasks = nullptr;
    int32_t *d_xsrc = nullptr;     // per stored column: its input (>= 0: x[.], else coefficient [-. - 1])
    float2 *d_mat = nullptr;
    int64_t *d_col0 = nullptr;     // per task: first stored column (scratch entry, d_xsrc entry)
    float2 *d_scratch = nullptr;
    int32_t *d_gptr = nullptr;     // per target cluster: range of gcol [ntarget + 1]
    int64_t *d_gcol = nullptr;     // scratch entry of column 0 of each (t, s), t < s
    int32_t *d_gout = nullptr;     // offset of yh^s in the coefficient buffer
    int32_t *d_gk = nullptr;       // rank of s
    int64_t stored_elems = 0;      // complex entries of the stored blocks
    int64_t scratch_entries = 0;
    float max_asym = 0.f;          // largest relative difference of a stored block from its partner's relation
    float2 *d_chi = nullptr;       // near field: chi per unknown (tree order)
    float2 *d_rs = nullptr;        // near field: 1 / chi
    float2 *d_xs = nullptr;        // near field: chi x of the current product
    int *d_err = nullptr;          // set when a bounded wait of the dual kernel ran out
    uint32_t wait_limit = 1u << 24;
    int warps = 8;                 // consumer warps of the dual kernel (4 or 8)
};

// FP64 Arnoldi state of restarted GMRES for R right-hand sides (h2_arnoldi.cu)
struct ArnDev {
    double2 *V;        // basis [(m+1)][R][n] (float4 hi/lo pairs in double-float mode, float2 in FP32 mode)
    double2 *w;        // [R][n] vector being orthogonalised (likewise)
    double2 *part;     // [R][np] partial sums of the reductions
    unsigned *ticket;  // [R][8] last-block counters
    double2 *h1, *h2;  // [R][m+2] projection coefficients (h1[j+1] = |w|^2); h2 follows h1
    double *scal;      // [R][8]: beta, -, -, reorthogonalised flag
    int *kact;         // [R] basis columns used by the update of x
    double eta2;       // second projection when |w'|^2 < eta2 |w|^2
    int n, m, R, np;
};

// Arnoldi arithmetic: FP64; double-float on the FP32 pipes; c64 basis with FP32 products
enum { ARN_FP64 = 0, ARN_DF = 1, ARN_F32 = 2 };

struct ArnWork {
    ArnDev K{};
    int n = 0, m = 0, R = 0, extra_cols = 0, mode = ARN_FP64;
    int rows = 0, nbu = 0;          // row blocks of the update and residual passes
    double2 *Z = nullptr;           // [extra_cols][R][n] preconditioned directions, c128 in every arithmetic (flexible GMRES)
    double2 *rr = nullptr, *tmp = nullptr;  // [R][n]
    float2 *x32 = nullptr, *y32 = nullptr;  // [R][n] product input / output
    double *h_scal = nullptr;       // pinned copy of scal
    int *h_kact = nullptr;          // pinned kact
    double2 *h_hh = nullptr;        // pinned copy of h1, h2 (and the least-squares solution)
    void *block = nullptr;
    // host FP64 least-squares state per right-hand side
    std::vector<std::complex<double>> H, g, sn;  // [R][m][m+1] rotated Hessenberg, [R][m+1], [R][m]
    std::vector<double> cs;                      // [R][m]
    std::vector<double> est, beta;               // after a step: |g_{j+1}|, |w|
    std::vector<char> bad, reorth;               // after a step: non-finite, second projection taken
};

h2_status arn_get(ArnWork **slot, int n, int m, int R, int extra_cols, int mode);
// reorthogonalisation threshold eta (0: the default 1/sqrt(2)); returns H2_ERR_ARG outside [0, 1]
h2_status arn_set_eta(ArnWork *w, double eta);
void arn_free(ArnWork *w);
// rr = b - y (y NULL: rr = b); scal[8 r] = |rr_r|
h2_status arn_residual(ArnWork *w, const double2 *b, int64_t ldb, const double2 *y, cudaStream_t st);
// v_0 = rr / |rr| (and x32 = c64(v_0) unless FP32 mode), g = |rr| e_1 (|rr| from h_scal: call arn_read first)
h2_status arn_start(ArnWork *w, cudaStream_t st);
// input of the product of step j: v_j in c64, [R][n] (x32, or the basis column itself in FP32 mode)
const float2 *arn_input(const ArnWork *w, int j);
// with y32 = A arn_input(j): orthogonalise, v_{j+1} (and x32 = c64(v_{j+1}) unless FP32 mode); then (host)
// Hessenberg column j, rotations, est / beta / bad / reorth per right-hand side
h2_status arn_step(ArnWork *w, int j, cudaStream_t st);
// copy scal to h_scal and synchronise
h2_status arn_read(ArnWork *w, cudaStream_t st);
// least-squares solve (host) with h_kact columns, x_r += basis_r y_r
h2_status arn_finish(ArnWork *w, const double2 *basis, double2 *x, int64_t ldx, cudaStream_t st);
h2_status arn_c128_to_c64(ArnWork *w, const double2 *a, int64_t lda, float2 *b, cudaStream_t st);
// basis column j of every right-hand side widened to c128, out [R][n]
h2_status arn_basis_c128(ArnWork *w, int j, double2 *out, cudaStream_t st);
h2_status arn_c64_to_c128(ArnWork *w, const float2 *a, double2 *b, cudaStream_t st);

}  // namespace h2

struct h2_handle {
    int device = 0;
    int32_t n = 0, nc = 0, nlev = 0;
    std::vector<int32_t> level_ptr, child, begin, size, rank, parent, level;
    std::vector<int32_t> xo;      // offset of xh^t in the coefficient buffer
    int64_t ktot = 0;             // sum of ranks; yh^t lives at ktot + xo[t]

    // device storage
    float2 *d_mat = nullptr;      // all task matrices
    int64_t mat_elems = 0;
    h2::Seg *d_segs = nullptr;
    h2::Task *d_tasks = nullptr;
    void *d_coef = nullptr;       // 2 * ktot coefficients (sized for c128)
    void *d_xbuf = nullptr;       // staging for the host-pointer entry point
    void *d_ybuf = nullptr;
    int64_t buf_bytes = 0;

    h2::Phase near, upleaf, leafexp, couple;
    std::vector<h2::Phase> up;    // per level (index = level of the output cluster)
    std::vector<h2::Phase> down;  // per level

    cudaStream_t s_aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_near = nullptr;

    h2_stats stats{};

    void *krylov = nullptr;       // GMRES workspace (h2_krylov.cu)
    void *d_coefm = nullptr;      // multi-RHS coefficients (2 ktot x R, h2_mrhs.cu)
    int32_t *d_colidx = nullptr;  // multi-RHS path: input index of every task column, all phases (h2_mrhs.cu)
    int64_t coefm_bytes = 0;
    std::vector<h2::Seg> segs_host;   // host copy of the input segments (split-bf16 packing)
    void *precond = nullptr;          // learned preconditioner (h2_precond.cu)
    void *bkrylov = nullptr;          // batched GMRES workspace (h2_bkrylov.cu)
    void *bicgstab = nullptr;         // BiCGStab workspace (h2_bicgstab.cu)
    // captured single-RHS FP32 products, one per (x, y) pair (h2_api.cu)
    struct GraphEntry {
        const void *x;
        void *y;
        cudaGraphExec_t exec;
        uint64_t last_use;
    };
    std::vector<GraphEntry> graphs;
    // captured split-bf16 products, one per (x, y, leading dimension, nrhs)
    struct SplitGraphEntry {
        const void *x;
        void *y;
        int64_t ld;
        int32_t nrhs;
        cudaGraphExec_t exec;
        uint64_t last_use;
    };
    std::vector<SplitGraphEntry> split_graphs;
    uint64_t graph_clock = 0;
    bool use_graphs = true;
    bool tc_pipeline = true;          // split-bf16: deepest tensor-core pipeline that fits (else two stages)
    uint32_t wait_limit = 1u << 24;   // polls of the tensor-core kernels' bounded waits
    cudaStream_t s_cap = nullptr;
    h2::SplitState *split = nullptr;  // split-bf16 tensor-core state (h2_umma.cu)
    bool sym_couple = false;          // single-RHS FP32 product: couplings stored once per pair
    h2::SymState *sym = nullptr;      // built on first use (h2_sym.cu)
    h2::SymState *symnear = nullptr;  // near field stored once per leaf pair (h2_sym_near)
    int sym_warps[2] = {8, 8};        // consumer warps of the dual kernel: couplings, near field (4 or 8)
    // device address of the static scratch array of h2_matvec_noalloc in the
    // context that owns this handle's memory (looked up by the first such call)
    float2 *noalloc_coef = nullptr;
};

void h2_free_krylov(h2_handle *h);
h2_status h2_ensure_coefm(h2_handle *h, int nrhs);
// column index tables of every phase for the multi-RHS kernels (built once)
h2_status h2_ensure_colidx(h2_handle *h);
void h2_free_split(h2_handle *h);
namespace h2 {
h2_status h2_sym_init(h2_handle *h);
h2_status h2_sym_error_flag(h2_handle *h, int *flag);
void h2_free_sym(h2_handle *h);
cudaError_t h2_sym_couple(h2_handle *h, float2 *coef, cudaStream_t st);
h2_status symnear_init(h2_handle *h, const std::vector<float2> &chi);
void symnear_free(h2_handle *h);
cudaError_t symnear_run(h2_handle *h, const float2 *x, float2 *y, cudaStream_t st);
// consumer warps (4 or 8) of the dual kernel for the couplings (near = false)
// or the near field; false for another count
bool sym_set_warps(h2_handle *h, bool near, int warps);
}  // namespace h2
h2_status h2_run_multi_split(h2_handle *h, const float2 *x, int64_t ldx, float2 *y, int64_t ldy, int nrhs,
                             cudaStream_t st);
h2_status h2_split_error_flag(h2_handle *h, int *flag);
h2_status h2_split_set_pipeline(h2_handle *h, int on);
// allocate the tensor-core state and planes for nrhs right-hand sides (never
// during a stream capture); *realloc = 1 when the planes moved
h2_status h2_split_prepare(h2_handle *h, int nrhs, int *realloc);
// time every pipeline depth of every tensor-core phase for nrhs right-hand
// sides and keep the fastest; appends "tc_<phase>": {...} entries to js
h2_status h2_split_autotune(h2_handle *h, int nrhs, std::string &js, bool &first);
// set the pipeline depth of a tensor-core phase by its report name; false if unknown
bool h2_split_set_ns(h2_handle *h, const std::string &name, int ns);
void h2_drop_split_graphs(h2_handle *h);
void h2_free_precond(h2_handle *h);
void h2_free_bkrylov(h2_handle *h);
void h2_free_bicgstab(h2_handle *h);
// z = M(v) for one c128 vector (v of unit norm or any norm); also writes c64 z32 when not NULL
h2_status h2_apply_precond(h2_handle *h, const double2 *v, double2 *z, float2 *z32, cudaStream_t st);
// z_r = M(v_r) for R c128 vectors (v, z: [R][n] with strides ldv, ldz; z32: [R][n] c64 or NULL): one
// pass of the network over a batch of R grids
h2_status h2_apply_precond_batched(h2_handle *h, const double2 *v, int64_t ldv, int R, double2 *z, int64_t ldz,
                                   float2 *z32, cudaStream_t st);
h2_status h2_run_multi_f32(h2_handle *h, const float2 *x, int64_t ldx, float2 *y, int64_t ldy, int nrhs,
                           cudaStream_t st);

namespace h2 {
// launch one phase; VT = float2 (FP32) or double2 (FP64 accumulation)
cudaError_t launch_phase_f32(const Phase &ph, const float2 *mat, const Seg *segs,
                             const float2 *in0, const float2 *in1, float2 *out,
                             int beta_one, cudaStream_t st);
cudaError_t launch_phase_mrhs_f32(const Phase &ph, const float2 *mat, const float2 *in0, int64_t ld0,
                                  const float2 *in1, int64_t ld1, float2 *out, int64_t ldo, int nrhs, int beta_one,
                                  cudaStream_t st);
cudaError_t launch_phase_f64(const Phase &ph, const float2 *mat, const Seg *segs,
                             const double2 *in0, const double2 *in1, double2 *out,
                             int beta_one, cudaStream_t st);
cudaError_t launch_phase_df(const Phase &ph, const float2 *mat, const Seg *segs,
                             const double2 *in0, const double2 *in1, double2 *out,
                             int beta_one, cudaStream_t st);
}  // namespace h2
