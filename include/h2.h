/*
 * libh2 -- minimal-rank H^2 matrix-vector product and Krylov solve on one GPU.
 *
 * The operator is the H^2 representation of a dense complex matrix A
 * (Omar & Jiao, Sec. III.C, Eqs. 8-9, and Sec. IV.A):
 *
 *   A = sum over near (inadmissible leaf) blocks        Z^{t,s}
 *     + sum over admissible blocks (t,s)   U^t S^{t,s} W^{sT}
 *
 * with nested cluster bases U^t = [U^{t1} T^{t1}; U^{t2} T^{t2}] and
 * W^t = [W^{t1} T^{t1}; W^{t2} T^{t2}] for a non-leaf t with children t1, t2
 * (Eq. 9). W = U gives the paper's symmetric form V^t S V^{sT} (Eq. 8).
 *
 * Conventions of every entry point:
 *   - complex numbers are interleaved (re, im): "c64" = two floats,
 *     "c128" = two doubles;
 *   - all matrices are column-major; all vectors are in tree order, i.e.
 *     every cluster is a contiguous index range [begin, begin + size);
 *   - host arrays passed to h2_load are owned by the caller and copied; every
 *     device buffer behind a handle is owned by the library;
 *   - vectors passed to h2_matvec / h2_gmres are caller-owned DEVICE
 *     pointers, except in the *_host variants, which take host pointers;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); all work is ordered on that stream;
 *   - no call exits, traps or prints; failures are returned as h2_status and
 *     the handle stays usable unless the status is H2_ERR_CUDA.
 */
#ifndef LIBH2_H2_H
#define LIBH2_H2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    H2_OK = 0,
    H2_ERR_ARG = 1,            /* invalid argument, shape or inconsistent tree/partition */
    H2_ERR_ALLOC = 2,          /* device or host allocation failed */
    H2_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    H2_ERR_NOT_CONVERGED = 4,  /* Krylov solve hit maxit before tol */
    H2_ERR_BREAKDOWN = 5,      /* Krylov breakdown or non-finite values */
    H2_ERR_TIMEOUT = 6,        /* a bounded device wait ran out */
    H2_ERR_STATE = 7           /* call not valid in the handle's state */
} h2_status;

typedef enum { H2_C64 = 0, H2_C128 = 1 } h2_dtype;

typedef enum {
    H2_PREC_FP32 = 0,      /* c64 vectors, FP32 products and accumulation */
    H2_PREC_SPLITBF16 = 1, /* c64 vectors; multi-RHS products on tensor cores
                              with operands split into two bf16 terms */
    H2_PREC_FP64ACC = 2,   /* c128 vectors, stored FP32 data, FP64 accumulation */
    H2_PREC_DFACC = 3      /* c128 vectors, stored FP32 data, double-float
                              accumulation on the FP32 pipes (each product
                              split exactly, compensated sums, FP64 reductions
                              of the per-thread sums); about ten times the
                              FP64ACC throughput on GB300 */
} h2_prec;

typedef struct h2_handle h2_handle;

/*
 * Binary cluster tree (Sec. III.A), clusters numbered in breadth-first
 * (level) order: cluster 0 is the root and covers [0, n); the clusters of
 * level l are [level_ptr[l], level_ptr[l+1]).
 */
typedef struct {
    int32_t n;                /* number of unknowns N > 0 */
    int32_t n_clusters;       /* number of clusters */
    int32_t n_levels;         /* number of levels */
    const int32_t *level_ptr; /* [n_levels + 1] */
    const int32_t *child;     /* [2 * n_clusters]: children of t at 2t, 2t+1; -1, -1 for a leaf */
    const int32_t *begin;     /* [n_clusters]: first unknown of each cluster */
    const int32_t *size;      /* [n_clusters]: number of unknowns, > 0 */
    const int32_t *rank;      /* [n_clusters]: rank k_t >= 0 of the cluster basis */
} h2_tree;

/*
 * Blocks of the H^2 representation. Every *_off array holds ELEMENT offsets
 * (complex elements, not bytes) into the matching data array, whose total
 * length in elements is *_len; entries for clusters that have no such block
 * are ignored. Elements are c64 or c128 according to `dtype`.
 */
typedef struct {
    h2_dtype dtype;
    /* leaf row bases U^t (n_t x k_t), Eqs. 11-12; indexed by cluster */
    const void *U; const int64_t *U_off; int64_t U_len;
    /* leaf column bases W^t (n_t x k_t); W == NULL means W = U */
    const void *W; const int64_t *W_off; int64_t W_len;
    /* transfer T^t (k_t x k_parent) of every non-root cluster t, Eq. 16 */
    const void *T; const int64_t *T_off; int64_t T_len;
    /* admissible blocks, row-cluster CSR: the partners of t are
       adm_col[adm_ptr[t] .. adm_ptr[t+1]); coupling S^{t,s} (k_t x k_s)
       at S_off[j] for the j-th entry, Eq. 18 */
    const int32_t *adm_ptr; const int32_t *adm_col;
    const void *S; const int64_t *S_off; int64_t S_len;
    /* near-field (inadmissible) blocks between leaves, same CSR form;
       Z^{t,s} (n_t x n_s) at Z_off[j] */
    const int32_t *near_ptr; const int32_t *near_col;
    const void *Z; const int64_t *Z_off; int64_t Z_len;
} h2_data;

/*
 * Validate a tree and its block partition, re-pack the blocks into the
 * device layout (FP32 complex) and upload them. Checks: tree shape and
 * index ranges, rank bounds (leaf k_t <= n_t, non-leaf k_t <= k_t1 + k_t2),
 * offsets within *_len, near blocks only between leaves, and that the
 * admissible and near blocks tile the N x N index square exactly once.
 * The upload is synchronous. On success *out receives a new handle; on
 * failure *out is set to NULL and nothing is leaked.
 * `opts` may be NULL or a string of "key=value" pairs separated by ';':
 * "device=<int>" (default 0), "graphs=0|1" (default 1: the single-RHS FP32
 * product is captured into a CUDA graph per (x, y) pair, and the split-bf16
 * product per (x, y, leading dimension, nrhs), on first use and replayed
 * afterwards; at most 8 graphs of each kind are kept, least recently used
 * first out), "tc_pipeline=0|1" (default 1: the split-bf16 tensor-core kernel runs
 * the deepest pipeline that fits in shared memory, up to 6 stages; 0: two),
 * "wait_limit=N" (polls of every bounded wait inside the tensor-core kernels
 * and the bulk-copy pipeline of the symmetric-storage kernel, default 2^24;
 * when one runs out the kernel waits for its copies and MMAs in flight, skips
 * its output, frees its tensor memory and flags the handle, so
 * that h2_device_status returns H2_ERR_TIMEOUT; 0 makes every first wait run
 * out, which tests that path), "sym_couple=0|1" (default 0; 1: the single-RHS
 * FP32 product keeps each coupling once per admissible pair, S^{t,s} with
 * s > t in cluster order, and reads it once for both S^{t,s} xh^s and
 * (S^{t,s})^T xh^t, since S^{s,t} = (S^{t,s})^T for the one-basis form of
 * the complex-symmetric kernel (Eq. 8); the transposed contributions go
 * through a scratch vector summed in a fixed order, so the product stays
 * deterministic. Built on the first such product, on the device, from the
 * loaded couplings: H2_ERR_STATE when some |S^{s,t} - (S^{t,s})^T| exceeds
 * 1e-5 of max |S^{t,s}| or a rank exceeds 128. Every other product path keeps
 * the full storage).
 */
h2_status h2_load(const h2_tree *tree, const h2_data *data, const char *opts,
                  h2_handle **out);

/*
 * As h2_load, with the block arrays of `data` (U, W, T, S, Z) in DEVICE
 * memory of the target device and of type H2_C64; the tree, the offset and
 * CSR arrays stay host arrays. Validation is the same; the blocks are packed
 * on the device (the non-finite check runs there too), so the H^2 data of a
 * large operator -- built on the GPU by the constructor -- never crosses to the
 * host. The caller keeps ownership of the block arrays and may free them when
 * the call returns. Synchronous.
 */
h2_status h2_load_device(const h2_tree *tree, const h2_data *data, const char *opts,
                         h2_handle **out);

/*
 * Write a loaded operator to a file and read it back without re-validating or
 * re-packing the blocks: the tree, the packed task and segment tables and the
 * FP32 device matrices, followed by an FNV-1a hash of the contents (file
 * layout in h2_api.cu). Construction of the H^2 data is the expensive step
 * for large N; a saved operator reloads at file-read speed. h2_load_file
 * takes the same `opts` as h2_load, checks the header, the hash and that
 * every task and segment stays inside the matrices and vectors, and returns
 * H2_ERR_ARG for a missing, truncated, corrupted or foreign file, before any
 * device work. Autotuned CTA sizes are not saved (call h2_autotune again).
 */
h2_status h2_save(const h2_handle *h, const char *path);
h2_status h2_load_file(const char *path, const char *opts, h2_handle **out);

/* Release every device and host resource of the handle (NULL is ignored).
   Synchronises the handle's internal streams first. */
void h2_free(h2_handle *h);

/*
 * y = A x for nrhs right-hand sides (Sec. IV.B): forward transformation,
 * coupling multiplication, backward transformation, plus the full products
 * with the inadmissible blocks. x and y are device arrays of nrhs columns of
 * length N with leading dimension ld >= N (elements); y is overwritten and
 * must not overlap x. Element type: c64 for H2_PREC_FP32 / H2_PREC_SPLITBF16,
 * c128 for H2_PREC_FP64ACC / H2_PREC_DFACC. nrhs >= 1.
 * Paths: nrhs = 1 FP32 runs level-batched GEMVs; nrhs > 1 FP32 runs complex
 * GEMMs on CUDA cores; H2_PREC_SPLITBF16 runs every pass -- leaf forward
 * transforms, upward transfers, couplings merged with the downward transfers,
 * and the near field merged with the leaf expansion -- on the tensor cores
 * (tcgen05, operands split into two bf16 terms, FP32 accumulation in tensor
 * memory; relative error ~1e-5). The first split-bf16 call packs the
 * tensor-core operand images of every stored matrix. FP64ACC and DFACC with
 * nrhs > 1 run one right-hand side after another.
 * Asynchronous on `stream`. Not thread-safe on one handle.
 */
h2_status h2_matvec(h2_handle *h, const void *x, void *y, int32_t nrhs,
                    int64_t ld, h2_prec prec, void *stream);

/* As h2_matvec, but x and y are HOST arrays: the call copies x to the device,
   runs the product and copies y back, and returns when y is complete. */
h2_status h2_matvec_host(h2_handle *h, const void *x_host, void *y_host,
                         int32_t nrhs, int64_t ld, h2_prec prec);

/* Synchronise the handle's device and report H2_ERR_TIMEOUT if a bounded wait
   inside a tensor-core kernel or the symmetric-storage kernel ran out since
   the handle was loaded (the kernel then skipped its output), else H2_OK. */
h2_status h2_device_status(h2_handle *h);

/*
 * Autotune the launch shape of every stage of the FP32 product: for each
 * block-row phase, time each admissible CTA size (128 ... 1024 threads) with
 * CUDA events and keep the fastest. With symmetric storage (sym_couple=1, and
 * the near field after h2_sym_near) it also times the two launch shapes of
 * the dual kernel (160 threads: 4 consumer warps, three CTAs per SM; 288: 8
 * consumer warps, two CTAs per SM), entries "sym_couple" and "sym_near";
 * building the symmetric couplings first if needed. Writes a JSON report
 * (phase -> chosen threads, time in microseconds, all candidates) into
 * report[0..report_len) when report is not NULL. Synchronous; drops cached
 * graphs.
 */
h2_status h2_autotune(h2_handle *h, char *report, int32_t report_len);

/*
 * Autotune the split-bf16 tensor-core product for nrhs right-hand sides: for
 * every phase (leaf forward transforms, upward transfers per level, merged
 * coupling / downward tiles per level, merged near-field / leaf-expansion
 * tiles) time each pipeline depth that fits in shared memory (2 ... 8
 * stages) with CUDA events and keep the fastest. Writes a JSON report
 * ("tc_<phase>": {"ns": depth, "us": time, "tiles": count, "tried": {...}})
 * into report[0..report_len) when report is not NULL. Allocates the
 * tensor-core state and planes for nrhs if needed; synchronous; drops
 * captured graphs. The paper has no counterpart (launch-shape tuning).
 */
h2_status h2_autotune_tc(h2_handle *h, int32_t nrhs, char *report, int32_t report_len);

/*
 * Apply a report of h2_autotune or h2_autotune_tc (for instance one cached
 * from an earlier run on the same GPU and operator shape) without timing
 * anything: "<phase>": {"threads": N} sets a CTA size (a multiple of 32 in
 * [rows / 2, 1024]; 160 or 288 for "sym_couple" and "sym_near"),
 * "<phase>": {"ns": N} a tensor-core pipeline depth (0 ... 8; 0 = deepest
 * that fits). H2_ERR_ARG for an unknown phase or a bad value. Drops captured
 * graphs.
 */
h2_status h2_apply_tuning(h2_handle *h, const char *report);

/*
 * Change options of a loaded handle: "graphs=0|1" (capture the single-RHS
 * FP32 product and the split-bf16 product into CUDA graphs keyed by their
 * arguments and replay them; both are rebuilt on next use) and
 * "tc_pipeline=0|1" (as in h2_load). H2_ERR_ARG when no known option is
 * given.
 */
h2_status h2_configure(h2_handle *h, const char *opts);

/* Sizes of the loaded representation (all counts in complex elements). */
typedef struct {
    int64_t n, n_clusters, n_leaves, n_levels;
    int64_t near_blocks, adm_blocks;
    int64_t near_elems;      /* sum of n_t n_s over near blocks */
    int64_t coupling_elems;  /* sum of k_t k_s over admissible blocks */
    int64_t transfer_elems;  /* sum of k_t k_parent over non-root clusters */
    int64_t leaf_elems;      /* sum of n_t k_t over leaves */
    int64_t device_bytes;    /* device memory held by the handle */
    int32_t max_rank;
    int32_t kernels_per_matvec; /* libh2 kernel launches of one single-RHS FP32 product */
} h2_stats;

h2_status h2_get_stats(const h2_handle *h, h2_stats *out);

/*
 * Symmetric coupling storage of a handle loaded with "sym_couple=1" (built
 * here if no product has built it yet): complex entries of the stored blocks
 * (about half of coupling_elems), scratch entries (one per stored column) and
 * the largest relative difference max |S^{s,t} - (S^{t,s})^T| / max |S^{t,s}|
 * over the pairs. H2_ERR_STATE for a handle without the option or with
 * non-symmetric couplings.
 */
h2_status h2_sym_stats(h2_handle *h, int64_t *stored_elems, int64_t *scratch_entries, double *max_asym);

/*
 * Near field stored once per pair of leaves for the single-RHS FP32 product.
 * The near blocks are Z^{t,s} = delta_ts I - K^{t,s} diag(chi_s) with K
 * complex symmetric (Sec. II; chi = eps_r - 1 per unknown), so
 *   Z^{s,t} = diag(1/chi_s) (Z^{t,s})^T diag(chi_t)   for t != s,
 * and one stored block serves both directions: Z^{t,s} x_s directly and
 * Z^{s,t} x_t = (1/chi_s) o (Z^{t,s})^T (chi_t o x_t), read once. chi: host
 * array of n complex values (c64 or c128 by dtype) in tree order, copied.
 * The structure is built here on the device from the loaded near blocks and
 * every pair is checked against that relation (H2_ERR_STATE beyond 1e-5
 * relative). H2_ERR_STATE as well when some chi is zero (a void voxel: its
 * near-field columns are zero and do not determine their transposes) or a
 * leaf has more than 128 unknowns. chi NULL returns to the full storage.
 * Captured product graphs are dropped; other product paths are unaffected.
 */
h2_status h2_sym_near(h2_handle *h, const void *chi, h2_dtype dtype);
/* Stored near-field entries (the diagonal blocks and one block per leaf
   pair), scratch entries and the largest relative difference from the
   relation above; H2_ERR_STATE when h2_sym_near has not been called. */
h2_status h2_sym_near_stats(h2_handle *h, int64_t *stored_elems, int64_t *scratch_entries, double *max_asym);

/*
 * Time the stages of a single-RHS FP32 product with CUDA events recorded on
 * the stream each stage is launched on. x, y: device c64 vectors. Runs `iters`
 * products (after one warm-up) and writes the mean duration in milliseconds
 * of each stage to ms[0..n_ms) in the order: near field, leaf forward,
 * upward transfers, couplings (all levels), downward transfers, leaf
 * expansion, whole product (stages on the concurrent path). Synchronous.
 */
h2_status h2_profile_matvec(h2_handle *h, const void *x, void *y, int32_t iters,
                            double *ms, int32_t n_ms);

/*
 * y = A x for one right-hand side in FP32 (c64 device vectors), like
 * h2_matvec with nrhs = 1 and H2_PREC_FP32, but without any memory the
 * handle allocated for scratch: the forward and backward coefficient vectors
 * live in one static device array of H2_NOALLOC_MAX_COEF complex64 entries
 * (8 MiB) that every GPU loading the library holds until the process exits.
 * The paper has no counterpart; this entry point exists for callers that must
 * not call the CUDA allocator once running -- a step embedded in another
 * framework whose caching allocator owns the device memory, or a real-time
 * loop that cannot take cudaMalloc's implicit synchronisation. Such a caller
 * loads the operator with h2_load at initialisation and afterwards passes
 * only x and y. This path always uses the full block storage (the symmetric
 * storage of sym_couple and h2_sym_near is not used here).
 * Operators needing more than H2_NOALLOC_MAX_COEF coefficients (2 x the sum
 * of the cluster ranks) are rejected with H2_ERR_ARG before any device work.
 * The first call on a handle looks up the array's device address in the
 * handle's context and keeps it in the handle; make that first call before
 * any stream capture. Every call shares the one array: calls that overlap on
 * the GPU (different streams, or concurrent host threads) race and give
 * wrong results. The array keeps the previous call's values, so every call
 * zeroes it first. Asynchronous on `stream`.
 */
#define H2_NOALLOC_MAX_COEF 1048576
h2_status h2_matvec_noalloc(h2_handle *h, const void *x, void *y, void *stream);

/* Options of h2_gmres. */
typedef struct {
    double tol;        /* stop when ||b - A x||_2 <= tol ||b||_2 (true residual) */
    int32_t restart;   /* Krylov subspace size m per cycle, 1..1024 */
    int32_t maxit;     /* maximum total number of Arnoldi steps */
    int32_t refine;    /* 1: restart residuals use the FP64-accumulated product
                          (iterative refinement of the FP32 inner cycles) */
    int32_t x0_given;  /* 1: x holds the initial guess on entry; 0: start from 0 */
    int32_t precond;   /* 0: none; 1: the handle's learned preconditioner as the
                          right preconditioner of flexible GMRES (Saad 1993):
                          z_j = M(v_j), A z_j enters the Arnoldi process and
                          x += Z y at the end of each cycle. A cycle that
                          reduces the true residual by less than 5% turns the
                          preconditioner off for the rest of the solve (plain
                          GMRES is the fallback). */
    int32_t arnoldi;   /* arithmetic of the Gram-Schmidt passes: 0 = FP64;
                          1 = double-float (each value an unevaluated sum of two
                          floats, 48-bit significand; exact product splitting
                          and compensated sums, Ogita-Rump-Oishi 2005) on the
                          FP32 pipes, with FP64 reductions, norms and least
                          squares. GB300 issues FP64 at about 1/58 of the FP32
                          rate. 2 = c64 basis and work vector (8 bytes per
                          entry, half the traffic of 0 and 1), FP32 products
                          summed with compensation, FP64 reductions, norms and
                          least squares; the stored vectors carry FP32
                          rounding, so tolerances well above 1e-7 only.
                          With precond = 1 the preconditioned directions are
                          kept as c128 in every arithmetic (n x m x 16 bytes
                          per right-hand side); with refine, 1 and 2 use the
                          DFACC residual, 0 FP64ACC. */
    double reorth_eta; /* selective reorthogonalisation threshold eta in [0, 1]:
                          a second Gram-Schmidt projection when the first
                          leaves |w'| < eta |w| (Daniel, Gragg, Kaufman &
                          Stewart 1976); one projection keeps w' orthogonal to
                          the basis to about u / eta. 0 selects 1/sqrt(2);
                          1 projects twice at every step (CGS2). */
} h2_solve_opts;

/* Per right-hand-side outcome of h2_gmres. */
typedef struct {
    int32_t iterations; /* Arnoldi steps taken */
    int32_t restarts;   /* completed cycles */
    double rel_res;     /* final true relative residual ||b - A x|| / ||b|| */
    int32_t status;     /* H2_OK, H2_ERR_NOT_CONVERGED or H2_ERR_BREAKDOWN */
    int32_t precond_cycles; /* cycles run with the preconditioner (flexible GMRES) */
    int32_t reorth_steps;   /* Arnoldi steps that needed the second Gram-Schmidt projection */
} h2_solve_info;

/*
 * Solve A x = b by restarted GMRES(m) (Saad & Schultz) around the H^2
 * product: Arnoldi on the device (arithmetic by opts->arnoldi; classical
 * Gram-Schmidt with selective reorthogonalisation: a second projection when
 * the first one leaves |w'| < eta |w|), FP32 H^2 products inside the cycles;
 * the projection coefficients of each step are copied to the host, where the
 * Hessenberg column, the Givens rotations, the residual estimate and the
 * least-squares back-substitution run in FP64. Each restart recomputes the
 * true residual (FP64-accumulated product when opts->refine). The paper's own
 * solver is BiCGStab (Sec. V); this is the Krylov method around the same
 * product (Sec. IV.B).
 * b, x: device c128 arrays of nrhs columns (leading dimension ld >= N);
 * right-hand sides are solved one after another. info: host array of nrhs
 * entries (may be NULL). Returns H2_OK when every right-hand side converged,
 * else the first failing status. Synchronises `stream` (convergence is read
 * back once per Arnoldi step). Device workspace (an N x (m+1) basis: 16
 * bytes per entry for arnoldi 0 and 1, 8 for arnoldi 2) is allocated on first
 * use and kept by the handle.
 */
h2_status h2_gmres(h2_handle *h, const void *b, void *x, int32_t nrhs, int64_t ld,
                   const h2_solve_opts *opts, h2_solve_info *info, void *stream);

/*
 * Batched restarted GMRES(m): the nrhs right-hand sides advance in lockstep,
 * each with its own Krylov basis, Hessenberg matrix and Givens rotations, so
 * every Arnoldi step runs ONE multi-RHS product (prec = H2_PREC_FP32: CUDA-core
 * complex GEMMs; H2_PREC_SPLITBF16: tensor cores) and the Gram-Schmidt passes
 * (arithmetic by opts->arnoldi, selective reorthogonalisation, as in
 * h2_gmres) are batched over the right-hand sides; the Hessenberg columns,
 * rotations and back-substitution run in FP64 on the host. A right-hand side
 * whose residual estimate drops below tol / 2 stops contributing at the end
 * of the cycle. Restart residuals: accumulated products when opts->refine
 * (one per right-hand side; FP64ACC for arnoldi 0, DFACC for 1 and 2), else
 * one batched product with `prec`. opts->precond = 1: flexible GMRES with the
 * handle's learned preconditioner (H2_ERR_STATE if none is loaded), applied
 * to the basis vectors of all right-hand sides in one batched pass of the
 * network; a right-hand side whose preconditioned cycle reduces its true
 * residual by less than 5 % continues with plain GMRES.
 * b, x: device c128, nrhs columns with leading dimension ld >= N.
 * Workspace: an N x (m+1) x nrhs basis (16 bytes per entry for arnoldi 0
 * and 1, 8 for arnoldi 2) plus O(N nrhs) vectors, allocated on first use and
 * kept by the handle. Synchronises `stream` once per step.
 */
h2_status h2_gmres_batched(h2_handle *h, const void *b, void *x, int32_t nrhs, int64_t ld,
                           const h2_solve_opts *opts, h2_prec prec, h2_solve_info *info, void *stream);

/*
 * Solve A x = b by BiCGStab (van der Vorst 1992), the paper's solver (Sec. V),
 * around the H^2 product: FP32 products inside the iteration, FP64 vectors,
 * inner products and scalars on the device (shadow residual r0, complex inner
 * products u^H v). One iteration is two products. opts: tol, maxit (maximum
 * iterations), refine (a recursive residual below tol is checked against the
 * true residual b - A x with the accumulated product, FP64ACC, or DFACC when
 * arnoldi = 1, and the iteration restarts from x while it is above tol),
 * x0_given; restart and reorth_eta are not used; precond must be 0. A
 * breakdown (rho, (r0, A p) or |A s| zero) restarts from the true residual.
 * b, x: device c128, nrhs columns (ld >= N), solved one after another;
 * info[c].iterations counts iterations, info[c].restarts the restarts.
 * Returns H2_OK when every right-hand side converged, H2_ERR_NOT_CONVERGED,
 * H2_ERR_BREAKDOWN, or an argument / CUDA error.
 */
h2_status h2_bicgstab(h2_handle *h, const void *b, void *x, int32_t nrhs, int64_t ld, const h2_solve_opts *opts,
                      h2_solve_info *info, void *stream);

/*
 * Load (or, with n_layers = 0, remove) the learned preconditioner used by
 * h2_gmres with precond = 1: a chain of 3x3x3 convolutions on the
 * Dx x Dy x Dz voxel grid (include/h2nn.h). Unknown 3 p + c of the operator is
 * field component c of the voxel at tree position p, and grid_of[p] is that
 * voxel's grid index. M(v): v is scaled to unit RMS and packed into 8
 * channels (Re, Im of the 3 components, aux[v] = a per-voxel input such as
 * chi, 0); the layers run in order (ReLU where layer_spec[3l+2] != 0); output
 * channels 0..5 are unpacked with the inverse scale and added to v: the
 * network N models the correction beyond the identity, M(v) = v + N(v).
 * layer_spec: [3 n_layers] (Cin, Cout, relu), channels in {8, 16, 32}, first
 * Cin = 8, last Cout = 8. weights: bf16 (uint16) [Cout][27][Cin] per layer,
 * concatenated; biases: f32 [Cout] per layer, concatenated; aux: f32 [V] or
 * NULL. All arrays are host memory, copied. Synchronous.
 */
h2_status h2_set_preconditioner(h2_handle *h, int32_t Dx, int32_t Dy, int32_t Dz, const int32_t *grid_of,
                                const float *aux, int32_t n_layers, const int32_t *layer_spec,
                                const void *weights, const float *biases);

const char *h2_status_string(h2_status s);

/* Text of the last CUDA or validation error seen by this thread ("" if none). */
const char *h2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBH2_H2_H */
