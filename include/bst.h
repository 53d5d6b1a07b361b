/*
 * bst.h -- C ABI of libbst, a GB300 (sm_103a) block-sparse matrix multiply and
 * block-sparse tensor contraction library following DBCSR (arXiv:1910.13555).
 *
 * The operations and where the paper defines them:
 *   - blocked-CSR matrices of small dense blocks with per-row/column block sizes
 *     (paper Sec. 2, first paragraph: "blocked compressed sparse row");
 *   - the local multiply C = C + A x B as pairwise products of (m x k) blocks of A
 *     with (k x n) blocks of B, grouped into batches ("stacks") that a small-GEMM
 *     kernel processes (paper Sec. 2, the local-computation paragraph);
 *   - the S_C << S_A,S_B rectangular product C~ = A^T B with the long K dimension
 *     split into parts whose partial results are reduced into C (paper Sec. 3.1,
 *     Eq. 2); here the parts are CTA groups of one GPU and the reduction is a fixed-
 *     order sum;
 *   - block-sparse tensors of rank 2..4 (up to 8 accepted) and their contraction
 *     over 1..3 index pairs, computed by mapping each tensor onto a matrix whose
 *     rows fold one set of modes and whose columns fold the other (paper Sec. 4).
 *
 * Additions that the paper does not define (each a reading of this library):
 *   - the block-norm filter eps: a product A_ik B_kj is computed iff
 *     ||A_ik||_F * ||B_kj||_F >= eps (alpha does not enter; eps = 0 keeps all);
 *   - pattern(C_out) = pattern(C_in) U {(i,j): some kept product}; no post-filter;
 *   - block elements are row-major (last index fastest);
 *   - stacks: one entry (a_off, b_off, c_off) per kept product, int32 element
 *     offsets of the stored blocks, bucketed by (m, n, k) sizes in lexicographic
 *     order and ordered by (i, j, k) block indices inside a bucket;
 *   - the adjoint of the computed function with the filter decisions held fixed;
 *   - FP64 emulation on BF16 tensor cores (Ozaki-scheme slices) and a 3xTF32 path.
 *
 * Conventions for every entry point:
 *   - Return value: BST_OK (0) or an error code below.  Nothing aborts and no C++
 *     exception crosses this boundary.  bst_last_error() gives a message for the
 *     calling thread's most recent failure.
 *   - Host-detectable errors (bad arguments, duplicates, shape mismatches, offset
 *     overflow) are reported synchronously before any device work is queued.
 *   - Element data (double*) is caller-owned DEVICE memory on the context's GPU.
 *     Index arrays passed in are HOST memory and are copied; the library keeps its
 *     own device copies.  Everything the library allocates goes through the
 *     context's allocator callbacks (or stream-ordered cudaMallocAsync when none
 *     are given) and is released by the matching destroy call.  One exception: the
 *     static split-K array of bst_multiply_execute_static, a __device__ array that
 *     each GPU which loads the library holds until the process exits.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it except where documented (plans synchronise the stream a few
 *     times to learn output and schedule sizes; the first emulated-FP64 or 3xTF32
 *     execute of a plan, the emulated execute that builds its panel schedule (the
 *     second by default, see BST_TUNE_EMU_PANEL) and the first execute after a tuning
 *     change synchronise too, while they build per-plan state; other executes only
 *     queue work).
 *   - Handles are not thread-safe; use one handle per thread or lock around it.
 *   - A matrix or tensor must outlive every plan built from it.
 */
#ifndef BST_H
#define BST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bst_status;

enum {
  BST_OK = 0,
  BST_ERR_INVALID_ARG = 1,      /* null/negative/inconsistent argument          */
  BST_ERR_OUT_OF_RANGE = 2,     /* block index outside the declared grid          */
  BST_ERR_DUPLICATE_BLOCK = 3,  /* the same block listed twice                    */
  BST_ERR_SHAPE_MISMATCH = 4,   /* block sizes of the operands do not line up     */
  BST_ERR_OVERFLOW = 5,         /* > 2^31-1 elements in a matrix, or stack entries */
  BST_ERR_ALLOC = 6,            /* an allocation failed                           */
  BST_ERR_CUDA = 7,             /* a CUDA runtime call failed                     */
  BST_ERR_TIMEOUT = 8,          /* a bounded device wait gave up                  */
  BST_ERR_UNSUPPORTED = 9,      /* valid but outside the library's limits         */
  BST_ERR_STATE = 10            /* wrong call order (e.g. C data not bound)       */
};

/* Message for the calling thread's last failing call (static storage). */
const char *bst_last_error(void);
/* Name of a status code, e.g. "BST_ERR_SHAPE_MISMATCH". */
const char *bst_status_name(bst_status s);
/* Library version string. */
const char *bst_version(void);
/* Number of CUDA kernels this library has launched in this process so far (all
 * contexts, all threads); lets a caller count the kernels of a timed region. */
int64_t bst_kernel_launches(void);

typedef struct bst_ctx bst_ctx;
typedef struct bst_matrix bst_matrix;
typedef struct bst_tensor bst_tensor;
typedef struct bst_plan bst_plan;
typedef struct bst_batch bst_batch;

/* Device allocator callbacks: return a device pointer of at least `bytes` bytes,
 * aligned to 256 bytes as cudaMalloc's are (the library's kernels use 16-byte vector
 * accesses on these buffers), usable on `stream` (NULL on failure); free it.  `user` is
 * passed through. */
typedef void *(*bst_alloc_fn)(size_t bytes, void *user, void *stream);
typedef void (*bst_free_fn)(void *ptr, void *user, void *stream);

/* Create a context on CUDA device `device`.  alloc/free may both be NULL, in which
 * case the library allocates stream-ordered (cudaMallocFromPoolAsync / cudaFreeAsync on
 * the call's stream) from a memory pool of its own that keeps freed memory for reuse
 * until bst_context_destroy (which synchronises the device and destroys the pool). */
bst_status bst_context_create(bst_ctx **out, int32_t device, bst_alloc_fn alloc,
                              bst_free_fn free_fn, void *user);
bst_status bst_context_destroy(bst_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Matrices (paper Sec. 2: blocked CSR of small dense blocks).
 *
 * nbr/nbc block rows/columns with sizes row_blk_sizes[nbr], col_blk_sizes[nbc]
 * (host, each >= 1).  The nblocks present blocks (blk_row[b], blk_col[b]) are host
 * arrays in any order; the library sorts them into canonical CSR order (row, then
 * column).  `data` (device, may be NULL until bound) holds the blocks packed in
 * that canonical order, each block row-major; its length is the sum of the block
 * areas (bst_matrix_info).  Errors: INVALID_ARG, OUT_OF_RANGE, DUPLICATE_BLOCK,
 * OVERFLOW (more than 2^31-1 elements or blocks).
 * ------------------------------------------------------------------------- */
bst_status bst_matrix_create(bst_ctx *ctx, bst_matrix **out, int32_t nbr,
                             const int32_t *row_blk_sizes, int32_t nbc,
                             const int32_t *col_blk_sizes, int64_t nblocks,
                             const int32_t *blk_row, const int32_t *blk_col, double *data,
                             void *stream);
/* Any pointer may be NULL.  nelem = number of doubles the data buffer holds. */
bst_status bst_matrix_info(const bst_matrix *m, int32_t *nbr, int32_t *nbc, int64_t *nblocks,
                           int64_t *nelem);
/* Host copies of the canonical block index and block element offsets
 * (arrays of nblocks; any may be NULL).  Synchronises the matrix's stream. */
bst_status bst_matrix_get_index(const bst_matrix *m, int32_t *blk_row, int32_t *blk_col,
                                int64_t *blk_off);
bst_status bst_matrix_bind_data(bst_matrix *m, double *data);
/* Number of doubles the matrix's data buffer holds (the packed block elements). */
bst_status bst_matrix_data_size(const bst_matrix *m, int64_t *n_elements);
bst_status bst_matrix_destroy(bst_matrix *m);

/* Block post-filter.  The paper names the sign-matrix iteration among the library's
 * operations (Sec. 2) but defines no filter on a product's result; dropping the blocks
 * of small norm between the products of such a chain is a reading of this library,
 * with the same Frobenius norm as the product filter.  bst_matrix_filter returns, in *out, a new
 * matrix with X's block sizes holding the blocks of X whose Frobenius norm is >= eps
 * (eps = 0 keeps every block), in canonical CSR order; its data is not bound.  It runs
 * on `stream` and synchronises it twice (to learn the kept block and element counts).
 * The caller binds nelem doubles (bst_matrix_info) to *out with bst_matrix_bind_data
 * and calls bst_matrix_filter_copy(X, *out), which copies the kept blocks' elements
 * (asynchronously on `stream`).  Errors: BST_ERR_INVALID_ARG (NULL, eps < 0),
 * BST_ERR_STATE (data not bound), BST_ERR_SHAPE_MISMATCH (Y is not a filter result of
 * X, or X's block count changed). */
bst_status bst_matrix_filter(bst_ctx *ctx, const bst_matrix *X, double eps, void *stream,
                             bst_matrix **out);
bst_status bst_matrix_filter_copy(const bst_matrix *X, bst_matrix *Y, void *stream);

/* ---------------------------------------------------------------------------
 * Multiply (paper Sec. 2 local multiply; Sec. 3.1 for transa = 'T').
 *
 * C_out = alpha * op(A) * op(B) + beta * C_in, op(X) = X ('N') or X^T ('T'), with
 * the block-norm filter eps >= 0 (see top).  C_in may be NULL.  Planning runs the
 * GPU symbolic phase on `stream`: block norms, pair matching + filter, pattern of
 * C_out, the stacks and the numeric schedule.  It synchronises `stream` several times
 * (about seven round trips) to learn the sizes of what it builds next.
 * The plan keeps pointers to A, B, C_in; their data are read at execute time.
 * Errors: INVALID_ARG, SHAPE_MISMATCH (inner block sizes differ, or C_in's grid
 * differs from op(A) rows x op(B) columns), OVERFLOW, UNSUPPORTED (more than 2^20
 * (m,n,k) size buckets, or a C row of more than 2^21 block columns).
 * ------------------------------------------------------------------------- */
bst_status bst_multiply_plan(bst_ctx *ctx, char transa, char transb, const bst_matrix *A,
                             const bst_matrix *B, const bst_matrix *C_in, double eps,
                             void *stream, bst_plan **out);

/* The result's pattern as a matrix owned by the plan (valid until the plan is
 * destroyed).  Bind a device buffer of its nelem doubles before executing. */
bst_status bst_plan_result(bst_plan *plan, bst_matrix **C_out);

typedef struct {
  int64_t n_candidates;   /* (i,k,j) pairs with both blocks present              */
  int64_t n_filtered;     /* of those, dropped by the norm filter                */
  int64_t n_stack;        /* kept products = stack entries                       */
  int64_t n_c_blocks;     /* blocks of C_out                                     */
  int64_t n_c_elements;   /* doubles of C_out                                    */
  int32_t n_buckets;      /* non-empty (m,n,k) buckets                           */
  int32_t split_k;        /* K parts used by the last execute (1 = unsplit)      */
  double flops;           /* sum over kept products of 2 m n k                   */
  double bytes;           /* algorithmic bytes of execute (see bst_plan_bytes)   */
} bst_stats;

/* Counters of the plan.  Also reports device-detected errors of the plan's earlier
 * executes: when a bounded wait inside the emulated-FP64 panel kernel ran out (the
 * kernel then stops, leaving that execute's result incomplete, and later executes of
 * the plan do nothing until the error is reported), it returns BST_ERR_TIMEOUT (with
 * *out filled) and clears the error.  Synchronises when the plan has run the panel
 * kernel. */
bst_status bst_plan_stats(const bst_plan *plan, bst_stats *out);

/* Host copies of the stacks: mnk[n_buckets*3], bucket_ptr[n_buckets+1] (int64),
 * a_off/b_off/c_off[n_stack].  Offsets index the STORED A, B data and C_out data.
 * Any pointer may be NULL.  Synchronises. */
bst_status bst_plan_get_stacks(const bst_plan *plan, int32_t *mnk, int64_t *bucket_ptr,
                               int32_t *a_off, int32_t *b_off, int32_t *c_off);

/* Work units of the native-FP64 staged kernel: hist[s] (s = 1..16) = row tiles of C
 * whose inner dimension is split over s lane groups (choice of BST_TUNE_F64_SPLIT and
 * the built-in cost rule, as of the last execute or plan build); hist[0] = C blocks
 * run by the direct-load kernel instead (plans whose blocks do not fit the staged
 * tiles).  hist has 17 entries.  Synchronises. */
bst_status bst_plan_split_histogram(const bst_plan *plan, int64_t *hist);

/* How the native-FP64 execute of a plan runs (for tests and tuning): info[0] = 1 when
 * the staged kernel runs its tiles (0: the direct-load kernel), info[1] = 1 when its
 * staging copies strided rows (row tiles, inner panels or slabs), info[2] = 1 when some
 * tile splits its inner dimension (BST_TUNE_F64_SPLIT), info[3] = 1 when A is read in
 * place as slabs of a contraction operand (BST_TUNE_CONTRACT_SLAB).  As of the last
 * execute or plan build; split-K executes (split_k > 1) run the same staged tiles. */
bst_status bst_plan_schedule_info(const bst_plan *plan, int32_t *info);

/* Cost model of the emulated-FP64 execute of a plan, for rooflines: out[0] = BF16
 * tensor-core flops one execute issues (the slice products on the MMA tiles the kernel
 * runs, padding included), out[1] = bytes its kernels move by design (FP64 operands
 * read by the slicing passes, digit planes written and read once, C written, the
 * schedule read; beta = 0), out[2] = bytes of intermediate partial products written
 * and read back (the int64 slots of the panel path; 0 for the C-block kernel), out[3]
 * = 1 when the plan's next execute runs the tcgen05 panel kernel, 0 for the C-block
 * kernel; the costs are those of that kernel.  Builds
 * the plan's emulation schedule when it has none yet; synchronises the legacy default
 * stream.  The paper is FP64 only: this is a reading. */
bst_status bst_plan_emu_costs(bst_plan *plan, double *out);

/* Arithmetic used by execute. */
enum {
  BST_FP64 = 0,          /* native FP64 FMA                                        */
  BST_FP64_EMU_BF16 = 1, /* Ozaki slices on BF16 tensor cores, FP64 recombination  */
  BST_TF32X3 = 2         /* 3xTF32 compensated products, FP32 accumulate per block */
};

/* Numeric phase into C_out's bound data.  split_k: 1 = each C block summed by one
 * warp; S > 1 = every C tile's products are cut into S contiguous parts (in product
 * order, so along K) whose partial sums go to a workspace and are added in the fixed
 * order 0..S-1 (paper Sec. 3.1: the K split with one reduction); 0 = choose S from
 * the plan's shape.  With beta == 0 C_in is not read.
 * Executes of one plan must not overlap on the GPU (e.g. on two streams at once):
 * they write the same C_out and share the plan's work counter, from which the
 * persistent kernels take their tiles; order them on one stream or with events.
 * Errors: STATE (C_out, A or B data not bound), INVALID_ARG, UNSUPPORTED. */
bst_status bst_multiply_execute(bst_plan *plan, double alpha, double beta, int32_t precision,
                                int32_t split_k, void *stream);

/* Native-FP64 execute (as bst_multiply_execute with BST_FP64 and split_k >= 1) that
 * allocates no device memory.  The paper has no counterpart: this entry point exists
 * for callers that may not allocate while they run -- services that reserve all GPU
 * memory up front and forbid later cudaMalloc (an allocation can synchronise the
 * device and stall every stream), or host frameworks that own the whole device heap.
 * The split-K partial sums live in a static __device__ array of
 * bst_static_scratch_doubles() doubles (32 MiB) that every GPU loading the library
 * holds until the process exits; split_k * nelem(C_out) above that returns
 * BST_ERR_UNSUPPORTED (split_k = 1 needs no scratch).  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not reset the
 * device (cudaDeviceReset) after it.  All calls share the one array: calls that overlap
 * on the GPU (different streams, or different plans on one device in flight together)
 * race.  Each call overwrites every scratch element it reads, so no clearing is needed.
 * Every argument and size check runs before any work is queued, so a failing call
 * queues nothing; the calling thread's current device is the same on return.
 * Errors: as bst_multiply_execute, plus UNSUPPORTED for a too-large workspace or a
 * device index above 63. */
bst_status bst_multiply_execute_static(bst_plan *plan, double alpha, double beta,
                                       int32_t split_k, void *stream);
/* Capacity of the static split-K array of bst_multiply_execute_static, in doubles. */
size_t bst_static_scratch_doubles(void);

/* Adjoint of execute's function with the filter decisions held fixed:
 *   dop(A)_ik = alpha sum_{j kept} dC_ij op(B)_kj^T on pattern(A),
 *   dop(B)_kj = alpha sum_{i kept} op(A)_ik^T dC_ij on pattern(B),
 *   dC_in = beta dC on pattern(C_in)  (dC_in may be NULL),
 * written (overwritten) in the stored layout of A, B, C_in.  dC is packed like
 * C_out.  For a contraction plan the buffers are the tensors' packings.  FP64. */
bst_status bst_plan_adjoint(bst_plan *plan, const double *dC, double *dA, double *dB,
                            double *dC_in, double alpha, double beta, void *stream);
/* The same without a C_in gradient: bst_plan_adjoint(plan, dC, dA, dB, NULL, alpha, 0). */
bst_status bst_multiply_adjoint(bst_plan *plan, const double *dC, double *dA, double *dB,
                                double alpha, void *stream);

bst_status bst_plan_destroy(bst_plan *plan);

/* Kernel choices of a context, set by the project's autotuner
 * (paper_1910_13555_gb300/tune.py) or by hand.
 *   BST_TUNE_EMU_ROW_SCALE (m, n ignored): 1 = emulated-FP64 digits scaled by the
 *     largest exponent of the whole op(A) row / op(B) column, so all products of a C
 *     element share a scale and their exact FP32 level sums run across products
 *     (default); 0 = scaled per block row / column, each product folded on its own
 *     (more robust to blocks of very different magnitudes in one row, slower).
 *   BST_TUNE_EMU_SWAP (per (m, n) C block class): thread mapping of the emulated-FP64
 *     kernel; 0 = the 16-row MMA tiles run over the C block's rows, 1 = over its columns
 *     (C^T = op(B)^T op(A)^T on the same digit planes, fewer tiles when n > m);
 *     -1 = back to the built-in rule (fewer 16 x 8 tiles wins).  Row-scaled mode only.
 *   BST_TUNE_F64_SPLIT (per (m, n) C block class): the largest number of lane groups
 *     over which the native-FP64 staged kernel may split the inner dimension of one
 *     C tile (1 = never split; 2..16); -1 = back to the built-in bound.  Within the
 *     bound each tile takes the split that needs the fewest FP64 instructions, and
 *     only when that saves at least 1/16 of them; the s partial sums of an output are
 *     added in a fixed order, so results stay deterministic.
 *   BST_TUNE_CONTRACT_SLAB (m, n ignored): 1 = when a contraction's first tensor is
 *     stored as (outer contracted modes, free modes, inner contracted modes), e.g.
 *     T(P, mu, nu) contracted over (P, nu), its matrix view is read in place as
 *     consecutive contiguous slabs by native-FP64 executes that run the staged kernel
 *     (no permuted copy is made before them) (default); 0 = always through the permuted
 *     copy.  Taken when a contraction plan is created; tune.tune_contract_slab times
 *     both on a given contraction.
 *   BST_TUNE_EMU_PANEL (m, n ignored): 1 = emulated-FP64 executes of a plan whose
 *     blocks fit the panel kernel (op(A) row blocks <= 128, op(B) column blocks <= 32,
 *     inner blocks <= 32 elements) run the tcgen05 panel kernel: per inner block k,
 *     the op(A) blocks of column k times the op(B) blocks of row k as one dense product
 *     on the tensor cores, digits scaled per stored block -- from the plan's second
 *     emulated execute on (the first runs the C-block kernel, so a plan executed once
 *     does not pay for building the panel schedule) (default); 2 = the panel kernel
 *     whenever the blocks fit, from the first execute; 0 = always the C-block kernel
 *     (BST_TUNE_EMU_ROW_SCALE and BST_TUNE_EMU_SWAP apply to it).  A batch decides
 *     when it is created: with 1 or 2 every matrix plan whose blocks fit runs in one
 *     panel launch over all those plans, its schedule built by bst_batch_create; the
 *     others run the C-block kernel.  A plan whose schedule exists (built by an
 *     execute or a batch) keeps the panel kernel at 1 and 2.
 * Changing a choice takes effect at the next execute of a plan; a batch built before
 * the change refuses emulated-FP64 execution (BST_ERR_STATE) and must be created again.
 * A plan or batch whose native-FP64 tiles must be split again after a change returns
 * BST_ERR_STATE when that execute is being captured into a CUDA graph: execute it once
 * outside capture first.
 * Errors: INVALID_ARG for an unknown key or value. */
enum {
  BST_TUNE_EMU_ROW_SCALE = 0,
  BST_TUNE_EMU_SWAP = 1,
  BST_TUNE_F64_SPLIT = 2,
  BST_TUNE_CONTRACT_SLAB = 3,
  BST_TUNE_EMU_PANEL = 4
};
bst_status bst_tune_set(bst_ctx *ctx, int32_t key, int32_t m, int32_t n, int32_t value);
bst_status bst_tune_get(const bst_ctx *ctx, int32_t key, int32_t m, int32_t n, int32_t *value);

/* ---------------------------------------------------------------------------
 * Tensors (paper Sec. 4).
 *
 * rank in 1..8; nblk[rank] blocks per mode; blk_sizes holds the block sizes of
 * mode 0, then mode 1, ... (host).  blk_idx[nblocks*rank] (host) lists the present
 * block tuples in any order; canonical order is lexicographic.  `data` (device)
 * packs the blocks in canonical order, each row-major (last mode fastest).
 * ------------------------------------------------------------------------- */
bst_status bst_tensor_create(bst_ctx *ctx, bst_tensor **out, int32_t rank, const int32_t *nblk,
                             const int32_t *blk_sizes, int64_t nblocks, const int32_t *blk_idx,
                             double *data, void *stream);
bst_status bst_tensor_info(const bst_tensor *t, int32_t *rank, int64_t *nblocks, int64_t *nelem);
/* host copies: blk_idx[nblocks*rank] canonical, blk_off[nblocks] */
bst_status bst_tensor_get_index(const bst_tensor *t, int32_t *blk_idx, int64_t *blk_off);
bst_status bst_tensor_bind_data(bst_tensor *t, double *data);
bst_status bst_tensor_destroy(bst_tensor *t);

/* Contraction R = alpha * sum over contracted indices of T1 * T2 + beta * R_in.
 * Mode c1[s] of T1 is summed against mode c2[s] of T2 (s < ncontract, 1..3); their
 * block sizes must agree (else SHAPE_MISMATCH).  f1 (f2) lists the free modes of
 * T1 (T2); every mode appears exactly once in c + f.  The result's modes are the
 * free modes in the order (f1..., f2...) permuted by result_order (NULL =
 * identity): result mode r is free slot result_order[r].  Computed on the GPU by
 * remapping T1 to a matrix with rows = f1 fold, cols = c1 fold (or its transpose,
 * or a permuted copy when neither is a pure fold of the stored layout), T2 to rows
 * = c2, cols = f2, then the multiply above.  The filter applies per tensor-block
 * pair (Frobenius norms do not change under reshaping).  R_in may be NULL. */
bst_status bst_contract_plan(bst_ctx *ctx, const bst_tensor *T1, const bst_tensor *T2,
                             int32_t ncontract, const int32_t *c1, const int32_t *c2,
                             int32_t nfree1, const int32_t *f1, int32_t nfree2,
                             const int32_t *f2, const int32_t *result_order,
                             const bst_tensor *R_in, double eps, void *stream, bst_plan **out);
/* The result tensor of a contraction plan (owned by the plan; bind its data). */
bst_status bst_plan_result_tensor(bst_plan *plan, bst_tensor **R);

/* ---------------------------------------------------------------------------
 * Batches: many independent plans executed by one persistent kernel launch,
 * capturable into a CUDA graph.  Tile choices per (m,n) class come from the
 * library's tune table (bst_tune_*).  alpha/beta are host arrays of n values.
 * Executes of one batch must not overlap on the GPU (they share its work counter),
 * nor overlap an execute of one of its plans (they write the same C_out).
 * alpha, beta and the plans' data pointers reach the GPU through a pinned host staging
 * buffer of the batch: an execute first waits (on the host) until the previous
 * execute's copy out of that buffer has run, so executes queued back to back each use
 * their own values.  An execute captured into a CUDA graph records that copy as a
 * graph node: a replay reads the buffer as the most recent execute call of the batch
 * left it (the captured call's values, until another execute call rewrites them).
 * Emulated-FP64 executes also write per-plan scratch of the plans on the panel kernel
 * (digit images and partial-sum slots, shared with the plans' own executes): executes
 * of such a plan, alone or in batches, must be ordered on the GPU (one stream).  A
 * device-side timeout of that batch launch is reported by bst_plan_stats of the
 * first plan on the panel kernel (in the batch's flops order) as BST_ERR_TIMEOUT.
 * ------------------------------------------------------------------------- */
bst_status bst_batch_create(bst_ctx *ctx, int32_t n, bst_plan *const *plans, bst_batch **out);
bst_status bst_batch_execute(bst_batch *batch, const double *alpha, const double *beta,
                             int32_t precision, void *stream);
bst_status bst_batch_destroy(bst_batch *batch);

/* ---------------------------------------------------------------------------
 * K-split reduction (paper Sec. 3.1, the case S_C << S_A, S_B: the inner dimension K is
 * divided among P processes, process i computes the partial product C~_i = op(A_i)
 * op(B_i) over its share of K, and C is the sum of the C~_i).
 *
 * bst_sum_parts adds up parts of C: for every output block u < nblocks, whose elements
 * are dst[dst_off[u] .. dst_off[u+1]-1], and every part i < nparts in increasing i, the
 * same number of elements of src starting at src_off[i * nblocks + u] (-1: part i has
 * no block u).  dst = ((first part present + next) + ...) in that fixed order, so the
 * bits do not depend on the launch; a block no part has is written as 0.
 * dst_off: device int64[nblocks + 1] (increasing), src_off: device int64[nparts *
 * nblocks], src and dst: device FP64, not overlapping, all owned by the caller.  Only
 * queues one kernel on `stream` (no allocation, no synchronisation).  The exchange
 * that brings each process its parts (an all-to-all over the processes, e.g. NCCL) and
 * the layout tables are the caller's; the package's ksplit module builds both.
 * Errors: INVALID_ARG for a NULL pointer (when nblocks > 0), nparts < 1 or nblocks < 0.
 * ------------------------------------------------------------------------- */
bst_status bst_sum_parts(bst_ctx *ctx, int32_t nparts, int64_t nblocks, const int64_t *dst_off,
                         const int64_t *src_off, const double *src, double *dst, void *stream);

/* ---------------------------------------------------------------------------
 * Test of the bounded device waits.  Every spin-wait of the library's kernels (the
 * panel kernel's mbarrier waits) gives up after a bound, records an error flag that the
 * host reads (bst_plan_stats reports it as BST_ERR_TIMEOUT) and lets the kernel drain
 * and return, so the context stays usable.  bst_debug_wait_probe runs a kernel whose
 * one wait, on an mbarrier nothing arrives at, is bounded by bound_ns (1e3 .. 1e9 ns),
 * and returns what that wait reports: BST_ERR_TIMEOUT.  Synchronises `stream`.
 * Errors: INVALID_ARG for a NULL context or a bound outside the range.
 * ------------------------------------------------------------------------- */
bst_status bst_debug_wait_probe(bst_ctx *ctx, int64_t bound_ns, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BST_H */
