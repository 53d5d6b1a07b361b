// Internal declarations of libbst: handle structs, device views, helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bst.h"

namespace bst {

// ---------------------------------------------------------------------------
// errors

void set_error(const std::string &msg);

struct Error {
  bst_status code;
  std::string msg;
};

#define BST_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess)                                                               \
      throw ::bst::Error{BST_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)}; \
  } while (0)

// every kernel launch site ends with BST_CHECK_LAUNCH(): it checks the launch and
// counts it (bst_kernel_launches)
void count_launch();
#define BST_CHECK_LAUNCH()          \
  do {                              \
    ::bst::count_launch();          \
    BST_CUDA(cudaGetLastError());   \
  } while (0)

#define BST_REQUIRE(cond, code, msg)                                      \
  do {                                                                    \
    if (!(cond)) throw ::bst::Error{(code), std::string(msg)};            \
  } while (0)

// Every extern "C" entry point wraps its body in API_BEGIN ... API_END: library errors
// become their status code and message, a failed host allocation BST_ERR_ALLOC, and no
// exception crosses the C boundary.
#define API_BEGIN try {
#define API_END                                          \
  }                                                      \
  catch (const ::bst::Error &e) {                        \
    ::bst::set_error(e.msg);                             \
    return e.code;                                       \
  }                                                      \
  catch (const std::bad_alloc &) {                       \
    ::bst::set_error("host allocation failed");          \
    return BST_ERR_ALLOC;                                \
  }                                                      \
  catch (...) {                                          \
    ::bst::set_error("unexpected internal error");       \
    return BST_ERR_INVALID_ARG;                          \
  }                                                      \
  return BST_OK;

// ---------------------------------------------------------------------------
// device memory through the context's allocator

struct Ctx;

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// A set of device allocations released together (by a plan, a matrix, ...).
struct Arena {
  Ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<DevBuf> bufs;
  void *alloc(size_t bytes);
  template <class T>
  T *alloc_n(size_t n) {
    return static_cast<T *>(alloc(sizeof(T) * (n ? n : 1)));
  }
  void release_all();
  ~Arena() { release_all(); }
};

}  // namespace bst

struct bst_ctx {
  int device = 0;
  bst_alloc_fn alloc = nullptr;
  bst_free_fn free_fn = nullptr;
  void *user = nullptr;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  cudaMemPool_t pool = nullptr;  // own allocations when no callbacks are given
  // mapped pinned staging for ReadBack (grown on demand), held for one ReadBack at a time
  void *rb_host = nullptr;
  size_t rb_cap = 0;
  std::mutex rb_mutex;
  // mapped pinned staging for Upload (grown on demand), held for one Upload at a time
  void *up_host = nullptr;
  size_t up_cap = 0;
  std::mutex up_mutex;
  // recorded after the copies of an Upload finished with done_async(); the next Upload
  // waits for it before it writes the staging buffer again
  cudaEvent_t up_event = nullptr;
  bool up_pending = false;
  // kernel choices (bst_tune_set): emulated-FP64 digit scaling per whole op row /
  // column (1) or per block row / column (0); per (m, n) C block class, the tile
  // orientation of the emulated kernel (1 = MMA rows run over the C block's columns);
  // tune_version changes whenever a choice does
  int tune_emu_row_scale = 1;
  std::map<std::pair<int32_t, int32_t>, int32_t> tune_emu_swap;
  // per (m, n) C block class, the largest inner split of the staged FP64 kernel's tiles
  // (1 = none); classes without an entry use the built-in bound
  std::map<std::pair<int32_t, int32_t>, int32_t> tune_f64_split;
  // contractions: read an operand whose matrix view is a sequence of contiguous slabs of
  // each tensor block in place (1) or through a permuted copy (0)
  int tune_contract_slab = 1;
  // emulated FP64: run the tcgen05 panel kernel on plans that suit it (1) or always the
  // C-block kernel (0)
  int tune_emu_panel = 1;
  int64_t tune_version = 0;
};

namespace bst {
struct Ctx : bst_ctx {};
}  // namespace bst

// Device view of a block-sparse matrix in canonical CSR order.  Blocks need not be
// packed in CSR order (a tensor view keeps the tensor's packing): off[] gives each
// block's element offset into data.  Element (p, q) of block b sits at
// data[off[b] + p * ld + q] with ld = column size of the block (row-major).
struct bst_matrix {
  bst_ctx *ctx = nullptr;
  int32_t nbr = 0, nbc = 0;
  std::vector<int32_t> h_rsz, h_csz;  // host copies of block sizes
  int64_t nblocks = 0;
  int64_t nelem = 0;
  // device arrays (owned by `arena` unless borrowed)
  int32_t *rsz = nullptr, *csz = nullptr;
  int32_t *rowptr = nullptr;  // nbr + 1
  int32_t *row = nullptr, *col = nullptr;
  int64_t *off = nullptr;
  double *data = nullptr;
  bst::Arena arena;
  bool owned_by_plan = false;
  // a post-filter result (bst_matrix_filter): source block in X of every block, and X's
  // block count when the filter ran
  int32_t *src = nullptr;
  int64_t src_nblocks = -1;
};

struct bst_tensor {
  bst_ctx *ctx = nullptr;
  int32_t rank = 0;
  std::vector<int32_t> h_nblk;
  std::vector<std::vector<int32_t>> h_sz;
  int64_t nblocks = 0, nelem = 0;
  std::vector<int32_t> h_idx;  // canonical, nblocks * rank (host copy)
  std::vector<int64_t> h_off;
  int32_t *idx = nullptr;      // device, canonical
  int64_t *off = nullptr;      // device
  int32_t *sz = nullptr;       // device, concatenated per-mode sizes
  double *data = nullptr;
  bst::Arena arena;
  bool owned_by_plan = false;
};

namespace bst {

// ---------------------------------------------------------------------------
// primitives (prims.cu)

// exclusive scan of n int32 counts into int64 (out has n + 1 entries, out[n] = total)
void exscan_i32_i64(const int32_t *in, int64_t *out, int64_t n, Arena &ar, cudaStream_t s);
// exclusive scan int64 -> int64 (n + 1 outputs)
void exscan_i64(const int64_t *in, int64_t *out, int64_t n, Arena &ar, cudaStream_t s);
// exclusive scan int32 -> int32 (n + 1 outputs); caller guarantees no overflow
void exscan_i32(const int32_t *in, int32_t *out, int64_t n, Arena &ar, cudaStream_t s);

// Stable counting sort of n items by a key in [0, nkeys): perm[out_pos] = in_pos and
// key_ptr[k] = first output position of key k (nkeys + 1 entries).
void stable_partition(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                      int32_t *key_ptr, Arena &ar, cudaStream_t s);

// Stable LSD radix sort of n (key, index) pairs on `bits` low bits of key;
// returns the permutation (out_pos -> in_pos).
void radix_sort_perm(const uint64_t *keys, int64_t n, int bits, int32_t *perm, Arena &ar,
                     cudaStream_t s);

void iota_i32(int32_t *p, int64_t n, cudaStream_t s);
void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);

// Device -> host reads of a few values (sizes, bucket and class pointers) during plan
// construction.  A kernel writes them into the context's mapped pinned buffer, so they
// do not queue on the copy engine behind a large transfer of another stream; finish()
// synchronises the stream and copies them to their host destinations.
struct ReadBack {
  bst_ctx *ctx;
  cudaStream_t s;
  struct Item {
    void *dst;
    size_t off, bytes;
  };
  std::vector<Item> items;
  size_t used = 0;
  bool locked = false;
  ReadBack(bst_ctx *c, cudaStream_t st);
  ~ReadBack();
  void add(void *host_dst, const void *dev_src, size_t bytes);
  void finish();  // values are in place afterwards
  void done();    // finish() and release the staging buffer to other threads
};
// Host -> device copies of index arrays the same way: the bytes are staged in the
// context's mapped pinned buffer and a kernel copies them to the device, so the upload
// never queues behind other streams' DMA transfers either.  done() waits for this
// stream's copies (the staging buffer is then free for the next Upload).
struct Upload {
  bst_ctx *ctx;
  cudaStream_t s;
  struct Item {
    void *dst;
    size_t off, bytes;
  };
  std::vector<Item> items;
  size_t used = 0;
  bool locked = false;
  Upload(bst_ctx *c, cudaStream_t st);
  ~Upload();
  void add(void *dev_dst, const void *host_src, size_t bytes);
  template <class T>
  T *add_vector(Arena &ar, const std::vector<T> &v) {
    T *d = ar.alloc_n<T>(v.size());
    add(d, v.data(), sizeof(T) * v.size());
    return d;
  }
  void flush();  // launch the copies staged so far and wait for them
  void done();   // flush() and release the staging buffer to other threads
  // launch the copies without waiting (the next Upload waits before it reuses the
  // buffer): only for data the same stream consumes, before a later synchronisation of
  // that stream hands the result to the caller
  void done_async();
  void launch();  // the copy kernels of the items staged so far
};
void gather_i32(const int32_t *src, const int32_t *idx, int32_t *dst, int64_t n, cudaStream_t s);

template <class T>
T read_scalar(const T *dptr, cudaStream_t s) {
  T v;
  BST_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  return v;
}

// ---------------------------------------------------------------------------
// block norms (symbolic.cu): Frobenius norm of each block of m, in its canonical order
void block_norms(const bst_matrix *m, double *norms, cudaStream_t s);

// A view of op(X) as CSR over its block rows (symbolic.cu)
struct OpView {
  int32_t nr = 0, nc = 0;
  const int32_t *rs = nullptr, *cs = nullptr;  // device block sizes of op(X)
  const int32_t *rowptr = nullptr;             // nr + 1
  const int32_t *col = nullptr;                // block column of op(X) per entry
  const int32_t *blk = nullptr;                // stored block id per entry (null = identity)
  std::vector<int32_t> h_rs, h_cs;
  bool trans = false;
};
OpView make_opview(const bst_matrix *m, bool trans, Arena &ar, cudaStream_t s);

}  // namespace bst

// ---------------------------------------------------------------------------
// plans

namespace bst {
struct EmuState;
struct PanelState;
struct AdjState;
struct Contract;
}  // namespace bst

struct bst_plan {
  bst_ctx *ctx = nullptr;
  const bst_matrix *A = nullptr, *B = nullptr, *Cin = nullptr;
  bool ta = false, tb = false;
  double eps = 0.0;
  bst::OpView oa, ob;
  // C_out (pattern owned by the plan)
  bst_matrix *C = nullptr;
  int32_t M = 0, N = 0, K = 0;
  // size classes
  std::vector<int32_t> m_vals, n_vals, k_vals;  // distinct sizes, ascending
  int32_t Dm = 0, Dn = 0, Dk = 0;
  int32_t *m_cls = nullptr, *n_cls = nullptr, *k_cls = nullptr;  // per block row/col/inner
  int32_t *cls_m = nullptr, *cls_n = nullptr;  // (m,n) class id -> m, n
  int32_t *kval = nullptr;                     // k class -> k
  // symbolic results (device)
  int32_t *c_cin = nullptr;    // per C block: C_in block id or -1
  int32_t *c_cls = nullptr;    // per C block: (m,n) class
  int64_t T = 0;               // kept products
  int32_t *t_start = nullptr;  // per C block: first triple in (i,j,k) order (nnzC + 1)
  // bucketed stacks
  int32_t nb_all = 0;                 // Dm*Dn*Dk buckets (incl. empty)
  std::vector<int64_t> h_bucket_ptr;  // nb_all + 1
  int32_t *s_a = nullptr, *s_b = nullptr, *s_c = nullptr;  // element offsets (int32)
  int32_t *s_cb = nullptr;            // C block of each entry
  int32_t *s_k = nullptr;             // k block index of each entry
  int32_t *s_ab = nullptr, *s_bb = nullptr;  // stored A / B block of each entry
  int32_t *run_start = nullptr;       // nnzC * Dk: first entry of (C block, k class) run
  int32_t *run_len = nullptr;         // nnzC * Dk
  // numeric task list: C blocks sorted by (m,n) class
  int32_t *task_c = nullptr;
  std::vector<int32_t> h_class_ptr;   // Dm*Dn + 1
  int32_t *class_ptr = nullptr;
  // persistent numeric schedule: C blocks by decreasing cost, counter of taken items
  int64_t *items = nullptr;
  unsigned long long *items_counter = nullptr;
  // staged numeric kernel: C-major entries, C block descriptors, doubles per slot
  // (0: products too large for a slot, the direct-load kernel runs)
  int4 *fents = nullptr;
  int32_t *fdesc = nullptr;
  int32_t stage_elems = 0;
  int64_t n_tiles = 0;         // row tiles of C blocks (the staged kernel's work units)
  bool stage_strided = false;  // some tile or panel is a strided part of a block
  int64_t *titems = nullptr;   // tiles by decreasing cost
  int32_t *tkeys = nullptr;    // each tile's cost key
  int64_t split_version = -1;  // tune_version the tiles' inner splits were chosen for
  bool stage_split = false;    // some tile splits its inner dimension
  bst::Arena sched_ar;         // the staged schedule's arrays (rebuilt for slab reading)
  // Slab reading of a contraction operand (set by the contraction before the staged
  // schedule is built): A's stored block (m x k, k = k_o * k_i) is k_o contiguous m x k_i
  // slabs of the tensor block, read in place.  Per k class k_i (empty: no slab reading),
  // per A view block its tensor element offset; a_slab_base = the tensor's data.
  std::vector<int32_t> a_slab_kin;
  int64_t *a_slab_toff = nullptr;
  bool a_slab = false;         // the staged schedule reads A as slabs
  double *a_slab_base = nullptr;
  // stats
  bst_stats stats{};
  // emulated-precision state (numeric_emu.cu), built on first use
  bst::EmuState *emu = nullptr;
  bst::PanelState *panel = nullptr;  // tcgen05 panel schedule (emu_panel.cu), built on first use
  int emu_executes = 0;              // emulated executes so far (panel schedule policy)
  bst::AdjState *adj = nullptr;  // adjoint grouping of the stacks (adjoint.cu)
  // contraction glue (remap.cu)
  bst::Contract *contract = nullptr;
  bst::Arena arena;
  bst::Arena work;  // execute-time workspaces (split-k partials, emulation slices)
  size_t work_bytes = 0;
};

namespace bst {

// symbolic phase (symbolic.cu): fills everything in the plan from oa/ob/Cin
void symbolic_phase(bst_plan *p, cudaStream_t s);

// numeric phase (numeric_fp64.cu / numeric_emu.cu)
struct NumArgs {
  const double *A, *B, *Cin;
  double *C;
  double alpha, beta;
};
void execute_fp64(bst_plan *p, const NumArgs &a, int split, cudaStream_t s);
void execute_fp64_workspace(bst_plan *p, const NumArgs &a, int split, double *W, cudaStream_t s);
void execute_emu_bf16(bst_plan *p, const NumArgs &a, cudaStream_t s);
void execute_tf32x3(bst_plan *p, const NumArgs &a, cudaStream_t s);
void emu_state_free(bst_plan *p);
// tcgen05 panel path of the emulated FP64 execute (emu_panel.cu)
// whether emulated executes run the panel kernel (builds its schedule when they do);
// count: this call is an execute (the default mode takes the panel from a plan's second)
bool panel_usable(bst_plan *p, cudaStream_t s, bool count = false);
void execute_emu_panel(bst_plan *p, const NumArgs &a, cudaStream_t s);
void panel_costs(bst_plan *p, cudaStream_t s, double *out);  // out[3]
void panel_state_free(bst_plan *p);
int panel_error(bst_plan *p);  // device error recorded by a panel launch (cleared)
// batches of panel plans (emu_panel.cu): one k_pan_mma launch over every plan's units
bool panel_batch_eligible(bst_plan *p, cudaStream_t s);  // builds the schedule now
size_t panel_plan_bytes();
void panel_fill_plan(bst_plan *p, const NumArgs &a, void *out);
int64_t panel_batch_units(const std::vector<bst_plan *> &plans, Arena &ar, int2 **out,
                          cudaStream_t s);
void panel_prepare(bst_plan *p, const NumArgs &a, cudaStream_t s);
void panel_finish(bst_plan *p, const NumArgs &a, cudaStream_t s);
void launch_panel_batch(const void *d_plans, const int2 *ulist, int64_t n, int *err, int num_sms,
                        cudaStream_t s);
int *panel_err_flag(bst_plan *p);
void emu_costs(bst_plan *p, cudaStream_t s, double *tensor_flops, double *bytes,
               double *intermediate);
void adj_state_free(bst_plan *p);
// contractions (contract.cu)
// throws BST_ERR_STATE when a tensor the execute reads or writes has no data bound
// (no device work)
void contract_check_bound(const bst_plan *p, bool read_cin);
void contract_prepare(bst_plan *p, bool read_cin, cudaStream_t s, bool a_copy = true);
// the native-FP64 execute with `split` K parts reads A in place (slab schedule)
bool fp64_reads_slabs(const bst_plan *p, int split);
void contract_finish(bst_plan *p, cudaStream_t s);
void contract_adjoint(bst_plan *p, const double *dR, double *dT1, double *dT2, double *dRin,
                      double alpha, double beta, cudaStream_t s);
void contract_free(bst_plan *p);
void adjoint_fp64(bst_plan *p, const double *A, const double *B, const double *dC, double *dA,
                  double *dB, double alpha, cudaStream_t s);
void scale_cin_grad(bst_plan *p, const double *dC, double *dCin, double beta, cudaStream_t s);

int choose_split(const bst_plan *p, int num_sms);
// persistent FP64 numeric (numeric_fp64.cu)
size_t num_params_bytes();
void fill_num_params(bst_plan *p, const NumArgs &a, void *out, bool staged);
void build_plan_items(bst_plan *p, int64_t base, int64_t *items, int32_t *keys, cudaStream_t s);
void sort_items(const int64_t *items, const int32_t *keys, int64_t n, int64_t *out, Arena &scratch,
                cudaStream_t s);
int persist_grid(int num_sms);
void launch_fp64_persist(const void *params, const int64_t *items, int64_t nitems,
                         unsigned long long *counter, int grid, cudaStream_t s);
void build_f64_schedule(bst_plan *p, cudaStream_t s);
void refresh_f64_split(bst_plan *p, cudaStream_t s);
constexpr int kF64DescWords = 8;  // descriptor words per staged tile
void build_plan_tile_items(bst_plan *p, int64_t base, int64_t *items, int32_t *keys,
                           cudaStream_t s);
void launch_fp64_staged(const void *params, const int64_t *items, int64_t nitems,
                        int slot_elems, bool strided, bool split, int num_sms,
                        unsigned long long *counter, cudaStream_t s);
// persistent emulated-FP64 numeric (numeric_emu.cu)
size_t emu_params_bytes();
int64_t emu_item_count(bst_plan *p, cudaStream_t s);
void emu_build_items(bst_plan *p, int64_t base, int64_t *items, cudaStream_t s);
void emu_prepare_and_fill(bst_plan *p, const NumArgs &a, void *out, cudaStream_t s);
int emu_persist_grid(int num_sms, int row_scale);
// true when row-scaled emulated tiles should take the pipelined loop: the C elements
// sum at least 64 inner elements on average (flops >= 128 nelem_c)
bool emu_pipelined(double flops, int64_t nelem_c);
void launch_emu_persist(const void *params, const int64_t *items, int64_t nitems,
                        unsigned long long *counter, int grid, int row_scale, bool pipe,
                        cudaStream_t s);

}  // namespace bst
