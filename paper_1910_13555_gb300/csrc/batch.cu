// Batches: many independent block-sparse products in one persistent kernel launch.
//
// A batch holds plans that were built with bst_multiply_plan / bst_contract_plan
// (their symbolic phases are done).  Its work list is every C block of every plan,
// tagged with the plan's index.  For native FP64 the list is sorted by decreasing cost
// across the batch, so one persistent grid balances products of very different sizes
// (the staged kernel takes chunks of items from a counter after two of its own, the
// direct-load kernel single items from a counter).  For emulated FP64, the plans whose
// blocks fit the tensor-core panel kernel (and, unless that kernel is forced, whose
// panels are full enough) run together in one launch of it: the units (one inner block
// of one plan each) of every such plan, by decreasing cost, with each plan's pointers
// in a small device table; their schedules are built here, at creation.  The other
// plans run on the C-block kernel: plans listed by decreasing flops and each plan's C
// blocks in CSR order, warps taking a few consecutive items at a time from a counter,
// so neighbouring warps share operand digits.  bst_batch_execute only queues work:
// parameter copies from the batch's pinned staging buffers, the counter reset and the
// launches (plus the per-plan slicing and reduction kernels for emulated FP64 and the
// permutations of contraction views), so a call can be captured into a CUDA graph and
// replayed; everything that allocates or synchronises happens in bst_batch_create.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bst_internal.h"

struct bst_batch {
  bst_ctx *ctx = nullptr;
  std::vector<bst_plan *> plans;
  bst::Arena ar;
  // native FP64 schedule (item = plan << 32 | C block)
  int64_t n_items = 0;
  int64_t *items = nullptr;
  unsigned long long *counter = nullptr;
  void *d_params = nullptr, *h_params = nullptr;
  size_t pbytes = 0;
  int grid = 0;
  int stage_elems = 0;  // staged FP64 kernel slot size (0: some plan needs direct loads)
  bool stage_strided = false;
  int64_t n_titems = 0;
  int64_t *titems = nullptr;  // staged kernel: every plan's tiles by decreasing cost
  // emulated FP64 schedule (item = plan << 32 | C block)
  int64_t n_items_e = 0;
  int64_t *items_e = nullptr;
  void *d_eparams = nullptr, *h_eparams = nullptr;
  size_t epbytes = 0;
  int grid_e = 0;
  // emulated FP64 on the panel kernel: the plans it runs, their (plan, unit) list and
  // the per-plan pointer table (staged like the parameters)
  std::vector<int32_t> panel_plans;
  std::vector<char> on_panel;
  int2 *ulist = nullptr;
  int64_t n_units = 0;
  void *d_pplans = nullptr, *h_pplans = nullptr;
  size_t ppbytes = 0;
  int *panel_err = nullptr;
  int64_t tune_version = 0;  // the context's tuning state the schedules were built for
  // recorded after each parameter copy out of h_params / h_eparams; the next execute
  // waits for it before it rewrites the staging buffers
  cudaEvent_t copied = nullptr;
  bool copy_pending = false;
  ~bst_batch() {
    if (copied) cudaEventDestroy(copied);
    if (h_params) cudaFreeHost(h_params);
    if (h_eparams) cudaFreeHost(h_eparams);
    if (h_pplans) cudaFreeHost(h_pplans);
  }
};

namespace {

struct Args {
  bst::NumArgs a;
  bool read_cin;
};

// a_copy: the execute reads A through the plan's permuted copy (not slab by slab in place)
Args plan_args(bst_plan *p, double alpha, double beta, cudaStream_t s, bool a_copy = true) {
  if (p->contract)
    bst::contract_prepare(p, beta != 0.0 && p->Cin && p->Cin->nblocks > 0, s, a_copy);
  const bst_matrix *C = p->C;
  BST_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), BST_ERR_INVALID_ARG,
              "alpha and beta must be finite");
  BST_REQUIRE(C->nelem == 0 || C->data, BST_ERR_STATE, "C_out data not bound");
  BST_REQUIRE(p->A->nblocks == 0 || p->A->data, BST_ERR_STATE, "A data not bound");
  BST_REQUIRE(p->B->nblocks == 0 || p->B->data, BST_ERR_STATE, "B data not bound");
  Args r;
  r.read_cin = beta != 0.0 && p->Cin && p->Cin->nblocks > 0;
  BST_REQUIRE(!r.read_cin || p->Cin->data, BST_ERR_STATE, "C_in data not bound");
  r.a.A = p->A->data;
  r.a.B = p->B->data;
  r.a.Cin = r.read_cin ? p->Cin->data : nullptr;
  r.a.C = C->data;
  r.a.alpha = alpha;
  r.a.beta = r.read_cin ? beta : 0.0;
  return r;
}

}  // namespace

extern "C" {

bst_status bst_batch_create(bst_ctx *ctx, int32_t n, bst_plan *const *plans, bst_batch **out) {
  try {
    BST_REQUIRE(ctx && out && n >= 1 && plans, BST_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    for (int32_t q = 0; q < n; ++q) {
      BST_REQUIRE(plans[q], BST_ERR_INVALID_ARG, "a plan is NULL");
      BST_REQUIRE(plans[q]->ctx == ctx, BST_ERR_INVALID_ARG, "plans of another context");
    }
    int cur = -1;
    BST_CUDA(cudaGetDevice(&cur));
    if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = nullptr;
    auto *b = new bst_batch();
    try {
      b->ctx = ctx;
      b->ar.ctx = static_cast<bst::Ctx *>(ctx);
      b->ar.stream = s;
      b->plans.assign(plans, plans + n);
      bst::Arena scratch;
      scratch.ctx = b->ar.ctx;
      scratch.stream = s;
      // plans by decreasing flops (the longest problems start first); inside a plan,
      // C blocks in CSR order for locality
      std::vector<int32_t> order(n);
      for (int32_t q = 0; q < n; ++q) order[q] = q;
      std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return b->plans[x]->stats.flops > b->plans[y]->stats.flops;
      });
      // native FP64: every C block of every plan, by decreasing cost across the batch
      for (auto *p : b->plans) b->n_items += p->C->nblocks;
      int64_t *it0 = scratch.alloc_n<int64_t>((size_t)b->n_items);
      int32_t *keys = scratch.alloc_n<int32_t>((size_t)b->n_items);
      int64_t off = 0;
      for (int32_t q : order) {
        bst::build_plan_items(b->plans[q], (int64_t)q << 32, it0 + off, keys + off, s);
        off += b->plans[q]->C->nblocks;
      }
      b->items = b->ar.alloc_n<int64_t>((size_t)b->n_items);
      bst::sort_items(it0, keys, b->n_items, b->items, scratch, s);
      b->counter = b->ar.alloc_n<unsigned long long>(1);
      b->pbytes = bst::num_params_bytes();
      b->d_params = b->ar.alloc(b->pbytes * n);
      BST_CUDA(cudaMallocHost(&b->h_params, b->pbytes * n));
      b->grid = bst::persist_grid(ctx->num_sms);
      b->stage_elems = 0;
      {
        bool all = true;
        int mx = 0;
        for (auto *p : b->plans) {
          if (p->C->nblocks == 0) continue;
          if (p->stage_elems == 0) all = false;
          mx = std::max(mx, (int)p->stage_elems);
        }
        if (all) b->stage_elems = std::max(mx, 1);
        for (auto *p : b->plans) b->stage_strided = b->stage_strided || p->stage_strided;
      }
      if (b->stage_elems > 0) {
        for (auto *p : b->plans) b->n_titems += p->n_tiles;
        int64_t *t0 = scratch.alloc_n<int64_t>((size_t)b->n_titems);
        int32_t *tk = scratch.alloc_n<int32_t>((size_t)b->n_titems);
        int64_t toff = 0;
        for (int32_t q : order) {
          bst::build_plan_tile_items(b->plans[q], (int64_t)q << 32, t0 + toff, tk + toff, s);
          toff += b->plans[q]->n_tiles;
        }
        b->titems = b->ar.alloc_n<int64_t>((size_t)b->n_titems);
        bst::sort_items(t0, tk, b->n_titems, b->titems, scratch, s);
      }
      // emulated FP64: plans on the panel kernel (schedule built here), every C block of
      // the others (slicing state built per plan here)
      b->on_panel.assign(n, 0);
      {
        std::vector<bst_plan *> pp;
        for (int32_t q : order) {
          bst_plan *p = b->plans[q];
          if (p->contract || p->C->nblocks == 0 || !bst::panel_batch_eligible(p, s)) continue;
          b->on_panel[q] = 1;
          b->panel_plans.push_back(q);
          pp.push_back(p);
        }
        if (!pp.empty()) {
          b->n_units = bst::panel_batch_units(pp, b->ar, &b->ulist, s);
          b->ppbytes = bst::panel_plan_bytes();
          b->d_pplans = b->ar.alloc(b->ppbytes * pp.size());
          BST_CUDA(cudaMallocHost(&b->h_pplans, b->ppbytes * pp.size()));
          b->panel_err = bst::panel_err_flag(pp[0]);
        }
      }
      std::vector<int64_t> cnt(n);
      for (int32_t q = 0; q < n; ++q) {
        cnt[q] = b->plans[q]->contract || b->on_panel[q] ? 0 : bst::emu_item_count(b->plans[q], s);
        b->n_items_e += cnt[q];
      }
      b->items_e = b->ar.alloc_n<int64_t>((size_t)std::max<int64_t>(b->n_items_e, 1));
      off = 0;
      for (int32_t q : order) {
        if (cnt[q]) bst::emu_build_items(b->plans[q], (int64_t)q << 32, b->items_e + off, s);
        off += cnt[q];
      }
      b->epbytes = bst::emu_params_bytes();
      b->d_eparams = b->ar.alloc(b->epbytes * n);
      BST_CUDA(cudaMallocHost(&b->h_eparams, b->epbytes * n));
      b->grid_e = bst::emu_persist_grid(ctx->num_sms, ctx->tune_emu_row_scale);
      b->tune_version = ctx->tune_version;
      BST_CUDA(cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming));
      BST_CUDA(cudaStreamSynchronize(s));
      scratch.release_all();
      BST_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      delete b;
      throw;
    }
    *out = b;
  } catch (const bst::Error &e) {
    bst::set_error(e.msg);
    return e.code;
  } catch (...) {
    bst::set_error("unexpected internal error");
    return BST_ERR_INVALID_ARG;
  }
  return BST_OK;
}

bst_status bst_batch_execute(bst_batch *b, const double *alpha, const double *beta,
                             int32_t precision, void *stream) {
  try {
    BST_REQUIRE(b && alpha && beta, BST_ERR_INVALID_ARG, "NULL argument");
    BST_REQUIRE(precision == BST_FP64 || precision == BST_FP64_EMU_BF16, BST_ERR_UNSUPPORTED,
                "batches run native FP64 or emulated FP64");
    int cur = -1;
    BST_CUDA(cudaGetDevice(&cur));
    if (cur != b->ctx->device) BST_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t n = (int32_t)b->plans.size();
    BST_REQUIRE(precision == BST_FP64 || b->tune_version == b->ctx->tune_version, BST_ERR_STATE,
                "the context's tuning changed after the batch was created; create it again");
    // The parameters travel through pinned host staging buffers.  An earlier execute's
    // copy out of them may still be queued: wait for it before they are rewritten, so
    // executes queued back to back each run with their own alpha, beta and data.  While
    // the stream is being captured the copy becomes a graph node that reads the buffers
    // when the graph is replayed (nothing is waited for or recorded then).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BST_CUDA(cudaStreamIsCapturing(s, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (b->copy_pending && !capturing) {
      BST_CUDA(cudaEventSynchronize(b->copied));
      b->copy_pending = false;
    }
    if (precision == BST_FP64) {
      bool split = false;
      for (int32_t q = 0; q < n; ++q) {
        if (b->stage_elems > 0) {
          bst::refresh_f64_split(b->plans[q], s);
          split = split || b->plans[q]->stage_split;
        }
        Args r = plan_args(b->plans[q], alpha[q], beta[q], s,
                           !(b->stage_elems > 0 && bst::fp64_reads_slabs(b->plans[q], 1)));
        bst::fill_num_params(b->plans[q], r.a, static_cast<char *>(b->h_params) + q * b->pbytes,
                             b->stage_elems > 0);
      }
      BST_CUDA(cudaMemcpyAsync(b->d_params, b->h_params, b->pbytes * n, cudaMemcpyHostToDevice, s));
      if (!capturing) {
        BST_CUDA(cudaEventRecord(b->copied, s));
        b->copy_pending = true;
      }
      if (b->stage_elems > 0)
        bst::launch_fp64_staged(b->d_params, b->titems, b->n_titems, b->stage_elems,
                                b->stage_strided, split, b->ctx->num_sms, b->counter, s);
      else
        bst::launch_fp64_persist(b->d_params, b->items, b->n_items, b->counter, b->grid, s);
    } else {
      for (int32_t q = 0; q < n; ++q)
        BST_REQUIRE(!b->plans[q]->contract, BST_ERR_UNSUPPORTED,
                    "emulated FP64 batches take matrix plans only");
      std::vector<bst::NumArgs> pargs(b->panel_plans.size());
      for (size_t i = 0; i < b->panel_plans.size(); ++i) {
        bst_plan *p = b->plans[b->panel_plans[i]];
        pargs[i] = plan_args(p, alpha[b->panel_plans[i]], beta[b->panel_plans[i]], s).a;
        bst::panel_prepare(p, pargs[i], s);
        bst::panel_fill_plan(p, pargs[i], static_cast<char *>(b->h_pplans) + i * b->ppbytes);
      }
      for (int32_t q = 0; q < n; ++q) {
        if (b->on_panel[q]) continue;
        Args r = plan_args(b->plans[q], alpha[q], beta[q], s);
        if (b->plans[q]->C->nblocks > 0)
          bst::emu_prepare_and_fill(b->plans[q], r.a,
                                    static_cast<char *>(b->h_eparams) + q * b->epbytes, s);
      }
      if (b->n_items_e > 0)
        BST_CUDA(cudaMemcpyAsync(b->d_eparams, b->h_eparams, b->epbytes * n,
                                 cudaMemcpyHostToDevice, s));
      if (!b->panel_plans.empty())
        BST_CUDA(cudaMemcpyAsync(b->d_pplans, b->h_pplans, b->ppbytes * b->panel_plans.size(),
                                 cudaMemcpyHostToDevice, s));
      if (!capturing) {
        BST_CUDA(cudaEventRecord(b->copied, s));
        b->copy_pending = true;
      }
      if (b->n_items_e > 0) {
        double flops = 0.0;
        int64_t nelem = 0;
        for (int32_t q = 0; q < n; ++q) {
          if (b->on_panel[q]) continue;
          flops += b->plans[q]->stats.flops;
          nelem += b->plans[q]->C->nelem;
        }
        bst::launch_emu_persist(b->d_eparams, b->items_e, b->n_items_e, b->counter, b->grid_e,
                                b->ctx->tune_emu_row_scale, bst::emu_pipelined(flops, nelem), s);
      }
      if (!b->panel_plans.empty()) {
        bst::launch_panel_batch(b->d_pplans, b->ulist, b->n_units, b->panel_err,
                                b->ctx->num_sms, s);
        for (size_t i = 0; i < b->panel_plans.size(); ++i)
          bst::panel_finish(b->plans[b->panel_plans[i]], pargs[i], s);
      }
    }
    for (int32_t q = 0; q < n; ++q) {
      if (b->plans[q]->contract) bst::contract_finish(b->plans[q], s);
      b->plans[q]->stats.split_k = 1;
    }
  } catch (const bst::Error &e) {
    bst::set_error(e.msg);
    return e.code;
  } catch (...) {
    bst::set_error("unexpected internal error");
    return BST_ERR_INVALID_ARG;
  }
  return BST_OK;
}

bst_status bst_batch_destroy(bst_batch *b) {
  delete b;
  return BST_OK;
}

}  // extern "C"
