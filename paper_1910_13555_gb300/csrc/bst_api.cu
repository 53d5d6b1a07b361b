// C ABI of libbst: contexts, matrices, multiply plans (see include/bst.h).
//
// Host work here is limited to argument validation, canonicalising the caller's
// block index (sort + duplicate check) at creation time, and orchestration; every
// step of the multiply itself runs in the CUDA kernels of symbolic.cu and
// numeric_*.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

#include "bst_internal.h"

namespace bst {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

void *Arena::alloc(size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 8;
  if (ctx && ctx->alloc) {
    p = ctx->alloc(bytes, ctx->user, stream);
    if (!p) throw Error{BST_ERR_ALLOC, "allocator callback returned NULL"};
    if (reinterpret_cast<uintptr_t>(p) & 255) {
      ctx->free_fn(p, ctx->user, stream);
      throw Error{BST_ERR_ALLOC, "allocator callback returned a pointer not aligned to 256 bytes"};
    }
  } else {
    cudaError_t e = ctx && ctx->pool ? cudaMallocFromPoolAsync(&p, bytes, ctx->pool, stream)
                                     : cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      throw Error{BST_ERR_ALLOC, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
    }
  }
  bufs.push_back({p, bytes});
  return p;
}

void Arena::release_all() {
  for (auto &b : bufs) {
    if (ctx && ctx->free_fn)
      ctx->free_fn(b.p, ctx->user, stream);
    else
      (void)cudaFreeAsync(b.p, stream);
  }
  bufs.clear();
}

}  // namespace bst

using bst::Error;


namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

void use_device(const bst_ctx *ctx) {
  int cur = -1;
  BST_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
}

}  // namespace

extern "C" {

const char *bst_last_error(void) { return bst::g_last_error.c_str(); }

const char *bst_status_name(bst_status s) {
  switch (s) {
    case BST_OK: return "BST_OK";
    case BST_ERR_INVALID_ARG: return "BST_ERR_INVALID_ARG";
    case BST_ERR_OUT_OF_RANGE: return "BST_ERR_OUT_OF_RANGE";
    case BST_ERR_DUPLICATE_BLOCK: return "BST_ERR_DUPLICATE_BLOCK";
    case BST_ERR_SHAPE_MISMATCH: return "BST_ERR_SHAPE_MISMATCH";
    case BST_ERR_OVERFLOW: return "BST_ERR_OVERFLOW";
    case BST_ERR_ALLOC: return "BST_ERR_ALLOC";
    case BST_ERR_CUDA: return "BST_ERR_CUDA";
    case BST_ERR_TIMEOUT: return "BST_ERR_TIMEOUT";
    case BST_ERR_UNSUPPORTED: return "BST_ERR_UNSUPPORTED";
    case BST_ERR_STATE: return "BST_ERR_STATE";
    default: return "BST_ERR_UNKNOWN";
  }
}

const char *bst_version(void) { return "bst 0.1 (sm_103a)"; }

int64_t bst_kernel_launches(void) { return bst::g_launches.load(std::memory_order_relaxed); }

bst_status bst_context_create(bst_ctx **out, int32_t device, bst_alloc_fn alloc,
                              bst_free_fn free_fn, void *user) {
  API_BEGIN
  BST_REQUIRE(out != nullptr, BST_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  BST_REQUIRE((alloc == nullptr) == (free_fn == nullptr), BST_ERR_INVALID_ARG,
              "alloc and free callbacks must be given together");
  int ndev = 0;
  BST_CUDA(cudaGetDeviceCount(&ndev));
  BST_REQUIRE(device >= 0 && device < ndev, BST_ERR_INVALID_ARG, "no such CUDA device");
  auto *c = new bst::Ctx();
  c->device = device;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  c->num_sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->max_smem_optin = (size_t)v;
  if (!alloc) {
    // the context's own stream-ordered pool, keeping freed memory for the next plan
    // (the device's default pool returns it to the driver at every synchronisation)
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      // no reuse of memory freed on another stream behind an inserted wait: that would
      // chain independent streams (a plan built on one stream behind another's copies)
      int no = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
      c->pool = pool;
    } else {
      (void)cudaGetLastError();
    }
  }
  *out = c;
  API_END
}

bst_status bst_context_destroy(bst_ctx *ctx) {
  API_BEGIN
  if (ctx && ctx->pool) {
    BST_CUDA(cudaDeviceSynchronize());
    cudaMemPoolDestroy(ctx->pool);
  }
  if (ctx && ctx->rb_host) cudaFreeHost(ctx->rb_host);
  if (ctx && ctx->up_host) cudaFreeHost(ctx->up_host);
  if (ctx && ctx->up_event) cudaEventDestroy(ctx->up_event);
  delete static_cast<bst::Ctx *>(ctx);
  API_END
}

bst_status bst_matrix_create(bst_ctx *ctx, bst_matrix **out, int32_t nbr,
                             const int32_t *row_blk_sizes, int32_t nbc,
                             const int32_t *col_blk_sizes, int64_t nblocks,
                             const int32_t *blk_row, const int32_t *blk_col, double *data,
                             void *stream) {
  API_BEGIN
  BST_REQUIRE(ctx && out, BST_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  BST_REQUIRE(nbr >= 0 && nbc >= 0 && nblocks >= 0, BST_ERR_INVALID_ARG, "negative size");
  BST_REQUIRE((nbr == 0 || row_blk_sizes) && (nbc == 0 || col_blk_sizes), BST_ERR_INVALID_ARG,
              "block size array is NULL");
  BST_REQUIRE(nblocks == 0 || (blk_row && blk_col), BST_ERR_INVALID_ARG, "block index is NULL");
  BST_REQUIRE(nblocks < INT32_MAX, BST_ERR_OVERFLOW, "more than 2^31-1 blocks");
  for (int32_t i = 0; i < nbr; ++i)
    BST_REQUIRE(row_blk_sizes[i] >= 1, BST_ERR_INVALID_ARG, "block row size < 1");
  for (int32_t j = 0; j < nbc; ++j)
    BST_REQUIRE(col_blk_sizes[j] >= 1, BST_ERR_INVALID_ARG, "block column size < 1");
  use_device(ctx);
  cudaStream_t s = as_stream(stream);
  std::vector<int64_t> key((size_t)nblocks);
  for (int64_t b = 0; b < nblocks; ++b) {
    BST_REQUIRE(blk_row[b] >= 0 && blk_row[b] < nbr && blk_col[b] >= 0 && blk_col[b] < nbc,
                BST_ERR_OUT_OF_RANGE, "block index outside the block grid");
    key[b] = (int64_t)blk_row[b] * nbc + blk_col[b];
  }
  std::vector<int32_t> ord((size_t)nblocks);
  std::iota(ord.begin(), ord.end(), 0);
  // blocks given in row-major order (the usual case) need no sort
  bool sorted = true;
  for (int64_t b = 1; b < nblocks && sorted; ++b) sorted = key[b - 1] < key[b];
  if (!sorted)
    std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return key[x] < key[y]; });
  std::vector<int32_t> row((size_t)nblocks), col((size_t)nblocks), rowptr((size_t)nbr + 1, 0);
  std::vector<int64_t> off((size_t)nblocks);
  int64_t acc = 0;
  for (int64_t b = 0; b < nblocks; ++b) {
    const int32_t o = ord[b];
    BST_REQUIRE(b == 0 || key[o] != key[ord[b - 1]], BST_ERR_DUPLICATE_BLOCK,
                "a block is listed twice");
    row[b] = blk_row[o];
    col[b] = blk_col[o];
    off[b] = acc;
    acc += (int64_t)row_blk_sizes[row[b]] * col_blk_sizes[col[b]];
    rowptr[row[b] + 1]++;
  }
  BST_REQUIRE(acc <= INT32_MAX, BST_ERR_OVERFLOW, "more than 2^31-1 elements");
  for (int32_t i = 0; i < nbr; ++i) rowptr[i + 1] += rowptr[i];
  auto *m = new bst_matrix();
  try {
    m->ctx = ctx;
    m->arena.ctx = static_cast<bst::Ctx *>(ctx);
    m->arena.stream = s;
    m->nbr = nbr;
    m->nbc = nbc;
    m->h_rsz.assign(row_blk_sizes, row_blk_sizes + nbr);
    m->h_csz.assign(col_blk_sizes, col_blk_sizes + nbc);
    m->nblocks = nblocks;
    m->nelem = acc;
    bst::Upload up(ctx, s);
    m->rsz = up.add_vector(m->arena, m->h_rsz);
    m->csz = up.add_vector(m->arena, m->h_csz);
    m->rowptr = up.add_vector(m->arena, rowptr);
    m->row = up.add_vector(m->arena, row);
    m->col = up.add_vector(m->arena, col);
    m->off = up.add_vector(m->arena, off);
    m->data = data;
    up.done();  // the host staging vectors end here
  } catch (...) {
    delete m;
    throw;
  }
  *out = m;
  API_END
}

bst_status bst_matrix_info(const bst_matrix *m, int32_t *nbr, int32_t *nbc, int64_t *nblocks,
                           int64_t *nelem) {
  API_BEGIN
  BST_REQUIRE(m, BST_ERR_INVALID_ARG, "matrix is NULL");
  if (nbr) *nbr = m->nbr;
  if (nbc) *nbc = m->nbc;
  if (nblocks) *nblocks = m->nblocks;
  if (nelem) *nelem = m->nelem;
  API_END
}

bst_status bst_matrix_data_size(const bst_matrix *m, int64_t *n_elements) {
  API_BEGIN
  BST_REQUIRE(m && n_elements, BST_ERR_INVALID_ARG, "NULL argument");
  *n_elements = m->nelem;
  API_END
}

bst_status bst_matrix_get_index(const bst_matrix *m, int32_t *blk_row, int32_t *blk_col,
                                int64_t *blk_off) {
  API_BEGIN
  BST_REQUIRE(m, BST_ERR_INVALID_ARG, "matrix is NULL");
  use_device(m->ctx);
  const size_t n = (size_t)m->nblocks;
  if (n) {
    if (blk_row) BST_CUDA(cudaMemcpy(blk_row, m->row, 4 * n, cudaMemcpyDeviceToHost));
    if (blk_col) BST_CUDA(cudaMemcpy(blk_col, m->col, 4 * n, cudaMemcpyDeviceToHost));
    if (blk_off) BST_CUDA(cudaMemcpy(blk_off, m->off, 8 * n, cudaMemcpyDeviceToHost));
  }
  API_END
}

bst_status bst_matrix_bind_data(bst_matrix *m, double *data) {
  API_BEGIN
  BST_REQUIRE(m, BST_ERR_INVALID_ARG, "matrix is NULL");
  m->data = data;
  API_END
}

bst_status bst_matrix_destroy(bst_matrix *m) {
  API_BEGIN
  if (!m) return BST_OK;
  BST_REQUIRE(!m->owned_by_plan, BST_ERR_STATE, "this matrix belongs to a plan");
  delete m;
  API_END
}

bst_status bst_multiply_plan(bst_ctx *ctx, char transa, char transb, const bst_matrix *A,
                             const bst_matrix *B, const bst_matrix *C_in, double eps,
                             void *stream, bst_plan **out) {
  API_BEGIN
  BST_REQUIRE(ctx && A && B && out, BST_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  const bool ta = transa == 'T' || transa == 't', tb = transb == 'T' || transb == 't';
  BST_REQUIRE(ta || transa == 'N' || transa == 'n', BST_ERR_INVALID_ARG, "transa must be N or T");
  BST_REQUIRE(tb || transb == 'N' || transb == 'n', BST_ERR_INVALID_ARG, "transb must be N or T");
  BST_REQUIRE(eps >= 0.0, BST_ERR_INVALID_ARG, "eps must be >= 0");
  BST_REQUIRE(A->nblocks == 0 || A->data, BST_ERR_STATE, "A data not bound");
  BST_REQUIRE(B->nblocks == 0 || B->data, BST_ERR_STATE, "B data not bound");
  // shapes: block columns of op(A) == block rows of op(B), with equal sizes
  const std::vector<int32_t> &a_rs = ta ? A->h_csz : A->h_rsz, &a_cs = ta ? A->h_rsz : A->h_csz;
  const std::vector<int32_t> &b_rs = tb ? B->h_csz : B->h_rsz, &b_cs = tb ? B->h_rsz : B->h_csz;
  BST_REQUIRE(a_cs == b_rs, BST_ERR_SHAPE_MISMATCH,
              "inner block sizes of op(A) and op(B) differ");
  if (C_in) {
    BST_REQUIRE(C_in->h_rsz == a_rs && C_in->h_csz == b_cs, BST_ERR_SHAPE_MISMATCH,
                "C_in block grid differs from op(A) rows x op(B) columns");
  }
  use_device(ctx);
  cudaStream_t s = as_stream(stream);
  auto *p = new bst_plan();
  try {
    p->ctx = ctx;
    p->arena.ctx = static_cast<bst::Ctx *>(ctx);
    p->arena.stream = s;
    p->work.ctx = static_cast<bst::Ctx *>(ctx);
    p->work.stream = s;
    p->A = A;
    p->B = B;
    p->Cin = C_in;
    p->ta = ta;
    p->tb = tb;
    p->eps = eps;
    p->oa = bst::make_opview(A, ta, p->arena, s);
    p->ob = bst::make_opview(B, tb, p->arena, s);
    p->M = p->oa.nr;
    p->N = p->ob.nc;
    p->K = p->oa.nc;
    p->C = new bst_matrix();
    p->C->ctx = ctx;
    p->C->owned_by_plan = true;
    bst::symbolic_phase(p, s);
  } catch (...) {
    if (p->C) {
      p->C->owned_by_plan = false;
      delete p->C;
    }
    delete p;
    throw;
  }
  *out = p;
  API_END
}

bst_status bst_plan_result(bst_plan *plan, bst_matrix **C_out) {
  API_BEGIN
  BST_REQUIRE(plan && C_out, BST_ERR_INVALID_ARG, "NULL argument");
  *C_out = plan->C;
  API_END
}

bst_status bst_plan_stats(const bst_plan *plan, bst_stats *out) {
  API_BEGIN
  BST_REQUIRE(plan && out, BST_ERR_INVALID_ARG, "NULL argument");
  *out = plan->stats;
  if (plan->panel) {
    use_device(plan->ctx);
    const int e = bst::panel_error(const_cast<bst_plan *>(plan));
    BST_REQUIRE(e == 0, BST_ERR_TIMEOUT,
                "a bounded wait of the emulated-FP64 panel kernel ran out; the results of the "
                "executes since the last check are incomplete");
  }
  API_END
}

bst_status bst_plan_split_histogram(const bst_plan *plan, int64_t *hist) {
  API_BEGIN
  BST_REQUIRE(plan && hist, BST_ERR_INVALID_ARG, "NULL argument");
  use_device(plan->ctx);
  for (int s = 0; s <= 16; ++s) hist[s] = 0;
  if (plan->n_tiles > 0) {
    std::vector<int32_t> w((size_t)plan->n_tiles);
    BST_CUDA(cudaMemcpy2D(w.data(), 4, plan->fdesc + 7, 4 * bst::kF64DescWords, 4,
                          (size_t)plan->n_tiles, cudaMemcpyDeviceToHost));
    for (int32_t v : w) ++hist[std::min(std::max(v, 1), 16)];
  } else if (plan->C) {
    hist[0] = plan->C->nblocks;
  }
  API_END
}

bst_status bst_plan_schedule_info(const bst_plan *plan, int32_t *info) {
  API_BEGIN
  BST_REQUIRE(plan && info, BST_ERR_INVALID_ARG, "NULL argument");
  info[0] = plan->stage_elems > 0;
  info[1] = plan->stage_elems > 0 && plan->stage_strided;
  info[2] = plan->stage_elems > 0 && plan->stage_split;
  info[3] = plan->stage_elems > 0 && plan->a_slab;
  API_END
}

bst_status bst_plan_emu_costs(bst_plan *plan, double *out) {
  API_BEGIN
  BST_REQUIRE(plan && out, BST_ERR_INVALID_ARG, "NULL argument");
  use_device(plan->ctx);
  cudaStream_t s = nullptr;
  bst::emu_costs(plan, s, &out[0], &out[1], &out[2]);
  out[3] = bst::panel_usable(plan, s) ? 1.0 : 0.0;  // as the next execute will run
  BST_CUDA(cudaStreamSynchronize(s));
  API_END
}

bst_status bst_plan_get_stacks(const bst_plan *plan, int32_t *mnk, int64_t *bucket_ptr,
                               int32_t *a_off, int32_t *b_off, int32_t *c_off) {
  API_BEGIN
  BST_REQUIRE(plan, BST_ERR_INVALID_ARG, "plan is NULL");
  use_device(plan->ctx);
  int32_t q = 0;
  const auto &hb = plan->h_bucket_ptr;
  for (int32_t b = 0; b < plan->nb_all; ++b) {
    if (hb[b + 1] == hb[b]) continue;
    const int32_t kc = b % plan->Dk, nc = (b / plan->Dk) % plan->Dn, mc = b / (plan->Dk * plan->Dn);
    if (mnk) {
      mnk[3 * q + 0] = plan->m_vals[mc];
      mnk[3 * q + 1] = plan->n_vals[nc];
      mnk[3 * q + 2] = plan->k_vals[kc];
    }
    if (bucket_ptr) bucket_ptr[q] = hb[b];
    ++q;
  }
  if (bucket_ptr) bucket_ptr[q] = plan->T;
  const size_t n = (size_t)plan->T;
  if (n) {
    if (a_off) BST_CUDA(cudaMemcpy(a_off, plan->s_a, 4 * n, cudaMemcpyDeviceToHost));
    if (b_off) BST_CUDA(cudaMemcpy(b_off, plan->s_b, 4 * n, cudaMemcpyDeviceToHost));
    if (c_off) BST_CUDA(cudaMemcpy(c_off, plan->s_c, 4 * n, cudaMemcpyDeviceToHost));
  }
  API_END
}

bst_status bst_multiply_execute(bst_plan *plan, double alpha, double beta, int32_t precision,
                                int32_t split_k, void *stream) {
  API_BEGIN
  BST_REQUIRE(plan, BST_ERR_INVALID_ARG, "plan is NULL");
  BST_REQUIRE(split_k >= 0 && split_k <= 64, BST_ERR_INVALID_ARG, "split_k must be in 0..64");
  BST_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), BST_ERR_INVALID_ARG,
              "alpha and beta must be finite");
  use_device(plan->ctx);
  int split = 1;
  if (precision == BST_FP64)
    split = split_k == 0 ? bst::choose_split(plan, plan->ctx->num_sms) : split_k;
  if (plan->contract)
    bst::contract_prepare(plan, beta != 0.0 && plan->Cin && plan->Cin->nblocks > 0,
                          as_stream(stream),
                          !(precision == BST_FP64 && bst::fp64_reads_slabs(plan, split)));
  const bst_matrix *C = plan->C;
  BST_REQUIRE(C->nelem == 0 || C->data, BST_ERR_STATE, "C_out data not bound");
  BST_REQUIRE(plan->A->nblocks == 0 || plan->A->data, BST_ERR_STATE, "A data not bound");
  BST_REQUIRE(plan->B->nblocks == 0 || plan->B->data, BST_ERR_STATE, "B data not bound");
  const bool read_cin = beta != 0.0 && plan->Cin && plan->Cin->nblocks > 0;
  BST_REQUIRE(!read_cin || plan->Cin->data, BST_ERR_STATE, "C_in data not bound");
  use_device(plan->ctx);
  cudaStream_t s = as_stream(stream);
  bst::NumArgs a;
  a.A = plan->A->data;
  a.B = plan->B->data;
  a.Cin = read_cin ? plan->Cin->data : nullptr;
  a.C = C->data;
  a.alpha = alpha;
  a.beta = read_cin ? beta : 0.0;
  switch (precision) {
    case BST_FP64:
      bst::execute_fp64(plan, a, split, s);
      break;
    case BST_FP64_EMU_BF16:
      bst::execute_emu_bf16(plan, a, s);
      break;
    case BST_TF32X3:
      bst::execute_tf32x3(plan, a, s);
      break;
    default:
      throw Error{BST_ERR_INVALID_ARG, "unknown precision"};
  }
  if (plan->contract) bst::contract_finish(plan, s);
  plan->stats.split_k = split;
  API_END
}

bst_status bst_plan_adjoint(bst_plan *plan, const double *dC, double *dA, double *dB,
                            double *dC_in, double alpha, double beta, void *stream) {
  API_BEGIN
  BST_REQUIRE(plan, BST_ERR_INVALID_ARG, "plan is NULL");
  BST_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), BST_ERR_INVALID_ARG,
              "alpha and beta must be finite");
  BST_REQUIRE(plan->C->nelem == 0 || dC, BST_ERR_INVALID_ARG, "dC is NULL");
  BST_REQUIRE(plan->contract || plan->A->nblocks == 0 || plan->A->data, BST_ERR_STATE,
              "A data not bound");
  BST_REQUIRE(plan->contract || plan->B->nblocks == 0 || plan->B->data, BST_ERR_STATE,
              "B data not bound");
  use_device(plan->ctx);
  cudaStream_t s = as_stream(stream);
  if (plan->contract) {
    bst::contract_adjoint(plan, dC, dA, dB, dC_in, alpha, beta, s);
    return BST_OK;
  }
  bst::adjoint_fp64(plan, plan->A->data, plan->B->data, dC, dA, dB, alpha, s);
  bst::scale_cin_grad(plan, dC, dC_in, beta, s);
  API_END
}

bst_status bst_multiply_adjoint(bst_plan *plan, const double *dC, double *dA, double *dB,
                                double alpha, void *stream) {
  return bst_plan_adjoint(plan, dC, dA, dB, nullptr, alpha, 0.0, stream);
}

bst_status bst_tune_set(bst_ctx *ctx, int32_t key, int32_t m, int32_t n, int32_t value) {
  API_BEGIN
  BST_REQUIRE(ctx, BST_ERR_INVALID_ARG, "ctx is NULL");
  switch (key) {
    case BST_TUNE_EMU_ROW_SCALE:
      BST_REQUIRE(value == 0 || value == 1, BST_ERR_INVALID_ARG, "value must be 0 or 1");
      ctx->tune_emu_row_scale = value;
      break;
    case BST_TUNE_EMU_SWAP:
      BST_REQUIRE(value >= -1 && value <= 1, BST_ERR_INVALID_ARG, "value must be -1, 0 or 1");
      BST_REQUIRE(m >= 1 && n >= 1, BST_ERR_INVALID_ARG, "m and n must be >= 1");
      if (value < 0)
        ctx->tune_emu_swap.erase({m, n});
      else
        ctx->tune_emu_swap[{m, n}] = value;
      break;
    case BST_TUNE_CONTRACT_SLAB:
      BST_REQUIRE(value == 0 || value == 1, BST_ERR_INVALID_ARG, "value must be 0 or 1");
      ctx->tune_contract_slab = value;
      break;
    case BST_TUNE_EMU_PANEL:
      BST_REQUIRE(value >= 0 && value <= 2, BST_ERR_INVALID_ARG, "value must be 0, 1 or 2");
      ctx->tune_emu_panel = value;
      break;
    case BST_TUNE_F64_SPLIT:
      BST_REQUIRE(value == -1 || (value >= 1 && value <= 16), BST_ERR_INVALID_ARG,
                  "value must be -1 or 1..16");
      BST_REQUIRE(m >= 1 && n >= 1, BST_ERR_INVALID_ARG, "m and n must be >= 1");
      if (value < 0)
        ctx->tune_f64_split.erase({m, n});
      else
        ctx->tune_f64_split[{m, n}] = value;
      break;
    default:
      throw Error{BST_ERR_INVALID_ARG, "unknown tuning key"};
  }
  ++ctx->tune_version;
  API_END
}

bst_status bst_tune_get(const bst_ctx *ctx, int32_t key, int32_t m, int32_t n, int32_t *value) {
  API_BEGIN
  BST_REQUIRE(ctx && value, BST_ERR_INVALID_ARG, "NULL argument");
  switch (key) {
    case BST_TUNE_EMU_ROW_SCALE:
      *value = ctx->tune_emu_row_scale;
      break;
    case BST_TUNE_EMU_SWAP: {
      auto it = ctx->tune_emu_swap.find({m, n});
      *value = it == ctx->tune_emu_swap.end() ? -1 : it->second;
      break;
    }
    case BST_TUNE_CONTRACT_SLAB:
      *value = ctx->tune_contract_slab;
      break;
    case BST_TUNE_EMU_PANEL:
      *value = ctx->tune_emu_panel;
      break;
    case BST_TUNE_F64_SPLIT: {
      auto it = ctx->tune_f64_split.find({m, n});
      *value = it == ctx->tune_f64_split.end() ? -1 : it->second;
      break;
    }
    default:
      throw Error{BST_ERR_INVALID_ARG, "unknown tuning key"};
  }
  API_END
}

bst_status bst_plan_destroy(bst_plan *plan) {
  API_BEGIN
  if (!plan) return BST_OK;
  bst::emu_state_free(plan);
  bst::panel_state_free(plan);
  bst::adj_state_free(plan);
  if (plan->C) {
    plan->C->owned_by_plan = false;
    delete plan->C;
  }
  plan->C = nullptr;
  bst::contract_free(plan);
  delete plan;
  API_END
}

}  // extern "C"
