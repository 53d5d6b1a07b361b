// Block post-filter of a matrix: keep the blocks whose Frobenius norm is >= eps.
//
// The paper names the sign-matrix iteration of linear-scaling DFT among the library's
// operations (Sec. 2) but defines no filter; dropping the result blocks of small norm
// between the products of such a chain is a reading of this library, beside the filter
// on the block products.  bst_matrix_filter builds the kept
// pattern on the GPU -- block norms (the filter's own norm kernel), a stable compaction in
// CSR order, per-row counts, element offsets -- and returns it as a new matrix;
// bst_matrix_filter_copy then moves the kept blocks' elements into the caller's buffer,
// one warp per kept block.
#include <cstring>

#include "bst_internal.h"

namespace bst {
namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_keep_flags(int64_t n, const double *__restrict__ norms, double eps,
                             int32_t *__restrict__ keep) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) keep[b] = norms[b] >= eps ? 1 : 0;
}

// kept block b of X -> block pos[b] of Y: row, column, source, size and row count
__global__ void k_compact(int64_t n, const int32_t *__restrict__ keep, const int32_t *__restrict__ pos,
                          const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ rsz, const int32_t *__restrict__ csz,
                          int32_t *__restrict__ yrow, int32_t *__restrict__ ycol,
                          int32_t *__restrict__ ysrc, int64_t *__restrict__ ysize,
                          int32_t *__restrict__ rowcnt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n || !keep[b]) return;
  const int32_t q = pos[b];
  yrow[q] = row[b];
  ycol[q] = col[b];
  ysrc[q] = (int32_t)b;
  ysize[q] = (int64_t)rsz[row[b]] * csz[col[b]];
  atomicAdd(&rowcnt[row[b]], 1);
}

__global__ void k_filter_copy(int64_t ny, const int32_t *__restrict__ src,
                              const int64_t *__restrict__ xoff, const int64_t *__restrict__ yoff,
                              const double *__restrict__ x, double *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= ny) return;
  const double *xs = x + xoff[src[q]];
  double *yd = y + yoff[q];
  const int64_t len = yoff[q + 1] - yoff[q];
  for (int64_t e = lane; e < len; e += 32) yd[e] = xs[e];
}

}  // namespace
}  // namespace bst

using bst::Error;

extern "C" {

bst_status bst_matrix_filter(bst_ctx *ctx, const bst_matrix *X, double eps, void *stream,
                             bst_matrix **out) {
  try {
    BST_REQUIRE(ctx && X && out, BST_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    BST_REQUIRE(eps >= 0.0, BST_ERR_INVALID_ARG, "eps must be >= 0");
    BST_REQUIRE(X->nblocks == 0 || X->data, BST_ERR_STATE, "X data not bound");
    int cur = -1;
    BST_CUDA(cudaGetDevice(&cur));
    if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = X->nblocks;
    auto *Y = new bst_matrix();
    try {
      Y->ctx = ctx;
      Y->arena.ctx = static_cast<bst::Ctx *>(ctx);
      Y->arena.stream = s;
      Y->nbr = X->nbr;
      Y->nbc = X->nbc;
      Y->h_rsz = X->h_rsz;
      Y->h_csz = X->h_csz;
      bst::Arena scratch;
      scratch.ctx = static_cast<bst::Ctx *>(ctx);
      scratch.stream = s;
      Y->rsz = Y->arena.alloc_n<int32_t>(Y->h_rsz.size());
      Y->csz = Y->arena.alloc_n<int32_t>(Y->h_csz.size());
      if (!Y->h_rsz.empty())
        BST_CUDA(cudaMemcpyAsync(Y->rsz, X->rsz, 4 * Y->h_rsz.size(), cudaMemcpyDeviceToDevice, s));
      if (!Y->h_csz.empty())
        BST_CUDA(cudaMemcpyAsync(Y->csz, X->csz, 4 * Y->h_csz.size(), cudaMemcpyDeviceToDevice, s));
      double *norms = scratch.alloc_n<double>((size_t)n);
      int32_t *keep = scratch.alloc_n<int32_t>((size_t)n);
      int32_t *pos = scratch.alloc_n<int32_t>((size_t)n + 1);
      int32_t *rowcnt = scratch.alloc_n<int32_t>((size_t)X->nbr);
      if (n > 0) {
        bst::block_norms(X, norms, s);
        bst::k_keep_flags<<<bst::nblk(n, 256), 256, 0, s>>>(n, norms, eps, keep);
        BST_CHECK_LAUNCH();
      }
      bst::exscan_i32(keep, pos, n, scratch, s);
      int32_t ny32 = 0;
      {
        bst::ReadBack rb(ctx, s);
        rb.add(&ny32, pos + n, 4);
        rb.done();
      }
      const int64_t ny = ny32;
      Y->nblocks = ny;
      Y->row = Y->arena.alloc_n<int32_t>((size_t)ny);
      Y->col = Y->arena.alloc_n<int32_t>((size_t)ny);
      Y->src = Y->arena.alloc_n<int32_t>((size_t)ny);
      Y->off = Y->arena.alloc_n<int64_t>((size_t)ny + 1);
      Y->rowptr = Y->arena.alloc_n<int32_t>((size_t)X->nbr + 1);
      int64_t *ysize = scratch.alloc_n<int64_t>((size_t)ny);
      bst::fill_i32(rowcnt, 0, X->nbr, s);
      if (n > 0) {
        bst::k_compact<<<bst::nblk(n, 256), 256, 0, s>>>(n, keep, pos, X->row, X->col, X->rsz,
                                                         X->csz, Y->row, Y->col, Y->src, ysize,
                                                         rowcnt);
        BST_CHECK_LAUNCH();
      }
      bst::exscan_i32(rowcnt, Y->rowptr, X->nbr, scratch, s);
      bst::exscan_i64(ysize, Y->off, ny, scratch, s);
      int64_t nelem = 0;
      {
        bst::ReadBack rb(ctx, s);
        rb.add(&nelem, Y->off + ny, 8);
        rb.done();
      }
      Y->nelem = nelem;
      Y->src_nblocks = n;
      scratch.release_all();
    } catch (...) {
      delete Y;
      throw;
    }
    *out = Y;
  } catch (const bst::Error &e) {
    bst::set_error(e.msg);
    return e.code;
  } catch (...) {
    bst::set_error("unexpected internal error");
    return BST_ERR_INVALID_ARG;
  }
  return BST_OK;
}

bst_status bst_matrix_filter_copy(const bst_matrix *X, bst_matrix *Y, void *stream) {
  try {
    BST_REQUIRE(X && Y, BST_ERR_INVALID_ARG, "NULL argument");
    BST_REQUIRE(Y->src != nullptr && Y->src_nblocks == X->nblocks && Y->nbr == X->nbr &&
                    Y->nbc == X->nbc,
                BST_ERR_SHAPE_MISMATCH, "Y is not a filter result of X");
    BST_REQUIRE(X->nblocks == 0 || X->data, BST_ERR_STATE, "X data not bound");
    BST_REQUIRE(Y->nelem == 0 || Y->data, BST_ERR_STATE, "Y data not bound");
    int cur = -1;
    BST_CUDA(cudaGetDevice(&cur));
    if (cur != X->ctx->device) BST_CUDA(cudaSetDevice(X->ctx->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (Y->nblocks > 0) {
      const int wpb = 8;
      bst::k_filter_copy<<<bst::nblk(Y->nblocks, wpb), 32 * wpb, 0, s>>>(
          Y->nblocks, Y->src, X->off, Y->off, X->data, Y->data);
      BST_CHECK_LAUNCH();
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

}  // extern "C"
