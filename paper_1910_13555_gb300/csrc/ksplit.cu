// bst_sum_parts: the reduction step of a K-split product, C = sum_i C~_i in a fixed
// order (paper Sec. 3.1: with S_C much smaller than S_A and S_B the inner dimension K is
// divided among the processes, each computes a partial product C~_i over its share of
// K, and the partial products are summed into C).
//
// Each process owns a contiguous range of the union C pattern and receives, from every
// process i, the blocks of C~_i that fall in that range (a contiguous run of C~_i, since
// every partial product keeps its blocks in CSR order).  This kernel adds them up: for
// every owned block u and every part i in increasing order, the block's elements in
// part i, located through src_off[i * nblocks + u] (-1: part i has no such block).  The
// order of the additions is the part order whatever the launch shape, so every process
// gets the same bits for the same inputs.  One warp per block, lanes over its elements
// (C blocks of a few hundred elements), read once and written once: bound by HBM, or by
// load latency when C is small.
#include "bst_internal.h"

namespace bst {
namespace {

constexpr int kWarps = 8;

// The block's part offsets are loaded once, 32 parts per round (lane i holds part i of
// the round), and the element loop issues the loads of up to 8 present parts before
// adding them in part order, so a warp keeps several loads in flight.
__global__ void __launch_bounds__(32 * kWarps)
    k_sum_parts(int32_t nparts, int64_t nblocks, const int64_t *__restrict__ dst_off,
                const int64_t *__restrict__ src_off, const double *__restrict__ src,
                double *__restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  for (int64_t u = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); u < nblocks; u += nwarps) {
    const int64_t d0 = dst_off[u], len = dst_off[u + 1] - d0;
    for (int64_t e0 = 0; e0 < len; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool live = e < len;
      double acc = 0.0;
      bool any = false;
      for (int32_t r0 = 0; r0 < nparts; r0 += 32) {
        const int64_t my = r0 + lane < nparts ? src_off[(int64_t)(r0 + lane) * nblocks + u] : -1;
        unsigned present = __ballot_sync(0xffffffffu, my >= 0);
        while (present) {
          // the next (up to) 8 present parts of this round, in part order
          int idx[8];
          int cnt = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            idx[k] = present ? __ffs(present) - 1 : -1;
            if (present) {
              present &= present - 1u;
              ++cnt;
            }
          }
          double v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const long long o = __shfl_sync(0xffffffffu, (long long)my, idx[k] < 0 ? 0 : idx[k]);
            v[k] = (k < cnt && live) ? __ldcs(src + o + e) : 0.0;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (k < cnt) {
              acc = any ? acc + v[k] : v[k];
              any = true;
            }
          }
        }
      }
      if (live) dst[d0 + e] = acc;
    }
  }
}

}  // namespace
}  // namespace bst

extern "C" {

bst_status bst_sum_parts(bst_ctx *ctx, int32_t nparts, int64_t nblocks, const int64_t *dst_off,
                         const int64_t *src_off, const double *src, double *dst, void *stream) {
  API_BEGIN
  BST_REQUIRE(ctx, BST_ERR_INVALID_ARG, "NULL context");
  BST_REQUIRE(nparts >= 1 && nblocks >= 0, BST_ERR_INVALID_ARG, "nparts < 1 or nblocks < 0");
  if (nblocks == 0) return BST_OK;
  BST_REQUIRE(dst_off && src_off && src && dst, BST_ERR_INVALID_ARG, "NULL argument");
  int cur = -1;
  BST_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t want = (nblocks + bst::kWarps - 1) / bst::kWarps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * 8);
  bst::k_sum_parts<<<grid, 32 * bst::kWarps, 0, s>>>(nparts, nblocks, dst_off, src_off, src, dst);
  BST_CHECK_LAUNCH();
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(cur));
  API_END
}

}  // extern "C"
