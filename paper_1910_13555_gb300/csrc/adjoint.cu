// Adjoint of the block-sparse multiply (sampled block-sparse products), native FP64.
//
// For C_out = alpha op(A) op(B) + beta C_in with the filter decisions held fixed (a
// kept product stays kept; its derivative through the filter threshold is zero):
//     dop(A)_ik = alpha sum_{j: (i,k,j) kept} dC_ij op(B)_kj^T   on pattern(A)
//     dop(B)_kj = alpha sum_{i: (i,k,j) kept} op(A)_ik^T dC_ij   on pattern(B)
//     dC_in     = beta dC                                        on pattern(C_in)
// The paper defines only the forward product; this is its exact adjoint.
//
// Each output block has one owner warp (no atomics): the plan's stack entries are
// grouped by stored A block and by stored B block once (stable counting sort, cached
// in the plan), and warp `a` sums over the entries of A block `a`.  Lanes own output
// elements (m x k of dop(A) column by column, k x n of dop(B) row by row) in passes of
// 32 RA = 128, a block of more than one pass spread over several warps (a pass each);
// every block product reads its dC block and the other operand's block from L1/L2.
#include <algorithm>

#include "bst_internal.h"

namespace bst {

struct AdjState {
  Arena ar;
  int32_t *by_a = nullptr, *a_ptr = nullptr;  // entries grouped by stored A block
  int32_t *by_b = nullptr, *b_ptr = nullptr;  // entries grouped by stored B block
};

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int RA = 4;  // outputs per lane per pass (8 and 2 measured: 4 the best balance)

struct AdjArgs {
  const double *A, *B, *dC;
  double *dA, *dB;
  double alpha;
  int ta, tb;
  const int32_t *grp, *ptr;        // entries of each output block
  const int32_t *s_a, *s_b, *s_c, *s_cb;
  const int32_t *c_row, *c_col, *c_rsz, *c_csz;  // C block index and sizes
  // stored blocks of the output side; each is cut into nch chunks of `span` outputs
  // (consecutive passes), one warp per (block, chunk), so that large blocks spread over
  // several warps
  int64_t nblocks;
  int32_t nch, span;
  const int32_t *row, *col, *rsz, *csz;
  const int64_t *off;
};

// dop(A) for stored A block b: lanes own (p, l) of the m x k op block, numbered column
// by column (o = l m + p), so that a pass of 32 RA outputs covers every row p of a few
// columns l and reads each op(B) row it needs once per product.  (Numbered row by row,
// a pass covered one or two rows p and every op(B) row came in again for each of the m
// rows: on the rank-3 adjoint the kernel read 14.6 GB from DRAM for about 2 GB of
// operands.)  The sums run over the entries, then q, in the same order either way.
__global__ void k_adj_a(AdjArgs P) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t b = w / P.nch;
  if (b >= P.nblocks) return;
  const int R = P.rsz[P.row[b]], Cc = P.csz[P.col[b]];
  const int m = P.ta ? Cc : R, k = P.ta ? R : Cc;
  const int64_t ob = (w - b * P.nch) * (int64_t)P.span;
  if (ob >= m * k) return;
  const int o1 = (int)min((int64_t)m * k, ob + P.span);
  const int e0 = P.ptr[b], e1 = P.ptr[b + 1];
  double *out = P.dA + P.off[b];
  for (int o0 = (int)ob; o0 < o1; o0 += 32 * RA) {
    double acc[RA];
    int pr[RA], lr[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int o = o0 + lane + 32 * r;
      lr[r] = o / m;
      pr[r] = o - lr[r] * m;
      acc[r] = 0.0;
    }
    for (int q0 = e0; q0 < e1; ++q0) {
      const int e = P.grp[q0];
      const int c = P.s_cb[e];
      const int n = P.c_csz[P.c_col[c]];
      const double *g = P.dC + P.s_c[e];   // m x n
      const double *bb = P.B + P.s_b[e];   // op(B): k x n
      const int b_sl = P.tb ? 1 : n, b_sq = P.tb ? k : 1;
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        if (o0 + lane + 32 * r < m * k) {
          const double *gr = g + pr[r] * n, *br = bb + lr[r] * b_sl;
          double s = acc[r];
          for (int q = 0; q < n; ++q) s = fma(__ldg(gr + q), __ldg(br + q * b_sq), s);
          acc[r] = s;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      if (o0 + lane + 32 * r < m * k)
        out[P.ta ? lr[r] * m + pr[r] : pr[r] * k + lr[r]] = P.alpha * acc[r];
    }
  }
}

// dop(B) for stored B block b: lanes own (l, q) of the k x n op block
__global__ void k_adj_b(AdjArgs P) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t b = w / P.nch;
  if (b >= P.nblocks) return;
  const int R = P.rsz[P.row[b]], Cc = P.csz[P.col[b]];
  const int k = P.tb ? Cc : R, n = P.tb ? R : Cc;
  const int64_t ob = (w - b * P.nch) * (int64_t)P.span;
  if (ob >= k * n) return;
  const int o1 = (int)min((int64_t)k * n, ob + P.span);
  const int e0 = P.ptr[b], e1 = P.ptr[b + 1];
  double *out = P.dB + P.off[b];
  for (int o0 = (int)ob; o0 < o1; o0 += 32 * RA) {
    double acc[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) acc[r] = 0.0;
    for (int q0 = e0; q0 < e1; ++q0) {
      const int e = P.grp[q0];
      const int c = P.s_cb[e];
      const int m = P.c_rsz[P.c_row[c]];
      const double *g = P.dC + P.s_c[e];  // m x n
      const double *aa = P.A + P.s_a[e];  // op(A): m x k
      const int a_sp = P.ta ? 1 : k, a_sl = P.ta ? m : 1;
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        const int o = o0 + lane + 32 * r;
        if (o < k * n) {
          const int l = o / n, q = o % n;
          const double *ar = aa + l * a_sl, *gq = g + q;
          double s = acc[r];
          if (m >= 32) {
            // long inner sums (e.g. the 169-row folds of a rank-4 contraction): eight p at
            // a time, their 16 loads issued before the dependent FMAs (rank-4 adjoint
            // 21.0 -> 20.2 ms; unrolled for short sums too, the rank-3 adjoint lost 5 %)
#pragma unroll 8
            for (int p = 0; p < m; ++p) s = fma(__ldg(ar + p * a_sp), __ldg(gq + p * n), s);
          } else {
            for (int p = 0; p < m; ++p) s = fma(__ldg(ar + p * a_sp), __ldg(gq + p * n), s);
          }
          acc[r] = s;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int o = o0 + lane + 32 * r;
      if (o < k * n) {
        const int l = o / n, q = o % n;
        out[P.tb ? q * k + l : l * n + q] = P.alpha * acc[r];
      }
    }
  }
}

// dC_in = beta dC on the C_in blocks (one warp per C block that carries a C_in block)
__global__ void k_adj_cin(int64_t nc, const int32_t *c_cin, const int64_t *c_off,
                          const int64_t *cin_off, const int32_t *c_row, const int32_t *c_col,
                          const int32_t *rsz, const int32_t *csz, const double *dC, double *dCin,
                          double beta) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= nc) return;
  const int ci = c_cin[c];
  if (ci < 0) return;
  const int len = rsz[c_row[c]] * csz[c_col[c]];
  for (int e = lane; e < len; e += 32) dCin[cin_off[ci] + e] = beta * dC[c_off[c] + e];
}

// Chunks of kAdjChunkPasses passes (of 32 RA outputs) per warp, as many per block as
// the largest stored block of the output side needs; a warp whose chunk lies past its
// block's end returns at once.  Without host block sizes: one chunk per block.  One
// pass per chunk: more warps and shorter tails than 4 (the rank-4 adjoint's dU grid
// was 3.4 waves of resident CTAs): rank-4 adjoint 20.2 -> 16.8 ms, rank-3 86 -> 80.5 ms
// with passes of 256 outputs; passes of 128 (RA = 4): 16.5 and 79.8 ms.
constexpr int kAdjChunkPasses = 1;

void chunking(AdjArgs &P, const bst_matrix &M) {
  int32_t r = 0, c = 0;
  for (int32_t v : M.h_rsz) r = std::max(r, v);
  for (int32_t v : M.h_csz) c = std::max(c, v);
  const int64_t span = (int64_t)kAdjChunkPasses * 32 * RA;
  const int64_t most = (int64_t)r * c;
  if (M.h_rsz.empty() || M.h_csz.empty() || most <= span) {
    P.nch = 1;
    P.span = 1 << 30;
  } else {
    P.nch = (int32_t)((most + span - 1) / span);
    P.span = (int32_t)span;
  }
}

}  // namespace

void adj_state_free(bst_plan *p) {
  delete p->adj;
  p->adj = nullptr;
}

void adjoint_fp64(bst_plan *p, const double *A, const double *B, const double *dC, double *dA,
                  double *dB, double alpha, cudaStream_t s) {
  const bst_matrix *Am = p->A, *Bm = p->B;
  if (!p->adj) {
    p->adj = new AdjState();
    AdjState &S = *p->adj;
    S.ar.ctx = static_cast<Ctx *>(p->ctx);
    S.ar.stream = s;
    Arena scratch;
    scratch.ctx = S.ar.ctx;
    scratch.stream = s;
    S.by_a = S.ar.alloc_n<int32_t>((size_t)p->T);
    S.a_ptr = S.ar.alloc_n<int32_t>((size_t)Am->nblocks + 1);
    S.by_b = S.ar.alloc_n<int32_t>((size_t)p->T);
    S.b_ptr = S.ar.alloc_n<int32_t>((size_t)Bm->nblocks + 1);
    stable_partition(p->s_ab, p->T, (int32_t)std::max<int64_t>(Am->nblocks, 1), S.by_a, S.a_ptr,
                     scratch, s);
    stable_partition(p->s_bb, p->T, (int32_t)std::max<int64_t>(Bm->nblocks, 1), S.by_b, S.b_ptr,
                     scratch, s);
    BST_CUDA(cudaStreamSynchronize(s));
  }
  AdjState &S = *p->adj;
  AdjArgs P{};
  P.A = A;
  P.B = B;
  P.dC = dC;
  P.dA = dA;
  P.dB = dB;
  P.alpha = alpha;
  P.ta = p->ta;
  P.tb = p->tb;
  P.s_a = p->s_a;
  P.s_b = p->s_b;
  P.s_c = p->s_c;
  P.s_cb = p->s_cb;
  P.c_row = p->C->row;
  P.c_col = p->C->col;
  P.c_rsz = p->C->rsz;
  P.c_csz = p->C->csz;
  const int wpb = 8;
  if (Am->nblocks > 0 && dA) {
    P.grp = S.by_a;
    P.ptr = S.a_ptr;
    P.nblocks = Am->nblocks;
    P.row = Am->row;
    P.col = Am->col;
    P.rsz = Am->rsz;
    P.csz = Am->csz;
    P.off = Am->off;
    chunking(P, *Am);
    k_adj_a<<<nblk(Am->nblocks * P.nch, wpb), 32 * wpb, 0, s>>>(P);
    BST_CHECK_LAUNCH();
  }
  if (Bm->nblocks > 0 && dB) {
    P.grp = S.by_b;
    P.ptr = S.b_ptr;
    P.nblocks = Bm->nblocks;
    P.row = Bm->row;
    P.col = Bm->col;
    P.rsz = Bm->rsz;
    P.csz = Bm->csz;
    P.off = Bm->off;
    chunking(P, *Bm);
    k_adj_b<<<nblk(Bm->nblocks * P.nch, wpb), 32 * wpb, 0, s>>>(P);
    BST_CHECK_LAUNCH();
  }
}

void scale_cin_grad(bst_plan *p, const double *dC, double *dCin, double beta, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (!p->Cin || !dCin || nc == 0) return;
  const int wpb = 8;
  k_adj_cin<<<nblk(nc, wpb), 32 * wpb, 0, s>>>(nc, p->c_cin, p->C->off, p->Cin->off, p->C->row,
                                               p->C->col, p->C->rsz, p->C->csz, dC, dCin, beta);
  BST_CHECK_LAUNCH();
}

}  // namespace bst
