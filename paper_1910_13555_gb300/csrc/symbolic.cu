// Symbolic phase of the block-sparse multiply on the GPU.
//
// Paper Sec. 2 describes the local multiplication as pairwise products of small
// blocks, organised by looping over the row blocks of A and, for each, over the
// matching blocks of B, with the products gathered into batches.  Here one warp owns
// one block row i of C = op(A) op(B) and walks every candidate pair (A_ik, B_kj) of
// that row (k ascending, then j ascending) three times:
//   count  -- a bitmap over the block columns of C marks the kept j (filter:
//             ||A_ik||_F ||B_kj||_F >= eps), giving the row's C blocks and products;
//   fill   -- the row's C block columns in order, per-C-block product counts, then
//             every kept product written at its place in (i, j, k) order;
// after which a stable counting sort by (m, n, k) size bucket turns the (i, j, k)
// list into the bucketed stacks (a_off, b_off, c_off) and, per (C block, k class),
// the run of entries that the numeric kernel of that C block reads.
//
// The candidate pairs of a row are walked 32 at a time in a flattened order: 32 A
// blocks of the row are loaded, the lengths of their B rows are scanned across the
// warp, and lane x takes pair number x, finding its A block by a binary search over
// the scanned lengths.  This keeps lanes busy whether B rows are long (square
// products) or hold one or two blocks (the tall-skinny A^T B of Sec. 3.1).
#include <algorithm>
#include <climits>

#include "bst_internal.h"

namespace bst {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ int warp_incl_scan_i(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// ---- block norms -------------------------------------------------------------------

// Matrices of small blocks (at most kNormSmall elements): one warp per group of 32
// consecutive blocks.  Lane j first loads the size and offset of block j of the group
// (one coalesced round of index loads).  For each block the lanes accumulate
// lane-strided squares and park their 32 partial sums in a row of shared memory; then
// lane j adds row j (the partials of block j) in lane order and takes its square root.
// GB300's FP64 pipe takes as long for a warp instruction with one active lane as with
// 32: a butterfly costs five full FP64 instructions per block, the transposed sum one
// per block, and the group's 32 square roots run together.  Matrices with larger blocks
// (a contraction's folded views, up to hundreds of thousands of elements a block): one
// warp per block, a butterfly at the end (grouping them left a few hundred warps
// streaming 32 large blocks each: 4.6 ms for the rank-4 operand against a few tens of
// microseconds).
constexpr int kNormGroup = 32;
constexpr int kNormWarps = 4;
constexpr int64_t kNormSmall = 1024;

__global__ void __launch_bounds__(32 * kNormWarps)
    k_block_norms1(int64_t nblocks, const int32_t *__restrict__ row,
                   const int32_t *__restrict__ col, const int32_t *__restrict__ rsz,
                   const int32_t *__restrict__ csz, const int64_t *__restrict__ off,
                   const double *__restrict__ data, double *__restrict__ norms) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kNormWarps + (threadIdx.x >> 5);
  if (b >= nblocks) return;
  const int64_t len = (int64_t)rsz[row[b]] * csz[col[b]];
  const double *x = data + off[b];
  double s = 0.0;
  for (int64_t e = lane; e < len; e += 32) {
    const double v = __ldg(x + e);
    s = fma(v, v, s);
  }
  s = warp_sum_d(s);
  if (lane == 0) norms[b] = sqrt(s);
}

__global__ void __launch_bounds__(32 * kNormWarps)
    k_block_norms(int64_t nblocks, const int32_t *__restrict__ row,
                  const int32_t *__restrict__ col, const int32_t *__restrict__ rsz,
                  const int32_t *__restrict__ csz, const int64_t *__restrict__ off,
                  const double *__restrict__ data, double *__restrict__ norms) {
  __shared__ double part[kNormWarps][kNormGroup][33];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t b0 = ((int64_t)blockIdx.x * kNormWarps + wl) * kNormGroup;
  if (b0 >= nblocks) return;
  const int nb = (int)min((int64_t)kNormGroup, nblocks - b0);
  int my_len = 0;
  long long my_off = 0;
  if (lane < nb) {
    my_len = rsz[row[b0 + lane]] * csz[col[b0 + lane]];
    my_off = off[b0 + lane];
  }
  double(*P)[33] = part[wl];
  for (int j = 0; j < nb; ++j) {
    const int len = __shfl_sync(0xffffffffu, my_len, j);
    const double *x = data + __shfl_sync(0xffffffffu, my_off, j);
    double s = 0.0;
    for (int e = lane; e < len; e += 32) {
      const double v = __ldg(x + e);
      s = fma(v, v, s);
    }
    P[j][lane] = s;
  }
  __syncwarp();
  if (lane < nb) {
    double t = P[lane][0];
    for (int q = 1; q < 32; ++q) t += P[lane][q];
    norms[b0 + lane] = sqrt(t);
  }
}

// ---- operand views -----------------------------------------------------------------

struct SymArgs {
  int32_t M, N;
  int32_t words;                 // 32-bit words of the per-row bitmap over N columns
  const int32_t *oa_rowptr, *oa_col, *oa_blk;
  const int32_t *ob_rowptr, *ob_col, *ob_blk;
  const double *nA, *nB;
  double eps;
  const int32_t *ci_rowptr, *ci_col;  // C_in (may be null)
};

// Walk the candidate pairs (a, b) of C row i, 32 per step, in (a, b) order.
// f(valid, sa, na, k, b) is called by all 32 lanes together (valid = lane has a pair).
template <class F>
__device__ __forceinline__ void for_row_pairs(const SymArgs &S, int i, F f) {
  const int lane = threadIdx.x & 31;
  const int a0 = S.oa_rowptr[i], a1 = S.oa_rowptr[i + 1];
  for (int ac = a0; ac < a1; ac += 32) {
    const int a = ac + lane;
    int len = 0, bstart = 0, k = 0, sa = 0;
    double na = 0.0;
    if (a < a1) {
      k = S.oa_col[a];
      sa = S.oa_blk ? S.oa_blk[a] : a;
      na = S.nA[sa];
      bstart = S.ob_rowptr[k];
      len = S.ob_rowptr[k + 1] - bstart;
    }
    const int incl = warp_incl_scan_i(len);
    const int excl = incl - len;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int x0 = 0; x0 < total; x0 += 32) {
      const int x = x0 + lane;
      // largest lane s with excl_s <= x (excl is non-decreasing and excl_0 = 0)
      int s = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        int e = __shfl_sync(0xffffffffu, excl, s + step);
        if (e <= x) s += step;
      }
      const int ks = __shfl_sync(0xffffffffu, k, s);
      const int sas = __shfl_sync(0xffffffffu, sa, s);
      const double nas = __shfl_sync(0xffffffffu, na, s);
      const int b = __shfl_sync(0xffffffffu, bstart, s) + (x - __shfl_sync(0xffffffffu, excl, s));
      f(x < total, sas, nas, ks, b);
    }
  }
}

__global__ void k_sym_count(SymArgs S, int32_t *__restrict__ c_rownnz,
                            int32_t *__restrict__ t_rowcnt, int32_t *__restrict__ cand_rowcnt) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + wl;
  if (i >= S.M) return;
  uint32_t *bm = smem + (size_t)wl * S.words;
  for (int w = lane; w < S.words; w += 32) bm[w] = 0u;
  __syncwarp();
  int tc = 0, cc = 0;
  for_row_pairs(S, i, [&](bool valid, int sa, double na, int k, int b) {
    if (!valid) return;
    ++cc;
    const int sb = S.ob_blk ? S.ob_blk[b] : b;
    if (na * S.nB[sb] >= S.eps) {
      const int j = S.ob_col[b];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
      ++tc;
    }
  });
  if (S.ci_rowptr) {
    for (int b = S.ci_rowptr[i] + lane; b < S.ci_rowptr[i + 1]; b += 32) {
      const int j = S.ci_col[b];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
  }
  __syncwarp();
  int pc = 0;
  for (int w = lane; w < S.words; w += 32) pc += __popc(bm[w]);
  pc = warp_sum_i(pc);
  tc = warp_sum_i(tc);
  cc = warp_sum_i(cc);
  if (lane == 0) {
    c_rownnz[i] = pc;
    t_rowcnt[i] = tc;
    cand_rowcnt[i] = cc;
  }
}

struct FillOut {
  const int32_t *c_rowptr;
  const int64_t *t_rowptr;
  int32_t *c_col, *c_row, *c_cin;
  int32_t *cnt;      // per C block: product count, then the write cursor
  int32_t *t_start;  // per C block: first product in (i, j, k) order
  int32_t *t_a, *t_b, *t_c, *t_k;
};

__global__ void k_sym_fill(SymArgs S, FillOut O) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + wl;
  if (i >= S.M) return;
  uint32_t *bm = smem + (size_t)wl * 2 * S.words;
  uint32_t *pre = bm + S.words;
  for (int w = lane; w < S.words; w += 32) bm[w] = 0u;
  __syncwarp();
  // 1. bitmap of the row's C block columns
  for_row_pairs(S, i, [&](bool valid, int sa, double na, int k, int b) {
    if (!valid) return;
    const int sb = S.ob_blk ? S.ob_blk[b] : b;
    if (na * S.nB[sb] >= S.eps) {
      const int j = S.ob_col[b];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
  });
  if (S.ci_rowptr) {
    for (int b = S.ci_rowptr[i] + lane; b < S.ci_rowptr[i + 1]; b += 32) {
      const int j = S.ci_col[b];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
  }
  __syncwarp();
  // 2. prefix popcounts per word -> rank of column j inside the row
  {
    int carry = 0;
    for (int w0 = 0; w0 < S.words; w0 += 32) {
      const int w = w0 + lane;
      const int v = w < S.words ? __popc(bm[w]) : 0;
      const int inc = warp_incl_scan_i(v);
      if (w < S.words) pre[w] = carry + inc - v;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncwarp();
  const int cr0 = O.c_rowptr[i], cr1 = O.c_rowptr[i + 1];
  for (int w = lane; w < S.words; w += 32) {
    uint32_t bits = bm[w];
    int pos = cr0 + pre[w];
    while (bits) {
      const int t = __ffs(bits) - 1;
      bits &= bits - 1u;
      O.c_col[pos] = w * 32 + t;
      O.c_row[pos] = i;
      ++pos;
    }
  }
  for (int c = cr0 + lane; c < cr1; c += 32) {
    O.c_cin[c] = -1;
    O.cnt[c] = 0;
  }
  __syncwarp();
  auto rank = [&](int j) {
    return pre[j >> 5] + __popc(bm[j >> 5] & ((1u << (j & 31)) - 1u));
  };
  if (S.ci_rowptr) {
    for (int b = S.ci_rowptr[i] + lane; b < S.ci_rowptr[i + 1]; b += 32)
      O.c_cin[cr0 + rank(S.ci_col[b])] = b;
  }
  // 3. products per C block
  for_row_pairs(S, i, [&](bool valid, int sa, double na, int k, int b) {
    if (!valid) return;
    const int sb = S.ob_blk ? S.ob_blk[b] : b;
    if (na * S.nB[sb] >= S.eps) atomicAdd(&O.cnt[cr0 + rank(S.ob_col[b])], 1);
  });
  __syncwarp();
  // 4. exclusive scan of the counts along the row -> start of each C block's run
  {
    int carry = (int)O.t_rowptr[i];
    for (int c0 = cr0; c0 < cr1; c0 += 32) {
      const int c = c0 + lane;
      const int v = c < cr1 ? O.cnt[c] : 0;
      const int inc = warp_incl_scan_i(v);
      if (c < cr1) {
        O.t_start[c] = carry + inc - v;
        O.cnt[c] = carry + inc - v;  // becomes the write cursor
      }
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncwarp();
  // 5. write the products; pairs arrive in (k, j) order, and each C block's cursor
  //    advances in k order, so every C block's products end up sorted by k.
  for_row_pairs(S, i, [&](bool valid, int sa, double na, int k, int b) {
    int sb = 0, c = -1;
    bool kept = false;
    if (valid) {
      sb = S.ob_blk ? S.ob_blk[b] : b;
      kept = na * S.nB[sb] >= S.eps;
      if (kept) c = cr0 + rank(S.ob_col[b]);
    }
    const unsigned km = __ballot_sync(0xffffffffu, kept);
    unsigned peers = 0;
    if (kept) {
      peers = __match_any_sync(km, c);
      const int pos = O.cnt[c] + __popc(peers & ((1u << lane) - 1u));
      O.t_a[pos] = sa;
      O.t_b[pos] = sb;
      O.t_c[pos] = c;
      O.t_k[pos] = k;
    }
    __syncwarp();
    if (kept && (int)(__ffs(peers) - 1) == lane) O.cnt[c] += __popc(peers);
    __syncwarp();
  });
}

__global__ void k_i64_to_i32_one(const int64_t *__restrict__ in, int32_t *__restrict__ out) {
  *out = (int32_t)*in;
}

__global__ void k_rowptr_i64_to_i32(const int64_t *__restrict__ in, int32_t *__restrict__ out,
                                    int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) out[i] = (int32_t)in[i];
}

__global__ void k_c_sizes(int64_t nc, const int32_t *__restrict__ c_row,
                          const int32_t *__restrict__ c_col, const int32_t *__restrict__ msz,
                          const int32_t *__restrict__ nsz, const int32_t *__restrict__ m_cls,
                          const int32_t *__restrict__ n_cls, int32_t Dn,
                          int64_t *__restrict__ size, int32_t *__restrict__ cls) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int r = c_row[c], q = c_col[c];
  size[c] = (int64_t)msz[r] * nsz[q];
  cls[c] = m_cls[r] * Dn + n_cls[q];
}

__global__ void k_bucket_keys(int64_t T, const int32_t *__restrict__ t_c,
                              const int32_t *__restrict__ t_k, const int32_t *__restrict__ c_cls,
                              const int32_t *__restrict__ k_cls, int32_t Dk,
                              int32_t *__restrict__ key) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < T) key[e] = c_cls[t_c[e]] * Dk + k_cls[t_k[e]];
}

struct EmitArgs {
  int64_t T;
  const int32_t *perm;
  const int32_t *t_a, *t_b, *t_c, *t_k;
  const int64_t *a_off, *b_off, *c_off;
  const int32_t *k_cls;
  int32_t Dk;
  int32_t *s_a, *s_b, *s_c, *s_cb, *s_k, *s_ab, *s_bb;
  int32_t *run_start, *run_len;
  int32_t *refA, *refB;
};

__global__ void k_emit_stacks(EmitArgs E) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= E.T) return;
  const int p = E.perm[q];
  const int a = E.t_a[p], b = E.t_b[p], c = E.t_c[p], k = E.t_k[p];
  E.s_a[q] = (int32_t)E.a_off[a];
  E.s_b[q] = (int32_t)E.b_off[b];
  E.s_c[q] = (int32_t)E.c_off[c];
  E.s_cb[q] = c;
  E.s_k[q] = k;
  E.s_ab[q] = a;
  E.s_bb[q] = b;
  const int64_t r = (int64_t)c * E.Dk + E.k_cls[k];
  atomicMin(&E.run_start[r], (int32_t)q);
  atomicAdd(&E.run_len[r], 1);
  E.refA[a] = 1;
  E.refB[b] = 1;
}

// referenced elements: sum over flagged blocks of their areas
__global__ void k_ref_elems(int64_t nblocks, const int32_t *__restrict__ flag,
                            const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ rsz, const int32_t *__restrict__ csz,
                            unsigned long long *__restrict__ out) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (b < nblocks && flag[b]) v = (unsigned long long)rsz[row[b]] * csz[col[b]];
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

}  // namespace

void block_norms(const bst_matrix *m, double *norms, cudaStream_t s) {
  if (m->nblocks == 0) return;
  BST_REQUIRE(m->data != nullptr, BST_ERR_STATE, "matrix data not bound");
  int64_t rmax = 0, cmax = 0;
  for (int32_t v : m->h_rsz) rmax = std::max<int64_t>(rmax, v);
  for (int32_t v : m->h_csz) cmax = std::max<int64_t>(cmax, v);
  if (m->h_rsz.empty() || m->h_csz.empty() || rmax * cmax > kNormSmall) {
    k_block_norms1<<<nblk(m->nblocks, kNormWarps), 32 * kNormWarps, 0, s>>>(
        m->nblocks, m->row, m->col, m->rsz, m->csz, m->off, m->data, norms);
  } else {
    const int64_t groups = (m->nblocks + kNormGroup - 1) / kNormGroup;
    k_block_norms<<<nblk(groups, kNormWarps), 32 * kNormWarps, 0, s>>>(
        m->nblocks, m->row, m->col, m->rsz, m->csz, m->off, m->data, norms);
  }
  BST_CHECK_LAUNCH();
}

OpView make_opview(const bst_matrix *m, bool trans, Arena &ar, cudaStream_t s) {
  OpView v;
  v.trans = trans;
  v.nr = trans ? m->nbc : m->nbr;
  v.nc = trans ? m->nbr : m->nbc;
  v.rs = trans ? m->csz : m->rsz;
  v.cs = trans ? m->rsz : m->csz;
  v.h_rs = trans ? m->h_csz : m->h_rsz;
  v.h_cs = trans ? m->h_rsz : m->h_csz;
  if (!trans) {
    v.rowptr = m->rowptr;
    v.col = m->col;
    v.blk = nullptr;
    return v;
  }
  // CSC of the stored matrix by a stable counting sort on the block column: within
  // each column the blocks stay in ascending row order.
  int32_t *perm = ar.alloc_n<int32_t>((size_t)m->nblocks);
  int32_t *rowptr = ar.alloc_n<int32_t>((size_t)std::max<int32_t>(m->nbc, 1) + 1);
  int32_t *col = ar.alloc_n<int32_t>((size_t)m->nblocks);
  stable_partition(m->col, m->nblocks, std::max<int32_t>(m->nbc, 1), perm, rowptr, ar, s);
  gather_i32(m->row, perm, col, m->nblocks, s);
  v.rowptr = rowptr;
  v.col = col;
  v.blk = perm;
  return v;
}

static std::vector<int32_t> distinct_sorted(const std::vector<int32_t> &v) {
  std::vector<int32_t> u(v);
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  return u;
}

static int32_t *upload_classes(const std::vector<int32_t> &sizes, const std::vector<int32_t> &vals,
                               Arena &ar, Upload &up) {
  std::vector<int32_t> cls(sizes.size());
  for (size_t i = 0; i < sizes.size(); ++i)
    cls[i] = (int32_t)(std::lower_bound(vals.begin(), vals.end(), sizes[i]) - vals.begin());
  return up.add_vector(ar, cls);
}

void symbolic_phase(bst_plan *p, cudaStream_t s) {
  Arena &ar = p->arena;
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  const bst_matrix *A = p->A, *B = p->B, *Ci = p->Cin;
  const OpView &oa = p->oa, &ob = p->ob;
  const int32_t M = p->M, N = p->N;

  // size classes of C rows (m), C columns (n) and the inner dimension (k)
  p->m_vals = distinct_sorted(oa.h_rs);
  p->n_vals = distinct_sorted(ob.h_cs);
  p->k_vals = distinct_sorted(oa.h_cs);
  p->Dm = std::max<int32_t>(1, (int32_t)p->m_vals.size());
  p->Dn = std::max<int32_t>(1, (int32_t)p->n_vals.size());
  p->Dk = std::max<int32_t>(1, (int32_t)p->k_vals.size());
  const int64_t nb_all = (int64_t)p->Dm * p->Dn * p->Dk;
  BST_REQUIRE(nb_all <= (1 << 20), BST_ERR_UNSUPPORTED, "more than 2^20 (m,n,k) size buckets");
  p->nb_all = (int32_t)nb_all;
  {
    Upload up(p->ctx, s);
    p->m_cls = upload_classes(oa.h_rs, p->m_vals, ar, up);
    p->n_cls = upload_classes(ob.h_cs, p->n_vals, ar, up);
    p->k_cls = upload_classes(oa.h_cs, p->k_vals, ar, up);
    std::vector<int32_t> cm((size_t)p->Dm * p->Dn), cn((size_t)p->Dm * p->Dn), kv(p->k_vals);
    for (int32_t a = 0; a < p->Dm; ++a)
      for (int32_t b = 0; b < p->Dn; ++b) {
        cm[(size_t)a * p->Dn + b] = p->m_vals.empty() ? 0 : p->m_vals[a];
        cn[(size_t)a * p->Dn + b] = p->n_vals.empty() ? 0 : p->n_vals[b];
      }
    if (kv.empty()) kv.push_back(0);
    p->cls_m = up.add_vector(ar, cm);
    p->cls_n = up.add_vector(ar, cn);
    p->kval = up.add_vector(ar, kv);
    up.done_async();  // staged on the host already; the plan synchronises later
  }

  // block norms (filter input)
  double *nA = scratch.alloc_n<double>((size_t)A->nblocks);
  double *nB = scratch.alloc_n<double>((size_t)B->nblocks);
  block_norms(A, nA, s);
  block_norms(B, nB, s);

  SymArgs S;
  S.M = M;
  S.N = N;
  S.words = (N + 31) / 32;
  S.oa_rowptr = oa.rowptr;
  S.oa_col = oa.col;
  S.oa_blk = oa.blk;
  S.ob_rowptr = ob.rowptr;
  S.ob_col = ob.col;
  S.ob_blk = ob.blk;
  S.nA = nA;
  S.nB = nB;
  S.eps = p->eps;
  S.ci_rowptr = Ci ? Ci->rowptr : nullptr;
  S.ci_col = Ci ? Ci->col : nullptr;

  // warps per CTA from the bitmap size (fill keeps bitmap + prefix per warp)
  const size_t per_warp = (size_t)S.words * 8;
  const size_t smem_cap = std::min<size_t>(p->ctx->max_smem_optin, 200 * 1024);
  BST_REQUIRE(per_warp <= smem_cap, BST_ERR_UNSUPPORTED,
              "C has too many block columns for the per-row bitmap");
  int wpc = (int)std::min<size_t>(8, std::max<size_t>(1, (48 * 1024) / std::max<size_t>(per_warp, 1)));
  if ((size_t)wpc * per_warp > smem_cap) wpc = 1;
  const size_t smem_count = (size_t)wpc * S.words * 4, smem_fill = (size_t)wpc * per_warp;
  BST_CUDA(cudaFuncSetAttribute(k_sym_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem_count, 1)));
  BST_CUDA(cudaFuncSetAttribute(k_sym_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem_fill, 1)));

  int32_t *c_rownnz = scratch.alloc_n<int32_t>((size_t)M);
  int32_t *t_rowcnt = scratch.alloc_n<int32_t>((size_t)M);
  int32_t *cand_rowcnt = scratch.alloc_n<int32_t>((size_t)M);
  if (M > 0) {
    k_sym_count<<<nblk(M, wpc), 32 * wpc, smem_count, s>>>(S, c_rownnz, t_rowcnt, cand_rowcnt);
    BST_CHECK_LAUNCH();
  }
  int64_t *c_rowptr64 = scratch.alloc_n<int64_t>((size_t)M + 1);
  int64_t *t_rowptr = scratch.alloc_n<int64_t>((size_t)M + 1);
  int64_t *cand_ptr = scratch.alloc_n<int64_t>((size_t)M + 1);
  exscan_i32_i64(c_rownnz, c_rowptr64, M, scratch, s);
  exscan_i32_i64(t_rowcnt, t_rowptr, M, scratch, s);
  exscan_i32_i64(cand_rowcnt, cand_ptr, M, scratch, s);
  int64_t tot[3];
  {
    ReadBack rb(p->ctx, s);
    rb.add(&tot[0], c_rowptr64 + M, 8);
    rb.add(&tot[1], t_rowptr + M, 8);
    rb.add(&tot[2], cand_ptr + M, 8);
    rb.done();
  }
  const int64_t nnzC = tot[0], T = tot[1], ncand = tot[2];
  BST_REQUIRE(nnzC < INT32_MAX && T < INT32_MAX, BST_ERR_OVERFLOW,
              "more than 2^31-1 C blocks or kept products");
  p->T = T;

  // C_out pattern
  bst_matrix *C = p->C;
  C->nbr = M;
  C->nbc = N;
  C->h_rsz = oa.h_rs;
  C->h_csz = ob.h_cs;
  C->nblocks = nnzC;
  C->rsz = const_cast<int32_t *>(oa.rs);
  C->csz = const_cast<int32_t *>(ob.cs);
  C->rowptr = ar.alloc_n<int32_t>((size_t)M + 1);
  C->row = ar.alloc_n<int32_t>((size_t)nnzC);
  C->col = ar.alloc_n<int32_t>((size_t)nnzC);
  C->off = ar.alloc_n<int64_t>((size_t)nnzC + 1);
  k_rowptr_i64_to_i32<<<nblk(M + 1, 256), 256, 0, s>>>(c_rowptr64, C->rowptr, M);
  BST_CHECK_LAUNCH();
  p->c_cin = ar.alloc_n<int32_t>((size_t)nnzC);
  p->c_cls = ar.alloc_n<int32_t>((size_t)nnzC);
  p->t_start = ar.alloc_n<int32_t>((size_t)nnzC + 1);
  int32_t *cnt = scratch.alloc_n<int32_t>((size_t)nnzC);
  int32_t *t_a = scratch.alloc_n<int32_t>((size_t)T);
  int32_t *t_b = scratch.alloc_n<int32_t>((size_t)T);
  int32_t *t_c = scratch.alloc_n<int32_t>((size_t)T);
  int32_t *t_k = scratch.alloc_n<int32_t>((size_t)T);
  FillOut O;
  O.c_rowptr = C->rowptr;
  O.t_rowptr = t_rowptr;
  O.c_col = C->col;
  O.c_row = C->row;
  O.c_cin = p->c_cin;
  O.cnt = cnt;
  O.t_start = p->t_start;
  O.t_a = t_a;
  O.t_b = t_b;
  O.t_c = t_c;
  O.t_k = t_k;
  if (M > 0) {
    k_sym_fill<<<nblk(M, wpc), 32 * wpc, smem_fill, s>>>(S, O);
    BST_CHECK_LAUNCH();
  }
  // t_start[nnzC] = T, from the device's own count (no host round trip)
  k_i64_to_i32_one<<<1, 1, 0, s>>>(t_rowptr + M, p->t_start + nnzC);
  BST_CHECK_LAUNCH();

  // element offsets and (m,n) class of every C block
  int64_t *csize = scratch.alloc_n<int64_t>((size_t)nnzC);
  if (nnzC > 0) {
    k_c_sizes<<<nblk(nnzC, 256), 256, 0, s>>>(nnzC, C->row, C->col, oa.rs, ob.cs, p->m_cls,
                                              p->n_cls, p->Dn, csize, p->c_cls);
    BST_CHECK_LAUNCH();
  }
  exscan_i64(csize, C->off, nnzC, scratch, s);
  int64_t nelemC = 0;  // read back with the class and bucket pointers below

  // numeric task list: C blocks grouped by (m, n) class, CSR order inside a class
  const int32_t ncls = p->Dm * p->Dn;
  p->task_c = ar.alloc_n<int32_t>((size_t)nnzC);
  p->class_ptr = ar.alloc_n<int32_t>((size_t)ncls + 1);
  stable_partition(p->c_cls, nnzC, ncls, p->task_c, p->class_ptr, scratch, s);
  p->h_class_ptr.assign((size_t)ncls + 1, 0);
  ReadBack rb_ptrs(p->ctx, s);  // class and bucket pointers, read together below
  rb_ptrs.add(p->h_class_ptr.data(), p->class_ptr, sizeof(int32_t) * (ncls + 1));

  // bucketed stacks
  int32_t *key = scratch.alloc_n<int32_t>((size_t)T);
  if (T > 0) {
    k_bucket_keys<<<nblk(T, 256), 256, 0, s>>>(T, t_c, t_k, p->c_cls, p->k_cls, p->Dk, key);
    BST_CHECK_LAUNCH();
  }
  int32_t *perm = scratch.alloc_n<int32_t>((size_t)T);
  int32_t *bptr = scratch.alloc_n<int32_t>((size_t)p->nb_all + 1);
  stable_partition(key, T, p->nb_all, perm, bptr, scratch, s);
  std::vector<int32_t> hb((size_t)p->nb_all + 1);
  rb_ptrs.add(hb.data(), bptr, sizeof(int32_t) * hb.size());
  p->s_a = ar.alloc_n<int32_t>((size_t)T);
  p->s_b = ar.alloc_n<int32_t>((size_t)T);
  p->s_c = ar.alloc_n<int32_t>((size_t)T);
  p->s_cb = ar.alloc_n<int32_t>((size_t)T);
  p->s_k = ar.alloc_n<int32_t>((size_t)T);
  p->s_ab = ar.alloc_n<int32_t>((size_t)T);
  p->s_bb = ar.alloc_n<int32_t>((size_t)T);
  const int64_t nruns = nnzC * (int64_t)p->Dk;
  BST_REQUIRE(nruns < INT32_MAX, BST_ERR_UNSUPPORTED, "run table too large");
  p->run_start = ar.alloc_n<int32_t>((size_t)nruns);
  p->run_len = ar.alloc_n<int32_t>((size_t)nruns);
  fill_i32(p->run_start, INT32_MAX, nruns, s);
  BST_CUDA(cudaMemsetAsync(p->run_len, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(nruns, 1), s));
  int32_t *refA = scratch.alloc_n<int32_t>((size_t)A->nblocks);
  int32_t *refB = scratch.alloc_n<int32_t>((size_t)B->nblocks);
  BST_CUDA(cudaMemsetAsync(refA, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(A->nblocks, 1), s));
  BST_CUDA(cudaMemsetAsync(refB, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(B->nblocks, 1), s));
  if (T > 0) {
    EmitArgs E;
    E.T = T;
    E.perm = perm;
    E.t_a = t_a;
    E.t_b = t_b;
    E.t_c = t_c;
    E.t_k = t_k;
    E.a_off = A->off;
    E.b_off = B->off;
    E.c_off = C->off;
    E.k_cls = p->k_cls;
    E.Dk = p->Dk;
    E.s_a = p->s_a;
    E.s_b = p->s_b;
    E.s_c = p->s_c;
    E.s_cb = p->s_cb;
    E.s_k = p->s_k;
    E.s_ab = p->s_ab;
    E.s_bb = p->s_bb;
    E.run_start = p->run_start;
    E.run_len = p->run_len;
    E.refA = refA;
    E.refB = refB;
    k_emit_stacks<<<nblk(T, 256), 256, 0, s>>>(E);
    BST_CHECK_LAUNCH();
  }
  p->items_counter = ar.alloc_n<unsigned long long>(1);
  unsigned long long *refel = scratch.alloc_n<unsigned long long>(2);
  BST_CUDA(cudaMemsetAsync(refel, 0, 16, s));
  if (A->nblocks > 0) {
    k_ref_elems<<<nblk(A->nblocks, 256), 256, 0, s>>>(A->nblocks, refA, A->row, A->col, A->rsz,
                                                      A->csz, refel);
    BST_CHECK_LAUNCH();
  }
  if (B->nblocks > 0) {
    k_ref_elems<<<nblk(B->nblocks, 256), 256, 0, s>>>(B->nblocks, refB, B->row, B->col, B->rsz,
                                                      B->csz, refel + 1);
    BST_CHECK_LAUNCH();
  }
  unsigned long long hrefel[2];
  rb_ptrs.add(hrefel, refel, 16);
  rb_ptrs.add(&nelemC, C->off + nnzC, 8);
  rb_ptrs.done();
  scratch.release_all();
  BST_REQUIRE(nelemC < INT32_MAX, BST_ERR_OVERFLOW, "C_out has more than 2^31-1 elements");
  C->nelem = nelemC;

  p->h_bucket_ptr.assign(hb.begin(), hb.end());
  // statistics
  bst_stats &st = p->stats;
  st.n_candidates = ncand;
  st.n_filtered = ncand - T;
  st.n_stack = T;
  st.n_c_blocks = nnzC;
  st.n_c_elements = nelemC;
  int32_t nbk = 0;
  double flops = 0.0;
  for (int32_t b = 0; b < p->nb_all; ++b) {
    const int64_t n = (int64_t)hb[b + 1] - hb[b];
    if (n <= 0) continue;
    ++nbk;
    const int32_t kc = b % p->Dk, nc = (b / p->Dk) % p->Dn, mc = b / (p->Dk * p->Dn);
    flops += 2.0 * p->m_vals[mc] * p->n_vals[nc] * p->k_vals[kc] * (double)n;
  }
  st.n_buckets = nbk;
  st.flops = flops;
  st.split_k = 1;
  // algorithmic bytes: referenced A and B elements, C_out written, 12 bytes per stack
  // entry, 8 bytes per norm (C_in read is added at execute time when beta != 0)
  st.bytes = 8.0 * ((double)hrefel[0] + (double)hrefel[1] + (double)nelemC) + 12.0 * (double)T +
             8.0 * (double)(A->nblocks + B->nblocks);
  build_f64_schedule(p, s);
}

}  // namespace bst
