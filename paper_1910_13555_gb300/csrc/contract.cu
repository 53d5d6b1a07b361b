// Block-sparse tensors and their contraction through the matrix multiply (paper Sec. 4).
//
// Paper Sec. 4: a contraction is computed by mapping each tensor onto a matrix whose
// one dimension holds the summed indices and the other all remaining ones, then calling
// the sparse matrix multiply; the caller controls the layout so that the conversion
// step can be skipped, and the matrix index is computed on the fly from the tensor
// index rather than stored for the whole folded dimension.
//
// Here a tensor view is built on the GPU (the "remap"): the block index of every tensor
// block is folded into a (row block, column block) pair by mixed radix over the row
// modes and the column modes (first listed mode most significant), the blocks are put
// in CSR order by a stable radix sort when the fold changes their order, and:
//   * when the view's modes (rows, then columns) are the tensor's own mode order, the
//     view is zero-copy: each block's row-major data already is the row-major
//     (row-fold x column-fold) matrix block;
//   * when they are that order reversed (columns first), the view is the zero-copy
//     transpose and the multiply takes op = 'T';
//   * otherwise the elements of every block are permuted into a plan-owned buffer
//     (once per execute; the inverse permutation maps gradients back) -- or, when the
//     tensor's modes are (outer contracted, free, inner contracted), the native-FP64
//     staged schedule reads each block in place as slabs (setup_slab_read below).
// The result is the matrix C = op(A) op(B) with rows = the free modes of T1 and columns
// = the free modes of T2; it is the result tensor itself when result_order is the
// identity, and is permuted block by block into the result tensor otherwise.
#include <algorithm>
#include <map>
#include <climits>
#include <cstring>
#include <numeric>

#include "bst_internal.h"

namespace bst {

constexpr int kMaxRank = 8;

// A matrix view of a tensor.
struct View {
  bst_matrix *M = nullptr;
  const bst_tensor *T = nullptr;
  int32_t rank = 0;
  int32_t ord[kMaxRank];  // view element layout: row-major over tensor modes in this order
  bool copy = false;      // data are a permuted copy in `buf`
  bool identity = false;  // view blocks are the tensor blocks in the same order
  int32_t *tblk = nullptr;  // view block -> tensor block
  double *buf = nullptr;
};

struct Contract {
  View A, B, Ci;
  bool has_cin = false;
  bst_tensor *R = nullptr;     // result tensor (owned by the plan)
  bool r_identity = false;     // R data == C data
  int32_t r_ord[kMaxRank];     // C block layout in terms of R modes
  int32_t *r_cblk = nullptr;   // R block -> C block
  double *cbuf = nullptr;      // C data when R is not the identity
  double *dcbuf = nullptr;     // dC buffer for the adjoint
  Arena ar;
};

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct FoldArgs {
  int64_t nblocks;
  int32_t rank;
  const int32_t *idx;
  int32_t nr, nc;
  int32_t rm[kMaxRank], cm[kMaxRank];
  int32_t rrad[kMaxRank], crad[kMaxRank];
  int64_t ncols;
  int32_t *row, *col;
  uint64_t *key;
};

// folded (row, column) block index of every tensor block
__global__ void k_fold(FoldArgs F) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= F.nblocks) return;
  const int32_t *t = F.idx + b * F.rank;
  int64_t r = 0, c = 0;
  for (int q = 0; q < F.nr; ++q) r = r * F.rrad[q] + t[F.rm[q]];
  for (int q = 0; q < F.nc; ++q) c = c * F.crad[q] + t[F.cm[q]];
  F.row[b] = (int32_t)r;
  F.col[b] = (int32_t)c;
  if (F.key) F.key[b] = (uint64_t)r * (uint64_t)F.ncols + (uint64_t)c;
}

__global__ void k_count_rows(int64_t n, const int32_t *row, int32_t *cnt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) atomicAdd(&cnt[row[b]], 1);
}

__global__ void k_i64_to_i32_n(const int64_t *in, int32_t *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

__global__ void k_gather_i64(const int64_t *src, const int32_t *idx, int64_t *dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

struct VolArgs {
  int64_t nblocks;
  int32_t rank;
  const int32_t *idx, *tblk, *sz;
  int32_t szoff[kMaxRank];
  int64_t *vol;
};

__global__ void k_volumes(VolArgs V) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= V.nblocks) return;
  const int32_t *t = V.idx + (int64_t)(V.tblk ? V.tblk[q] : q) * V.rank;
  int64_t v = 1;
  for (int d = 0; d < V.rank; ++d) v *= V.sz[V.szoff[d] + t[d]];
  V.vol[q] = v;
}

// element permutation between tensor blocks (row-major over modes 0..rank-1) and view
// blocks (row-major over modes ord[0..rank-1]); to_view: view <- tensor, else
// tensor <- view
constexpr int kPermThreads = 256;  // threads per tensor block in k_permute

struct PermArgs {
  int64_t nblocks;
  int32_t rank;
  const int32_t *tblk, *idx, *sz;
  int32_t szoff[kMaxRank], ord[kMaxRank];
  const int64_t *toff, *voff;
  const double *src;
  double *dst;
  int to_view;
};

// One CTA per tensor block: its elements are visited in view order, which reads (or
// writes) the tensor layout out of order; with one block in flight per CTA (a few per
// SM) its lines stay in L1 / L2 until every element is used.  A warp per block, with
// dozens of blocks of up to ~175 KB in flight per SM, re-fetched them from DRAM.
__global__ void k_permute(PermArgs P) {
  const int64_t q = blockIdx.x;
  if (q >= P.nblocks) return;
  const int64_t tb = P.tblk ? P.tblk[q] : q;
  const int32_t *t = P.idx + tb * P.rank;
  // block-local index arithmetic in 32 bits (a tensor block holds fewer than 2^31
  // elements; 64-bit division costs several times more)
  int32_t s[kMaxRank], st[kMaxRank];
  int32_t len = 1;
  for (int d = P.rank - 1; d >= 0; --d) {
    s[d] = P.sz[P.szoff[d] + t[d]];
    st[d] = len;
    len *= s[d];
  }
  const int64_t to = P.toff[tb], vo = P.voff[q];
  if ((int32_t)threadIdx.x >= len) return;
  // the thread's elements e = threadIdx.x + i * blockDim.x in view order, as mixed-radix
  // digits over the view's modes (slowest first): decoded once by division, then
  // advanced by the step's own digits with one carry per mode (an element costs a few
  // adds instead of one division per mode)
  // (loops over all kMaxRank modes with the unused ones as size-1 modes, so that the
  // digit arrays live in registers)
  int32_t dig[kMaxRank], inc[kMaxRank], sv[kMaxRank], tv[kMaxRank];
  {
    int32_t rem = (int32_t)threadIdx.x, stp = (int32_t)blockDim.x;
#pragma unroll
    for (int j = kMaxRank - 1; j >= 0; --j) {
      const bool used = j < P.rank;
      const int d = used ? P.ord[j] : 0;
      sv[j] = used ? s[d] : 1;
      tv[j] = used ? st[d] : 0;
      dig[j] = rem % sv[j];
      rem /= sv[j];
      inc[j] = stp % sv[j];
      stp /= sv[j];
    }
  }
  for (int32_t e = threadIdx.x; e < len; e += blockDim.x) {
    int32_t src = 0;
#pragma unroll
    for (int j = 0; j < kMaxRank; ++j) src += dig[j] * tv[j];
    if (P.to_view)
      P.dst[vo + e] = P.src[to + src];
    else
      P.dst[to + src] = P.src[vo + e];
    int32_t carry = 0;
#pragma unroll
    for (int j = kMaxRank - 1; j >= 0; --j) {
      const int32_t v = dig[j] + inc[j] + carry;
      carry = v >= sv[j];
      dig[j] = carry ? v - sv[j] : v;
    }
  }
}

// R tuple of every C block: decode folded row / column, reorder by result_order
struct UnfoldArgs {
  int64_t nc;
  const int32_t *row, *col;
  int32_t nf1, nf2, rr;
  int32_t rad1[kMaxRank], rad2[kMaxRank];
  int32_t ro[2 * kMaxRank];
  int32_t rrad[2 * kMaxRank];
  int32_t *idx;
  uint64_t *key;
};

__global__ void k_unfold(UnfoldArgs U) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= U.nc) return;
  int32_t slot[2 * kMaxRank];
  int64_t r = U.row[c];
  for (int q = U.nf1 - 1; q >= 0; --q) {
    slot[q] = (int32_t)(r % U.rad1[q]);
    r /= U.rad1[q];
  }
  int64_t cc = U.col[c];
  for (int q = U.nf2 - 1; q >= 0; --q) {
    slot[U.nf1 + q] = (int32_t)(cc % U.rad2[q]);
    cc /= U.rad2[q];
  }
  uint64_t key = 0;
  for (int q = 0; q < U.rr; ++q) {
    const int32_t v = slot[U.ro[q]];
    U.idx[c * U.rr + q] = v;
    key = key * (uint64_t)U.rrad[q] + (uint64_t)v;
  }
  if (U.key) U.key[c] = key;
}

__global__ void k_gather_tuples(const int32_t *src, const int32_t *perm, int32_t *dst, int64_t n,
                                int32_t rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < rank; ++d) dst[i * rank + d] = src[(int64_t)perm[i] * rank + d];
}

int bits_for(uint64_t n) {
  int b = 0;
  while (b < 64 && (n >> b) > 0) ++b;
  return b;
}

void szoffsets(const bst_tensor *T, int32_t *szoff) {
  int32_t o = 0;
  for (int d = 0; d < T->rank; ++d) {
    szoff[d] = o;
    o += T->h_nblk[d];
  }
}

// Build the matrix view of T with rows = fold of `rm`, columns = fold of `cm`.
void build_view(bst_ctx *ctx, const bst_tensor *T, const std::vector<int32_t> &rm,
                const std::vector<int32_t> &cm, View &V, Arena &ar, cudaStream_t s) {
  V.T = T;
  V.rank = T->rank;
  std::vector<int32_t> order(rm);
  order.insert(order.end(), cm.begin(), cm.end());
  for (int d = 0; d < T->rank; ++d) V.ord[d] = order[d];
  bool ident = true;
  for (int d = 0; d < T->rank; ++d) ident &= order[d] == d;
  V.identity = ident;
  V.copy = !ident;
  // folded grid and block sizes (computed from the per-mode sizes; never stored per
  // tensor block row beyond the folded dimension itself)
  auto fold_sizes = [&](const std::vector<int32_t> &modes, std::vector<int32_t> &out) {
    int64_t n = 1;
    for (int32_t d : modes) n *= T->h_nblk[d];
    BST_REQUIRE(n < INT32_MAX, BST_ERR_UNSUPPORTED, "a folded tensor dimension exceeds 2^31-1 blocks");
    out.assign((size_t)n, 1);
    for (int64_t x = 0; x < n; ++x) {
      int64_t rem = x, v = 1;
      for (int q = (int)modes.size() - 1; q >= 0; --q) {
        const int32_t d = modes[q];
        v *= T->h_sz[d][rem % T->h_nblk[d]];
        rem /= T->h_nblk[d];
      }
      BST_REQUIRE(v < INT32_MAX, BST_ERR_OVERFLOW, "folded block size exceeds 2^31-1");
      out[(size_t)x] = (int32_t)v;
    }
  };
  auto *M = new bst_matrix();
  V.M = M;
  M->ctx = ctx;
  M->owned_by_plan = true;
  fold_sizes(rm, M->h_rsz);
  fold_sizes(cm, M->h_csz);
  M->nbr = (int32_t)M->h_rsz.size();
  M->nbc = (int32_t)M->h_csz.size();
  M->nblocks = T->nblocks;
  M->nelem = T->nelem;
  {
    Upload up(ctx, s);
    M->rsz = up.add_vector(ar, M->h_rsz);
    M->csz = up.add_vector(ar, M->h_csz);
    up.done();
  }
  const int64_t n = T->nblocks;
  FoldArgs F{};
  F.nblocks = n;
  F.rank = T->rank;
  F.idx = T->idx;
  F.nr = (int32_t)rm.size();
  F.nc = (int32_t)cm.size();
  for (int q = 0; q < F.nr; ++q) {
    F.rm[q] = rm[q];
    F.rrad[q] = T->h_nblk[rm[q]];
  }
  for (int q = 0; q < F.nc; ++q) {
    F.cm[q] = cm[q];
    F.crad[q] = T->h_nblk[cm[q]];
  }
  F.ncols = M->nbc;
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(ctx);
  scratch.stream = s;
  int32_t *frow = ar.alloc_n<int32_t>((size_t)n), *fcol = ar.alloc_n<int32_t>((size_t)n);
  uint64_t *key = ident ? nullptr : scratch.alloc_n<uint64_t>((size_t)n);
  F.row = frow;
  F.col = fcol;
  F.key = key;
  if (n > 0) {
    k_fold<<<nblk(n, 256), 256, 0, s>>>(F);
    BST_CHECK_LAUNCH();
  }
  if (ident) {
    // tensor order is already (row fold, column fold) lexicographic
    M->row = frow;
    M->col = fcol;
    M->off = const_cast<int64_t *>(T->off);
    V.tblk = nullptr;
  } else {
    V.tblk = ar.alloc_n<int32_t>((size_t)n);
    radix_sort_perm(key, n, bits_for((uint64_t)M->nbr * (uint64_t)M->nbc), V.tblk, scratch, s);
    M->row = ar.alloc_n<int32_t>((size_t)n);
    M->col = ar.alloc_n<int32_t>((size_t)n);
    gather_i32(frow, V.tblk, M->row, n, s);
    gather_i32(fcol, V.tblk, M->col, n, s);
    // packed offsets of the permuted copy, in view order
    VolArgs VA{};
    VA.nblocks = n;
    VA.rank = T->rank;
    VA.idx = T->idx;
    VA.tblk = V.tblk;
    VA.sz = T->sz;
    szoffsets(T, VA.szoff);
    int64_t *vol = scratch.alloc_n<int64_t>((size_t)n);
    VA.vol = vol;
    if (n > 0) {
      k_volumes<<<nblk(n, 256), 256, 0, s>>>(VA);
      BST_CHECK_LAUNCH();
    }
    M->off = ar.alloc_n<int64_t>((size_t)n + 1);
    exscan_i64(vol, M->off, n, scratch, s);
    V.buf = ar.alloc_n<double>((size_t)std::max<int64_t>(T->nelem, 1));
  }
  // CSR row pointer of the view
  int32_t *cnt = scratch.alloc_n<int32_t>((size_t)M->nbr);
  BST_CUDA(cudaMemsetAsync(cnt, 0, 4 * (size_t)std::max<int32_t>(M->nbr, 1), s));
  if (n > 0) {
    k_count_rows<<<nblk(n, 256), 256, 0, s>>>(n, M->row, cnt);
    BST_CHECK_LAUNCH();
  }
  int64_t *rp64 = scratch.alloc_n<int64_t>((size_t)M->nbr + 1);
  exscan_i32_i64(cnt, rp64, M->nbr, scratch, s);
  M->rowptr = ar.alloc_n<int32_t>((size_t)M->nbr + 1);
  k_i64_to_i32_n<<<nblk((int64_t)M->nbr + 1, 256), 256, 0, s>>>(rp64, M->rowptr, (int64_t)M->nbr + 1);
  BST_CHECK_LAUNCH();
  BST_CUDA(cudaStreamSynchronize(s));
  scratch.release_all();
  M->data = ident ? T->data : V.buf;
}

void permute_view(const View &V, const double *src, double *dst, bool to_view, cudaStream_t s) {
  if (!V.copy || V.T->nblocks == 0) return;
  PermArgs P{};
  P.nblocks = V.T->nblocks;
  P.rank = V.rank;
  P.tblk = V.tblk;
  P.idx = V.T->idx;
  P.sz = V.T->sz;
  szoffsets(V.T, P.szoff);
  for (int d = 0; d < V.rank; ++d) P.ord[d] = V.ord[d];
  P.toff = V.T->off;
  P.voff = V.M->off;
  P.src = src;
  P.dst = dst;
  P.to_view = to_view;
  k_permute<<<(unsigned)P.nblocks, kPermThreads, 0, s>>>(P);
  BST_CHECK_LAUNCH();
}

// Slab reading of T1 (the second remap of a non-fold view).  When T1's modes are stored
// as (outer contracted modes, free modes, inner contracted modes), each in the order the
// view folds them, the view's m x k block (rows = free fold, k = outer fold x inner fold)
// is the tensor block itself read as k / k_i consecutive m x k_i slabs (k_i = the inner
// fold's size): column o k_i + i of row r sits at o m k_i + r k_i + i.  The native-FP64
// staged schedule can then read A in place instead of through the permuted copy.  Needs
// k_i to be a function of the k block size (one slab width per k class).
void setup_slab_read(bst_plan *p, const View &V, const std::vector<int32_t> &F1,
                     const std::vector<int32_t> &C1, Arena &ar, cudaStream_t s) {
  const bst_tensor *T = V.T;
  const int nc = (int)C1.size();
  int j = -1;
  for (int q = 1; q < nc && j < 0; ++q) {
    std::vector<int32_t> o(C1.begin(), C1.begin() + q);
    o.insert(o.end(), F1.begin(), F1.end());
    o.insert(o.end(), C1.begin() + q, C1.end());
    bool id = true;
    for (int d = 0; d < (int)o.size(); ++d) id &= o[d] == d;
    if (id) j = q;
  }
  if (j < 0 || V.M->nblocks == 0) return;
  // k_i of every k block (mixed radix over C1, first listed most significant)
  std::map<int32_t, int32_t> kin_of;
  const int64_t nk = (int64_t)V.M->h_csz.size();
  for (int64_t x = 0; x < nk; ++x) {
    int64_t rem = x, ki = 1;
    for (int q = nc - 1; q >= 0; --q) {
      const int32_t d = C1[q];
      if (q >= j) ki *= T->h_sz[d][rem % T->h_nblk[d]];
      rem /= T->h_nblk[d];
    }
    const int32_t k = V.M->h_csz[(size_t)x];
    auto it = kin_of.find(k);
    if (it == kin_of.end())
      kin_of[k] = (int32_t)ki;
    else if (it->second != ki)
      return;  // two slab widths for one k class
  }
  std::vector<int32_t> kin(p->k_vals.size());
  for (size_t kc = 0; kc < kin.size(); ++kc) {
    auto it = kin_of.find(p->k_vals[kc]);
    kin[kc] = it == kin_of.end() ? p->k_vals[kc] : it->second;
  }
  const int64_t n = V.M->nblocks;
  int64_t *toff = ar.alloc_n<int64_t>((size_t)n);
  k_gather_i64<<<nblk(n, 256), 256, 0, s>>>(T->off, V.tblk, toff, n);
  BST_CHECK_LAUNCH();
  p->a_slab_kin = kin;
  p->a_slab_toff = toff;
  p->a_slab_base = T->data;
  build_f64_schedule(p, s);
}

void free_view(View &V) {
  if (V.M) {
    V.M->owned_by_plan = false;
    delete V.M;
    V.M = nullptr;
  }
}

}  // namespace

void contract_free(bst_plan *p) {
  if (!p->contract) return;
  Contract *c = p->contract;
  free_view(c->A);
  free_view(c->B);
  free_view(c->Ci);
  if (c->R) {
    c->R->owned_by_plan = false;
    delete c->R;
  }
  delete c;
  p->contract = nullptr;
}

// Refresh the views' data before an execute: permute the inputs that are copies and
// point the C matrix at the result data.  Returns the C data pointer to use.
void contract_check_bound(const bst_plan *p, bool read_cin) {
  const Contract &K = *p->contract;
  BST_REQUIRE(K.A.T->nblocks == 0 || K.A.T->data, BST_ERR_STATE, "T1 data not bound");
  BST_REQUIRE(K.B.T->nblocks == 0 || K.B.T->data, BST_ERR_STATE, "T2 data not bound");
  BST_REQUIRE(!(K.has_cin && read_cin) || K.Ci.T->nblocks == 0 || K.Ci.T->data, BST_ERR_STATE,
              "R_in data not bound");
  BST_REQUIRE(K.R->nelem == 0 || K.R->data, BST_ERR_STATE, "result tensor data not bound");
}

void contract_prepare(bst_plan *p, bool read_cin, cudaStream_t s, bool a_copy) {
  Contract &K = *p->contract;
  contract_check_bound(p, read_cin);
  K.A.M->data = K.A.copy ? K.A.buf : K.A.T->data;
  K.B.M->data = K.B.copy ? K.B.buf : K.B.T->data;
  p->a_slab_base = K.A.T->data;
  if (a_copy) permute_view(K.A, K.A.T->data, K.A.buf, true, s);
  permute_view(K.B, K.B.T->data, K.B.buf, true, s);
  if (K.has_cin) {
    K.Ci.M->data = K.Ci.copy ? K.Ci.buf : K.Ci.T->data;
    if (read_cin) {
      BST_REQUIRE(K.Ci.T->nblocks == 0 || K.Ci.T->data, BST_ERR_STATE, "R_in data not bound");
      permute_view(K.Ci, K.Ci.T->data, K.Ci.buf, true, s);
    }
  }
  BST_REQUIRE(K.R->nelem == 0 || K.R->data, BST_ERR_STATE, "result tensor data not bound");
  p->C->data = K.r_identity ? K.R->data : K.cbuf;
}

// C (view layout) -> R (tensor layout) after an execute
void contract_finish(bst_plan *p, cudaStream_t s) {
  Contract &K = *p->contract;
  if (K.r_identity || K.R->nblocks == 0) return;
  PermArgs P{};
  P.nblocks = K.R->nblocks;
  P.rank = K.R->rank;
  P.tblk = nullptr;  // view block q == C block r_cblk... handled through voff below
  P.idx = K.R->idx;
  P.sz = K.R->sz;
  szoffsets(K.R, P.szoff);
  for (int d = 0; d < K.R->rank; ++d) P.ord[d] = K.r_ord[d];
  P.toff = K.R->off;
  P.voff = K.R->off + K.R->nblocks;  // C offsets gathered into R order (second half)
  P.src = K.cbuf;
  P.dst = K.R->data;
  P.to_view = 0;
  k_permute<<<(unsigned)P.nblocks, kPermThreads, 0, s>>>(P);
  BST_CHECK_LAUNCH();
}

// adjoint of a contraction: dR (tensor layout) -> dC, matrix adjoint, views -> tensors
void contract_adjoint(bst_plan *p, const double *dR, double *dT1, double *dT2, double *dRin,
                      double alpha, double beta, cudaStream_t s) {
  Contract &K = *p->contract;
  contract_prepare(p, false, s);
  const double *dC = dR;
  if (!K.r_identity && K.R->nblocks > 0) {
    PermArgs P{};
    P.nblocks = K.R->nblocks;
    P.rank = K.R->rank;
    P.tblk = nullptr;
    P.idx = K.R->idx;
    P.sz = K.R->sz;
    szoffsets(K.R, P.szoff);
    for (int d = 0; d < K.R->rank; ++d) P.ord[d] = K.r_ord[d];
    P.toff = K.R->off;
    P.voff = K.R->off + K.R->nblocks;
    P.src = dR;
    P.dst = K.dcbuf;
    P.to_view = 1;
    k_permute<<<(unsigned)P.nblocks, kPermThreads, 0, s>>>(P);
    BST_CHECK_LAUNCH();
    dC = K.dcbuf;
  }
  // view-layout gradients: straight into the tensors when zero-copy, else through a
  // scratch buffer and the inverse permutation
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  double *dA = dT1, *dB = dT2;
  if (K.A.copy && dT1) dA = scratch.alloc_n<double>((size_t)std::max<int64_t>(K.A.T->nelem, 1));
  if (K.B.copy && dT2) dB = scratch.alloc_n<double>((size_t)std::max<int64_t>(K.B.T->nelem, 1));
  adjoint_fp64(p, p->A->data, p->B->data, dC, dA, dB, alpha, s);
  if (K.A.copy && dT1) permute_view(K.A, dA, dT1, false, s);
  if (K.B.copy && dT2) permute_view(K.B, dB, dT2, false, s);
  if (K.has_cin && dRin) {
    double *dCi = dRin;
    if (K.Ci.copy) dCi = scratch.alloc_n<double>((size_t)std::max<int64_t>(K.Ci.T->nelem, 1));
    scale_cin_grad(p, dC, dCi, beta, s);
    if (K.Ci.copy) permute_view(K.Ci, dCi, dRin, false, s);
  }
  scratch.release_all();
}

}  // namespace bst

using bst::Error;


extern "C" {

bst_status bst_tensor_create(bst_ctx *ctx, bst_tensor **out, int32_t rank, const int32_t *nblk,
                             const int32_t *blk_sizes, int64_t nblocks, const int32_t *blk_idx,
                             double *data, void *stream) {
  API_BEGIN
  BST_REQUIRE(ctx && out, BST_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  BST_REQUIRE(rank >= 1 && rank <= bst::kMaxRank, BST_ERR_INVALID_ARG, "rank must be in 1..8");
  BST_REQUIRE(nblk && nblocks >= 0, BST_ERR_INVALID_ARG, "bad block counts");
  BST_REQUIRE(nblocks == 0 || blk_idx, BST_ERR_INVALID_ARG, "block index is NULL");
  BST_REQUIRE(nblocks < INT32_MAX, BST_ERR_OVERFLOW, "more than 2^31-1 blocks");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int cur = -1;
  BST_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
  std::vector<std::vector<int32_t>> sz(rank);
  int64_t so = 0;
  for (int d = 0; d < rank; ++d) {
    BST_REQUIRE(nblk[d] >= 0, BST_ERR_INVALID_ARG, "negative block count");
    BST_REQUIRE(nblk[d] == 0 || blk_sizes, BST_ERR_INVALID_ARG, "block sizes are NULL");
    sz[d].assign(blk_sizes + so, blk_sizes + so + nblk[d]);
    for (int32_t v : sz[d]) BST_REQUIRE(v >= 1, BST_ERR_INVALID_ARG, "block size < 1");
    so += nblk[d];
  }
  for (int64_t b = 0; b < nblocks; ++b)
    for (int d = 0; d < rank; ++d)
      BST_REQUIRE(blk_idx[b * rank + d] >= 0 && blk_idx[b * rank + d] < nblk[d],
                  BST_ERR_OUT_OF_RANGE, "block index outside the block grid");
  std::vector<int32_t> ord((size_t)nblocks);
  std::iota(ord.begin(), ord.end(), 0);
  auto less = [&](int32_t x, int32_t y) {
    return std::lexicographical_compare(blk_idx + (int64_t)x * rank, blk_idx + (int64_t)x * rank + rank,
                                        blk_idx + (int64_t)y * rank, blk_idx + (int64_t)y * rank + rank);
  };
  std::sort(ord.begin(), ord.end(), less);
  auto *t = new bst_tensor();
  try {
    t->ctx = ctx;
    t->arena.ctx = static_cast<bst::Ctx *>(ctx);
    t->arena.stream = s;
    t->rank = rank;
    t->h_nblk.assign(nblk, nblk + rank);
    t->h_sz = sz;
    t->nblocks = nblocks;
    t->h_idx.resize((size_t)nblocks * rank);
    t->h_off.resize((size_t)nblocks);
    int64_t acc = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
      const int32_t o = ord[b];
      if (b > 0)
        BST_REQUIRE(std::memcmp(blk_idx + (int64_t)o * rank, blk_idx + (int64_t)ord[b - 1] * rank,
                                sizeof(int32_t) * rank) != 0,
                    BST_ERR_DUPLICATE_BLOCK, "a block is listed twice");
      int64_t v = 1;
      for (int d = 0; d < rank; ++d) {
        t->h_idx[(size_t)b * rank + d] = blk_idx[(int64_t)o * rank + d];
        v *= sz[d][blk_idx[(int64_t)o * rank + d]];
      }
      t->h_off[(size_t)b] = acc;
      acc += v;
    }
    BST_REQUIRE(acc <= INT32_MAX, BST_ERR_OVERFLOW, "more than 2^31-1 elements");
    t->nelem = acc;
    std::vector<int32_t> flat;
    for (auto &v : sz) flat.insert(flat.end(), v.begin(), v.end());
    t->idx = t->arena.alloc_n<int32_t>(t->h_idx.size());
    t->off = t->arena.alloc_n<int64_t>(t->h_off.size() + 1);
    {
      bst::Upload up(ctx, s);
      up.add(t->idx, t->h_idx.data(), 4 * t->h_idx.size());
      up.add(t->off, t->h_off.data(), 8 * t->h_off.size());
      t->sz = up.add_vector(t->arena, flat);
      up.done();
    }
    t->data = data;
  } catch (...) {
    delete t;
    throw;
  }
  *out = t;
  API_END
}

bst_status bst_tensor_info(const bst_tensor *t, int32_t *rank, int64_t *nblocks, int64_t *nelem) {
  API_BEGIN
  BST_REQUIRE(t, BST_ERR_INVALID_ARG, "tensor is NULL");
  if (rank) *rank = t->rank;
  if (nblocks) *nblocks = t->nblocks;
  if (nelem) *nelem = t->nelem;
  API_END
}

bst_status bst_tensor_get_index(const bst_tensor *t, int32_t *blk_idx, int64_t *blk_off) {
  API_BEGIN
  BST_REQUIRE(t, BST_ERR_INVALID_ARG, "tensor is NULL");
  if (blk_idx && !t->h_idx.empty()) std::memcpy(blk_idx, t->h_idx.data(), 4 * t->h_idx.size());
  if (blk_off && !t->h_off.empty()) std::memcpy(blk_off, t->h_off.data(), 8 * t->h_off.size());
  API_END
}

bst_status bst_tensor_bind_data(bst_tensor *t, double *data) {
  API_BEGIN
  BST_REQUIRE(t, BST_ERR_INVALID_ARG, "tensor is NULL");
  t->data = data;
  API_END
}

bst_status bst_tensor_destroy(bst_tensor *t) {
  API_BEGIN
  if (!t) return BST_OK;
  BST_REQUIRE(!t->owned_by_plan, BST_ERR_STATE, "this tensor belongs to a plan");
  delete t;
  API_END
}

bst_status bst_contract_plan(bst_ctx *ctx, const bst_tensor *T1, const bst_tensor *T2,
                             int32_t ncontract, const int32_t *c1, const int32_t *c2,
                             int32_t nfree1, const int32_t *f1, int32_t nfree2,
                             const int32_t *f2, const int32_t *result_order,
                             const bst_tensor *R_in, double eps, void *stream, bst_plan **out) {
  API_BEGIN
  BST_REQUIRE(ctx && T1 && T2 && out, BST_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  BST_REQUIRE(ncontract >= 1 && ncontract <= 3, BST_ERR_INVALID_ARG, "contract over 1..3 index pairs");
  BST_REQUIRE(c1 && c2, BST_ERR_INVALID_ARG, "contracted modes are NULL");
  BST_REQUIRE(nfree1 >= 0 && nfree2 >= 0 && nfree1 + nfree2 >= 1, BST_ERR_INVALID_ARG,
              "bad free mode counts");
  BST_REQUIRE((nfree1 == 0 || f1) && (nfree2 == 0 || f2), BST_ERR_INVALID_ARG, "free modes are NULL");
  BST_REQUIRE(ncontract + nfree1 == T1->rank && ncontract + nfree2 == T2->rank, BST_ERR_INVALID_ARG,
              "every mode must be listed once as contracted or free");
  BST_REQUIRE(eps >= 0.0, BST_ERR_INVALID_ARG, "eps must be >= 0");
  BST_REQUIRE((T1->nblocks == 0 || T1->data) && (T2->nblocks == 0 || T2->data), BST_ERR_STATE,
              "T1 / T2 data not bound");
  std::vector<int> seen1(T1->rank, 0), seen2(T2->rank, 0);
  for (int q = 0; q < ncontract; ++q) {
    BST_REQUIRE(c1[q] >= 0 && c1[q] < T1->rank && c2[q] >= 0 && c2[q] < T2->rank,
                BST_ERR_INVALID_ARG, "contracted mode out of range");
    BST_REQUIRE(!seen1[c1[q]]++ && !seen2[c2[q]]++, BST_ERR_INVALID_ARG, "mode listed twice");
  }
  for (int q = 0; q < nfree1; ++q) {
    BST_REQUIRE(f1[q] >= 0 && f1[q] < T1->rank && !seen1[f1[q]]++, BST_ERR_INVALID_ARG,
                "bad free mode of T1");
  }
  for (int q = 0; q < nfree2; ++q) {
    BST_REQUIRE(f2[q] >= 0 && f2[q] < T2->rank && !seen2[f2[q]]++, BST_ERR_INVALID_ARG,
                "bad free mode of T2");
  }
  for (int q = 0; q < ncontract; ++q)
    BST_REQUIRE(T1->h_sz[c1[q]] == T2->h_sz[c2[q]], BST_ERR_SHAPE_MISMATCH,
                "contracted modes have different block sizes");
  const int rr = nfree1 + nfree2;
  BST_REQUIRE(rr <= bst::kMaxRank, BST_ERR_UNSUPPORTED, "result rank above 8");
  std::vector<int32_t> ro(rr), inv(rr, -1);
  for (int r = 0; r < rr; ++r) {
    ro[r] = result_order ? result_order[r] : r;
    BST_REQUIRE(ro[r] >= 0 && ro[r] < rr && inv[ro[r]] < 0, BST_ERR_INVALID_ARG,
                "result_order is not a permutation");
    inv[ro[r]] = r;
  }
  // free slot q -> (tensor, mode)
  auto slot_nblk = [&](int q) { return q < nfree1 ? T1->h_nblk[f1[q]] : T2->h_nblk[f2[q - nfree1]]; };
  auto slot_sz = [&](int q) -> const std::vector<int32_t> & {
    return q < nfree1 ? T1->h_sz[f1[q]] : T2->h_sz[f2[q - nfree1]];
  };
  if (R_in) {
    BST_REQUIRE(R_in->rank == rr, BST_ERR_SHAPE_MISMATCH, "R_in rank differs from the result's");
    for (int r = 0; r < rr; ++r)
      BST_REQUIRE(R_in->h_sz[r] == slot_sz(ro[r]), BST_ERR_SHAPE_MISMATCH,
                  "R_in block sizes differ from the result's");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int cur = -1;
  BST_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));

  auto *K = new bst::Contract();
  bst_plan *p = nullptr;
  try {
    K->ar.ctx = static_cast<bst::Ctx *>(ctx);
    K->ar.stream = s;
    std::vector<int32_t> F1(f1, f1 + nfree1), F2(f2, f2 + nfree2), C1(c1, c1 + ncontract),
        C2(c2, c2 + ncontract);
    auto is_ident = [](const std::vector<int32_t> &a, const std::vector<int32_t> &b) {
      std::vector<int32_t> o(a);
      o.insert(o.end(), b.begin(), b.end());
      for (size_t d = 0; d < o.size(); ++d)
        if (o[d] != (int32_t)d) return false;
      return true;
    };
    // T1 -> A = rows f1, cols c1 (or its zero-copy transpose)
    bool ta = false, tb = false;
    if (is_ident(F1, C1) || !is_ident(C1, F1)) {
      bst::build_view(ctx, T1, F1, C1, K->A, K->ar, s);
    } else {
      bst::build_view(ctx, T1, C1, F1, K->A, K->ar, s);
      ta = true;
    }
    // T2 -> B = rows c2, cols f2 (or its zero-copy transpose)
    if (is_ident(C2, F2) || !is_ident(F2, C2)) {
      bst::build_view(ctx, T2, C2, F2, K->B, K->ar, s);
    } else {
      bst::build_view(ctx, T2, F2, C2, K->B, K->ar, s);
      tb = true;
    }
    // R_in -> C_in view: rows = result modes of the f1 slots, cols = those of f2 slots
    if (R_in) {
      std::vector<int32_t> rm, cm;
      for (int q = 0; q < nfree1; ++q) rm.push_back(inv[q]);
      for (int q = nfree1; q < rr; ++q) cm.push_back(inv[q]);
      bst::build_view(ctx, R_in, rm, cm, K->Ci, K->ar, s);
      K->has_cin = true;
    }
    // the symbolic phase reads the operand norms: fill the permuted copies first
    bst::permute_view(K->A, T1->data, K->A.buf, true, s);
    bst::permute_view(K->B, T2->data, K->B.buf, true, s);
    bst_status st = bst_multiply_plan(ctx, ta ? 'T' : 'N', tb ? 'T' : 'N', K->A.M, K->B.M,
                                      R_in ? K->Ci.M : nullptr, eps, stream, &p);
    if (st != BST_OK) throw Error{st, bst_last_error()};
    p->contract = K;
    if (!ta && K->A.copy && static_cast<bst::Ctx *>(ctx)->tune_contract_slab)
      bst::setup_slab_read(p, K->A, F1, C1, K->ar, s);
    // result tensor: blocks of C unfolded into result-order tuples
    const bst_matrix *C = p->C;
    auto *R = new bst_tensor();
    K->R = R;
    R->ctx = ctx;
    R->owned_by_plan = true;
    R->rank = rr;
    R->h_nblk.resize(rr);
    R->h_sz.resize(rr);
    std::vector<int32_t> flat;
    for (int r = 0; r < rr; ++r) {
      R->h_nblk[r] = slot_nblk(ro[r]);
      R->h_sz[r] = slot_sz(ro[r]);
      flat.insert(flat.end(), R->h_sz[r].begin(), R->h_sz[r].end());
    }
    R->nblocks = C->nblocks;
    R->nelem = C->nelem;
    {
      bst::Upload up(ctx, s);
      R->sz = up.add_vector(K->ar, flat);
      up.done();
    }
    bool rid = true;
    for (int r = 0; r < rr; ++r) rid &= ro[r] == r;
    K->r_identity = rid;
    for (int q = 0; q < rr; ++q) K->r_ord[q] = inv[q];
    const int64_t nc = C->nblocks;
    bst::UnfoldArgs U{};
    U.nc = nc;
    U.row = C->row;
    U.col = C->col;
    U.nf1 = nfree1;
    U.nf2 = nfree2;
    U.rr = rr;
    for (int q = 0; q < nfree1; ++q) U.rad1[q] = T1->h_nblk[f1[q]];
    for (int q = 0; q < nfree2; ++q) U.rad2[q] = T2->h_nblk[f2[q]];
    uint64_t span = 1;
    for (int r = 0; r < rr; ++r) {
      U.ro[r] = ro[r];
      U.rrad[r] = R->h_nblk[r];
      span *= (uint64_t)R->h_nblk[r];
    }
    bst::Arena scratch;
    scratch.ctx = static_cast<bst::Ctx *>(ctx);
    scratch.stream = s;
    int32_t *cidx = scratch.alloc_n<int32_t>((size_t)nc * rr);
    uint64_t *key = rid ? nullptr : scratch.alloc_n<uint64_t>((size_t)nc);
    U.idx = cidx;
    U.key = key;
    if (nc > 0) {
      bst::k_unfold<<<bst::nblk(nc, 256), 256, 0, s>>>(U);
      BST_CHECK_LAUNCH();
    }
    R->idx = K->ar.alloc_n<int32_t>((size_t)nc * rr);
    // R offsets; when R is a permutation of C the second half of R->off holds the C
    // offset of each R block, for the block permutation kernels
    R->off = K->ar.alloc_n<int64_t>(2 * (size_t)nc + 1);
    if (rid) {
      BST_CUDA(cudaMemcpyAsync(R->idx, cidx, 4 * (size_t)nc * rr, cudaMemcpyDeviceToDevice, s));
      BST_CUDA(cudaMemcpyAsync(R->off, C->off, 8 * (size_t)nc, cudaMemcpyDeviceToDevice, s));
    } else {
      K->r_cblk = K->ar.alloc_n<int32_t>((size_t)nc);
      bst::radix_sort_perm(key, nc, bst::bits_for(span), K->r_cblk, scratch, s);
      if (nc > 0) {
        bst::k_gather_tuples<<<bst::nblk(nc, 256), 256, 0, s>>>(cidx, K->r_cblk, R->idx, nc, rr);
        BST_CHECK_LAUNCH();
      }
      bst::VolArgs VA{};
      VA.nblocks = nc;
      VA.rank = rr;
      VA.idx = R->idx;
      VA.tblk = nullptr;
      VA.sz = R->sz;
      bst::szoffsets(R, VA.szoff);
      int64_t *vol = scratch.alloc_n<int64_t>((size_t)nc);
      VA.vol = vol;
      if (nc > 0) {
        bst::k_volumes<<<bst::nblk(nc, 256), 256, 0, s>>>(VA);
        BST_CHECK_LAUNCH();
      }
      bst::exscan_i64(vol, R->off, nc, scratch, s);
      if (nc > 0) {
        bst::k_gather_i64<<<bst::nblk(nc, 256), 256, 0, s>>>(C->off, K->r_cblk, R->off + nc, nc);
        BST_CHECK_LAUNCH();
      }
      K->cbuf = K->ar.alloc_n<double>((size_t)std::max<int64_t>(C->nelem, 1));
      K->dcbuf = K->ar.alloc_n<double>((size_t)std::max<int64_t>(C->nelem, 1));
    }
    R->h_idx.resize((size_t)nc * rr);
    R->h_off.resize((size_t)nc);
    {
      bst::ReadBack rb(ctx, s);
      rb.add(R->h_idx.data(), R->idx, 4 * (size_t)nc * rr);
      rb.add(R->h_off.data(), R->off, 8 * (size_t)nc);
      rb.done();
    }
    scratch.release_all();
  } catch (...) {
    if (p) {
      bst_plan_destroy(p);  // also frees K through contract_free
    } else {
      bst::free_view(K->A);
      bst::free_view(K->B);
      bst::free_view(K->Ci);
      delete K;
    }
    throw;
  }
  *out = p;
  API_END
}

bst_status bst_plan_result_tensor(bst_plan *plan, bst_tensor **R) {
  API_BEGIN
  BST_REQUIRE(plan && R, BST_ERR_INVALID_ARG, "NULL argument");
  BST_REQUIRE(plan->contract, BST_ERR_STATE, "not a contraction plan");
  *R = plan->contract->R;
  API_END
}

}  // extern "C"
