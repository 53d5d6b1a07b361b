// Numeric phase, native FP64: batched small-block products of the stacks.
//
// Paper Sec. 2: the stacks of block products are processed by small-GEMM kernels
// specialised per (m, n, k).  On GB300 FP64 runs at about 1 TFLOP/s on the CUDA
// cores (FP64 DMMA measures the same), so this path is bound by the FP64 pipe, and
// what matters is how many lanes of every FP64 FMA do useful work and that C is
// written once.  Every plan whose block sizes fit its tiles runs the staged persistent
// kernel (k_num_fp64_staged1, "staged persistent kernel" below: row tiles of C blocks
// from a cost-ordered list, operands staged through shared memory, one runtime-size
// product body).  The direct-load kernels described here serve the other plans and the
// split-K path:
//   * one warp owns one C block (the "task"); its lanes own the m*n outputs
//     (ceil(m n / 32) accumulators per lane), so no two warps write the same C block
//     and no atomics are needed (the paper's static assignment of whole A rows to
//     threads serves the same purpose);
//   * the warp walks, k class by k class, the run of stack entries of its C block in
//     each (m, n, k) bucket (entries inside a run ascend in k), calling the product
//     code specialised at compile time for (m, n) in {5, 13, 23}^2 and k in
//     {5, 13, 23} (runtime k and runtime (m, n) otherwise);
//   * C = alpha * acc + beta * C_in is written once per element (C_in unread when
//     beta == 0);
//   * split-K (paper Sec. 3.1, Eq. 2): with S parts, warp (task, s) sums only the
//     entries whose k block index lies in part s of the K range into a workspace
//     slice; a second kernel adds the S slices in the fixed order 0..S-1.
#include <algorithm>
#include <cstring>

#include "bst_internal.h"

namespace bst {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct NumParams {
  const double *A, *B, *Cin;
  double *C, *W;
  double alpha, beta;
  int64_t nelemC;
  int64_t ntasks;
  int32_t split, K;
  int32_t Dk;
  int32_t ta, tb;
  int32_t alpha_one, has_beta;  // alpha == 1, beta != 0 (host-side: FP64 compares would
                                // occupy the slow FP64 pipe once per C block)
  const int32_t *task_c, *c_cls, *c_cin;
  const int64_t *c_off, *cin_off;
  const int32_t *run_start, *run_len;
  const int32_t *s_a, *s_b, *s_k;
  const int32_t *cls_m, *cls_n, *kval;
  const int32_t *fdesc;  // staged kernel: C block descriptors (kF64Desc words each)
  const int4 *fents;     // staged kernel: C-major entries
};

// first entry in [lo, hi) whose k block index is >= kb (entries ascend in k)
__device__ __forceinline__ int lower_k(const int32_t *__restrict__ s_k, int lo, int hi, int kb) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s_k[mid] < kb)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// entry range of run r restricted to split part s
__device__ __forceinline__ void run_range(const NumParams &P, int64_t r, int s, int &e0, int &e1) {
  const int len = P.run_len[r];
  if (len == 0) {
    e0 = e1 = 0;
    return;
  }
  e0 = P.run_start[r];
  e1 = e0 + len;
  if (P.split > 1) {
    const int kb0 = (int)((int64_t)s * P.K / P.split), kb1 = (int)((int64_t)(s + 1) * P.K / P.split);
    const int a = lower_k(P.s_k, e0, e1, kb0);
    const int b = lower_k(P.s_k, a, e1, kb1);
    e0 = a;
    e1 = b;
  }
}

// acc[r] += sum over entries [e0,e1) of op(A)(p_r, :) . op(B)(:, q_r), where output
// o = lane + 32 r sits at (p_r, q_r) = (o / N, o % N).  Offsets are recomputed from
// the lane id inside the loop: integer work is free next to the FP64 pipe, registers
// are not.
template <int M, int N, int KC>
__device__ __forceinline__ void products_mn(const NumParams &P, int e0, int e1, int kk,
                                            double (&acc)[(M * N + 31) / 32]) {
  constexpr int MN = M * N, R = (MN + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int k = KC ? KC : kk;
  // element strides inside op(A) (m x k) and op(B) (k x n) blocks
  const int a_sp = P.ta ? 1 : k, a_sl = P.ta ? M : 1;
  const int b_sl = P.tb ? 1 : N, b_sq = P.tb ? k : 1;
  for (int e = e0; e < e1; ++e) {
    const double *__restrict__ a = P.A + P.s_a[e];
    const double *__restrict__ b = P.B + P.s_b[e];
#pragma unroll 1
    for (int l = 0; l < k; ++l) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int o = lane + 32 * r;
        if (r < R - 1 || o < MN)
          acc[r] = fma(__ldg(a + (o / N) * a_sp + l * a_sl), __ldg(b + (o % N) * b_sq + l * b_sl),
                       acc[r]);
      }
    }
  }
}

template <int M, int N>
__device__ __forceinline__ void task_mn(const NumParams &P, int c, int s) {
  constexpr int MN = M * N, R = (MN + 31) / 32;
  const int lane = threadIdx.x & 31;
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  for (int kc = 0; kc < P.Dk; ++kc) {
    int e0, e1;
    run_range(P, (int64_t)c * P.Dk + kc, s, e0, e1);
    if (e0 >= e1) continue;
    const int k = P.kval[kc];
    switch (k) {
      case 5: products_mn<M, N, 5>(P, e0, e1, k, acc); break;
      case 13: products_mn<M, N, 13>(P, e0, e1, k, acc); break;
      case 23: products_mn<M, N, 23>(P, e0, e1, k, acc); break;
      default: products_mn<M, N, 0>(P, e0, e1, k, acc); break;
    }
  }
  const int64_t off = P.c_off[c];
  if (P.split > 1) {
    double *w = P.W + (int64_t)s * P.nelemC + off;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < MN) w[lane + 32 * r] = acc[r];
    return;
  }
  const int cin = P.c_cin[c];
  const double *ci = (P.has_beta && cin >= 0) ? P.Cin + P.cin_off[cin] : nullptr;
  if (!P.alpha_one || ci) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int o = lane + 32 * r;
      if (o < MN) {
        double v = P.alpha * acc[r];
        if (ci) v = fma(P.beta, ci[o], v);
        P.C[off + o] = v;
      }
    }
  } else {  // alpha == 1, no C_in: store the sums without an FP64 multiply
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < MN) P.C[off + lane + 32 * r] = acc[r];
  }
}

// any (m, n): outputs in passes of 32 * RG per lane group
constexpr int RG = 8;

__device__ void task_generic(const NumParams &P, int c, int s, int m, int n) {
  const int lane = threadIdx.x & 31;
  const int mn = m * n;
  const int64_t off = P.c_off[c];
  const int cin = P.c_cin[c];
  const double *ci = (P.split == 1 && P.has_beta && cin >= 0) ? P.Cin + P.cin_off[cin] : nullptr;
  for (int o0 = 0; o0 < mn; o0 += 32 * RG) {
    double acc[RG];
    int pr[RG], qr[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      acc[r] = 0.0;
      const int o = min(o0 + lane + 32 * r, mn - 1);
      pr[r] = o / n;
      qr[r] = o % n;
    }
    for (int kc = 0; kc < P.Dk; ++kc) {
      int e0, e1;
      run_range(P, (int64_t)c * P.Dk + kc, s, e0, e1);
      if (e0 >= e1) continue;
      const int k = P.kval[kc];
      const int a_sp = P.ta ? 1 : k, a_sl = P.ta ? m : 1;
      const int b_sl = P.tb ? 1 : n, b_sq = P.tb ? k : 1;
      for (int e = e0; e < e1; ++e) {
        const double *a = P.A + P.s_a[e];
        const double *b = P.B + P.s_b[e];
        for (int l = 0; l < k; ++l) {
#pragma unroll
          for (int r = 0; r < RG; ++r)
            if (o0 + lane + 32 * r < mn)
              acc[r] = fma(__ldg(a + pr[r] * a_sp + l * a_sl), __ldg(b + qr[r] * b_sq + l * b_sl), acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      const int o = o0 + lane + 32 * r;
      if (o < mn) {
        if (P.split > 1) {
          P.W[(int64_t)s * P.nelemC + off + o] = acc[r];
        } else {
          double v = P.alpha * acc[r];
          if (ci) v = fma(P.beta, ci[o], v);
          P.C[off + o] = v;
        }
      }
    }
  }
}

__device__ __forceinline__ void dispatch_task(const NumParams &P, int c, int s) {
  const int cls = P.c_cls[c];
  const int m = P.cls_m[cls], n = P.cls_n[cls];
#define BST_MN(MM, NN) \
  if (m == MM && n == NN) { task_mn<MM, NN>(P, c, s); return; }
  BST_MN(5, 5)
  BST_MN(5, 13)
  BST_MN(5, 23)
  BST_MN(13, 5)
  BST_MN(13, 13)
  BST_MN(13, 23)
  BST_MN(23, 5)
  BST_MN(23, 13)
  BST_MN(23, 23)
#undef BST_MN
  task_generic(P, c, s, m, n);
}

// one warp per (C block, K part): used with split-K
__global__ void __launch_bounds__(256, 2) k_num_fp64(NumParams P) {
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= P.ntasks * P.split) return;
  const int64_t t = gw / P.split;
  const int s = (int)(gw % P.split);
  dispatch_task(P, P.task_c[t], s);
}

// Persistent form: a grid sized to fill the GPU once; every warp takes the next work
// item (plan << 32 | C block) from a global counter until the list is exhausted.  The
// items are ordered by decreasing cost, so the long C blocks start first and the warps
// finish together -- with one launch-time task per warp, a CTA holding one long task
// would keep its SM slot while its other warps sat idle.  No waits: a warp that finds
// the counter past the end returns.
template <class GetP>
__device__ __forceinline__ void persist_loop(const int64_t *__restrict__ items, int64_t nitems,
                                             unsigned long long *counter, GetP get) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned long long)nitems) return;
    const int64_t v = items[it];
    dispatch_task(get(v >> 32), (int)(v & 0xffffffffll), 0);
  }
}

// one plan, parameters by value
__global__ void __launch_bounds__(256, 2)
    k_num_fp64_persist1(NumParams P, const int64_t *__restrict__ items, int64_t nitems,
                        unsigned long long *counter) {
  persist_loop(items, nitems, counter, [&](int64_t) -> const NumParams & { return P; });
}

// many plans (a batch), parameters in device memory
__global__ void __launch_bounds__(256, 2)
    k_num_fp64_persist(const NumParams *__restrict__ plans, const int64_t *__restrict__ items,
                       int64_t nitems, unsigned long long *counter) {
  persist_loop(items, nitems, counter, [&](int64_t pl) -> const NumParams & { return plans[pl]; });
}

// ---- staged persistent kernel ---------------------------------------------------------
//
// The work units are row tiles of C blocks (whole blocks up to 32 * kMaxR elements) and
// their entries are (product, inner panel) pairs, both cut on the host so that one
// entry's operands always fit a shared-memory slot (kStageMax doubles).  A warp walks a
// stream of jobs (the entries of its tiles, tile by tile) and keeps two slots: while it
// multiplies the op(A) and op(B) panels of job j from one slot, those of job j + 1 --
// possibly the first job of its next tile -- arrive in the other through cp.async, so
// the FP64 pipe never waits on an L2 round trip inside a product.  The operands are then
// read from shared memory (broadcast for A, consecutive for B).  Tiles come from the
// cost-ordered list in chunks of `chunk` consecutive items: warp w of W takes chunks w
// and W + w, then the next free chunk from a counter each time it has used up one, so
// a warp that drew expensive tiles takes fewer of the cheaper ones later (a fixed
// stride left the most expensive tile of every round to the same warps: 27 % above
// the mean load on the rank-4 contraction's 28 000 tiles).  A warp knows its next two
// tiles ahead: the descriptor of the next tile is loaded one tile ahead and its first
// entries while the current tile runs, and the counter is read one tile before its
// value is needed, so the atomic's latency is hidden too.  Which warp runs a tile does
// not change its result: every tile is summed by one warp in its entry order.

constexpr int kMaxR = 17;         // accumulators per lane: tiles up to 544 elements
constexpr int kTile = 32 * kMaxR;
// doubles per slot (two slots per warp): at most 1184 keeps three 4-warp CTAs resident
// per SM (3 x (2 x 4 x 1184 x 8 B + 1 KB) <= 228 KB); the panels get narrower, but with
// 1536 the contraction plans ran 2 CTAs per SM and lost 8-9 % (FP64 pipe 68-82 % busy)
constexpr int kStageMax = 1184;
constexpr int kStageWarps = 4;    // warps per CTA
constexpr int kF64Desc = kF64DescWords;

// Work unit: a row tile of a C block (the whole block when it has at most 32 * kMaxR
// elements).  Descriptor: 0 element offset of the tile in C, 1 first entry, 2 entry
// count, 3 tile rows m | n << 12, 4 C_in block (-1: none), 5 element offset of the tile
// inside the C_in block, 6 C block, 7 inner split s (>= 1).
struct F64Blk {
  int off, eb, ne, m, n, cin, cio, s;
};

__device__ __forceinline__ F64Blk f64_blk(int dw) {
  F64Blk b;
  b.off = __shfl_sync(0xffffffffu, dw, 0);
  b.eb = __shfl_sync(0xffffffffu, dw, 1);
  b.ne = __shfl_sync(0xffffffffu, dw, 2);
  const int mn = __shfl_sync(0xffffffffu, dw, 3);
  b.cin = __shfl_sync(0xffffffffu, dw, 4);
  b.cio = __shfl_sync(0xffffffffu, dw, 5);
  b.s = max(__shfl_sync(0xffffffffu, dw, 7), 1);
  b.m = mn & 0xfff;
  b.n = (mn >> 12) & 0xfff;
  return b;
}

__device__ __forceinline__ void cp_async8(double *smem, const double *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// `rows` segments of `len` doubles, `stride` apart, packed into dst (out of line: only
// panels and tiles of large products take it).  stride < len: the source is len / stride
// consecutive slabs of rows x stride doubles (a slab-read operand), one contiguous range
// whose slab j supplies columns j stride .. (j + 1) stride - 1 of every row.
__device__ __noinline__ void stage_strided(double *dst, const double *src, int rows, int len,
                                           int stride) {
  const int lane = threadIdx.x & 31;
  if (stride < len) {
    const int per = rows * stride;
    for (int i = lane; i < rows * len; i += 32) {
      const int j = i / per, rem = i - j * per, r = rem / stride;
      cp_async8(dst + r * len + j * stride + (rem - r * stride), src + i);
    }
    return;
  }
  for (int r = 0; r < rows; ++r)
    for (int c = lane; c < len; c += 32) cp_async8(dst + r * len + c, src + (int64_t)r * stride + c);
}

template <bool STRIDED>
__device__ __forceinline__ void stage_2d(double *dst, const double *src, int rows, int len,
                                         int stride) {
  const int lane = threadIdx.x & 31;
  if (!STRIDED || len == stride) {
    for (int i = lane; i < rows * len; i += 32) cp_async8(dst + i, src + i);
  } else {
    stage_strided(dst, src, rows, len, stride);
  }
}

// One job's operands into a slot in their stored layouts, restricted to the job's tile
// rows and inner panel: op(A) is m x w (stored as m rows of w, or w rows of m when
// transposed), op(B) is w x n (w rows of n, or n rows of w).  The entry gives the first
// element of each and the stored row strides (sa | sb << 16); contiguous when a stride
// equals the row length.
template <bool STRIDED>
__device__ __forceinline__ void stage_product(double *slot, const double *a, const double *b,
                                              int m, int n, int w, int strides, int ta, int tb) {
  const int sa = strides & 0xffff, sb = strides >> 16;
  if (ta)
    stage_2d<STRIDED>(slot, a, w, m, sa);
  else
    stage_2d<STRIDED>(slot, a, m, w, sa);
  if (tb)
    stage_2d<STRIDED>(slot + m * w, b, n, w, sb);
  else
    stage_2d<STRIDED>(slot + m * w, b, w, n, sb);
}

// acc[r] += op(A)(p_r, :) . op(B)(:, q_r) from a slot for o = lane + 32 r = p_r n + q_r:
// any (m, n) with m n <= 32 kMaxR, runtime sizes, one body for every size.  Bodies
// specialised at compile time per (m, n) in {5, 13, 23}^2 and k in {5, 13, 23} were no
// faster on GB300 (the FP64 pipe, not the index arithmetic, bounds the product) and their
// code cost instruction-fetch stalls; one body per accumulator count thrashed the
// instruction cache outright.
__device__ __forceinline__ void slot_product_rt(const NumParams &P, const double *__restrict__ As,
                                                int m, int n, int k, double (&acc)[kMaxR]) {
  const int lane = threadIdx.x & 31, mn = m * n;
  const double *__restrict__ Bs = As + m * k;
  const int a_sp = P.ta ? 1 : k, a_sl = P.ta ? m : 1;
  const int b_sl = P.tb ? 1 : n, b_sq = P.tb ? k : 1;
  const int R = (mn + 31) >> 5;
  // output by output: the element's row and column are found once (incrementally from
  // the previous accumulator's: o grows by 32), then its whole dot product runs
  int p = lane / n, q = lane - p * n;
  const int dp = 32 / n, dq = 32 - dp * n;
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) {
    if (r >= R) break;
    if (lane + 32 * r < mn) {
      const double *a = As + p * a_sp, *b = Bs + q * b_sq;
      double s = acc[r];
#pragma unroll 4
      for (int l = 0; l < k; ++l) s = fma(a[l * a_sl], b[l * b_sl], s);
      acc[r] = s;
    }
    p += dp;
    q += dq;
    if (q >= n) {
      q -= n;
      ++p;
    }
  }
}

// The inner dimension split s ways over the lanes, for tiles whose m n leaves lanes idle
// (65 outputs on 3 x 32 lanes): virtual output v = lane + 32 r = g m n + o (o = p n + q)
// accumulates op(A)(p, l) op(B)(l, q) over l = g, g + s, g + 2s, ... < k.  The s partial
// sums of an output are added once, at the end of the tile (split_reduce).
__device__ __forceinline__ void slot_product_split(const NumParams &P,
                                                   const double *__restrict__ As, int m, int n,
                                                   int k, int s, double (&acc)[kMaxR]) {
  const int lane = threadIdx.x & 31, nv = s * m * n;
  const double *__restrict__ Bs = As + m * k;
  const int a_sp = P.ta ? 1 : k, a_sl = P.ta ? m : 1;
  const int b_sl = P.tb ? 1 : n, b_sq = P.tb ? k : 1;
  const int mn = m * n;
  int g = lane / mn;
  const int o = lane - g * mn;
  int p = o / n, q = o - p * n;
  const int dp = 32 / n, dq = 32 - dp * n;
  const int da = s * a_sl, db = s * b_sl;
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) {
    if (32 * r >= nv) break;
    if (lane + 32 * r < nv) {
      const double *a = As + p * a_sp + g * a_sl, *b = Bs + q * b_sq + g * b_sl;
      double t = acc[r];
#pragma unroll 1
      for (int l = g; l < k; l += s) {
        t = fma(*a, *b, t);
        a += da;
        b += db;
      }
      acc[r] = t;
    }
    // the virtual output 32 further on
    p += dp;
    q += dq;
    if (q >= n) {
      q -= n;
      ++p;
    }
    while (p >= m) {
      p -= m;
      ++g;
    }
  }
}

// acc[r] <- sum over g = 0 .. s - 1 (in that order) of the partial sums of output
// o = lane + 32 r, through `red` (s m n doubles of a free slot)
__device__ __forceinline__ void split_reduce(double *red, int mn, int s, double (&acc)[kMaxR]) {
  const int lane = threadIdx.x & 31, nv = s * mn;
#pragma unroll
  for (int r = 0; r < kMaxR; ++r)
    if (lane + 32 * r < nv) red[lane + 32 * r] = acc[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) {
    const int o = lane + 32 * r;
    if (o < mn) {
      double t = red[o];
      for (int g = 1; g < s; ++g) t += red[g * mn + o];
      acc[r] = t;
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void slot_dispatch(const NumParams &P, const double *As, int m, int n,
                                              int k, double (&acc)[kMaxR]) {
  slot_product_rt(P, As, m, n, k, acc);
}

// C = alpha * acc + beta * C_in for one C block (C_in unread when beta == 0)
__device__ __forceinline__ void store_block(const NumParams &P, const F64Blk &b,
                                            const double (&acc)[kMaxR]) {
  const int lane = threadIdx.x & 31, mn = b.m * b.n;
  const double *ci = (P.has_beta && b.cin >= 0) ? P.Cin + P.cin_off[b.cin] + b.cio : nullptr;
  double *C = P.C + b.off;
  if (!P.alpha_one || ci) {
#pragma unroll
    for (int r = 0; r < kMaxR; ++r) {
      const int o = lane + 32 * r;
      if (o < mn) {
        double v = P.alpha * acc[r];
        if (ci) v = fma(P.beta, ci[o], v);
        C[o] = v;
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < kMaxR; ++r)
      if (lane + 32 * r < mn) C[lane + 32 * r] = acc[r];
  }
}

// A K split (ksplit > 1, single plans only): item i is part i % ksplit of tile
// items[i / ksplit]; the part takes its share of the tile's entries (contiguous, in
// entry order) and writes its partial sums, without alpha, to W + part * nelem(C), which
// k_splitk_reduce adds in part order.
__device__ __forceinline__ void store_part(const NumParams &P, const F64Blk &b, int part,
                                           const double (&acc)[kMaxR]) {
  const int lane = threadIdx.x & 31, mn = b.m * b.n;
  double *W = P.W + (int64_t)part * P.nelemC + b.off;
#pragma unroll
  for (int r = 0; r < kMaxR; ++r)
    if (lane + 32 * r < mn) W[lane + 32 * r] = acc[r];
}

template <bool STRIDED, bool SPLIT, class GetP>
__device__ __forceinline__ void staged_loop(const int64_t *__restrict__ items, int64_t nitems,
                                            int slot_elems, unsigned long long *__restrict__ counter,
                                            int chunk, int ksplit, GetP get) {
  extern __shared__ double smem_stage[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double *slots = smem_stage + (size_t)wid * 2 * slot_elems;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
  auto item = [&](int64_t i) -> int64_t {
    if (i >= nitems) return -1;
    if (ksplit <= 1) return items[i];
    return items[i / ksplit] | ((i % ksplit) << 32);
  };
  // a K part's share of its tile's entries
  auto part_of = [&](F64Blk b, int64_t v) -> F64Blk {
    if (ksplit > 1 && v >= 0) {
      const int q = (int)(v >> 32);
      const int e0 = (int)((int64_t)b.ne * q / ksplit), e1 = (int)((int64_t)b.ne * (q + 1) / ksplit);
      b.eb += e0;
      b.ne = e1 - e0;
    }
    return b;
  };
  // item positions [pos, end) left of the current chunk.  Chunks w and W + w are the
  // warp's own; on opening a chunk lane 0 requests the next one from the counter
  // (`ticket`, chunk 2 W + ticket), whose value is first read when that chunk opens.
  int64_t pos = gw * chunk, end = pos + chunk;
  bool second = true;
  unsigned long long ticket = 0;
  auto next_pos = [&]() -> int64_t {
    if (pos == end) {
      int64_t c = nw + gw;
      if (!second) c = 2 * nw + (int64_t)__shfl_sync(0xffffffffu, ticket, 0);
      second = false;
      if (lane == 0) ticket = atomicAdd(counter, 1ull);
      pos = c * chunk;
      end = pos + chunk;
    }
    return pos++;
  };
  auto word = [&](int64_t v) -> int {
    return (v >= 0 && lane < kF64Desc)
               ? get(v >> 32).fdesc[(v & 0xffffffffll) * kF64Desc + lane]
               : 0;
  };
  // entries g0 .. g0 + 31 of a block, one per lane
  auto group = [&](int64_t v, const F64Blk &b, int g0) -> int4 {
    return (v >= 0 && g0 + lane < b.ne) ? get(v >> 32).fents[(int64_t)b.eb + g0 + lane]
                                        : make_int4(0, 0, 0, 0);
  };
  int64_t v = item(next_pos());
  if (v < 0) return;
  int64_t vn = item(next_pos());
  int dw = word(v), dwn = word(vn);
  F64Blk b = part_of(f64_blk(dw), v);
  int4 ent = group(v, b, 0);
  int slot = 0;
  bool staged = false;  // slot holds the first product of the current block
  for (;;) {
    const NumParams &P = get(v >> 32);
    const F64Blk bn = part_of(f64_blk(dwn), vn);
    const int4 entn = group(vn, bn, 0);
    const int64_t vnn = vn >= 0 ? item(next_pos()) : -1;
    const int dwnn = word(vnn);
    if (!staged && b.ne > 0) {
      stage_product<STRIDED>(slots + slot * slot_elems, P.A + __shfl_sync(0xffffffffu, ent.x, 0),
                    P.B + __shfl_sync(0xffffffffu, ent.y, 0), b.m, b.n,
                    __shfl_sync(0xffffffffu, ent.z, 0), __shfl_sync(0xffffffffu, ent.w, 0), P.ta,
                    P.tb);
      cp_commit();
    }
    double acc[kMaxR];
#pragma unroll
    for (int r = 0; r < kMaxR; ++r) acc[r] = 0.0;
    int g0 = 0;
    for (int e = 0; e < b.ne; ++e) {
      if (e - g0 == 32) {
        g0 += 32;
        ent = group(v, b, g0);
      }
      const int k = __shfl_sync(0xffffffffu, ent.z, e - g0);
      // the next job into the other slot: this block's next product, else the first
      // product of the next block
      double *nxt = slots + (slot ^ 1) * slot_elems;
      if (e + 1 < b.ne) {
        int j = e + 1 - g0;
        int4 src = ent;
        if (j == 32) {
          src = group(v, b, g0 + 32);
          j = 0;
        }
        stage_product<STRIDED>(nxt, P.A + __shfl_sync(0xffffffffu, src.x, j),
                      P.B + __shfl_sync(0xffffffffu, src.y, j), b.m, b.n,
                      __shfl_sync(0xffffffffu, src.z, j), __shfl_sync(0xffffffffu, src.w, j), P.ta,
                      P.tb);
      } else if (vn >= 0 && bn.ne > 0) {
        const NumParams &Pn = get(vn >> 32);
        stage_product<STRIDED>(nxt, Pn.A + __shfl_sync(0xffffffffu, entn.x, 0),
                      Pn.B + __shfl_sync(0xffffffffu, entn.y, 0), bn.m, bn.n,
                      __shfl_sync(0xffffffffu, entn.z, 0), __shfl_sync(0xffffffffu, entn.w, 0),
                      Pn.ta, Pn.tb);
      }
      cp_commit();
      cp_wait_prev();
      __syncwarp();
      if (SPLIT && b.s > 1)
        slot_product_split(P, slots + slot * slot_elems, b.m, b.n, k, b.s, acc);
      else
        slot_dispatch(P, slots + slot * slot_elems, b.m, b.n, k, acc);
      __syncwarp();
      slot ^= 1;
    }
    staged = b.ne > 0 && vn >= 0 && bn.ne > 0;
    // the slot of the tile's last job is free: the next tile's first job went to the other
    if (SPLIT && b.s > 1 && b.ne > 0) split_reduce(slots + (slot ^ 1) * slot_elems, b.m * b.n, b.s, acc);
    if (ksplit > 1)
      store_part(P, b, (int)(v >> 32), acc);
    else
      store_block(P, b, acc);
    if (vn < 0) break;
    v = vn;
    vn = vnn;
    dw = dwn;
    dwn = dwnn;
    b = bn;
    ent = entn;
  }
  cp_wait_all();
}

// STRIDED: the plan has row tiles or inner panels (staging copies strided rows);
// SPLIT: some tile spreads its inner dimension over lane groups.  Each is a separate
// instance so that plans without them run none of their code (a larger loop body costs
// instruction-fetch stalls on every tile).
template <bool STRIDED, bool SPLIT>
__global__ void __launch_bounds__(32 * kStageWarps, 3)
    k_num_fp64_staged1(NumParams P, const int64_t *__restrict__ items, int64_t nitems,
                       int slot_elems, unsigned long long *counter, int chunk, int ksplit) {
  staged_loop<STRIDED, SPLIT>(items, nitems, slot_elems, counter, chunk, ksplit,
                              [&](int64_t) -> const NumParams & { return P; });
}

template <bool STRIDED, bool SPLIT>
__global__ void __launch_bounds__(32 * kStageWarps, 3)
    k_num_fp64_staged(const NumParams *__restrict__ plans, const int64_t *__restrict__ items,
                      int64_t nitems, int slot_elems, unsigned long long *counter, int chunk,
                      int ksplit) {
  staged_loop<STRIDED, SPLIT>(items, nitems, slot_elems, counter, chunk, 1,
                              [&](int64_t pl) -> const NumParams & { return plans[pl]; });
}

// ---- schedule of the staged kernel (built with the plan) ----------------------------
//
// Work units ("tiles") are row ranges of C blocks: a block of m x n elements with
// m n > 32 * kMaxR is cut into tiles of floor(32 kMaxR / n) rows.  A product whose
// tile operands exceed a slot ((tile rows + n) k > kStageMax) is cut into panels of the
// inner dimension of width floor(kStageMax / (tile rows + n)).  Each tile lists its
// (product, panel) entries {first A element, first B element, panel width w, row
// strides}, in the product order of the stacks; per (m, n) class the host passes the
// tile rows, and per (class, k class) the panel width.

struct SchedTabs {
  const int32_t *cls_m, *cls_n, *tile_rows;  // per (m, n) class
  const int32_t *wpanel;                     // per (class, k class): panel width
  const int32_t *kval;
  int32_t Dk, ta, tb;
  // slab reading of A (null: none): per k class the slab width k_i, per entry its stored
  // A block, per stored A block its element offset in the tensor
  const int32_t *kin, *s_ab;
  const int64_t *a_toff;
};

// panels of one product of inner size k at panel width w: whole panels, or with slab
// width ki > 0 panels that never cross a slab (several whole slabs when w >= ki)
__device__ __forceinline__ int panel_count(int k, int w, int ki) {
  if (ki <= 0) return (k + w - 1) / w;
  if (w >= ki) {
    const int ws = (w / ki) * ki;
    return (k + ws - 1) / ws;
  }
  return (k / ki) * ((ki + w - 1) / w);
}

__device__ __forceinline__ int ntiles_of(const SchedTabs &S, int cls) {
  const int tr = S.tile_rows[cls];
  return (S.cls_m[cls] + tr - 1) / tr;
}

__global__ void k_f64_tile_count(int64_t nc, const int32_t *__restrict__ c_cls, SchedTabs S,
                                 int32_t *__restrict__ cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) cnt[c] = ntiles_of(S, c_cls[c]);
}

// entries of every tile of block c: sum over its products of the panel count
__global__ void k_f64_ent_count(int64_t nc, const int32_t *__restrict__ c_cls,
                                const int32_t *__restrict__ run_len, const int64_t *__restrict__ tbeg,
                                SchedTabs S, int32_t *__restrict__ cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int cls = c_cls[c];
  int s = 0;
  for (int kc = 0; kc < S.Dk; ++kc) {
    const int w = S.wpanel[cls * S.Dk + kc], k = S.kval[kc];
    s += run_len[c * S.Dk + kc] * panel_count(k, w, S.kin ? S.kin[kc] : 0);
  }
  const int nt = ntiles_of(S, cls);
  for (int t = 0; t < nt; ++t) cnt[tbeg[c] + t] = s;
}

// Inner split of every tile (descriptor word 7): the s <= smax of the tile's class that
// needs the fewest FP64 warp instructions -- ceil(s mt n / 32) for each of the
// ceil(w / s) steps of a panel of width w, plus (s - 1) ceil(mt n / 32) adds for the
// final sums -- when it saves anything on a tile with at least kSplitLongInner inner
// elements in all, at least 1/8 of the unsplit count on one with kSplitMinInner or more,
// else 1 (on short tiles the final sums cost more than the idle lanes).  The plan-wide
// sums of the unsplit counts and of the savings decide whether the plan splits at all
// (refresh_f64_split).
constexpr int kMaxSplit = 16;
constexpr int kSplitMinInner = 48;
constexpr int kSplitLongInner = 128;

__device__ int f64_split_of(int32_t *__restrict__ d, const int4 *__restrict__ ents, int smax,
                            int slot_elems, long long &c1, long long &saved) {
  const int mn = (d[3] & 0xfff) * ((d[3] >> 12) & 0xfff), ne = d[2];
  // s m n partial sums fit the accumulators and, for the final sums, one slot
  smax = min(min(smax, kMaxSplit), min(kTile, slot_elems) / max(mn, 1));
  const long long v1 = (mn + 31) / 32;
  int best = 1;
  c1 = 0;
  saved = 0;
  // short tiles (most of a plan of small products) never split: one pass over the widths
  long long w1 = 0;
  for (int e = 0; e < ne; ++e) w1 += ents[(int64_t)d[1] + e].z;
  if (w1 < kSplitMinInner || smax < 2) {
    c1 = v1 * w1;
    return 1;
  }
  long long W[kMaxSplit + 1];
  for (int s = 1; s <= max(smax, 1); ++s) W[s] = 0;
  for (int e = 0; e < ne; ++e) {
    const int w = ents[(int64_t)d[1] + e].z;
    for (int s = 1; s <= max(smax, 1); ++s) W[s] += (w + s - 1) / s;
  }
  c1 = v1 * W[1];
  long long cb = c1;
  for (int s = 2; s <= smax; ++s) {
    const long long c = (long long)((s * mn + 31) / 32) * W[s] + (s - 1) * v1;
    if (c < cb) {
      cb = c;
      best = s;
    }
  }
  if ((W[1] >= kSplitLongInner ? cb >= c1 : 8 * cb > 7 * c1) || W[1] < kSplitMinInner) best = 1;
  if (best > 1) saved = c1 - cb;
  return best;
}

// descriptors and entries of every tile of C block c, each tile's cost key
// (63 - floor(log2(flops)): a stable partition on it lists costly tiles first) and its
// inner split, with its FP64 instruction counts added to c1_sum / saved_sum
__device__ __forceinline__ void f64_tiles_of(
    int64_t c, const int32_t *__restrict__ c_cls, const int32_t *__restrict__ run_start,
    const int32_t *__restrict__ run_len, const int32_t *__restrict__ s_a,
    const int32_t *__restrict__ s_b, const int64_t *__restrict__ c_off,
    const int32_t *__restrict__ c_cin, const int64_t *__restrict__ tbeg,
    const int64_t *__restrict__ ebeg, const SchedTabs &S, int32_t *__restrict__ desc,
    int4 *__restrict__ ents, int32_t *__restrict__ key, const int32_t *__restrict__ cls_smax,
    int slot_elems, long long &c1_sum, long long &saved_sum) {
  const int cls = c_cls[c];
  const int m = S.cls_m[cls], n = S.cls_n[cls], tr = S.tile_rows[cls];
  const int nt = (m + tr - 1) / tr;
  for (int t = 0; t < nt; ++t) {
    const int64_t tile = tbeg[c] + t;
    const int p0 = t * tr, mt = min(tr, m - p0);
    int64_t q = ebeg[tile];
    unsigned long long flops = 0;
    long long w1 = 0;  // the tile's inner elements (sum of its entries' panel widths)
    for (int kc = 0; kc < S.Dk; ++kc) {
      const int len = run_len[c * S.Dk + kc];
      if (len == 0) continue;
      const int e0 = run_start[c * S.Dk + kc];
      const int k = S.kval[kc], w = S.wpanel[cls * S.Dk + kc];
      // stored row strides of the panels: A is m x k (k x m when transposed), B is k x n
      // (n x k when transposed)
      const int strides = (S.ta ? m : k) | ((S.tb ? k : n) << 16);
      const int ki = S.kin ? S.kin[kc] : 0;
      for (int e = e0; e < e0 + len; ++e) {
        if (ki > 0) {
          // slabs of the tensor block (whole blocks only: p0 == 0): stored row stride ki
          const int64_t ab = S.a_toff[S.s_ab[e]];
          const int st = ki | ((S.tb ? k : n) << 16);
          if (w >= ki) {
            const int ws = (w / ki) * ki;
            for (int l0 = 0; l0 < k; l0 += ws) {
              const int b = s_b[e] + (S.tb ? l0 : l0 * n);
              ents[q++] = make_int4((int)(ab + (int64_t)(l0 / ki) * m * ki), b, min(ws, k - l0), st);
              w1 += min(ws, k - l0);
            }
          } else {
            for (int l0 = 0; l0 < k; l0 += ki)
              for (int c0 = 0; c0 < ki; c0 += w) {
                const int b = s_b[e] + (S.tb ? l0 + c0 : (l0 + c0) * n);
                ents[q++] = make_int4((int)(ab + (int64_t)(l0 / ki) * m * ki + c0), b,
                                      min(w, ki - c0), st);
                w1 += min(w, ki - c0);
              }
          }
          continue;
        }
        for (int l0 = 0; l0 < k; l0 += w) {
          const int wl = min(w, k - l0);
          const int a = s_a[e] + (S.ta ? l0 * m + p0 : p0 * k + l0);
          const int b = s_b[e] + (S.tb ? l0 : l0 * n);
          ents[q++] = make_int4(a, b, wl, strides);
          w1 += wl;
        }
      }
      flops += (unsigned long long)len * mt * n * k;
    }
    // the descriptor as two 16-byte stores (word 7, the split, once it is known)
    int32_t *d = desc + tile * kF64Desc;
    int4 *dv = reinterpret_cast<int4 *>(d);
    dv[0] = make_int4((int32_t)(c_off[c] + (int64_t)p0 * n), (int32_t)ebeg[tile],
                      (int32_t)(q - ebeg[tile]), mt | (n << 12));
    key[tile] = __clzll(flops + 1ull);
    // a short tile never splits (the test f64_split_of starts with), decided here
    // without reading its entries back
    const int mn = mt * n;
    const int smax = min(min(cls_smax[cls], kMaxSplit), min(kTile, slot_elems) / max(mn, 1));
    long long c1, saved = 0;
    int split = 1;
    if (w1 < kSplitMinInner || smax < 2)
      c1 = (long long)((mn + 31) / 32) * w1;
    else
      split = f64_split_of(d, ents, cls_smax[cls], slot_elems, c1, saved);
    dv[1] = make_int4(c_cin[c], p0 * n, (int32_t)c, split);
    c1_sum += c1;
    saved_sum += saved;
  }
}

// all C blocks; sums[0] += unsplit FP64 instruction counts, sums[1] += split savings
__global__ void k_f64_tiles(int64_t nc, const int32_t *__restrict__ c_cls,
                            const int32_t *__restrict__ run_start, const int32_t *__restrict__ run_len,
                            const int32_t *__restrict__ s_a, const int32_t *__restrict__ s_b,
                            const int64_t *__restrict__ c_off, const int32_t *__restrict__ c_cin,
                            const int64_t *__restrict__ tbeg, const int64_t *__restrict__ ebeg,
                            SchedTabs S, int32_t *__restrict__ desc, int4 *__restrict__ ents,
                            int32_t *__restrict__ key, const int32_t *__restrict__ cls_smax,
                            int slot_elems, unsigned long long *__restrict__ sums) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long c1_sum = 0, saved_sum = 0;
  if (c < nc) f64_tiles_of(c, c_cls, run_start, run_len, s_a, s_b, c_off, c_cin, tbeg, ebeg, S,
                           desc, ents, key, cls_smax, slot_elems, c1_sum, saved_sum);
  for (int o = 16; o > 0; o >>= 1) {
    c1_sum += __shfl_down_sync(0xffffffffu, c1_sum, o);
    saved_sum += __shfl_down_sync(0xffffffffu, saved_sum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], (unsigned long long)c1_sum);
    if (saved_sum) atomicAdd(&sums[1], (unsigned long long)saved_sum);
  }
}

// sums[0] += unsplit FP64 instruction counts, sums[1] += savings of the chosen splits
__global__ void k_f64_split(int64_t ntiles, const int4 *__restrict__ ents,
                            const int32_t *__restrict__ c_cls, const int32_t *__restrict__ cls_smax,
                            int slot_elems, int32_t *__restrict__ desc,
                            unsigned long long *__restrict__ sums) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long c1 = 0, saved = 0;
  if (t < ntiles) {
    int32_t *d = desc + t * kF64Desc;
    d[7] = f64_split_of(d, ents, cls_smax[c_cls[d[6]]], slot_elems, c1, saved);
  }
  for (int o = 16; o > 0; o >>= 1) {
    c1 += __shfl_down_sync(0xffffffffu, c1, o);
    saved += __shfl_down_sync(0xffffffffu, saved, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], (unsigned long long)c1);
    atomicAdd(&sums[1], (unsigned long long)saved);
  }
}

__global__ void k_f64_nosplit(int64_t ntiles, int32_t *__restrict__ desc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntiles) desc[t * kF64Desc + 7] = 1;
}

__global__ void k_plan_items(int64_t nc, int64_t base, int64_t *__restrict__ item) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) item[c] = base | c;
}

// cost of every C block (flops of its products) as a descending-order key
// 63 - floor(log2(cost)): a stable partition on it lists costly blocks first
__global__ void k_task_cost_keys(int64_t nc, int32_t Dk, const int32_t *__restrict__ run_len,
                                 const int32_t *__restrict__ kval, const int32_t *__restrict__ c_cls,
                                 const int32_t *__restrict__ cls_m, const int32_t *__restrict__ cls_n,
                                 int32_t *__restrict__ key) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  unsigned long long k = 0;
  for (int q = 0; q < Dk; ++q) k += (unsigned long long)run_len[c * Dk + q] * kval[q];
  const int cls = c_cls[c];
  key[c] = __clzll(k * (unsigned long long)cls_m[cls] * cls_n[cls] + 1ull);
}

__global__ void k_gather_items(const int64_t *__restrict__ in, const int32_t *__restrict__ perm,
                               int64_t n, int64_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[perm[i]];
}

// C = alpha * sum_{s=0..S-1} W_s + beta * C_in, one warp per C block
__global__ void k_splitk_reduce(NumParams P, int64_t nc, const int32_t *__restrict__ c_row,
                                const int32_t *__restrict__ c_col, const int32_t *__restrict__ msz,
                                const int32_t *__restrict__ nsz) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= nc) return;
  const int64_t off = P.c_off[c];
  const int len = msz[c_row[c]] * nsz[c_col[c]];
  const int cin = P.c_cin[c];
  const double *ci = (P.has_beta && cin >= 0) ? P.Cin + P.cin_off[cin] : nullptr;
  for (int o = lane; o < len; o += 32) {
    double v = 0.0;
    for (int s = 0; s < P.split; ++s) v += P.W[(int64_t)s * P.nelemC + off + o];
    v = P.alpha * v;
    if (ci) v = fma(P.beta, ci[o], v);
    P.C[off + o] = v;
  }
}

NumParams make_params(bst_plan *p, const NumArgs &a, int split) {
  NumParams P;
  P.A = (p->a_slab && p->stage_elems > 0) ? p->a_slab_base : a.A;
  P.B = a.B;
  P.Cin = a.Cin;
  P.C = a.C;
  P.W = nullptr;
  P.alpha = a.alpha;
  P.alpha_one = a.alpha == 1.0;
  P.has_beta = a.beta != 0.0;
  P.beta = a.beta;
  P.nelemC = p->C->nelem;
  P.ntasks = p->C->nblocks;
  P.split = std::max(1, split);
  P.K = p->K;
  P.Dk = p->Dk;
  P.ta = p->ta;
  P.tb = p->tb;
  P.task_c = p->task_c;
  P.c_cls = p->c_cls;
  P.c_cin = p->c_cin;
  P.c_off = p->C->off;
  P.cin_off = p->Cin ? p->Cin->off : nullptr;
  P.run_start = p->run_start;
  P.run_len = p->run_len;
  P.s_a = p->s_a;
  P.s_b = p->s_b;
  P.s_k = p->s_k;
  P.cls_m = p->cls_m;
  P.cls_n = p->cls_n;
  P.kval = p->kval;
  P.fdesc = p->fdesc;
  P.fents = p->fents;
  return P;
}

}  // namespace

// every native-FP64 execute of a plan with a staged schedule runs the staged kernel (a
// K split too), which reads a slab plan's first tensor in place
bool fp64_reads_slabs(const bst_plan *p, int split) {
  (void)split;
  return p->a_slab && p->stage_elems > 0;
}

size_t num_params_bytes() { return sizeof(NumParams); }

void fill_num_params(bst_plan *p, const NumArgs &a, void *out, bool staged) {
  NumParams P = make_params(p, a, 1);
  if (!staged) P.A = a.A;  // the direct-load kernel reads A through the stacks
  std::memcpy(out, &P, sizeof(P));
}

// Work items of one plan's C blocks in CSR order (item = base | c) and their
// decreasing-cost keys.
void build_plan_items(bst_plan *p, int64_t base, int64_t *items, int32_t *keys, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  k_plan_items<<<nblk(nc, 256), 256, 0, s>>>(nc, base, items);
  BST_CHECK_LAUNCH();
  if (keys) {
    k_task_cost_keys<<<nblk(nc, 256), 256, 0, s>>>(nc, p->Dk, p->run_len, p->kval, p->c_cls,
                                                   p->cls_m, p->cls_n, keys);
    BST_CHECK_LAUNCH();
  }
}

// items reordered by their keys (stable): costly C blocks first
void sort_items(const int64_t *items, const int32_t *keys, int64_t n, int64_t *out, Arena &scratch,
                cudaStream_t s) {
  if (n == 0) return;
  int32_t *perm = scratch.alloc_n<int32_t>((size_t)n);
  int32_t *kp = scratch.alloc_n<int32_t>(65);
  stable_partition(keys, n, 64, perm, kp, scratch, s);
  k_gather_items<<<nblk(n, 256), 256, 0, s>>>(items, perm, n, out);
  BST_CHECK_LAUNCH();
}

// Tiles, entries, descriptors and slot size of the staged kernel; false (stage_elems
// stays 0) when a block size does not fit the descriptor's 12 bits or a row of C (n
// elements) exceeds one output tile.
static std::vector<int32_t> class_split_bounds(const bst_plan *p);
static void apply_split_gate(bst_plan *p, const unsigned long long sums[2], cudaStream_t s);

static bool build_staged(bst_plan *p, cudaStream_t s) {
  p->stage_elems = 0;
  p->n_tiles = 0;
  p->a_slab = false;
  p->sched_ar.ctx = static_cast<Ctx *>(p->ctx);
  p->sched_ar.stream = s;
  p->sched_ar.release_all();
  const int64_t nc = p->C->nblocks;
  if (nc == 0 || p->T == 0) return false;
  const int32_t ncls = p->Dm * p->Dn, Dk = p->Dk;
  std::vector<int32_t> tile_rows((size_t)ncls, 1), wpanel((size_t)ncls * Dk, 1);
  for (int32_t c = 0; c < ncls; ++c) {
    if (p->h_class_ptr[c + 1] == p->h_class_ptr[c]) continue;
    const int64_t m = p->m_vals[c / p->Dn], n = p->n_vals[c % p->Dn];
    if (m >= 4096 || n >= 4096 || n > kTile) return false;
    const int64_t tr = m * n <= kTile ? m : kTile / n;
    if (tr + n > kStageMax) return false;
    tile_rows[(size_t)c] = (int32_t)tr;
  }
  bool strided = false;
  for (int32_t c = 0; c < ncls; ++c)
    if (p->h_class_ptr[c + 1] > p->h_class_ptr[c] && tile_rows[(size_t)c] < p->m_vals[c / p->Dn])
      strided = true;
  // slab reading of A: whole C blocks only (a slab holds all m rows), op(A) = A
  const bool slab = !p->a_slab_kin.empty() && !strided && !p->ta && p->a_slab_toff;
  if (slab) strided = true;
  int64_t slot = 1;
  for (int32_t b = 0; b < p->nb_all; ++b) {
    if (p->h_bucket_ptr[b + 1] == p->h_bucket_ptr[b]) continue;
    const int32_t kc = b % Dk, ncl = (b / Dk) % p->Dn, mc = b / (Dk * p->Dn);
    const int32_t cls = mc * p->Dn + ncl;
    const int64_t n = p->n_vals[ncl], k = p->k_vals[kc], tr = tile_rows[(size_t)cls];
    const int64_t w = (tr + n) * k <= kStageMax ? k : kStageMax / (tr + n);
    wpanel[(size_t)cls * Dk + kc] = (int32_t)w;
    if (w < k) strided = true;
    slot = std::max(slot, (tr + n) * w);
  }
  Arena &ar = p->sched_ar;
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  int32_t *d_tr, *d_wp, *d_kin = nullptr, *d_smax;
  {
    Upload up(p->ctx, s);
    d_tr = up.add_vector(scratch, tile_rows);
    d_wp = up.add_vector(scratch, wpanel);
    d_smax = up.add_vector(scratch, class_split_bounds(p));
    if (slab) d_kin = up.add_vector(scratch, p->a_slab_kin);
    up.done_async();  // read by this stream's kernels below; the plan synchronises later
  }
  unsigned long long *d_sums = scratch.alloc_n<unsigned long long>(2);
  BST_CUDA(cudaMemsetAsync(d_sums, 0, 2 * sizeof(unsigned long long), s));
  SchedTabs S;
  S.cls_m = p->cls_m;
  S.cls_n = p->cls_n;
  S.tile_rows = d_tr;
  S.wpanel = d_wp;
  S.kval = p->kval;
  S.Dk = Dk;
  S.ta = p->ta;
  S.tb = p->tb;
  S.kin = d_kin;
  S.s_ab = p->s_ab;
  S.a_toff = p->a_slab_toff;
  int32_t *tcnt = scratch.alloc_n<int32_t>((size_t)nc);
  int64_t *tbeg = scratch.alloc_n<int64_t>((size_t)nc + 1);
  k_f64_tile_count<<<nblk(nc, 256), 256, 0, s>>>(nc, p->c_cls, S, tcnt);
  BST_CHECK_LAUNCH();
  exscan_i32_i64(tcnt, tbeg, nc, scratch, s);
  int64_t ntiles = 0;
  {
    ReadBack rb(p->ctx, s);
    rb.add(&ntiles, tbeg + nc, 8);
    rb.done();
  }
  int32_t *ecnt = scratch.alloc_n<int32_t>((size_t)ntiles);
  int64_t *ebeg = scratch.alloc_n<int64_t>((size_t)ntiles + 1);
  k_f64_ent_count<<<nblk(nc, 256), 256, 0, s>>>(nc, p->c_cls, p->run_len, tbeg, S, ecnt);
  BST_CHECK_LAUNCH();
  exscan_i32_i64(ecnt, ebeg, ntiles, scratch, s);
  int64_t nents = 0;
  {
    ReadBack rb(p->ctx, s);
    rb.add(&nents, ebeg + ntiles, 8);
    rb.done();
  }
  BST_REQUIRE(nents < INT32_MAX && ntiles < INT32_MAX, BST_ERR_OVERFLOW,
              "more than 2^31-1 staged tiles or entries");
  p->fents = ar.alloc_n<int4>((size_t)nents);
  p->fdesc = ar.alloc_n<int32_t>((size_t)ntiles * kF64Desc);
  p->tkeys = ar.alloc_n<int32_t>((size_t)ntiles);
  k_f64_tiles<<<nblk(nc, 256), 256, 0, s>>>(nc, p->c_cls, p->run_start, p->run_len, p->s_a,
                                            p->s_b, p->C->off, p->c_cin, tbeg, ebeg, S, p->fdesc,
                                            p->fents, p->tkeys, d_smax, (int)slot, d_sums);
  BST_CHECK_LAUNCH();
  // tiles by decreasing cost
  int64_t *it0 = scratch.alloc_n<int64_t>((size_t)ntiles);
  p->titems = ar.alloc_n<int64_t>((size_t)ntiles);
  k_plan_items<<<nblk(ntiles, 256), 256, 0, s>>>(ntiles, 0, it0);
  BST_CHECK_LAUNCH();
  sort_items(it0, p->tkeys, ntiles, p->titems, scratch, s);
  unsigned long long sums[2] = {0, 0};
  {
    ReadBack rb(p->ctx, s);
    rb.add(sums, d_sums, sizeof(sums));
    rb.done();
  }
  scratch.release_all();
  p->n_tiles = ntiles;
  p->stage_elems = (int32_t)slot;
  p->stage_strided = strided;
  p->a_slab = slab;
  apply_split_gate(p, sums, s);
  return true;
}

// per (m, n) class of the plan, the largest inner split the context's tuning allows
static std::vector<int32_t> class_split_bounds(const bst_plan *p) {
  const Ctx *ctx = static_cast<const Ctx *>(p->ctx);
  const int32_t ncls = p->Dm * p->Dn;
  std::vector<int32_t> smax((size_t)ncls, kMaxSplit);
  for (int32_t c = 0; c < ncls; ++c) {
    auto it = ctx->tune_f64_split.find({(int32_t)p->m_vals[c / p->Dn], (int32_t)p->n_vals[c % p->Dn]});
    if (it != ctx->tune_f64_split.end()) smax[(size_t)c] = it->second;
  }
  return smax;
}

// The plan runs the split instance only when the chosen splits save at least 1/25 of all
// its FP64 instructions (a safeguard: a longer loop body once cost every tile a few per
// cent); otherwise every tile is set back to s = 1.
static void apply_split_gate(bst_plan *p, const unsigned long long sums[2], cudaStream_t s) {
  p->stage_split = sums[1] > 0 && 25 * sums[1] >= sums[0];
  if (!p->stage_split && sums[1] > 0) {  // with no saving every tile already has s = 1
    k_f64_nosplit<<<nblk(p->n_tiles, 256), 256, 0, s>>>(p->n_tiles, p->fdesc);
    BST_CHECK_LAUNCH();
  }
  p->split_version = static_cast<const Ctx *>(p->ctx)->tune_version;
}

// (Re)choose the inner split of every staged tile for the context's current tuning.
void refresh_f64_split(bst_plan *p, cudaStream_t s) {
  Ctx *ctx = static_cast<Ctx *>(p->ctx);
  if (p->n_tiles == 0 || p->split_version == ctx->tune_version) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  BST_CUDA(cudaStreamIsCapturing(s, &cap));
  BST_REQUIRE(cap == cudaStreamCaptureStatusNone, BST_ERR_STATE,
              "the context's tuning changed since the plan's FP64 tiles were split; "
              "execute once outside stream capture");
  const std::vector<int32_t> smax = class_split_bounds(p);
  Arena scratch;
  scratch.ctx = ctx;
  scratch.stream = s;
  int32_t *d_smax;
  {
    Upload up(p->ctx, s);
    d_smax = up.add_vector(scratch, smax);
    up.done();
  }
  unsigned long long *d_sums = scratch.alloc_n<unsigned long long>(2);
  BST_CUDA(cudaMemsetAsync(d_sums, 0, 2 * sizeof(unsigned long long), s));
  k_f64_split<<<nblk(p->n_tiles, 128), 128, 0, s>>>(p->n_tiles, p->fents, p->c_cls, d_smax,
                                                   p->stage_elems, p->fdesc, d_sums);
  BST_CHECK_LAUNCH();
  unsigned long long sums[2] = {0, 0};
  {
    ReadBack rb(p->ctx, s);
    rb.add(sums, d_sums, sizeof(sums));
    rb.done();
  }
  apply_split_gate(p, sums, s);
}

// C blocks by decreasing cost, for the direct-load persistent kernel
static void build_cost_items(bst_plan *p, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  int64_t *it0 = scratch.alloc_n<int64_t>((size_t)nc);
  int32_t *keys = scratch.alloc_n<int32_t>((size_t)nc);
  p->items = p->arena.alloc_n<int64_t>((size_t)nc);
  build_plan_items(p, 0, it0, keys, s);
  sort_items(it0, keys, nc, p->items, scratch, s);
  BST_CUDA(cudaStreamSynchronize(s));
  scratch.release_all();
}

// The numeric schedule of a plan: the staged kernel's, else the direct-load kernel's
void build_f64_schedule(bst_plan *p, cudaStream_t s) {
  if (!build_staged(p, s)) build_cost_items(p, s);
}

// the staged kernel's tiles of a plan for a batch (item = base | tile) and their keys
void build_plan_tile_items(bst_plan *p, int64_t base, int64_t *items, int32_t *keys,
                           cudaStream_t s) {
  if (p->n_tiles == 0) return;
  k_plan_items<<<nblk(p->n_tiles, 256), 256, 0, s>>>(p->n_tiles, base, items);
  BST_CHECK_LAUNCH();
  BST_CUDA(cudaMemcpyAsync(keys, p->tkeys, 4 * (size_t)p->n_tiles, cudaMemcpyDeviceToDevice, s));
}

// resident CTAs per SM of a staged kernel instance for a slot size; raises its dynamic
// shared-memory limit on first use
template <class K>
static int staged_ctas_per_sm(K kernel, bool &attr_set, int slot_elems, size_t &smem) {
  const size_t max_smem = sizeof(double) * 2 * kStageMax * kStageWarps;
  if (!attr_set) {
    BST_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)max_smem));
    attr_set = true;
  }
  smem = sizeof(double) * 2 * (size_t)slot_elems * kStageWarps;
  int nb = 0;
  BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 32 * kStageWarps, smem));
  return std::max(1, nb);
}

// one launch of a staged kernel instance: as many CTAs as fit (all resident), at most
// one warp per chunk of work items.  Chunks hold about 1/64 of a warp's share of the
// items (1 .. 32 items): one counter request per chunk, fine enough that the last
// chunks are small.  The counter is cleared on the launch's stream.
template <class K, class Arg>
static void staged_launch(K kernel, bool &attr_set, Arg params, const int64_t *items,
                          int64_t nitems, int slot_elems, int num_sms,
                          unsigned long long *counter, cudaStream_t s, int ksplit = 1) {
  BST_REQUIRE(counter, BST_ERR_STATE, "staged kernel without a work counter");
  size_t smem = 0;
  const int per = staged_ctas_per_sm(kernel, attr_set, slot_elems, smem);
  const int64_t full = (int64_t)per * num_sms * kStageWarps;
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(32, nitems / (64 * full)));
  const int64_t nchunks = (nitems + chunk - 1) / chunk;
  const int g = (int)std::min<int64_t>((int64_t)per * num_sms,
                                       (nchunks + kStageWarps - 1) / kStageWarps);
  BST_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  kernel<<<g, 32 * kStageWarps, smem, s>>>(params, items, nitems, slot_elems, counter, chunk,
                                           ksplit);
  BST_CHECK_LAUNCH();
}

static bool g_attr[2][4] = {};  // [batch, single plan][strided | split << 1]

void launch_fp64_staged(const void *params, const int64_t *items, int64_t nitems,
                        int slot_elems, bool strided, bool split, int num_sms,
                        unsigned long long *counter, cudaStream_t s) {
  if (nitems == 0) return;
  const NumParams *P = static_cast<const NumParams *>(params);
  const int v = (strided ? 1 : 0) | (split ? 2 : 0);
  switch (v) {
    case 0: staged_launch(k_num_fp64_staged<false, false>, g_attr[0][v], P, items, nitems, slot_elems, num_sms, counter, s); break;
    case 1: staged_launch(k_num_fp64_staged<true, false>, g_attr[0][v], P, items, nitems, slot_elems, num_sms, counter, s); break;
    case 2: staged_launch(k_num_fp64_staged<false, true>, g_attr[0][v], P, items, nitems, slot_elems, num_sms, counter, s); break;
    default: staged_launch(k_num_fp64_staged<true, true>, g_attr[0][v], P, items, nitems, slot_elems, num_sms, counter, s); break;
  }
}

int persist_grid(int num_sms) {
  int nb = 0;
  BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_fp64_persist, 256, 0));
  return std::max(1, nb) * num_sms;
}

int persist1_grid(int num_sms) {
  int nb = 0;
  BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_fp64_persist1, 256, 0));
  return std::max(1, nb) * num_sms;
}

void launch_fp64_persist(const void *params, const int64_t *items, int64_t nitems,
                         unsigned long long *counter, int grid, cudaStream_t s) {
  if (nitems == 0) return;
  BST_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  const int64_t need = (nitems + 7) / 8;
  const int g = (int)std::min<int64_t>(grid, need);
  k_num_fp64_persist<<<g, 256, 0, s>>>(static_cast<const NumParams *>(params), items, nitems,
                                       counter);
  BST_CHECK_LAUNCH();
}

int choose_split(const bst_plan *p, int num_sms) {
  const int64_t nc = p->C->nblocks;
  if (nc <= 0 || p->T <= 0) return 1;
  // enough work units to fill every SM: the staged kernel's 12 resident warps eight
  // items each (its tiles; on a 40 x 40-block C of 1600 tiles, parts 1, 2, 4, 8 ran
  // 611, 748, 803, 930 GFLOP/s), else the direct-load kernel's 32 resident warps (its C
  // blocks); never more parts than the average number of products per unit
  const bool staged = p->stage_elems > 0;
  const int64_t units = staged ? std::max<int64_t>(p->n_tiles, 1) : nc;
  const int64_t per_sm = staged ? (int64_t)kStageWarps * 3 * 8 : 32;
  const int64_t want = ((int64_t)num_sms * per_sm + units - 1) / units;
  const int64_t avg = p->T / units;
  int64_t s = std::min<int64_t>(want, std::max<int64_t>(1, avg));
  s = std::max<int64_t>(1, std::min<int64_t>(s, 16));
  return (int)s;
}

namespace {

// The direct-load kernel over every (C block, K part), then, for S > 1 parts, the
// fixed-order reduction of the parts' partial sums (P.W) into C.
void launch_direct_splitk(bst_plan *p, const NumParams &P, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  const int wpb = 8;
  k_num_fp64<<<nblk(nc * P.split, wpb), 32 * wpb, 0, s>>>(P);
  BST_CHECK_LAUNCH();
  if (P.split > 1) {
    k_splitk_reduce<<<nblk(nc, wpb), 32 * wpb, 0, s>>>(P, nc, p->C->row, p->C->col, p->C->rsz,
                                                       p->C->csz);
    BST_CHECK_LAUNCH();
  }
}

}  // namespace

// The staged kernel over every tile (split = 1: into C), or over every (tile, K part)
// into W followed by the fixed-order reduction of the parts (split > 1).
static void staged_single(bst_plan *p, const NumParams &P, int split, cudaStream_t s) {
  const int v = (p->stage_strided ? 1 : 0) | (p->stage_split ? 2 : 0);
  const int ns = p->ctx->num_sms, se = p->stage_elems;
  const int64_t nt = p->n_tiles * split;
  switch (v) {
    case 0: staged_launch(k_num_fp64_staged1<false, false>, g_attr[1][v], P, p->titems, nt, se, ns, p->items_counter, s, split); break;
    case 1: staged_launch(k_num_fp64_staged1<true, false>, g_attr[1][v], P, p->titems, nt, se, ns, p->items_counter, s, split); break;
    case 2: staged_launch(k_num_fp64_staged1<false, true>, g_attr[1][v], P, p->titems, nt, se, ns, p->items_counter, s, split); break;
    default: staged_launch(k_num_fp64_staged1<true, true>, g_attr[1][v], P, p->titems, nt, se, ns, p->items_counter, s, split); break;
  }
  if (split > 1) {
    const int wpb = 8;
    const int64_t nc = p->C->nblocks;
    k_splitk_reduce<<<nblk(nc, wpb), 32 * wpb, 0, s>>>(P, nc, p->C->row, p->C->col, p->C->rsz,
                                                       p->C->csz);
    BST_CHECK_LAUNCH();
  }
}

void execute_fp64(bst_plan *p, const NumArgs &a, int split, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  if (p->stage_elems > 0) {
    refresh_f64_split(p, s);
    NumParams P = make_params(p, a, std::max(split, 1));
    if (P.split > 1) {
      const size_t need = sizeof(double) * (size_t)P.split * (size_t)P.nelemC;
      if (p->work_bytes < need) {
        p->work.release_all();
        p->work.ctx = static_cast<Ctx *>(p->ctx);
        p->work.stream = s;
        p->work.alloc(need);
        p->work_bytes = need;
      }
      P.W = static_cast<double *>(p->work.bufs.back().p);
    }
    staged_single(p, P, P.split, s);
    return;
  }
  if (split <= 1 && p->items) {
    BST_CUDA(cudaMemsetAsync(p->items_counter, 0, sizeof(unsigned long long), s));
    const int64_t need = (nc + 7) / 8;
    const int g = (int)std::min<int64_t>(persist1_grid(p->ctx->num_sms), need);
    k_num_fp64_persist1<<<g, 256, 0, s>>>(make_params(p, a, 1), p->items, nc, p->items_counter);
    BST_CHECK_LAUNCH();
    return;
  }
  NumParams P = make_params(p, a, split);
  P.A = a.A;  // the direct-load kernel never reads slabs in place
  if (P.split > 1) {
    const size_t need = sizeof(double) * (size_t)P.split * (size_t)P.nelemC;
    if (p->work_bytes < need) {
      p->work.release_all();
      p->work.ctx = static_cast<Ctx *>(p->ctx);
      p->work.stream = s;
      p->work.alloc(need);
      p->work_bytes = need;
    }
    P.W = static_cast<double *>(p->work.bufs.back().p);
  }
  launch_direct_splitk(p, P, s);
}

// Same launches as execute_fp64's split-K path, with the partial sums in a caller-
// provided workspace W of at least split * nelem(C) doubles (no allocation here).
void execute_fp64_workspace(bst_plan *p, const NumArgs &a, int split, double *W, cudaStream_t s) {
  if (p->C->nblocks == 0) return;
  if (p->stage_elems > 0) {
    // the tiles' inner splits were chosen when the plan was built (a later tuning change
    // is taken by the next bst_multiply_execute, which may synchronise)
    NumParams P = make_params(p, a, std::max(split, 1));
    P.W = P.split > 1 ? W : nullptr;
    staged_single(p, P, P.split, s);
    return;
  }
  NumParams P = make_params(p, a, split);
  P.A = a.A;  // the direct-load kernel never reads slabs in place
  P.W = P.split > 1 ? W : nullptr;
  launch_direct_splitk(p, P, s);
}

}  // namespace bst
