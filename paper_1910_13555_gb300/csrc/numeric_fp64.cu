// Numeric phase, native FP64: batched small-block products of the stacks.
//
// Paper Sec. 2: the stacks of block products are processed by small-GEMM kernels
// specialised per (m, n, k).  On GB300 FP64 runs at about 1 TFLOP/s on the CUDA
// cores (FP64 DMMA measures the same), so this path is bound by the FP64 pipe, and
// what matters is how many lanes of every FP64 FMA do useful work and that C is
// written once.  The design:
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
  P.A = a.A;
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
  return P;
}

}  // namespace

size_t num_params_bytes() { return sizeof(NumParams); }

void fill_num_params(bst_plan *p, const NumArgs &a, void *out) {
  NumParams P = make_params(p, a, 1);
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
  // enough warps to fill every SM with 32 resident warps; never more parts than the
  // average number of products per C block
  const int64_t want = ((int64_t)num_sms * 32 + nc - 1) / nc;
  const int64_t avg = p->T / nc;
  int64_t s = std::min<int64_t>(want, std::max<int64_t>(1, avg));
  s = std::max<int64_t>(1, std::min<int64_t>(s, 16));
  return (int)s;
}

void execute_fp64(bst_plan *p, const NumArgs &a, int split, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  if (split <= 1 && p->items) {
    BST_CUDA(cudaMemsetAsync(p->items_counter, 0, sizeof(unsigned long long), s));
    const int64_t need = (nc + 7) / 8;
    const int g = (int)std::min<int64_t>(persist1_grid(p->ctx->num_sms), need);
    k_num_fp64_persist1<<<g, 256, 0, s>>>(make_params(p, a, 1), p->items, nc, p->items_counter);
    BST_CHECK_LAUNCH();
    return;
  }
  NumParams P;
  P.A = a.A;
  P.B = a.B;
  P.Cin = a.Cin;
  P.C = a.C;
  P.W = nullptr;
  P.alpha = a.alpha;
  P.alpha_one = a.alpha == 1.0;
  P.has_beta = a.beta != 0.0;
  P.beta = a.beta;
  P.nelemC = p->C->nelem;
  P.ntasks = nc;
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
  const int wpb = 8;
  k_num_fp64<<<nblk(nc * P.split, wpb), 32 * wpb, 0, s>>>(P);
  BST_CHECK_LAUNCH();
  if (P.split > 1) {
    k_splitk_reduce<<<nblk(nc, wpb), 32 * wpb, 0, s>>>(P, nc, p->C->row, p->C->col, p->C->rsz,
                                                       p->C->csz);
    BST_CHECK_LAUNCH();
  }
}

// Same launches as execute_fp64, with the split-K partial sums in a caller-provided
// workspace W of at least split * nelem(C) doubles (no allocation here).
void execute_fp64_workspace(bst_plan *p, const NumArgs &a, int split, double *W, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  NumParams P;
  P.A = a.A;
  P.B = a.B;
  P.Cin = a.Cin;
  P.C = a.C;
  P.W = W;
  P.alpha = a.alpha;
  P.alpha_one = a.alpha == 1.0;
  P.has_beta = a.beta != 0.0;
  P.beta = a.beta;
  P.nelemC = p->C->nelem;
  P.ntasks = nc;
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
  const int wpb = 8;
  k_num_fp64<<<nblk(nc * P.split, wpb), 32 * wpb, 0, s>>>(P);
  BST_CHECK_LAUNCH();
  if (P.split > 1) {
    k_splitk_reduce<<<nblk(nc, wpb), 32 * wpb, 0, s>>>(P, nc, p->C->row, p->C->col, p->C->rsz,
                                                       p->C->csz);
    BST_CHECK_LAUNCH();
  }
}

}  // namespace bst
