// Numeric phase on the tensor cores: FP64 emulated with BF16 slices (Ozaki scheme),
// and a 3xTF32 compensated path.
//
// Emulated FP64 (BST_FP64_EMU_BF16).  The error-free splitting of Ozaki, Ogita, Oishi
// and Rump (Numer. Algorithms 59, 2012) cuts every operand into slices whose pairwise
// products a low-precision unit computes exactly.  Each op(A) row (op(B) column) is
// scaled by a power of two 2^E with E its largest exponent -- over the whole op(A) row
// of the matrix (row-scaled mode, the default) or over the row of one block
// (block-scaled mode) -- and written in fixed point with 48 fraction bits,
//     a = 2^E * sum_{s=0..5} d_s 2^{-8(s+1)},  d_s integers, |d_0| <= 256, |d_s| <= 255,
// so every digit is exact in BF16 (8 significant bits).  A digit product is at most
// 2^16 and exact in FP32; a sum of 6 * 32 of them stays below 2^24, so the tensor core's
// FP32 accumulation is exact over 32 inner elements.  Slice products are grouped by
// level w = s + t and levels w <= 5 are kept (21 of 36; the dropped ones weigh about
// 2^-48 of the scale).  Every 32 inner elements the six exact level sums are folded into
// one integer I = sum_w D_w 2^{8(5-w)} (|I| < 2^62) and added into an int64 accumulator
// at the element's common scale 2^{ref - 56 + G}: in row-scaled mode all products of a C
// element share ref = E_row + F_col, in block-scaled mode each product's I is first
// shifted (with rounding) from its own scale ea + eb to the element's ref = the largest
// E_row + F_col; G guard bits keep K_tot * 2^56 below 2^62.  The int64 sum becomes FP64
// through the hardware conversion and an exponent-field add; no FP64 multiply-add is
// issued -- GB300's FP64 pipe runs at 1/64 of the FP32 rate.
//
// 3xTF32 (BST_TF32X3), after Ootomo and Yokota (IJHPCA 2022): x = hi + lo with hi, lo
// TF32; per block product hi*hi + hi*lo + lo*hi on the TF32 tensor cores with FP32
// accumulation, and the products summed as an unevaluated FP32 pair (TwoSum), then
// converted to FP64 and combined with alpha, beta.
//
// Both use warp-level mma.sync tiles (m16n8k16 BF16, m16n8k8 TF32).  The BF16 kernel
// runs one warp per C block (its 16 x 8 tiles one after another; no two warps write the
// same element), taking consecutive C blocks in chunks from a counter; the tile rows may
// run over the C block's columns instead (C^T = op(B)^T op(A)^T on the same slices),
// chosen per (m, n) class by the autotuner.  The 3xTF32 kernel runs one warp per 16 x 16
// tile.  The operand slices are staged once per execute in a padded, permuted layout that
// makes every fragment a single 8-byte load at a fixed offset (inner dimension padded
// with zeros to the MMA K, a chunk's slices side by side, and permuted inside each chunk
// so a thread's four values are adjacent).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <cmath>

#include "bst_internal.h"

namespace bst {

constexpr int kSlices = 6;     // BF16 digits per operand
constexpr int kBeta = 8;       // bits per digit
constexpr int kSegChunks = 2;  // 16-wide K chunks per exact FP32 segment (32 elements)
constexpr int kExpNone = -4000;
constexpr int kDescWords = 8;  // int32 words per C block descriptor of the BF16 kernel

struct EmuState {
  Arena ar;
  bool index_ready = false;
  // per stored block: offsets of its digit block, its exponents
  int64_t *a_doff = nullptr, *b_doff = nullptr, *a_toff = nullptr, *b_toff = nullptr;
  int64_t *a_eoff = nullptr, *b_eoff = nullptr;
  int64_t a_dsize = 0, b_dsize = 0, a_tsize = 0, b_tsize = 0, a_esize = 0, b_esize = 0;
  int64_t nwarps = 0;            // 3xTF32 warps (one per 16 x 16 tile)
  int64_t nitems_b = 0;          // BF16 work items (one per C block)
  int64_t *wstart = nullptr;    // per (m,n) class: first warp, 16 x 16 tiles (3xTF32)
  int32_t ncls = 0;
  // global start of every op(A) row block / op(B) column block, and the largest
  // exponent of every op(A) row / op(B) column over all blocks
  int64_t *a_rowstart = nullptr, *b_colstart = nullptr;
  int64_t nrows = 0, ncols = 0;
  int32_t *row_exp = nullptr, *col_exp = nullptr;
  // data-dependent buffers (rebuilt per execute)
  __nv_bfloat16 *a_dig = nullptr, *b_dig = nullptr;
  float *a_tf = nullptr, *b_tf = nullptr;
  int32_t *a_exp = nullptr, *b_exp = nullptr;
  bool dig_alloc = false, tf_alloc = false;
  // C-major stack entries of the BF16 kernel (int4 each) and where each C block's start
  int4 *ents = nullptr;
  int64_t *ebeg = nullptr;
  // C block descriptors, built for one tuning state (the tile orientation per class)
  int32_t *desc = nullptr;
  int32_t *cls_swap = nullptr;
  unsigned long long *counter = nullptr;  // work counter of the persistent kernel
  int64_t sched_version = -1;
  int sched_rows = -1;
};

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- exponents and slices ------------------------------------------------------------

// E(x): the smallest E with |x| < 2^E, for normal x; kExpNone for zero and subnormals
__device__ __forceinline__ int exp_of(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  return ex == 0 ? kExpNone : ex - 1022;
}

// same for m16n8k8 TF32 (thread t holds k = t, t+4 -> positions 2t, 2t+1)
__device__ __forceinline__ int perm8(int l) {
  const int j = l & 7;
  return (l & ~7) + 2 * (j & 3) + (j >> 2);
}

struct SideArgs {
  int64_t nblocks;
  const int32_t *row, *col, *rsz, *csz;  // stored block index and sizes
  const int64_t *off;                    // element offset of stored block
  const double *data;
  int trans;       // op(X) = X^T
  int is_b;        // 0: exponents per op row (A side), 1: per op column (B side)
  const int64_t *eoff;   // per block exponent offset
  const int64_t *doff;   // per block digit / tf32 offset
  int32_t *bexp;         // per block exponents
  const int64_t *start;  // global start of each op row block (A) / op column block (B)
  int32_t *gexp;         // largest exponent of each whole op row (A) / op column (B)
  int row_scale;         // digits scaled by the whole op row / column (1) or the block's (0)
  __nv_bfloat16 *dig;
  float *tf;
};

// decompose stored element e of block b into op coordinates: (r, l) for the A side
// (op row r, inner l), (l, q) for the B side (inner l, op column q); `outer` is r or q
__device__ __forceinline__ void op_coords(const SideArgs &S, int rs, int cs, int &outer,
                                          int &inner) {
  // stored element (rs, cs); op(X) element = (rs, cs) or (cs, rs)
  const int opr = S.trans ? cs : rs, opc = S.trans ? rs : cs;
  if (S.is_b) {
    inner = opr;
    outer = opc;
  } else {
    outer = opr;
    inner = opc;
  }
}

// Both side kernels run one warp per stored block; four lanes share one 16-wide chunk of
// one op row (A side) or op column (B side) and lane t of the four takes the inner
// indices 2t, 2t+1, 2t+8, 2t+9 of the chunk -- the four values that the digit layout
// stores next to each other (positions 4t..4t+3).  Elements are read in the stored
// block's layout: element (outer, inner) sits at outer * Cc + inner when the op keeps
// the stored rows as outer (op(A) = A, op(B) = B^T), else at inner * Cc + outer.
struct SideBlock {
  const double *x;
  int Cc, nouter, ninner, nch;
  bool outer_major;
  int64_t gbase;
};

__device__ __forceinline__ SideBlock side_block(const SideArgs &S, int64_t b) {
  SideBlock B;
  const int R = S.rsz[S.row[b]], Cc = S.csz[S.col[b]];
  B.x = S.data + S.off[b];
  B.Cc = Cc;
  B.nouter = S.is_b ? (S.trans ? R : Cc) : (S.trans ? Cc : R);
  B.ninner = S.is_b ? (S.trans ? Cc : R) : (S.trans ? R : Cc);
  B.nch = (B.ninner + 15) >> 4;
  B.outer_major = S.is_b == S.trans;
  // op block index along the exponent dimension (rows of op(A), columns of op(B))
  const int obr = S.trans ? S.col[b] : S.row[b], obc = S.trans ? S.row[b] : S.col[b];
  B.gbase = S.start[S.is_b ? obc : obr];
  return B;
}

__device__ __forceinline__ double side_value(const SideBlock &B, int outer, int inner) {
  if (inner >= B.ninner) return 0.0;
  return B.x[B.outer_major ? outer * B.Cc + inner : inner * B.Cc + outer];
}

// inner index (within its 16-chunk) stored at digit position 4t + u: thread t of an
// m16n8k16 fragment holds k = 2t, 2t+1, 2t+8, 2t+9, stored next to each other
__device__ __forceinline__ int chunk_inner(int t, int u) { return 2 * t + (u & 1) + 8 * (u >> 1); }

// largest exponent of every op row (column) of a block and of the whole op row (column):
// the four lanes of a chunk combine their maxima, then one atomic per chunk and target
__global__ void k_emu_exponents(SideArgs S) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= S.nblocks) return;
  const SideBlock B = side_block(S, b);
  const int total = B.nouter * B.nch;
  for (int q0 = 0; q0 < total; q0 += 8) {  // uniform trip count: every lane shuffles
    const int q = q0 + (lane >> 2);
    const bool ok = q < total;
    const int outer = ok ? q / B.nch : 0, ch = ok ? q - outer * B.nch : 0;
    int E = kExpNone;
    if (ok)
#pragma unroll
      for (int u = 0; u < 4; ++u) E = max(E, exp_of(side_value(B, outer, ch * 16 + chunk_inner(t, u))));
    E = max(E, __shfl_xor_sync(0xffffffffu, E, 1));
    E = max(E, __shfl_xor_sync(0xffffffffu, E, 2));
    if (ok && t == 0 && E != kExpNone) {
      atomicMax(&S.bexp[S.eoff[b] + outer], E);
      atomicMax(&S.gexp[B.gbase + outer], E);
    }
  }
}

// The six digit planes of a block, every position written (zero padding included), one
// 8-byte store per plane and lane.  With 2^E the scale of the element's op row (column),
// N = round(|v| 2^(48 - E)) < 2^48 (+1) is cut into 8-bit digits, the leading one taking
// the rounding carry (it may reach 2^8); all are exact in BF16.
__global__ void k_emu_digits(SideArgs S) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= S.nblocks) return;
  const SideBlock B = side_block(S, b);
  __nv_bfloat16 *d = S.dig + S.doff[b];
  const int total = B.nouter * B.nch;
  for (int q = lane >> 2; q < total; q += 8) {
    const int outer = q / B.nch, ch = q - outer * B.nch;
    const int E = S.row_scale ? S.gexp[B.gbase + outer] : S.bexp[S.eoff[b] + outer];
    uint32_t w[kSlices][2];
#pragma unroll
    for (int s = 0; s < kSlices; ++s) w[s][0] = w[s][1] = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long bits = __double_as_longlong(side_value(B, outer, ch * 16 + chunk_inner(t, u)));
      const int ex = (int)((bits >> 52) & 0x7ff);
      unsigned long long N = 0;
      if (ex != 0 && E != kExpNone) {
        const unsigned long long M = (unsigned long long)(bits & 0xfffffffffffffLL) | (1ull << 52);
        // N = round(M 2^(ex - 1075 + 48 - E)); |v| < 2^E makes the shift >= 5
        const int rsh = 1075 - kSlices * kBeta - ex + E;
        if (rsh < 64) N = (M + (1ull << (rsh - 1))) >> rsh;
      }
      const bool neg = bits < 0;
#pragma unroll
      for (int s = 0; s < kSlices; ++s) {
        const unsigned mask = s == 0 ? (2u << kBeta) - 1u : (1u << kBeta) - 1u;
        int dg = (int)((N >> (kBeta * (kSlices - 1 - s))) & mask);
        if (neg) dg = -dg;
        const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn((float)dg));
        w[s][u >> 1] |= h << (16 * (u & 1));
      }
    }
    // chunk q = outer * nch + ch holds its six digit slices side by side
    __nv_bfloat16 *p = d + (int64_t)q * (kSlices * 16) + 4 * t;
#pragma unroll
    for (int s = 0; s < kSlices; ++s)
      *reinterpret_cast<uint2 *>(p + s * 16) = make_uint2(w[s][0], w[s][1]);
  }
}

// round a double to TF32 (10 explicit mantissa bits), nearest with ties away
__device__ __forceinline__ float to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void k_tf32_split(SideArgs S) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= S.nblocks) return;
  const int R = S.rsz[S.row[b]], Cc = S.csz[S.col[b]];
  const int nouter = S.is_b ? (S.trans ? R : Cc) : (S.trans ? Cc : R);
  const int ninner = S.is_b ? (S.trans ? Cc : R) : (S.trans ? R : Cc);
  const int kp = (ninner + 7) & ~7;
  const int64_t plane = (int64_t)nouter * kp;
  const double *x = S.data + S.off[b];
  float *t = S.tf + S.doff[b];
  for (int e = lane; e < R * Cc; e += 32) {
    int outer, inner;
    op_coords(S, e / Cc, e % Cc, outer, inner);
    const double v = x[e];
    const float hi = to_tf32((float)v);
    const float lo = to_tf32((float)(v - (double)hi));
    const int64_t pos = (int64_t)outer * kp + perm8(inner);
    t[pos] = hi;
    t[plane + pos] = lo;
  }
}

// per stored block: digit / tf32 / exponent sizes
__global__ void k_side_sizes(SideArgs S, int64_t *dsz, int64_t *tsz, int64_t *esz) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.nblocks) return;
  const int R = S.rsz[S.row[b]], Cc = S.csz[S.col[b]];
  const int nouter = S.is_b ? (S.trans ? R : Cc) : (S.trans ? Cc : R);
  const int ninner = S.is_b ? (S.trans ? Cc : R) : (S.trans ? R : Cc);
  dsz[b] = (int64_t)kSlices * nouter * ((ninner + 15) & ~15);
  tsz[b] = (int64_t)2 * nouter * ((ninner + 7) & ~7);
  esz[b] = nouter;
}

// ---- per-plan index of the BF16 kernel ------------------------------------------------

// number of stack entries of every C block (over all its k classes)
__global__ void k_emu_ent_count(int64_t nc, int32_t Dk, const int32_t *__restrict__ run_len,
                                int32_t *__restrict__ cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int s = 0;
  for (int kc = 0; kc < Dk; ++kc) s += run_len[c * Dk + kc];
  cnt[c] = s;
}

// C-major entry list: the entries of C block c at [ebeg[c], ebeg[c+1]), k classes in
// order; entry = {A digit block offset / 16, B digit block offset / 16, 16-chunks of the
// inner size, stack entry}.  Digit blocks start on multiples of 16 elements (every
// block's digit size is 6 * outer * inner rounded up to 16).
__global__ void k_emu_ents(int64_t nc, int32_t Dk, const int32_t *__restrict__ run_start,
                           const int32_t *__restrict__ run_len, const int32_t *__restrict__ kval,
                           const int32_t *__restrict__ s_ab, const int32_t *__restrict__ s_bb,
                           const int64_t *__restrict__ a_doff, const int64_t *__restrict__ b_doff,
                           const int64_t *__restrict__ ebeg, int4 *__restrict__ ents) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int64_t q = ebeg[c];
  for (int kc = 0; kc < Dk; ++kc) {
    const int len = run_len[c * Dk + kc];
    if (len == 0) continue;
    const int e0 = run_start[c * Dk + kc], nch = (kval[kc] + 15) >> 4;
    for (int e = e0; e < e0 + len; ++e)
      ents[q++] = make_int4((int)(unsigned)(a_doff[s_ab[e]] >> 4),
                            (int)(unsigned)(b_doff[s_bb[e]] >> 4), nch, e);
  }
}

// C block descriptors (kDescWords words each; see EmuBlk).  The guard G of a block keeps
// its K_tot products of at most 2^56 units each below 2^62 after the shift by G.
__global__ void k_emu_desc(int64_t nc, int32_t Dk, const int32_t *__restrict__ run_len,
                           const int32_t *__restrict__ kval, const int64_t *__restrict__ ebeg,
                           const int64_t *__restrict__ c_off, const int32_t *__restrict__ c_row,
                           const int32_t *__restrict__ c_col, const int32_t *__restrict__ c_cls,
                           const int32_t *__restrict__ cls_m, const int32_t *__restrict__ cls_n,
                           const int32_t *__restrict__ cls_swap, const int32_t *__restrict__ c_cin,
                           const int64_t *__restrict__ a_rowstart,
                           const int64_t *__restrict__ b_colstart, int32_t *__restrict__ desc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  long long ktot = 0;
  for (int kc = 0; kc < Dk; ++kc) ktot += (long long)run_len[c * Dk + kc] * kval[kc];
  int lg = 0;
  while (lg < 63 && (1ll << lg) <= ktot) ++lg;
  const int guard = max(0, lg - (62 - (kSlices + 1) * kBeta));
  const int cls = c_cls[c];
  int32_t *d = desc + c * kDescWords;
  d[0] = (int32_t)c_off[c];
  d[1] = (int32_t)ebeg[c];
  d[2] = (int32_t)(ebeg[c + 1] - ebeg[c]);
  d[3] = (int32_t)a_rowstart[c_row[c]];
  d[4] = (int32_t)b_colstart[c_col[c]];
  d[5] = cls_m[cls] | (cls_n[cls] << 12) | (cls_swap[cls] << 24) | (guard << 25);
  d[6] = c_cin[c];
  d[7] = (int32_t)c;
}

// items of a plan in a batch: base | C block
__global__ void k_emu_items(int64_t nc, int64_t base, int64_t *__restrict__ items) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) items[c] = base | c;
}

// ---- integer -> FP64 ---------------------------------------------------------------

// results outside the normal binary64 range (not met by the test workloads)
__device__ __noinline__ double i64_ldexp_slow(double d, int e2) { return ldexp(d, e2); }

// v * 2^e2 rounded to nearest-even binary64: the hardware int64 -> FP64 conversion
// (correctly rounded; it runs on the FP64 unit, which the emulated kernel otherwise
// leaves idle) and the scale added to the exponent field, exact while the result stays
// normal.  This keeps the epilogue's integer work, which competes with the MMA loop for
// issue slots, to a handful of instructions per element.
__device__ __forceinline__ double i64_ldexp(long long v, int e2) {
  if (v == 0) return 0.0;
  const double d = __ll2double_rn(v);
  const long long bits = __double_as_longlong(d);
  const int be = (int)((bits >> 52) & 0x7ff) + e2;
  if (be <= 0 || be >= 2047) return i64_ldexp_slow(d, e2);
  return __longlong_as_double(bits + ((long long)e2 << 52));
}

// FP32 -> FP64 from the binary32 / binary64 encodings (normal numbers and zero; FP32
// subnormals flush to zero), integer operations only
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  if (ex == 0) return 0.0;
  if (ex == 0xffu) return (double)f;
  const unsigned long long bits = ((unsigned long long)(b >> 31) << 63) |
                                  ((unsigned long long)(ex - 127 + 1023) << 52) |
                                  ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ long long round_shift(long long v, int sh) {
  if (sh <= 0) return v;
  if (sh >= 62) return 0;
  return (v + (1ll << (sh - 1))) >> sh;
}

// ---- the numeric kernels -----------------------------------------------------------

struct EmuParams {
  const double *Cin;
  double *C;
  double alpha, beta;
  int32_t Dk, ncls;
  const int64_t *wstart;
  int32_t tiles_n;  // N-tiles of 8 columns per warp (1 or 2)
  int32_t alpha_one, has_beta;  // alpha == 1, beta != 0 (set on the host: FP64 compares
                                // would occupy GB300's slow FP64 pipe in every tile)
  int32_t row_scale;  // 1: digits scaled per whole op row / column (shared by all products)
  const int64_t *a_rowstart, *b_colstart;
  const int32_t *row_exp, *col_exp;
  const int32_t *class_ptr, *task_c, *cls_m, *cls_n, *kval;
  const int32_t *c_row, *c_col, *c_cin, *c_cls;
  const int64_t *c_off, *cin_off;
  const int32_t *run_start, *run_len, *s_ab, *s_bb;
  const int32_t *desc;  // BF16 kernel: C block descriptors (kDescWords each)
  const int4 *ents;     // BF16 kernel: C-major entries
  const int64_t *a_doff, *b_doff, *a_eoff, *b_eoff;
  const __nv_bfloat16 *a_dig, *b_dig;
  const float *a_tf, *b_tf;
  const int32_t *a_exp, *b_exp;
};

struct WarpTask {
  int c, m, n, mt, ng, ntn;
  int sw = 0;  // 1: tile rows run over the C block's columns (C^T = op(B)^T op(A)^T)
};

__device__ __forceinline__ WarpTask find_task(const EmuParams &P, int64_t gw) {
  // class of this warp: last class whose start <= gw (classes with no warps are skipped)
  int lo = 0, hi = P.ncls;  // wstart has ncls + 1 entries, wstart[ncls] = total
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.wstart[mid] <= gw)
      lo = mid;
    else
      hi = mid;
  }
  WarpTask w;
  const int cls = lo;
  w.m = P.cls_m[cls];
  w.n = P.cls_n[cls];
  const int MT = (w.m + 15) >> 4, NT = (w.n + 7) >> 3, NG = (NT + P.tiles_n - 1) / P.tiles_n;
  // warps of one class number below 2^31 (a class holds < 2^31 C blocks x a few tiles)
  const unsigned local = (unsigned)(gw - P.wstart[cls]), per = (unsigned)(MT * NG);
  const unsigned task = local / per, sub = local - task * per;
  w.mt = (int)(sub / (unsigned)NG);
  w.ng = (int)(sub - (unsigned)w.mt * (unsigned)NG);
  w.ntn = min(P.tiles_n, NT - P.tiles_n * w.ng);
  w.c = P.task_c[P.class_ptr[cls] + (int)task];
  return w;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint2 ld8(const void *p) {
  return __ldg(reinterpret_cast<const uint2 *>(p));
}

// element (row, col) of this warp's tile owned by accumulator slot h of N-tile nt
__device__ __forceinline__ void slot_rc(const WarpTask &w, int nt, int h, int &r, int &c) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  r = w.mt * 16 + g + (h >= 2 ? 8 : 0);
  c = (2 * w.ng + nt) * 8 + 2 * t + (h & 1);
}

// ---- the BF16 slice kernel: one warp per C block -----------------------------------
//
// Warps take C blocks in chunks of kChunk consecutive blocks from a counter over the
// work list (C block order, so warps running at the same time share op(A) digit rows
// in L2) and prefetch the descriptors of their next chunk while they compute the
// current one.  A block's stack entries (most blocks have one or two) are loaded once,
// one per lane, and broadcast with shuffles; the warp then runs the block's 16 x 8
// tiles one after another.

constexpr unsigned kFull = 0xffffffffu;

// a C block as the kernel sees it, decoded from its descriptor words
//   0 element offset, 1 first entry, 2 entry count, 3 first global op(A) row of its
//   block row, 4 first global op(B) column of its block column,
//   5 m | n << 12 | swap << 24 | guard << 25, 6 C_in block (-1: none), 7 C block
struct EmuBlk {
  int off, eb, ne, rbase, cbase, m, n, sw, guard, cin;
};

__device__ __forceinline__ EmuBlk emu_blk(int dw) {
  EmuBlk b;
  b.off = __shfl_sync(kFull, dw, 0);
  b.eb = __shfl_sync(kFull, dw, 1);
  b.ne = __shfl_sync(kFull, dw, 2);
  b.rbase = __shfl_sync(kFull, dw, 3);
  b.cbase = __shfl_sync(kFull, dw, 4);
  const int mn = __shfl_sync(kFull, dw, 5);
  b.cin = __shfl_sync(kFull, dw, 6);
  b.m = mn & 0xfff;
  b.n = (mn >> 12) & 0xfff;
  b.sw = (mn >> 24) & 1;
  b.guard = (mn >> 25) & 0x3f;
  return b;
}

// The four elements a lane owns in tile (mt, ng): tile rows r0, r1 = mt*16 + g (+8),
// tile columns cc0, cc1 = ng*8 + 2t (+1); tile space is the C block, or its transpose
// when the class runs swapped.
struct TileLane {
  int r0, r1, cc0, cc1, colB;
  bool v0, v1, vB;
  bool valid[4];
  int ref[4];  // exponent of each element's common scale (whole op row + op column)
};

__device__ __forceinline__ TileLane tile_lane(const EmuParams &P, const EmuBlk &b, int mt, int ng) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int RM = b.sw ? b.n : b.m, RN = b.sw ? b.m : b.n;
  TileLane L;
  L.r0 = mt * 16 + g;
  L.r1 = L.r0 + 8;
  L.v0 = L.r0 < RM;
  L.v1 = L.r1 < RM;
  L.colB = ng * 8 + g;
  L.vB = L.colB < RN;
  L.cc0 = ng * 8 + 2 * t;
  L.cc1 = L.cc0 + 1;
  const bool vc0 = L.cc0 < RN, vc1 = L.cc1 < RN;
  L.valid[0] = L.v0 && vc0;
  L.valid[1] = L.v0 && vc1;
  L.valid[2] = L.v1 && vc0;
  L.valid[3] = L.v1 && vc1;
  const int32_t *ER = b.sw ? P.col_exp + b.cbase : P.row_exp + b.rbase;  // tile rows
  const int32_t *EC = b.sw ? P.row_exp + b.rbase : P.col_exp + b.cbase;  // tile columns
  const int E0 = L.v0 ? ER[L.r0] : kExpNone, E1 = L.v1 ? ER[L.r1] : kExpNone;
  const int F0 = vc0 ? EC[L.cc0] : kExpNone, F1 = vc1 ? EC[L.cc1] : kExpNone;
  L.ref[0] = E0 + F0;
  L.ref[1] = E0 + F1;
  L.ref[2] = E1 + F0;
  L.ref[3] = E1 + F1;
  return L;
}

// C = alpha * acc * 2^(ref - 56 + G) + beta * C_in for the lane's valid elements
__device__ __forceinline__ void emu_store(const EmuParams &P, const EmuBlk &b, const TileLane &L,
                                          const long long (&acc)[4]) {
  const double *ci = (P.has_beta && b.cin >= 0) ? P.Cin + P.cin_off[b.cin] : nullptr;
  const int sh = (kSlices + 1) * kBeta - b.guard;
  // element (x, y) of the tile is C(x, y), or C(y, x) when swapped
  auto cidx = [&](int h) {
    const int x = h < 2 ? L.r0 : L.r1, y = (h & 1) ? L.cc1 : L.cc0;
    return b.sw ? y * b.n + x : x * b.n + y;
  };
  if (P.alpha_one && !ci) {  // plain stores: no FP64 instruction at all
#pragma unroll
    for (int h = 0; h < 4; ++h)
      if (L.valid[h]) P.C[b.off + cidx(h)] = i64_ldexp(acc[h], L.ref[h] - sh);
  } else {
#pragma unroll
    for (int h = 0; h < 4; ++h)
      if (L.valid[h]) {
        double v = P.alpha * i64_ldexp(acc[h], L.ref[h] - sh);
        if (ci) v = fma(P.beta, ci[cidx(h)], v);
        P.C[b.off + cidx(h)] = v;
      }
  }
}

// the six exact FP32 level sums of element h as one integer in units of 2^-56 of the
// scale: I = sum_w D_w 2^(8(5 - w)), |I| < 2^62.  Levels weighted below 2^32 go
// through 32 x 32 -> 64-bit multiply-adds; the two top levels (|D_0| < 2^21.1,
// |D_1| < 2^22) are combined in 32 bits and added to the upper word.
__device__ __forceinline__ long long fold_levels(const float (&lv)[kSlices][4], int h) {
  long long lo = __float2int_rn(lv[kSlices - 1][h]);
  int hi = 0;
#pragma unroll
  for (int s = kSlices - 2; s >= 0; --s) {
    const int sh = kBeta * (kSlices - 1 - s);
    const int d = __float2int_rn(lv[s][h]);
    if (sh < 32)
      lo += (long long)d * (long long)(1u << sh);
    else
      hi += d * (1 << (sh - 32));
  }
  return lo + (long long)((unsigned long long)(unsigned)hi << 32);
}

__device__ __forceinline__ int4 load_ent(const EmuParams &P, const EmuBlk &b, int q) {
  return q < b.ne ? P.ents[(int64_t)b.eb + q] : make_int4(0, 0, 0, 0);
}

// Row-scaled tile, direct loads: per entry, the row operand's six digit fragments
// (two 8-byte loads each) and the column operand's six (one each) feed the 21 kept slice products into
// six FP32 level sums.  All products of an element share its scale, so the level sums
// run across entries and are folded into the int64 accumulators every 32 inner
// elements (or at the end).
__device__ __forceinline__ void emu_tile_rs_direct(const EmuParams &P, const EmuBlk &b, int mt, int ng,
                                            const int4 &ent0) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const TileLane L = tile_lane(P, b, mt, ng);
  const __nv_bfloat16 *Xa = b.sw ? P.b_dig : P.a_dig, *Xb = b.sw ? P.a_dig : P.b_dig;
  long long acc[4] = {0, 0, 0, 0};
  float lv[kSlices][4];
#pragma unroll
  for (int s = 0; s < kSlices; ++s)
#pragma unroll
    for (int h = 0; h < 4; ++h) lv[s][h] = 0.f;
  int used = 0;  // 16-wide chunks summed into lv since the last fold
  auto fold = [&]() {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (L.valid[h]) {
        const long long I = fold_levels(lv, h);
        acc[h] += b.guard ? round_shift(I, b.guard) : I;
      }
#pragma unroll
      for (int s = 0; s < kSlices; ++s) lv[s][h] = 0.f;
    }
    used = 0;
  };
  const uint2 zero = make_uint2(0u, 0u);
  for (int g0 = 0; g0 < b.ne; g0 += 32) {
    const int4 ent = g0 == 0 ? ent0 : load_ent(P, b, g0 + lane);
    const int cnt = min(32, b.ne - g0);
    for (int j = 0; j < cnt; ++j) {
      const unsigned ea = (unsigned)__shfl_sync(kFull, ent.x, j);
      const unsigned eb = (unsigned)__shfl_sync(kFull, ent.y, j);
      const int nch = __shfl_sync(kFull, ent.z, j);
      const __nv_bfloat16 *Ad = Xa + 16 * (size_t)(b.sw ? eb : ea);
      const __nv_bfloat16 *Bd = Xb + 16 * (size_t)(b.sw ? ea : eb);
      // per-thread digit pointers of the row / column operand: chunk ch of outer row r
      // starts at (r * nch + ch) * 96, slice s of it 16 elements further per s
      const int rs = nch * (kSlices * 16);
      const __nv_bfloat16 *a0 = Ad + (L.r0 * rs + 4 * t), *a1 = Ad + (L.r1 * rs + 4 * t);
      const __nv_bfloat16 *b0 = Bd + (L.colB * rs + 4 * t);
      for (int ch = 0; ch < nch; ++ch) {
        if (used == kSegChunks) fold();
        const int cofs = ch * (kSlices * 16);
        uint2 bf[kSlices];
#pragma unroll
        for (int tt = 0; tt < kSlices; ++tt) bf[tt] = L.vB ? ld8(b0 + cofs + tt * 16) : zero;
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
          const uint2 x0 = L.v0 ? ld8(a0 + cofs + s * 16) : zero;
          const uint2 x1 = L.v1 ? ld8(a1 + cofs + s * 16) : zero;
          const uint32_t af[4] = {x0.x, x1.x, x0.y, x1.y};
#pragma unroll
          for (int tt = 0; s + tt < kSlices; ++tt) mma_bf16(lv[s + tt], af, bf[tt].x, bf[tt].y);
        }
        ++used;
      }
    }
  }
  fold();
  emu_store(P, b, L, acc);
}

// digit fragments of one (entry, 16-wide chunk) job of a row-scaled tile: the row
// operand's six slices for the lane's two tile rows and the column operand's six
struct EmuFrag {
  uint2 a0[kSlices], a1[kSlices], b[kSlices];
};

__device__ __forceinline__ void emu_frag_load(EmuFrag &f, const TileLane &L,
                                              const __nv_bfloat16 *a0, const __nv_bfloat16 *a1,
                                              const __nv_bfloat16 *b0) {
  const uint2 zero = make_uint2(0u, 0u);
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    f.b[s] = L.vB ? ld8(b0 + s * 16) : zero;
    f.a0[s] = L.v0 ? ld8(a0 + s * 16) : zero;
    f.a1[s] = L.v1 ? ld8(a1 + s * 16) : zero;
  }
}

// the 21 kept slice products (levels s + t <= 5) of one job into the six level sums
__device__ __forceinline__ void emu_frag_mma(float (&lv)[kSlices][4], const EmuFrag &f) {
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const uint32_t af[4] = {f.a0[s].x, f.a1[s].x, f.a0[s].y, f.a1[s].y};
#pragma unroll
    for (int tt = 0; s + tt < kSlices; ++tt) mma_bf16(lv[s + tt], af, f.b[tt].x, f.b[tt].y);
  }
}

// Row-scaled tile, pipelined: the tile's jobs -- (entry, 16-wide chunk) pairs, entry by
// entry -- each feed the 21 kept slice products into six FP32 level sums; the fragments
// of the next job are loaded while the current job's products run, so the MMAs do not
// wait on L2 for their operands.  The second fragment set costs registers (52 bytes of
// spills at the 128-register limit), which plans with short inner sums pay for without
// gaining: the launch takes this loop only when a C element sums at least
// kPipeMinInner inner elements on average (measured: tall-skinny A^T B, 311 per
// element, 1088 -> 1181 GFLOP/s; banded, 21 per element, 2347 -> 2154 with it).  All products of an element share its scale, so the level
// sums run across entries and are folded into the int64 accumulators every 32 inner
// elements (or at the end).
__device__ __forceinline__ void emu_tile_rs_pipe(const EmuParams &P, const EmuBlk &b, int mt, int ng,
                                                 const int4 &ent0) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const TileLane L = tile_lane(P, b, mt, ng);
  const __nv_bfloat16 *Xa = b.sw ? P.b_dig : P.a_dig, *Xb = b.sw ? P.a_dig : P.b_dig;
  long long acc[4] = {0, 0, 0, 0};
  float lv[kSlices][4];
#pragma unroll
  for (int s = 0; s < kSlices; ++s)
#pragma unroll
    for (int h = 0; h < 4; ++h) lv[s][h] = 0.f;
  int used = 0;  // 16-wide chunks summed into lv since the last fold
  auto fold = [&]() {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (L.valid[h]) {
        const long long I = fold_levels(lv, h);
        acc[h] += b.guard ? round_shift(I, b.guard) : I;
      }
#pragma unroll
      for (int s = 0; s < kSlices; ++s) lv[s][h] = 0.f;
    }
    used = 0;
  };
  // per-thread digit pointers of entry j of the loaded group: chunk ch of outer row r
  // starts at (r * nch + ch) * 96, slice s of it 16 elements further per s
  auto entry = [&](const int4 &e, int j, const __nv_bfloat16 *&pa0, const __nv_bfloat16 *&pa1,
                   const __nv_bfloat16 *&pb0, int &nch) {
    const unsigned ea = (unsigned)__shfl_sync(kFull, e.x, j);
    const unsigned eb = (unsigned)__shfl_sync(kFull, e.y, j);
    nch = __shfl_sync(kFull, e.z, j);
    const __nv_bfloat16 *Ad = Xa + 16 * (size_t)(b.sw ? eb : ea);
    const __nv_bfloat16 *Bd = Xb + 16 * (size_t)(b.sw ? ea : eb);
    const int rs = nch * (kSlices * 16);
    pa0 = Ad + (L.r0 * rs + 4 * t);
    pa1 = Ad + (L.r1 * rs + 4 * t);
    pb0 = Bd + (L.colB * rs + 4 * t);
  };
  if (b.ne > 0) {
    int4 ent = ent0;
    int g0 = 0, j = 0, ch = 0, nch = 0;
    const __nv_bfloat16 *a0, *a1, *b0;
    entry(ent, 0, a0, a1, b0, nch);
    EmuFrag cur;
    emu_frag_load(cur, L, a0, a1, b0);
    for (;;) {
      int jn = j, chn = ch + 1, nnch = nch;
      const __nv_bfloat16 *na0 = a0, *na1 = a1, *nb0 = b0;
      bool more = true;
      if (chn == nch) {
        chn = 0;
        jn = j + 1;
        if (g0 + jn >= b.ne) {
          more = false;
        } else {
          if (jn == 32) {
            g0 += 32;
            jn = 0;
            ent = load_ent(P, b, g0 + lane);
          }
          entry(ent, jn, na0, na1, nb0, nnch);
        }
      }
      EmuFrag nxt;
      if (more) {
        const int cofs = chn * (kSlices * 16);
        emu_frag_load(nxt, L, na0 + cofs, na1 + cofs, nb0 + cofs);
      }
      if (used == kSegChunks) fold();
      emu_frag_mma(lv, cur);
      ++used;
      if (!more) break;
      cur = nxt;
      j = jn;
      ch = chn;
      nch = nnch;
      a0 = na0;
      a1 = na1;
      b0 = nb0;
    }
  }
  fold();
  emu_store(P, b, L, acc);
}

// Block-scaled tile (never swapped): each product has its own scale 2^(ea + eb) per
// element, so its level sums are folded after every 32 inner elements of that product
// and shifted (with rounding) to the element's common scale.
__device__ __forceinline__ void emu_tile_bs(const EmuParams &P, const EmuBlk &b, int mt, int ng,
                                            const int4 &ent0) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const TileLane L = tile_lane(P, b, mt, ng);
  long long acc[4] = {0, 0, 0, 0};
  const uint2 zero = make_uint2(0u, 0u);
  for (int g0 = 0; g0 < b.ne; g0 += 32) {
    const int4 ent = g0 == 0 ? ent0 : load_ent(P, b, g0 + lane);
    const int cnt = min(32, b.ne - g0);
    for (int j = 0; j < cnt; ++j) {
      const unsigned ea = (unsigned)__shfl_sync(kFull, ent.x, j);
      const unsigned eb = (unsigned)__shfl_sync(kFull, ent.y, j);
      const int nch = __shfl_sync(kFull, ent.z, j);
      const int e = __shfl_sync(kFull, ent.w, j);
      const __nv_bfloat16 *Ad = P.a_dig + 16 * (size_t)ea;
      const __nv_bfloat16 *Bd = P.b_dig + 16 * (size_t)eb;
      const int rs = nch * (kSlices * 16);
      const __nv_bfloat16 *a0 = Ad + (L.r0 * rs + 4 * t), *a1 = Ad + (L.r1 * rs + 4 * t);
      const __nv_bfloat16 *b0 = Bd + (L.colB * rs + 4 * t);
      const int64_t aeo = P.a_eoff[P.s_ab[e]], beo = P.b_eoff[P.s_bb[e]];
      const bool vc0 = L.valid[0] || L.valid[2], vc1 = L.valid[1] || L.valid[3];
      const int ea0 = L.v0 ? P.a_exp[aeo + L.r0] : kExpNone, ea1 = L.v1 ? P.a_exp[aeo + L.r1] : kExpNone;
      const int eb0 = vc0 ? P.b_exp[beo + L.cc0] : kExpNone, eb1 = vc1 ? P.b_exp[beo + L.cc1] : kExpNone;
      const int eas[4] = {ea0 + eb0, ea0 + eb1, ea1 + eb0, ea1 + eb1};
      for (int cs = 0; cs < nch; cs += kSegChunks) {
        float lv[kSlices][4];
#pragma unroll
        for (int s = 0; s < kSlices; ++s)
#pragma unroll
          for (int h = 0; h < 4; ++h) lv[s][h] = 0.f;
        const int ce = min(nch, cs + kSegChunks);
        for (int ch = cs; ch < ce; ++ch) {
          const int cofs = ch * (kSlices * 16);
          uint2 bf[kSlices];
#pragma unroll
          for (int tt = 0; tt < kSlices; ++tt) bf[tt] = L.vB ? ld8(b0 + cofs + tt * 16) : zero;
#pragma unroll
          for (int s = 0; s < kSlices; ++s) {
            const uint2 x0 = L.v0 ? ld8(a0 + cofs + s * 16) : zero;
            const uint2 x1 = L.v1 ? ld8(a1 + cofs + s * 16) : zero;
            const uint32_t af[4] = {x0.x, x1.x, x0.y, x1.y};
#pragma unroll
            for (int tt = 0; s + tt < kSlices; ++tt) mma_bf16(lv[s + tt], af, bf[tt].x, bf[tt].y);
          }
        }
#pragma unroll
        for (int h = 0; h < 4; ++h)
          if (L.valid[h]) acc[h] += round_shift(fold_levels(lv, h), L.ref[h] - eas[h] + b.guard);
      }
    }
  }
  emu_store(P, b, L, acc);
}

// ROWS: 0 block-scaled tiles, 1 row-scaled with direct loads, 2 row-scaled pipelined
template <int ROWS>
__device__ __forceinline__ void emu_block(const EmuParams &P, const EmuBlk &b) {
  const int lane = threadIdx.x & 31;
  const int4 ent0 = load_ent(P, b, lane);
  const int RM = b.sw ? b.n : b.m, RN = b.sw ? b.m : b.n;
  const int MT = (RM + 15) >> 4, NT = (RN + 7) >> 3;
  for (int mt = 0; mt < MT; ++mt)
    for (int ng = 0; ng < NT; ++ng) {
      if (ROWS == 2)
        emu_tile_rs_pipe(P, b, mt, ng, ent0);
      else if (ROWS == 1)
        emu_tile_rs_direct(P, b, mt, ng, ent0);
      else
        emu_tile_bs(P, b, mt, ng, ent0);
    }
}

// Persistent: warps take kChunk consecutive work items at a time from one counter, so
// the blocks in flight stay within a narrow window of the C order (their op(A) digit
// rows and op(B) digit columns stay in L2) and one atomic serves kChunk blocks.  An item
// is plan << 32 | C block (the identity when `items` is null).  The next chunk's index
// is requested when a chunk starts, and its descriptors (lane l holds word l % 8 of
// block l / 8) are loaded after the chunk's first block, so both arrive off the critical
// path.  No waits: a warp whose chunk starts past the end returns.
constexpr int kChunk = 4;
static_assert(kChunk * kDescWords == 32, "one descriptor word per lane");

// average inner length per C element (flops / 2 nelem(C)) from which row-scaled tiles
// take the pipelined loop
constexpr double kPipeMinInner = 64.0;

template <int ROWS, class GetP>
__device__ __forceinline__ void emu_persist(const int64_t *__restrict__ items, int64_t nitems,
                                            unsigned long long *counter, GetP get) {
  const int lane = threadIdx.x & 31;
  // lane 0 issues the atomic; the result is shuffled to the warp only when needed
  auto request = [&]() -> unsigned long long {
    return lane == 0 ? atomicAdd(counter, (unsigned long long)kChunk) : 0ull;
  };
  auto item = [&](int64_t i) -> int64_t { return i < nitems ? (items ? items[i] : i) : -1; };
  // lane l: word l % 8 of the descriptor of item c0 + l / 8
  auto words = [&](int64_t c0) -> int {
    const int64_t v = item(c0 + lane / kDescWords);
    return v >= 0 ? get(v >> 32).desc[(v & 0xffffffffll) * kDescWords + lane % kDescWords] : 0;
  };
  int64_t c0 = (int64_t)__shfl_sync(kFull, request(), 0);
  if (c0 >= nitems) return;
  int dw = words(c0);
  for (;;) {
    const unsigned long long req = request();  // the next chunk, in flight during block 0
    int64_t cn = 0;
    int dwn = 0;
    for (int q = 0; q < kChunk && c0 + q < nitems; ++q) {
      const int64_t v = item(c0 + q);
      const int w = __shfl_sync(kFull, dw, q * kDescWords + (lane & (kDescWords - 1)));
      emu_block<ROWS>(get(v >> 32), emu_blk(w));
      if (q == 0) {
        cn = (int64_t)__shfl_sync(kFull, req, 0);
        dwn = words(cn);
      }
    }
    if (cn >= nitems) return;
    c0 = cn;
    dw = dwn;
  }
}

template <int ROWS>
__global__ void __launch_bounds__(256, 2)
    k_num_emu_bf16_persist1(EmuParams P, int64_t nitems, unsigned long long *counter) {
  emu_persist<ROWS>(nullptr, nitems, counter, [&](int64_t) -> const EmuParams & { return P; });
}

template <int ROWS>
__global__ void __launch_bounds__(256, 2)
    k_num_emu_bf16_persist(const EmuParams *__restrict__ plans, const int64_t *__restrict__ items,
                           int64_t nitems, unsigned long long *counter) {
  emu_persist<ROWS>(items, nitems, counter,
                    [&](int64_t pl) -> const EmuParams & { return plans[pl]; });
}

__global__ void __launch_bounds__(256) k_num_tf32x3(EmuParams P, int64_t nwarps) {
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= nwarps) return;
  const WarpTask w = find_task(P, gw);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = w.mt * 16 + g, r1 = r0 + 8;
  const bool v0 = r0 < w.m, v1 = r1 < w.m;
  int colB[2];
  bool vB[2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    colB[nt] = (2 * w.ng + nt) * 8 + g;
    vB[nt] = nt < w.ntn && colB[nt] < w.n;
  }
  // running sum over the block products as an unevaluated FP32 pair (hi + lo), each
  // product added with an error-free TwoSum, so the sum over many products keeps about
  // twice FP32's precision
  float hi[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  float lo[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int kc = 0; kc < P.Dk; ++kc) {
    const int64_t rr = (int64_t)w.c * P.Dk + kc;
    const int len = P.run_len[rr];
    if (len == 0) continue;
    const int e0 = P.run_start[rr];
    const int k = P.kval[kc], kp = (k + 7) & ~7, nch = kp >> 3;
    for (int e = e0; e < e0 + len; ++e) {
      const float *At = P.a_tf + P.a_doff[P.s_ab[e]];
      const float *Bt = P.b_tf + P.b_doff[P.s_bb[e]];
      const int64_t pa = (int64_t)w.m * kp, pb = (int64_t)w.n * kp;
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      for (int ch = 0; ch < nch; ++ch) {
        const uint2 ah0 = v0 ? ld8(At + (int64_t)r0 * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
        const uint2 ah1 = v1 ? ld8(At + (int64_t)r1 * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
        const uint2 al0 = v0 ? ld8(At + pa + (int64_t)r0 * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
        const uint2 al1 = v1 ? ld8(At + pa + (int64_t)r1 * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          if (nt >= w.ntn) break;
          const uint2 bh = vB[nt] ? ld8(Bt + (int64_t)colB[nt] * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
          const uint2 bl = vB[nt] ? ld8(Bt + pb + (int64_t)colB[nt] * kp + ch * 8 + 2 * t) : make_uint2(0, 0);
          mma_tf32(acc[nt], al0.x, al1.x, al0.y, al1.y, bh.x, bh.y);
          mma_tf32(acc[nt], ah0.x, ah1.x, ah0.y, ah1.y, bl.x, bl.y);
          mma_tf32(acc[nt], ah0.x, ah1.x, ah0.y, ah1.y, bh.x, bh.y);
        }
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float a = hi[nt][h], b = acc[nt][h];
          const float s = __fadd_rn(a, b);
          const float bb = __fsub_rn(s, a);
          const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
          hi[nt][h] = s;
          lo[nt][h] = __fadd_rn(lo[nt][h], err);
        }
    }
  }
  const int64_t off = P.c_off[w.c];
  const int cin = P.c_cin[w.c];
  const double *ci = (P.has_beta && cin >= 0) ? P.Cin + P.cin_off[cin] : nullptr;
  const bool scale = !P.alpha_one;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int r, c;
      slot_rc(w, nt, h, r, c);
      if (nt < w.ntn && r < w.m && c < w.n) {
        double v = f32_to_f64(hi[nt][h]) + f32_to_f64(lo[nt][h]);
        if (scale) v *= P.alpha;
        if (ci) v = fma(P.beta, ci[r * w.n + c], v);
        P.C[off + r * w.n + c] = v;
      }
    }
}

SideArgs side_args(const bst_matrix *X, bool trans, bool is_b) {
  SideArgs S{};
  S.nblocks = X->nblocks;
  S.row = X->row;
  S.col = X->col;
  S.rsz = X->rsz;
  S.csz = X->csz;
  S.off = X->off;
  S.data = X->data;
  S.trans = trans;
  S.is_b = is_b;
  return S;
}

// plan-shape dependent index data (built once per plan)
void emu_index(bst_plan *p, EmuState &E, cudaStream_t s) {
  if (E.index_ready) return;
  Arena &ar = E.ar;
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  auto side = [&](const bst_matrix *X, bool trans, bool is_b, int64_t *&doff, int64_t *&toff,
                  int64_t *&eoff, int64_t &dsize, int64_t &tsize, int64_t &esize) {
    SideArgs S = side_args(X, trans, is_b);
    const int64_t n = X->nblocks;
    int64_t *dsz = scratch.alloc_n<int64_t>((size_t)n), *tsz = scratch.alloc_n<int64_t>((size_t)n),
            *esz = scratch.alloc_n<int64_t>((size_t)n);
    doff = ar.alloc_n<int64_t>((size_t)n + 1);
    toff = ar.alloc_n<int64_t>((size_t)n + 1);
    eoff = ar.alloc_n<int64_t>((size_t)n + 1);
    if (n > 0) {
      k_side_sizes<<<nblk(n, 256), 256, 0, s>>>(S, dsz, tsz, esz);
      BST_CHECK_LAUNCH();
    }
    exscan_i64(dsz, doff, n, scratch, s);
    exscan_i64(tsz, toff, n, scratch, s);
    exscan_i64(esz, eoff, n, scratch, s);
    int64_t tot[3];
    ReadBack rb(p->ctx, s);
    rb.add(&tot[0], doff + n, 8);
    rb.add(&tot[1], toff + n, 8);
    rb.add(&tot[2], eoff + n, 8);
    rb.done();
    dsize = tot[0];
    tsize = tot[1];
    esize = tot[2];
  };
  side(p->A, p->ta, false, E.a_doff, E.a_toff, E.a_eoff, E.a_dsize, E.a_tsize, E.a_esize);
  side(p->B, p->tb, true, E.b_doff, E.b_toff, E.b_eoff, E.b_dsize, E.b_tsize, E.b_esize);
  // entries hold digit offsets in units of 16 elements as 32-bit values
  BST_REQUIRE(E.a_dsize < (1ll << 36) && E.b_dsize < (1ll << 36), BST_ERR_UNSUPPORTED,
              "emulated FP64 digit planes above 2^36 elements");
  // C-major entries of the BF16 kernel
  const int64_t nc = p->C->nblocks;
  E.ebeg = ar.alloc_n<int64_t>((size_t)nc + 1);
  E.ents = ar.alloc_n<int4>((size_t)std::max<int64_t>(p->T, 1));
  {
    int32_t *cnt = scratch.alloc_n<int32_t>((size_t)std::max<int64_t>(nc, 1));
    if (nc > 0) {
      k_emu_ent_count<<<nblk(nc, 256), 256, 0, s>>>(nc, p->Dk, p->run_len, cnt);
      BST_CHECK_LAUNCH();
    }
    exscan_i32_i64(cnt, E.ebeg, nc, scratch, s);
    if (nc > 0) {
      k_emu_ents<<<nblk(nc, 256), 256, 0, s>>>(nc, p->Dk, p->run_start, p->run_len, p->kval,
                                               p->s_ab, p->s_bb, E.a_doff, E.b_doff, E.ebeg,
                                               E.ents);
      BST_CHECK_LAUNCH();
    }
  }
  // 3xTF32 warps per (m,n) class: one per 16-row x 16-column tile of each C block
  const int32_t ncls = p->Dm * p->Dn;
  std::vector<int64_t> ws((size_t)ncls + 1, 0);
  for (int32_t c = 0; c < ncls; ++c) {
    const int64_t cnt = (int64_t)p->h_class_ptr[c + 1] - p->h_class_ptr[c];
    const int m = p->m_vals.empty() ? 0 : p->m_vals[c / p->Dn];
    const int n = p->n_vals.empty() ? 0 : p->n_vals[c % p->Dn];
    const int64_t mt = (m + 15) / 16, nt = (n + 7) / 8;
    ws[c + 1] = ws[c] + cnt * mt * ((nt + 1) / 2);
  }
  E.ncls = ncls;
  E.nwarps = ws.back();
  // global element starts of op(A) row blocks and op(B) column blocks
  auto starts = [&](const std::vector<int32_t> &sz, int64_t &total) {
    std::vector<int64_t> h(sz.size() + 1, 0);
    for (size_t q = 0; q < sz.size(); ++q) h[q + 1] = h[q] + sz[q];
    total = h.back();
    return h;
  };
  {
    const std::vector<int64_t> ha = starts(p->oa.h_rs, E.nrows), hb = starts(p->ob.h_cs, E.ncols);
    Upload up(p->ctx, s);
    E.wstart = up.add_vector(ar, ws);
    E.a_rowstart = up.add_vector(ar, ha);
    E.b_colstart = up.add_vector(ar, hb);
    up.done();
  }
  BST_CUDA(cudaStreamSynchronize(s));
  scratch.release_all();
  E.index_ready = true;
}

EmuState &emu_state(bst_plan *p, cudaStream_t s) {
  if (!p->emu) {
    p->emu = new EmuState();
    p->emu->ar.ctx = static_cast<Ctx *>(p->ctx);
    p->emu->ar.stream = s;
  }
  emu_index(p, *p->emu, s);
  return *p->emu;
}

EmuParams emu_params(bst_plan *p, const EmuState &E, const NumArgs &a) {
  EmuParams P{};
  P.Cin = a.Cin;
  P.C = a.C;
  P.alpha = a.alpha;
  P.alpha_one = a.alpha == 1.0;
  P.has_beta = a.beta != 0.0;
  P.beta = a.beta;
  P.Dk = p->Dk;
  P.ncls = E.ncls;
  P.wstart = E.wstart;
  P.tiles_n = 2;
  P.a_rowstart = E.a_rowstart;
  P.b_colstart = E.b_colstart;
  P.row_exp = E.row_exp;
  P.col_exp = E.col_exp;
  P.class_ptr = p->class_ptr;
  P.task_c = p->task_c;
  P.cls_m = p->cls_m;
  P.cls_n = p->cls_n;
  P.kval = p->kval;
  P.c_row = p->C->row;
  P.c_cls = p->c_cls;
  P.c_col = p->C->col;
  P.c_cin = p->c_cin;
  P.c_off = p->C->off;
  P.cin_off = p->Cin ? p->Cin->off : nullptr;
  P.run_start = p->run_start;
  P.run_len = p->run_len;
  P.s_ab = p->s_ab;
  P.s_bb = p->s_bb;
  P.desc = E.desc;
  P.ents = E.ents;
  P.a_eoff = E.a_eoff;
  P.b_eoff = E.b_eoff;
  P.a_dig = E.a_dig;
  P.b_dig = E.b_dig;
  P.a_tf = E.a_tf;
  P.b_tf = E.b_tf;
  P.a_exp = E.a_exp;
  P.b_exp = E.b_exp;
  return P;
}

}  // namespace

void emu_state_free(bst_plan *p) {
  delete p->emu;
  p->emu = nullptr;
}

// digit buffers of a plan (allocated once; outside any stream capture)
static void emu_alloc_digits(EmuState &E) {
  if (E.dig_alloc) return;
  E.a_dig = E.ar.alloc_n<__nv_bfloat16>((size_t)E.a_dsize);
  E.b_dig = E.ar.alloc_n<__nv_bfloat16>((size_t)E.b_dsize);
  E.a_exp = E.ar.alloc_n<int32_t>((size_t)E.a_esize);
  E.b_exp = E.ar.alloc_n<int32_t>((size_t)E.b_esize);
  E.row_exp = E.ar.alloc_n<int32_t>((size_t)E.nrows);
  E.col_exp = E.ar.alloc_n<int32_t>((size_t)E.ncols);
  E.dig_alloc = true;
}

// slices and exponents of the current operand data (launches only)
static void emu_prepare(bst_plan *p, EmuState &E, const NumArgs &a, cudaStream_t s) {
  fill_i32(E.a_exp, kExpNone, E.a_esize, s);
  fill_i32(E.b_exp, kExpNone, E.b_esize, s);
  fill_i32(E.row_exp, kExpNone, E.nrows, s);
  fill_i32(E.col_exp, kExpNone, E.ncols, s);
  const int wpb = 8;
  for (int side = 0; side < 2; ++side) {
    const bst_matrix *X = side ? p->B : p->A;
    if (X->nblocks == 0) continue;
    SideArgs S = side_args(X, side ? p->tb : p->ta, side == 1);
    S.data = side ? a.B : a.A;
    S.eoff = side ? E.b_eoff : E.a_eoff;
    S.doff = side ? E.b_doff : E.a_doff;
    S.bexp = side ? E.b_exp : E.a_exp;
    S.start = side ? E.b_colstart : E.a_rowstart;
    S.gexp = side ? E.col_exp : E.row_exp;
    S.dig = side ? E.b_dig : E.a_dig;
    S.row_scale = p->ctx->tune_emu_row_scale;
    k_emu_exponents<<<nblk(X->nblocks, wpb), 32 * wpb, 0, s>>>(S);
    BST_CHECK_LAUNCH();
    k_emu_digits<<<nblk(X->nblocks, wpb), 32 * wpb, 0, s>>>(S);
    BST_CHECK_LAUNCH();
  }
}

static EmuParams bf16_params(bst_plan *p, const EmuState &E, const NumArgs &a) {
  EmuParams P = emu_params(p, E, a);
  P.a_doff = E.a_doff;
  P.b_doff = E.b_doff;
  P.tiles_n = 1;
  P.row_scale = p->ctx->tune_emu_row_scale;
  return P;
}

size_t emu_params_bytes() { return sizeof(EmuParams); }

void emu_build_items(bst_plan *p, int64_t base, int64_t *items, cudaStream_t s);

// Tile orientation of class (m, n): the tuned choice when there is one, else the one
// with fewer 16 x 8 tiles (ties keep rows over rows).  Block-scaled mode never swaps.
static int class_swap(const bst_ctx *ctx, int m, int n) {
  if (!ctx->tune_emu_row_scale) return 0;
  auto it = ctx->tune_emu_swap.find({m, n});
  if (it != ctx->tune_emu_swap.end()) return it->second;
  const int plain = ((m + 15) / 16) * ((n + 7) / 8), swapped = ((n + 15) / 16) * ((m + 7) / 8);
  return swapped < plain ? 1 : 0;
}

// (Re)build the BF16 C block descriptors when the tuning state changed since the last
// build (they carry each class's tile orientation).  Launches only, no synchronisation.
static void emu_schedule(bst_plan *p, EmuState &E, cudaStream_t s) {
  const bst_ctx *ctx = p->ctx;
  if (E.desc && E.sched_version == ctx->tune_version && E.sched_rows == ctx->tune_emu_row_scale)
    return;
  const int32_t ncls = p->Dm * p->Dn;
  std::vector<int32_t> sw((size_t)std::max(ncls, 1), 0);
  for (int32_t c = 0; c < ncls; ++c) {
    const int m = p->m_vals.empty() ? 0 : p->m_vals[c / p->Dn];
    const int n = p->n_vals.empty() ? 0 : p->n_vals[c % p->Dn];
    const int64_t cnt = (int64_t)p->h_class_ptr[c + 1] - p->h_class_ptr[c];
    // the descriptor holds m and n in 12 bits each
    BST_REQUIRE(cnt == 0 || (m < 4096 && n < 4096), BST_ERR_UNSUPPORTED,
                "emulated FP64 takes C blocks of at most 4095 x 4095 elements");
    if (cnt > 0 && m > 0 && n > 0) sw[(size_t)c] = class_swap(ctx, m, n);
  }
  const int64_t nc = p->C->nblocks;
  if (!E.cls_swap) E.cls_swap = E.ar.alloc_n<int32_t>(sw.size());
  if (!E.desc) E.desc = E.ar.alloc_n<int32_t>((size_t)std::max<int64_t>(nc, 1) * kDescWords);
  if (!E.counter) E.counter = E.ar.alloc_n<unsigned long long>(1);
  {
    Upload up(p->ctx, s);
    up.add(E.cls_swap, sw.data(), 4 * sw.size());
    up.done();
  }
  if (nc > 0) {
    k_emu_desc<<<nblk(nc, 256), 256, 0, s>>>(nc, p->Dk, p->run_len, p->kval, E.ebeg, p->C->off,
                                             p->C->row, p->C->col, p->c_cls, p->cls_m, p->cls_n,
                                             E.cls_swap, p->c_cin, E.a_rowstart, E.b_colstart,
                                             E.desc);
    BST_CHECK_LAUNCH();
  }
  E.nitems_b = nc;
  E.sched_version = ctx->tune_version;
  E.sched_rows = ctx->tune_emu_row_scale;
}

int64_t emu_item_count(bst_plan *p, cudaStream_t s) {
  if (p->C->nblocks == 0) return 0;
  EmuState &E = emu_state(p, s);
  emu_alloc_digits(E);
  emu_schedule(p, E, s);
  return E.nitems_b;
}

// the BF16 work items of a plan in a batch: base | C block, in C block order
void emu_build_items(bst_plan *p, int64_t base, int64_t *items, cudaStream_t s) {
  const int64_t nc = p->C->nblocks;
  if (nc == 0) return;
  k_emu_items<<<nblk(nc, 256), 256, 0, s>>>(nc, base, items);
  BST_CHECK_LAUNCH();
}

void emu_prepare_and_fill(bst_plan *p, const NumArgs &a, void *out, cudaStream_t s) {
  EmuState &E = *p->emu;
  emu_prepare(p, E, a, s);
  EmuParams P = bf16_params(p, E, a);
  std::memcpy(out, &P, sizeof(P));
}

// resident CTAs of 256 threads per SM for the BF16 kernels (both scaling modes)
static int emu_ctas_per_sm(bool batch, int row_scale) {
  int nb = 0;
  if (batch) {
    if (row_scale)
      BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_emu_bf16_persist<1>, 256, 0));
    else
      BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_emu_bf16_persist<0>, 256, 0));
  } else {
    if (row_scale)
      BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_emu_bf16_persist1<1>, 256, 0));
    else
      BST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_num_emu_bf16_persist1<0>, 256, 0));
  }
  return std::max(1, nb);
}

int emu_persist_grid(int num_sms, int row_scale) { return emu_ctas_per_sm(true, row_scale) * num_sms; }

bool emu_pipelined(double flops, int64_t nelem_c) {
  return nelem_c > 0 && flops >= 2.0 * kPipeMinInner * (double)nelem_c;
}

void launch_emu_persist(const void *params, const int64_t *items, int64_t nitems,
                        unsigned long long *counter, int grid, int row_scale, bool pipe,
                        cudaStream_t s) {
  if (nitems == 0) return;
  BST_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  const int g = (int)std::min<int64_t>(grid, (nitems + 8 * kChunk - 1) / (8 * kChunk));
  const EmuParams *P = static_cast<const EmuParams *>(params);
  if (row_scale && pipe)
    k_num_emu_bf16_persist<2><<<g, 256, 0, s>>>(P, items, nitems, counter);
  else if (row_scale)
    k_num_emu_bf16_persist<1><<<g, 256, 0, s>>>(P, items, nitems, counter);
  else
    k_num_emu_bf16_persist<0><<<g, 256, 0, s>>>(P, items, nitems, counter);
  BST_CHECK_LAUNCH();
}

void execute_emu_bf16(bst_plan *p, const NumArgs &a, cudaStream_t s) {
  if (p->C->nblocks == 0) return;
  if (panel_usable(p, s, true)) {
    execute_emu_panel(p, a, s);
    return;
  }
  EmuState &E = emu_state(p, s);
  emu_alloc_digits(E);
  emu_schedule(p, E, s);  // C block descriptors, rebuilt when tuning changed
  emu_prepare(p, E, a, s);
  const EmuParams P = bf16_params(p, E, a);
  if (E.nitems_b > 0) {
    const int g = (int)std::min<int64_t>((int64_t)emu_ctas_per_sm(false, P.row_scale) * p->ctx->num_sms,
                                         (E.nitems_b + 8 * kChunk - 1) / (8 * kChunk));
    BST_CUDA(cudaMemsetAsync(E.counter, 0, sizeof(unsigned long long), s));
    if (P.row_scale && emu_pipelined(p->stats.flops, p->C->nelem))
      k_num_emu_bf16_persist1<2><<<g, 256, 0, s>>>(P, E.nitems_b, E.counter);
    else if (P.row_scale)
      k_num_emu_bf16_persist1<1><<<g, 256, 0, s>>>(P, E.nitems_b, E.counter);
    else
      k_num_emu_bf16_persist1<0><<<g, 256, 0, s>>>(P, E.nitems_b, E.counter);
    BST_CHECK_LAUNCH();
  }
}

// Cost model of one emulated-FP64 execute (for rooflines): BF16 tensor flops issued
// (21 slice products per MMA tile the kernel runs, padding included), the bytes its
// kernels move by design -- the FP64 operands read by the exponent and digit passes,
// the digit planes written once and read once, C written, the schedule read -- and the
// intermediate bytes of partial products (the panel path's int64 slots).
void emu_costs(bst_plan *p, cudaStream_t s, double *tensor_flops, double *bytes,
               double *intermediate) {
  *tensor_flops = 0.0;
  *bytes = 0.0;
  *intermediate = 0.0;
  if (p->C->nblocks == 0) return;
  if (panel_usable(p, s)) {
    double o[3];
    panel_costs(p, s, o);
    *tensor_flops = o[0];
    *bytes = o[1];
    *intermediate = o[2];
    return;
  }
  EmuState &E = emu_state(p, s);
  const auto &hb = p->h_bucket_ptr;
  double fl = 0.0;
  for (int32_t b = 0; b < p->nb_all; ++b) {
    const int64_t cnt = hb[b + 1] - hb[b];
    if (cnt == 0) continue;
    const int kc = b % p->Dk, nc = (b / p->Dk) % p->Dn, mc = b / (p->Dk * p->Dn);
    const int m = p->m_vals[mc], n = p->n_vals[nc], k = p->k_vals[kc];
    const int sw = p->ctx->tune_emu_row_scale ? class_swap(p->ctx, m, n) : 0;
    const double tiles = sw ? (double)((n + 15) / 16) * ((m + 7) / 8)
                            : (double)((m + 15) / 16) * ((n + 7) / 8);
    fl += (double)cnt * 21.0 * 2.0 * tiles * 16 * 8 * 16 * ((k + 15) / 16);
  }
  *tensor_flops = fl;
  *bytes = 16.0 * (double)(p->A->nelem + p->B->nelem) +
           2.0 * 2.0 * (double)(E.a_dsize + E.b_dsize) + 8.0 * (double)p->C->nelem +
           16.0 * (double)p->T + 4.0 * kDescWords * (double)p->C->nblocks;
}

void execute_tf32x3(bst_plan *p, const NumArgs &a, cudaStream_t s) {
  if (p->C->nblocks == 0) return;
  EmuState &E = emu_state(p, s);
  if (!E.tf_alloc) {
    E.a_tf = E.ar.alloc_n<float>((size_t)E.a_tsize);
    E.b_tf = E.ar.alloc_n<float>((size_t)E.b_tsize);
    E.tf_alloc = true;
  }
  BST_CUDA(cudaMemsetAsync(E.a_tf, 0, 4 * (size_t)std::max<int64_t>(E.a_tsize, 1), s));
  BST_CUDA(cudaMemsetAsync(E.b_tf, 0, 4 * (size_t)std::max<int64_t>(E.b_tsize, 1), s));
  const int wpb = 8;
  for (int side = 0; side < 2; ++side) {
    const bst_matrix *X = side ? p->B : p->A;
    if (X->nblocks == 0) continue;
    SideArgs S = side_args(X, side ? p->tb : p->ta, side == 1);
    S.data = side ? a.B : a.A;
    S.doff = side ? E.b_toff : E.a_toff;
    S.tf = side ? E.b_tf : E.a_tf;
    k_tf32_split<<<nblk(X->nblocks, wpb), 32 * wpb, 0, s>>>(S);
    BST_CHECK_LAUNCH();
  }
  EmuParams P = emu_params(p, E, a);
  P.a_doff = E.a_toff;
  P.b_doff = E.b_toff;
  if (E.nwarps > 0) {
    k_num_tf32x3<<<nblk(E.nwarps, wpb), 32 * wpb, 0, s>>>(P, E.nwarps);
    BST_CHECK_LAUNCH();
  }
}

}  // namespace bst
