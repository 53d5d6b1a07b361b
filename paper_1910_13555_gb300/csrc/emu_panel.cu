// Emulated FP64 on the fifth-generation tensor cores (tcgen05, TMEM accumulators), by
// inner-block panels.
//
// The local multiply sums, for every kept triple (i, k, j), the product of the op(A)
// block (i, k) with the op(B) block (k, j) (paper Sec. 2).  For a fixed inner block k
// every present op(A) block of block column k meets every present op(B) block of block
// row k, so the products of panel k form one dense outer product: the op(A) blocks of
// column k stacked into M_k rows times the op(B) blocks of row k side by side in N_k
// columns, over the k inner elements.  With blocks of 5-23 elements and ~1 % occupancy
// a C block has only one or two products, but a panel is hundreds of rows by hundreds
// of columns: a dense contraction the tcgen05 tensor cores can run in 128 x 32 tiles,
// where a C-block-centred schedule would pad 5-row blocks to 16-row tiles.
//
// Arithmetic (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012: error-free
// splitting).  Every stored block X is scaled by 2^-E with E its largest exponent
// (|x| < 2^E) and each element is rounded to 47 fraction bits and written as six
// balanced 8-bit digits, x = 2^(E-47) sum_s d_s 2^(8(5-s)), |d_s| <= 128, all exact in
// BF16.  A digit product is at most 2^14 and exact in FP32; the slice products of
// level w = s + t <= 5 (21 of 36; the dropped ones weigh about 2^-48 of the scale) are
// summed per level by the tensor cores into FP32 TMEM accumulators.  A level sum over
// at most 32 inner elements holds at most 6 * 32 * 2^14 < 2^22 in magnitude, so every
// partial sum is an integer below 2^24 and exact.  The epilogue adds 1.5 * 2^23 to each
// level sum (exact: the result stays in [2^23, 2^24), where the FP32 encoding minus that
// of 1.5 * 2^23 is the integer itself -- no float-to-int conversion), folds the six
// levels into one integer I = sum_w D_w 2^(8(5-w)) (|I| < 2^59.1) and the product
// block is I * 2^(Ea + Eb - 54).
//
// Output.  A C block with exactly one product and no C_in block is written directly
// (I converted to FP64 with the hardware int64 -> FP64 conversion, correctly rounded).
// The products of every other C block go to int64 slots (one m x n slot per product,
// in the C block's product order), each shifted with rounding from its own scale
// Ea + Eb to the C block's common scale S (the largest Ea + Eb of its products plus
// guard bits for their count); a second kernel adds a C block's slots in a fixed order
// (exact integer sums), converts once and applies alpha and beta C_in.  Results do not
// depend on scheduling; each C block keeps its own scale, so a block many decades below
// the other blocks of its rows keeps full relative accuracy.
//
// The MMA kernel is persistent, one CTA of 18 warps per SM, warp-specialised: warp 16
// loads each unit's A tile image, each N-tile's B image and the epilogue's records with
// cp.async.bulk (completion on mbarriers); warp 17 allocates 512 TMEM columns and one
// elected lane of it issues the tcgen05.mma instructions into two accumulator buffers
// (6 levels x 32 columns each); warps 0-15 are two epilogue groups of 8 warps, group g
// draining buffer g: they read the levels back with tcgen05.ld (thread t of a group:
// TMEM lane t mod 128, half of the columns), fold them, stage the tile in shared memory
// and write whole C-block rows with coalesced stores.  Units, in decreasing cost, are
// dealt to the CTAs in serpentine order (odd rounds backwards); one grid serves the
// units of one plan or of a whole batch of plans (per-plan pointers in a table).
// Every wait is bounded: a wait that runs out (2 s) records an error flag, and the
// kernel's roles stop, drain their copies and MMAs, free TMEM and return.
//
// Operand images.  The digits are written once per execute directly in the layout the
// tensor core reads from shared memory (K-major; each row's inner values contiguous, 32
// or 64 bytes for nq = 1 or 2 K-steps of 16, in 8-row atoms with the 32- or 64-byte
// swizzle), per unit (panel k, 128-row tile) slice by slice, so a unit's A operand is
// one contiguous bulk copy of 6 * nq * 4 KB and an N-tile's B operand 6 * nq * 1 KB.
// Tiles are cut at block boundaries (at most 32 blocks per A tile, 8 per N-tile, packed
// first-fit decreasing), so each (A block, B block) pair of a tile is one whole product.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "bst_internal.h"

namespace bst {

namespace {

constexpr int kDig = 6;             // digits per operand element
constexpr int kTM = 128;            // rows of an A tile (TMEM lanes)
constexpr int kTN = 32;             // columns of an N-tile
constexpr int kMaxAB = 32;          // A blocks per tile
constexpr int kMaxBB = 8;           // B blocks per N-tile
constexpr int kStages = 3;          // B operand stages
constexpr int kRecStages = 4;       // tile record stages (epilogue tables of an N-tile)
constexpr int kURec = kMaxAB;       // int4 entries of a unit record
constexpr int kNTRec = 17;          // int4 entries of an N-tile record
constexpr int kAStep = kTM * 16 * 2;               // bytes of one A K-step image (4096)
constexpr int kBStep = kTN * 16 * 2;               // bytes of one B K-step image (1024)
constexpr int kABuf = kDig * 2 * kAStep;           // A buffer: 6 slices x 2 K-steps
constexpr int kBBuf = kDig * 2 * kBStep;
constexpr int kStgLd = kTN + 1;                    // staging row stride (8-byte words)
constexpr int kFrac = 47;                          // fraction bits of the digits
constexpr int kNoExp = -4000;                      // exponent of an all-zero block
constexpr int kAccCols = 256;                      // TMEM columns per accumulator buffer
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every wait
constexpr int kErrWait = 1;                        // error code: a wait ran out

// unit = (panel k, 128-row tile); sorted by decreasing cost on the host
struct PUnit {
  long long a_img;  // byte offset of the tile's digit image
  long long pb;     // first pair entry of its first N-tile
  int ab0, nab;     // its A blocks in alist
  int v0, nN;       // the panel's N-tiles
  int nq, pad;
};

struct PNTile {
  long long b_img;  // byte offset of the N-tile's digit image
  int bb0, nbb;     // its B blocks in blist
  int cum;          // B blocks of the panel's earlier N-tiles
  int nq;
};

}  // namespace

struct PanelState {
  Arena ar;
  bool built = false, eligible = false;
  int64_t nunits = 0, nntiles = 0, npairs = 0, nred = 0;
  PUnit *units = nullptr;
  PNTile *ntiles = nullptr;
  int4 *alist = nullptr, *blist = nullptr;  // {stored block, row / column offset, m / n, 0}
  int2 *a_where = nullptr, *b_where = nullptr;  // per stored block: {unit / N-tile, index}
  int64_t a_img_bytes = 0, b_img_bytes = 0;
  char *a_img = nullptr, *b_img = nullptr;
  // per (unit, N-tile) pair {dst lo, dst hi, shift, 0}: dst >= 0 C offset, <= -2 slot
  // -(dst + 2), -1 filtered; shift (per execute) of a slot product to its C block's scale
  int4 *pairs = nullptr;
  int4 *urec = nullptr;   // per unit: kURec {row offset, m, exponent (per execute), block}
  int4 *ntrec = nullptr;  // per N-tile: {nbb}, column table, {col offset, n, exponent, block}
  int32_t *pair_pos = nullptr;  // per C-major product: its pair entry
  int64_t *cbeg = nullptr;      // per C block: first C-major product (nc + 1)
  int32_t *red = nullptr;       // C blocks summed from slots (several products or C_in)
  int4 *red_desc = nullptr;     // their descriptors (two int4 each)
  int64_t *slot_base = nullptr;
  int64_t slot_elems = 0;
  int64_t *slots = nullptr;
  int32_t *c_scale = nullptr;   // per C block: common exponent of its slots
  int32_t *a_exp = nullptr, *b_exp = nullptr;  // per stored block (per execute)
  int *err = nullptr;
  double tensor_flops = 0.0;
  double fill = 0.0;  // credited multiply-adds / the tiles' multiply-adds
};

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- small device helpers --------------------------------------------------------

__device__ __forceinline__ int exp_of(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  return ex == 0 ? kNoExp : ex - 1022;
}

__device__ __noinline__ double ldexp_slow(double d, int e2) { return ldexp(d, e2); }

// v * 2^e2, rounded to nearest-even: hardware int64 -> FP64, then the scale added to the
// exponent field (exact while the result stays normal)
__device__ __forceinline__ double i64_scaled(long long v, int e2) {
  if (v == 0) return 0.0;
  const double d = __ll2double_rn(v);
  const long long bits = __double_as_longlong(d);
  const int be = (int)((bits >> 52) & 0x7ff) + e2;
  if (be <= 0 || be >= 2047) return ldexp_slow(d, e2);
  return __longlong_as_double(bits + ((long long)e2 << 52));
}

// The same with integer instructions only (GB300's FP64 unit, where the hardware
// conversion runs, is slow to return results; measured faster in the reduction kernel,
// slower than the hardware conversion in the panel kernel's copy-out, where the extra
// integer instructions compete for issue slots): |v| normalised by its leading-zero
// count, its top 53 bits rounded to nearest-even on the 11 below, the exponent field
// 1086 - lz + e2 assembled (a rounding carry into bit 53 raises it by one).  Checked
// against the correctly rounded conversion on 600 000 values; results outside the
// normal range go through ldexp.
__device__ __forceinline__ double i64_scaled_int(long long v, int e2) {
  if (v == 0) return 0.0;
  const unsigned long long sg = (unsigned long long)v & (1ull << 63);
  unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long m = a >> 11;
  const unsigned rem = (unsigned)a & 0x7FFu;
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  const int be = 1086 - lz + e2;
  if (be <= 0 || be >= 2046) return ldexp_slow(__ll2double_rn(v), e2);
  return __longlong_as_double((long long)(sg | (((unsigned long long)(be - 1) << 52) + m)));
}

__device__ __forceinline__ long long round_shift(long long v, int sh) {
  if (sh <= 0) return v;
  if (sh >= 62) return 0;
  return (v + (1ll << (sh - 1))) >> sh;
}

// ---- per-plan index kernels -------------------------------------------------------

__global__ void k_pan_count(int64_t nc, int32_t Dk, const int32_t *__restrict__ run_len,
                            int32_t *__restrict__ cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int s = 0;
  for (int kc = 0; kc < Dk; ++kc) s += run_len[c * Dk + kc];
  cnt[c] = s;
}

// C blocks written by the reduction (all but single-product blocks without C_in) and
// their slot sizes
__global__ void k_pan_red_flags(int64_t nc, const int32_t *__restrict__ cnt,
                                const int32_t *__restrict__ c_cin, const int32_t *__restrict__ crow,
                                const int32_t *__restrict__ ccol, const int32_t *__restrict__ rsz,
                                const int32_t *__restrict__ csz, int32_t *__restrict__ flag,
                                int64_t *__restrict__ ssz) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const bool r = cnt[c] != 1 || c_cin[c] >= 0;
  flag[c] = r;
  ssz[c] = r ? (int64_t)cnt[c] * rsz[crow[c]] * csz[ccol[c]] : 0;
}

__global__ void k_pan_compact(int64_t nc, const int32_t *__restrict__ flag,
                              const int32_t *__restrict__ pos, int32_t *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && flag[c]) out[pos[c]] = (int32_t)c;
}

// descriptors of the reduced C blocks (the scale word is filled per execute)
__global__ void k_pan_red_desc(int64_t nred, const int32_t *__restrict__ red,
                               const int32_t *__restrict__ cnt, const int32_t *__restrict__ c_cin,
                               const int32_t *__restrict__ crow, const int32_t *__restrict__ ccol,
                               const int32_t *__restrict__ rsz, const int32_t *__restrict__ csz,
                               const int64_t *__restrict__ slot_base, const int64_t *__restrict__ c_off,
                               int4 *__restrict__ desc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nred) return;
  const int c = red[i];
  const unsigned long long sb = (unsigned long long)slot_base[c], co = (unsigned long long)c_off[c];
  desc[2 * i] = make_int4((int)(unsigned)sb, (int)(unsigned)(sb >> 32), (int)(unsigned)co,
                          (int)(unsigned)(co >> 32));
  desc[2 * i + 1] = make_int4(rsz[crow[c]] * csz[ccol[c]], cnt[c], 0, c_cin[c]);
}

struct PairArgs {
  int64_t nc;
  int32_t Dk;
  const int32_t *run_start, *run_len, *s_ab, *s_bb;
  const int32_t *flag, *crow, *ccol, *rsz, *csz;
  const int64_t *c_off, *cbeg, *slot_base;
  const PUnit *units;
  const PNTile *ntiles;
  const int2 *a_where, *b_where;
  int4 *pairs;
  int32_t *pair_pos;
};

// pair entry of every kept product: its destination and, per C-major product, where
// its entry is
__global__ void k_pan_pairs(PairArgs P) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  const int64_t mn = (int64_t)P.rsz[P.crow[c]] * P.csz[P.ccol[c]];
  const bool r = P.flag[c] != 0;
  int64_t q = 0;
  const int64_t e0 = P.cbeg[c];
  for (int kc = 0; kc < P.Dk; ++kc) {
    const int len = P.run_len[c * P.Dk + kc];
    const int es = P.run_start[c * P.Dk + kc];
    for (int e = es; e < es + len; ++e, ++q) {
      const int2 aw = P.a_where[P.s_ab[e]], bw = P.b_where[P.s_bb[e]];
      const PUnit &U = P.units[aw.x];
      const PNTile &V = P.ntiles[bw.x];
      const int64_t pos = U.pb + (int64_t)U.nab * V.cum + (int64_t)aw.y * V.nbb + bw.y;
      const long long dst = r ? -(P.slot_base[c] + q * mn) - 2 : P.c_off[c];
      P.pairs[pos] = make_int4((int)(unsigned)(unsigned long long)dst,
                               (int)(unsigned)((unsigned long long)dst >> 32), 0, -1);
      P.pair_pos[e0 + q] = (int32_t)pos;
    }
  }
}

// ---- per-execute kernels ----------------------------------------------------------

struct SideP {
  int64_t nblocks;
  const int32_t *row, *col, *rsz, *csz;
  const int64_t *off;
  const double *data;
  int trans, is_b;
  int32_t *bexp;
  const int2 *where;
  const PUnit *units;
  const PNTile *ntiles;
  const int4 *list;
  char *img;
};

// Digits of every stored block of a panel into its tile image, after its largest
// exponent (one warp per stored block; blocks no kept product uses are skipped, their
// exponent is never read).  Item (outer row r of
// the tile, 8-group g of the inner index): 8 consecutive inner values -> six 16-byte
// core-matrix rows, one per slice (inner positions at and above the inner size are
// written as zeros).
__global__ void k_pan_digits(SideP S) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= S.nblocks) return;
  const int2 wh = S.where[b];
  if (wh.x < 0) return;  // no product uses this block
  const int R = S.rsz[S.row[b]], Cc = S.csz[S.col[b]];
  const int nouter = S.is_b ? (S.trans ? R : Cc) : (S.trans ? Cc : R);
  const int ninner = S.is_b ? (S.trans ? Cc : R) : (S.trans ? R : Cc);
  const bool outer_major = S.is_b == S.trans;  // element (o, l) at o * Cc + l
  long long img;
  int nq, first;
  if (S.is_b) {
    const PNTile &V = S.ntiles[wh.x];
    img = V.b_img;
    nq = V.nq;
    first = S.list[V.bb0 + wh.y].y;
  } else {
    const PUnit &U = S.units[wh.x];
    img = U.a_img;
    nq = U.nq;
    first = S.list[U.ab0 + wh.y].y;
  }
  const int stepb = S.is_b ? kBStep : kAStep;
  const double *x = S.data + S.off[b];
  // the block's largest exponent (also kept for the records and the slot shifts)
  int E = kNoExp;
  {
    const int n = R * Cc;
    for (int e = lane; e < n; e += 32) E = max(E, exp_of(x[e]));
#pragma unroll
    for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) S.bexp[b] = E;
  }
  const int ng = 2 * nq;
  const int total = nouter * ng;
  for (int it = lane; it < total; it += 32) {
    const int o = it / ng, g = it - o * ng;
    uint32_t w[kDig][4];
#pragma unroll
    for (int s = 0; s < kDig; ++s) w[s][0] = w[s][1] = w[s][2] = w[s][3] = 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int l = 8 * g + u;
      if (l >= ninner || E == kNoExp) continue;
      const double v = x[outer_major ? o * Cc + l : l * Cc + o];
      const long long bits = __double_as_longlong(v);
      const int ex = (int)((bits >> 52) & 0x7ff);
      unsigned long long N = 0;
      if (ex != 0) {
        const unsigned long long M = (unsigned long long)(bits & 0xfffffffffffffLL) | (1ull << 52);
        const int rsh = 1075 - kFrac - ex + E;  // >= 6 since |v| < 2^E
        if (rsh < 64) N = (M + (1ull << (rsh - 1))) >> rsh;
      }
      const bool neg = bits < 0;
      int d[kDig];
#pragma unroll
      for (int s = kDig - 1; s >= 1; --s) {
        int r = (int)(N & 255ull);
        N >>= 8;
        if (r >= 128) {
          r -= 256;
          N += 1;
        }
        d[s] = r;
      }
      d[0] = (int)N;  // <= 128
#pragma unroll
      for (int s = 0; s < kDig; ++s) {
        const int dv = neg ? -d[s] : d[s];
        const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn((float)dv));
        w[s][u >> 1] |= h << (16 * (u & 1));
      }
    }
    // tile row (A) / tile column (B) r, 16-byte chunk g of its row: rows of 32 B (nq = 1)
    // or 64 B (nq = 2) in 8-row atoms; the chunk index is XORed with row bits as the
    // 32-byte (bit 2 of r) or 64-byte (bits 1-2 of r) swizzle places it
    const int r = first + o;
    const int rowb = 32 * nq;
    const int sw = nq == 1 ? ((r >> 2) & 1) : ((r >> 1) & 3);
    const long long base = img + (long long)(r >> 3) * (8 * rowb) + (r & 7) * rowb + ((g ^ sw) << 4);
#pragma unroll
    for (int s = 0; s < kDig; ++s)
      *reinterpret_cast<uint4 *>(S.img + base + (long long)s * nq * stepb) =
          make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// the per-execute block exponents copied into the unit and N-tile records
__global__ void k_pan_recexp(int64_t nunits, int64_t nntiles, int4 *__restrict__ urec,
                             int4 *__restrict__ ntrec, const PNTile *__restrict__ ntiles,
                             const int4 *__restrict__ blist, const int32_t *__restrict__ a_exp,
                             const int32_t *__restrict__ b_exp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nunits * kURec) {
    int4 &e = urec[i];
    if (e.y > 0) e.z = a_exp[e.w];
  } else if (i < nunits * kURec + nntiles * kMaxBB) {
    const int64_t j = i - nunits * kURec, v = j / kMaxBB;
    const int jb = (int)(j % kMaxBB);
    const PNTile &V = ntiles[v];
    if (jb < V.nbb) ntrec[v * kNTRec + 9 + jb].z = b_exp[blist[V.bb0 + jb].x];
  }
}

struct ShiftArgs {
  int64_t nred;
  int32_t Dk;
  const int32_t *red, *run_start, *run_len, *s_ab, *s_bb, *pair_pos;
  const int64_t *cbeg;
  const int32_t *a_exp, *b_exp;
  int4 *pairs;
  int32_t *c_scale;
  int4 *desc;
};

// common scale of every reduced C block and each of its products' shift to it
__global__ void k_pan_shift(ShiftArgs P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.nred) return;
  const int c = P.red[i];
  int S = -2 * 4096, np = 0;
  for (int kc = 0; kc < P.Dk; ++kc) {
    const int len = P.run_len[(int64_t)c * P.Dk + kc], es = P.run_start[(int64_t)c * P.Dk + kc];
    for (int e = es; e < es + len; ++e, ++np) S = max(S, P.a_exp[P.s_ab[e]] + P.b_exp[P.s_bb[e]]);
  }
  int lg = 0;
  while ((1 << lg) <= np) ++lg;
  const int G = max(0, lg - 3);  // np values below 2^59.1 each sum below 2^62.1
  S += G;
  P.c_scale[c] = S;
  P.desc[2 * i + 1].z = S;
  int q = 0;
  const int64_t e0 = P.cbeg[c];
  for (int kc = 0; kc < P.Dk; ++kc) {
    const int len = P.run_len[(int64_t)c * P.Dk + kc], es = P.run_start[(int64_t)c * P.Dk + kc];
    for (int e = es; e < es + len; ++e, ++q) {
      const int d = S - (P.a_exp[P.s_ab[e]] + P.b_exp[P.s_bb[e]]);
      P.pairs[P.pair_pos[e0 + q]].z = min(63, max(0, d));
    }
  }
}

struct RedArgs {
  int64_t nred;
  const int4 *desc;  // per reduced C block: {slot base, C offset}, {m n, products, scale, C_in}
  const int32_t *red, *crow, *ccol, *rsz, *csz, *c_cin;
  const int64_t *cbeg, *slot_base, *c_off, *cin_off;
  const int32_t *c_scale;
  const long long *slots;
  const double *Cin;
  double *C;
  double alpha, beta;
  int alpha_one, has_beta;
};

// C blocks with several products or a C_in block: their slots added in product order
// (exact integer sums), converted once, alpha and beta C_in applied.  One warp per C
// block, each lane summing two elements' slots at a time with the loads issued before
// the adds.
__global__ void k_pan_reduce(RedArgs P) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= P.nred) return;
  const int4 d0 = P.desc[2 * i], d1 = P.desc[2 * i + 1];
  const int mn = d1.x, np = d1.y, sc = d1.z - 54, cin = d1.w;
  const long long *sl =
      P.slots + (long long)(((unsigned long long)(unsigned)d0.y << 32) | (unsigned)d0.x);
  const double *ci = (P.has_beta && cin >= 0) ? P.Cin + P.cin_off[cin] : nullptr;
  double *out = P.C + (long long)(((unsigned long long)(unsigned)d0.w << 32) | (unsigned)d0.z);
  // two elements per lane and iteration (e, e + 32); the common product counts spelled
  // out so that all loads of both are in flight before the adds
  auto sum_at = [&](int e) -> long long {
    long long acc = 0;
    int q = 0;
    for (; q + 4 <= np; q += 4) {
      const long long x0 = __ldcs(sl + (int64_t)q * mn + e), x1 = __ldcs(sl + (int64_t)(q + 1) * mn + e);
      const long long x2 = __ldcs(sl + (int64_t)(q + 2) * mn + e), x3 = __ldcs(sl + (int64_t)(q + 3) * mn + e);
      acc += (x0 + x1) + (x2 + x3);
    }
    for (; q < np; ++q) acc += __ldcs(sl + (int64_t)q * mn + e);
    return acc;
  };
  auto finish = [&](long long acc, int e) {
    double v = np > 0 ? i64_scaled_int(acc, sc) : 0.0;
    if (!P.alpha_one) v *= P.alpha;
    if (ci) v = fma(P.beta, ci[e], v);
    out[e] = v;
  };
  for (int e = lane; e < mn; e += 64) {
    const bool v1 = e + 32 < mn;
    const int e1 = v1 ? e + 32 : e;  // a valid index for the second element's loads
    long long a0 = 0, a1 = 0;
    if (np == 1) {
      a0 = __ldcs(sl + e);
      a1 = __ldcs(sl + e1);
    } else if (np == 2) {
      const long long x0 = __ldcs(sl + e), x1 = __ldcs(sl + mn + e);
      const long long y0 = __ldcs(sl + e1), y1 = __ldcs(sl + mn + e1);
      a0 = x0 + x1;
      a1 = y0 + y1;
    } else if (np == 3) {
      const long long x0 = __ldcs(sl + e), x1 = __ldcs(sl + mn + e), x2 = __ldcs(sl + 2 * mn + e);
      const long long y0 = __ldcs(sl + e1), y1 = __ldcs(sl + mn + e1), y2 = __ldcs(sl + 2 * mn + e1);
      a0 = x0 + x1 + x2;
      a1 = y0 + y1 + y2;
    } else if (np > 0) {
      a0 = sum_at(e);
      if (v1) a1 = sum_at(e1);
    }
    finish(a0, e);
    if (v1) finish(a1, e1);
  }
}

// ---- the tcgen05 panel kernel -----------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of the phase; the thread may sleep up to 0.2 ms inside it while the phase is
// incomplete (a suspend-time hint), so waiting threads do not spin on issue slots that
// the MMA-issuing and loading threads need.
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(200000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of the phase of `bar` with parity `parity`, for at most
// kWaitNs; gives up early once another role has recorded an error.  Returns false
// (and records kErrWait) when it gives up.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                       bool drain = false,
                                       unsigned long long bound = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    {
      // a drain (copies or MMAs in flight) waits out its bound even after an error
      if (!drain && *reinterpret_cast<volatile int *>(err) != 0) return false;
      if (gtimer() - t0 > bound) {
        atomicCAS(err, 0, kErrWait);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// A wait that cannot complete (an mbarrier nothing arrives at), bounded by bound_ns: lets
// a test check on the GPU that a wait which runs out is reported the way every bounded
// wait of the panel kernel reports it, and that the context stays usable afterwards.
__global__ void k_pan_wait_probe(int *err, unsigned long long bound_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0, err, false, bound_ns);
  }
}

// shared-memory matrix descriptor, K-major and swizzled: rows of 32 B (one K-step of 16
// BF16 values, 32-byte swizzle) or 64 B (two K-steps, 64-byte swizzle), 8-row atoms of
// 256 or 512 B one after another (stride byte offset), leading byte offset unused (1).
// An unswizzled layout with 256-byte row-group strides put the 16-byte chunks that the
// tensor core reads together into the same shared-memory banks.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t nq) {
  const uint64_t sbo = nq == 1 ? 256 : 512;
  const uint64_t layout = nq == 1 ? 6 : 4;  // SWIZZLE_32B : SWIZZLE_64B
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((sbo >> 4) << 32) | (1ull << 46) |
         (layout << 61);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N = 32, M = 128
constexpr uint32_t kIDesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(kIDesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// named barrier of the epilogue group of accumulator buffer b (its eight warps)
__device__ __forceinline__ void epi_bar(int b) {
  asm volatile("bar.sync %0, 256;" ::"r"(1 + b) : "memory");
}

// barrier of the epilogue group of buffer b that also ANDs a predicate over its 256
// threads, so that they all take the same branch after a wait
__device__ __forceinline__ bool epi_bar_and(int b, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + b)
      : "memory");
  return r != 0;
}

// the 21 slice pairs (s, tt) of levels s + tt <= 5, in level-major order per s
template <int NQ>
__device__ __forceinline__ void issue_tile(uint32_t d0, uint64_t da, uint64_t db) {
  // slice s starts NQ * 4 KB (A) / NQ * 1 KB (B) further; K-step kq 32 bytes further
  // along the rows.  The first product into level w, pair (0, w) K-step 0, overwrites it.
#pragma unroll
  for (int s = 0; s < kDig; ++s)
#pragma unroll
    for (int tt = 0; s + tt < kDig; ++tt)
#pragma unroll
      for (int kq = 0; kq < NQ; ++kq)
        umma(d0 + (uint32_t)((s + tt) * kTN), da + (uint64_t)(s * NQ * (kAStep >> 4) + kq * 2),
             db + (uint64_t)(tt * NQ * (kBStep >> 4) + kq * 2), (s == 0 && kq == 0) ? 0u : 1u);
}

__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "elect.sync _|p, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(pred));
  return pred != 0;
}

// One plan's panel schedule and this execute's output.
struct PanPlan {
  const PUnit *units;
  const PNTile *ntiles;
  const char *a_img, *b_img;
  const int4 *urec;   // per unit: kURec int4 {row offset, m, exponent, stored block}
  const int4 *ntrec;  // per N-tile: kNTRec int4 (header, column table, B blocks)
  const int4 *pairs;  // per (unit, N-tile) pair: {dst lo, dst hi, shift, -1}
  double *C;
  long long *slots;
  double alpha;
  int alpha_one, pad;
};

struct PanArgs {
  PanPlan one;           // the plan of a single execute
  const PanPlan *plans;  // a batch: its plans (null: `one`)
  const int2 *ulist;     // a batch: (plan, unit) in decreasing cost (null: units of `one`)
  int64_t nunits;
  int *err;
};

// unit u of the launch: its plan and its index in that plan's schedule
__device__ __forceinline__ const PanPlan &unit_plan(const PanArgs &P, int64_t u, int &lu) {
  if (!P.ulist) {
    lu = (int)u;
    return P.one;
  }
  const int2 w = P.ulist[u];
  lu = w.y;
  return P.plans[w.x];
}

// the units of this CTA: snake order over the cost-sorted list
__device__ __forceinline__ int64_t unit_at(int64_t r, int G, int b) {
  return r * G + ((r & 1) ? (G - 1 - b) : b);
}

struct PanBars {
  uint64_t full_a[2], empty_a[2], full_b[kStages], empty_b[kStages], full_acc[2], empty_acc[2];
  uint64_t full_u[2], empty_u[2], full_r[kRecStages], empty_r[kRecStages];
  uint64_t done;
  uint32_t tmem;
  int skip;
};

constexpr size_t kRecBytes = 16 * (size_t)(kNTRec + kMaxAB * kMaxBB);
constexpr size_t kSmemBytes = 1024 + 2 * (size_t)kABuf + (size_t)kStages * kBBuf +
                              2 * (size_t)kTM * kStgLd * 8 + (size_t)kRecStages * kRecBytes +
                              2 * 16 * (size_t)kURec + sizeof(PanBars);

// Warps 0-7 and 8-15: the epilogue groups of accumulator buffers 0 and 1 (tiles t with
// t % 2 = b); in each, warps 0-3 fold tile columns 0-15 and warps 4-7 columns 16-31 (a
// warp reads the TMEM lanes 32 (warp % 4) .. + 31), then all eight write the tile's
// products.  Warp 16: loader; warp 17: TMEM allocation and MMA issue.
__global__ void __launch_bounds__(576, 1) k_pan_mma(PanArgs P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = sA + 2 * kABuf;
  unsigned long long *stg0 = reinterpret_cast<unsigned long long *>(sB + kStages * kBBuf);
  int4 *srec = reinterpret_cast<int4 *>(stg0 + 2 * kTM * kStgLd);
  int4 *surec = srec + kRecStages * (kRecBytes / 16);
  PanBars &S = *reinterpret_cast<PanBars *>(surec + 2 * kURec);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, cta = blockIdx.x;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.full_a[i], 1);
      mbar_init(&S.empty_a[i], 1);
      mbar_init(&S.full_acc[i], 1);
      mbar_init(&S.empty_acc[i], 256);
      mbar_init(&S.full_u[i], 1);
      mbar_init(&S.empty_u[i], 2);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&S.full_b[i], 1);
      mbar_init(&S.empty_b[i], 1);
    }
    for (int i = 0; i < kRecStages; ++i) {
      mbar_init(&S.full_r[i], 1);
      mbar_init(&S.empty_r[i], 1);
    }
    mbar_init(&S.done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // an error recorded by an earlier launch and not yet reported: do nothing
    S.skip = *reinterpret_cast<volatile int *>(P.err) != 0;
  }
  if (warp == 17) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&S.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tmem;

  if (S.skip) {
    // nothing issued, nothing to drain
  } else if (warp == 16) {
    // ---- loader: one thread issues every bulk copy
    if (lane == 0) {
      int64_t t = 0, q = 0;
      bool ok = true;
      for (int64_t r = 0; ok; ++r) {
        const int64_t u = unit_at(r, G, cta);
        if (u >= P.nunits) break;
        int lu;
        const PanPlan &Q = unit_plan(P, u, lu);
        const PUnit U = Q.units[lu];
        const int ab = (int)(q & 1);
        if (q >= 2) {
          if (!(ok = mbar_wait(&S.empty_u[ab], (uint32_t)(((q >> 1) - 1) & 1), P.err))) break;
          if (!(ok = mbar_wait(&S.empty_a[ab], (uint32_t)(((q >> 1) - 1) & 1), P.err))) break;
        }
        mbar_expect_tx(&S.full_u[ab], 16 * kURec);
        bulk_g2s(surec + ab * kURec, Q.urec + (int64_t)lu * kURec, 16 * kURec, &S.full_u[ab]);
        const uint32_t abytes = (uint32_t)(kDig * U.nq * kAStep);
        mbar_expect_tx(&S.full_a[ab], abytes);
        bulk_g2s(sA + ab * kABuf, Q.a_img + U.a_img, abytes, &S.full_a[ab]);
        ++q;
        long long pb = U.pb;
        PNTile Vn = Q.ntiles[U.v0];  // descriptors loaded one N-tile ahead
        for (int nt = 0; nt < U.nN; ++nt) {
          const PNTile V = Vn;
          if (nt + 1 < U.nN) Vn = Q.ntiles[U.v0 + nt + 1];
          const int st = (int)(t % kStages), rs = (int)(t % kRecStages);
          if (t >= kStages &&
              !(ok = mbar_wait(&S.empty_b[st], (uint32_t)(((t / kStages) - 1) & 1), P.err)))
            break;
          const uint32_t bbytes = (uint32_t)(kDig * V.nq * kBStep);
          mbar_expect_tx(&S.full_b[st], bbytes);
          bulk_g2s(sB + st * kBBuf, Q.b_img + V.b_img, bbytes, &S.full_b[st]);
          if (t >= kRecStages &&
              !(ok = mbar_wait(&S.empty_r[rs], (uint32_t)(((t / kRecStages) - 1) & 1), P.err)))
            break;
          const int np = U.nab * V.nbb;
          int4 *rec = srec + rs * (kRecBytes / 16);
          mbar_expect_tx(&S.full_r[rs], (uint32_t)(16 * (kNTRec + np)));
          bulk_g2s(rec, Q.ntrec + (int64_t)(U.v0 + nt) * kNTRec, 16 * kNTRec, &S.full_r[rs]);
          bulk_g2s(rec + kNTRec, Q.pairs + pb, (uint32_t)(16 * np), &S.full_r[rs]);
          pb += np;
          ++t;
        }
      }
      // copies still in flight (after an error) complete before the CTA ends: wait for
      // the last copy issued into every buffer (returns at once when it was consumed)
      for (int st = 0; st < kStages; ++st) {
        const int64_t n = t > st ? (t - 1 - st) / kStages + 1 : 0;
        if (n > 0) mbar_wait(&S.full_b[st], (uint32_t)((n - 1) & 1), P.err, true);
      }
      for (int rs = 0; rs < kRecStages; ++rs) {
        const int64_t n = t > rs ? (t - 1 - rs) / kRecStages + 1 : 0;
        if (n > 0) mbar_wait(&S.full_r[rs], (uint32_t)((n - 1) & 1), P.err, true);
      }
      for (int ab = 0; ab < 2; ++ab) {
        const int64_t n = q > ab ? (q - 1 - ab) / 2 + 1 : 0;
        if (n > 0) {
          mbar_wait(&S.full_a[ab], (uint32_t)((n - 1) & 1), P.err, true);
          mbar_wait(&S.full_u[ab], (uint32_t)((n - 1) & 1), P.err, true);
        }
      }
    }
    __syncwarp();
  } else if (warp == 17) {
    // ---- MMA issuer: the warp runs the loop converged, one elected lane issues every
    // tcgen05.mma and commit (lane 0 waits on the barriers for the warp)
    int64_t t = 0, q = 0;
    bool ok = true;
    for (int64_t r = 0; ok; ++r) {
      const int64_t u = unit_at(r, G, cta);
      if (u >= P.nunits) break;
      int lu;
      const PUnit U = unit_plan(P, u, lu).units[lu];
      const int ab = (int)(q & 1);
      ok = __shfl_sync(0xffffffffu, lane != 0 || mbar_wait(&S.full_a[ab], (uint32_t)((q >> 1) & 1), P.err), 0);
      if (!ok) break;
      const uint32_t a0 = smem_u32(sA + ab * kABuf);
      for (int nt = 0; nt < U.nN; ++nt, ++t) {
        const int st = (int)(t % kStages), acc = (int)(t & 1);
        ok = __shfl_sync(0xffffffffu,
                         lane != 0 || (mbar_wait(&S.full_b[st], (uint32_t)((t / kStages) & 1), P.err) &&
                                       (t < 2 || mbar_wait(&S.empty_acc[acc], (uint32_t)(((t >> 1) - 1) & 1), P.err))),
                         0);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d0 = tbase + (uint32_t)(acc * kAccCols);
        const uint32_t nq = (uint32_t)U.nq;
        const uint64_t da = sdesc(a0, nq), db = sdesc(smem_u32(sB + st * kBBuf), nq);
        if (elect_one()) {
          if (nq == 1)
            issue_tile<1>(d0, da, db);
          else
            issue_tile<2>(d0, da, db);
          umma_commit(&S.empty_b[st]);
          umma_commit(&S.full_acc[acc]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (elect_one()) umma_commit(&S.empty_a[ab]);
      __syncwarp();
      ++q;
    }
    // every MMA issued has completed before TMEM is freed
    if (elect_one()) umma_commit(&S.done);
    __syncwarp();
    if (lane == 0) mbar_wait(&S.done, 0, P.err, true);
    __syncwarp();
  } else {
    // ---- epilogue group g (accumulator buffer g): thread tr reads TMEM lane tr, half
    // hf of the tile's columns
    const int g = warp >> 3, hf = (warp >> 2) & 1, wg = warp & 7, tr = threadIdx.x & 127;
    const int gt = threadIdx.x & 255;  // thread index within the group
    unsigned long long *stg = stg0 + g * kTM * kStgLd;
    int64_t t = 0, q = 0;
    bool ok = true;
    for (int64_t r = 0; ok; ++r) {
      const int64_t u = unit_at(r, G, cta);
      if (u >= P.nunits) break;
      int lu;
      const PanPlan &Q = unit_plan(P, u, lu);
      const int nN = Q.units[lu].nN, nab = Q.units[lu].nab;
      double *const QC = Q.C;
      long long *const Qslots = Q.slots;
      const double Qalpha = Q.alpha;
      const int Qalpha_one = Q.alpha_one;
      const int us = (int)(q & 1);
      if (!(ok = epi_bar_and(g, gt != 0 || mbar_wait(&S.full_u[us], (uint32_t)((q >> 1) & 1), P.err))))
        break;
      const int4 *ur = surec + us * kURec;
      for (int nt = 0; nt < nN; ++nt, ++t) {
        if ((int)(t & 1) != g) continue;
        const int rs = (int)(t % kRecStages);
        // one thread of the group waits (the rest sleep at the barrier); the copies and
        // MMAs it observed complete are visible to the group after the barrier
        if (!(ok = epi_bar_and(g, gt != 0 || (mbar_wait(&S.full_r[rs], (uint32_t)((t / kRecStages) & 1), P.err) &&
                                              mbar_wait(&S.full_acc[g], (uint32_t)((t >> 1) & 1), P.err)))))
          break;
        tc_fence_after();
        const int4 *rec = srec + rs * (kRecBytes / 16);
        const int nbb = rec[0].x;
        const int4 *bb = rec + 9;
        const int4 *pr = rec + kNTRec;
        const uint32_t ta = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * kAccCols);
        // fold phase: the 16 slots of the thread's tile row in its half, no branches
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int c0 = hf * 16 + h * 8;
          uint32_t lv[kDig][8];
#pragma unroll
          for (int w = 0; w < kDig; ++w) tmem_ld8(ta + (uint32_t)(w * kTN + c0), lv[w]);
          tmem_wait_ld();
          if (h == 1) {
            tc_fence_before();
            mbar_arrive(&S.empty_acc[g]);
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            // level sums as integers: x + 1.5 * 2^23 keeps them in [2^23, 2^24)
            int D[kDig];
#pragma unroll
            for (int w = 0; w < kDig; ++w)
              D[w] = __float_as_int(__uint_as_float(lv[w][c]) + 12582912.0f) - 0x4B400000;
            const int hi = D[0] * 256 + D[1];
            const long long lo = (long long)D[5] + (long long)D[4] * 256ll +
                                 (long long)D[3] * 65536ll + (long long)D[2] * 16777216ll;
            stg[tr * kStgLd + c0 + c] =
                (unsigned long long)(lo + (long long)((unsigned long long)(unsigned)hi << 32));
          }
        }
        const int np = nab * nbb, inv = rec[0].y;  // ib = x / nbb = (x * inv) >> 16, x < 256
        epi_bar(g);
        // copy-out phase: the eight warps of the group take the tile's products in turn
        // (round robin measured faster than giving each warp an equal share of elements
        // in consecutive products); every (A block, B block) product is m x n contiguous
        // values, written coalesced
        for (int x = wg; x < np; x += 8) {
          {
            const int ib = (x * inv) >> 16, jb = x - ib * nbb;
            const int4 ar = ur[ib];  // {row offset, m, exponent}
            const int4 pe = pr[x];
            const long long dst =
                (long long)(((unsigned long long)(unsigned)pe.y << 32) | (unsigned)pe.x);
            if (dst == -1) continue;
            const int4 bq = bb[jb];  // {col offset, n, exponent, ceil(2^20 / n)}
            const int mn = ar.y * bq.y;
            const unsigned long long *src = stg + ar.x * kStgLd + bq.x;
            // element e of the product: row p = e / n, column qq = e - p n of the block;
            // four elements per iteration (e, e + 32, e + 64, e + 96) as independent chains
            const unsigned n = (unsigned)bq.y, mg = (unsigned)bq.w;
            auto at = [&](int e) -> long long {
              const int p = (int)(((unsigned)e * mg) >> 20);
              return (long long)src[p * kStgLd + (e - p * (int)n)];
            };
            if (dst >= 0) {
              // the C block's only product: converted and written
              const int e2 = ar.z + bq.z - 54;
              double *o = QC + dst;
              if (Qalpha_one) {
                for (int e = lane; e < mn; e += 128) {
                  const bool v1 = e + 32 < mn, v2 = e + 64 < mn, v3 = e + 96 < mn;
                  const long long x0 = at(e), x1 = v1 ? at(e + 32) : 0, x2 = v2 ? at(e + 64) : 0,
                                  x3 = v3 ? at(e + 96) : 0;
                  o[e] = i64_scaled(x0, e2);
                  if (v1) o[e + 32] = i64_scaled(x1, e2);
                  if (v2) o[e + 64] = i64_scaled(x2, e2);
                  if (v3) o[e + 96] = i64_scaled(x3, e2);
                }
              } else {
                for (int e = lane; e < mn; e += 32) o[e] = Qalpha * i64_scaled(at(e), e2);
              }
            } else {
              // one of several products (or a block with C_in): its slot, at the C
              // block's common scale; the reduction kernel adds a block's slots
              long long *sl = Qslots + (-(dst + 2));
              const int sh = pe.z;
              for (int e = lane; e < mn; e += 128) {
                const bool v1 = e + 32 < mn, v2 = e + 64 < mn, v3 = e + 96 < mn;
                const long long x0 = at(e), x1 = v1 ? at(e + 32) : 0, x2 = v2 ? at(e + 64) : 0,
                                x3 = v3 ? at(e + 96) : 0;
                sl[e] = round_shift(x0, sh);
                if (v1) sl[e + 32] = round_shift(x1, sh);
                if (v2) sl[e + 64] = round_shift(x2, sh);
                if (v3) sl[e + 96] = round_shift(x3, sh);
              }
            }
          }
        }
        epi_bar(g);
        if (gt == 0) mbar_arrive(&S.empty_r[rs]);
      }
      if (!ok) break;
      if (gt == 0) mbar_arrive(&S.empty_u[us]);
      ++q;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 17) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

SideP side_p(const bst_matrix *X, bool trans, bool is_b, const double *data) {
  SideP S{};
  S.nblocks = X->nblocks;
  S.row = X->row;
  S.col = X->col;
  S.rsz = X->rsz;
  S.csz = X->csz;
  S.off = X->off;
  S.data = data;
  S.trans = trans;
  S.is_b = is_b;
  return S;
}

// host copy of an op view: per CSR entry, its block column and stored block
struct HostView {
  std::vector<int32_t> rowptr, col, blk;
};

HostView host_view(const bst_plan *p, const OpView &v, int64_t nnz, cudaStream_t s) {
  HostView h;
  h.rowptr.resize((size_t)v.nr + 1);
  h.col.resize((size_t)nnz);
  h.blk.resize((size_t)nnz);
  ReadBack rb(p->ctx, s);
  rb.add(h.rowptr.data(), v.rowptr, 4 * h.rowptr.size());
  rb.add(h.col.data(), v.col, 4 * h.col.size());
  if (v.blk)
    rb.add(h.blk.data(), v.blk, 4 * h.blk.size());
  else
    std::iota(h.blk.begin(), h.blk.end(), 0);
  rb.done();
  return h;
}

}  // namespace

// Build the panel schedule of a plan (once).  Sets eligible = false when the plan does
// not suit it: blocks larger than a tile (m > 128, n > 32) or inner blocks above 32
// elements.  Thin panels are taken too: on the 64 problems of the batched workload run
// one by one, the plans whose panels fill under 15 % of their tiles' multiply-adds
// took 2.20 ms on this kernel against 2.41 ms on the C-block kernel, in all.
static void panel_build(bst_plan *p, PanelState &PS, cudaStream_t s) {
  PS.built = true;
  PS.eligible = false;
  const int64_t nc = p->C->nblocks;
  if (nc == 0 || p->T == 0) return;
  for (int v : p->m_vals)
    if (v > kTM) return;
  for (int v : p->n_vals)
    if (v > kTN) return;
  for (int v : p->k_vals)
    if (v > 32) return;
  const int64_t na = p->A->nblocks, nbk = p->B->nblocks;
  const HostView va = host_view(p, p->oa, na, s), vb = host_view(p, p->ob, nbk, s);
  const std::vector<int32_t> &ars = p->oa.h_rs, &acs = p->oa.h_cs, &bcs = p->ob.h_cs;
  const int32_t K = p->oa.nc;
  // A panels: op(A) blocks grouped by block column k, in block-row order
  std::vector<int64_t> kcnt((size_t)K + 1, 0);
  for (int64_t e = 0; e < na; ++e) kcnt[(size_t)va.col[e] + 1]++;
  for (int32_t k = 0; k < K; ++k) kcnt[k + 1] += kcnt[k];
  std::vector<int32_t> apan((size_t)na), arowi((size_t)na);
  {
    std::vector<int64_t> fillp(kcnt.begin(), kcnt.end() - 1);
    for (int32_t i = 0; i < p->oa.nr; ++i)
      for (int32_t e = va.rowptr[i]; e < va.rowptr[i + 1]; ++e) {
        const int64_t pos = fillp[va.col[e]]++;
        apan[pos] = va.blk[e];
        arowi[pos] = i;
      }
  }
  // Bins of a panel: first-fit decreasing of the blocks (sizes sz[x], x < n) into bins
  // of capacity cap holding at most maxn blocks; returns the bin of each block (blocks
  // of one bin keep their panel order).  Fewer, fuller tiles than cutting the panel in
  // order: the 5/13/23-element blocks of the 4000 x 4000 banded product fill 88 % of
  // the 32-column N-tiles this way against 76 % (67 134 N-tiles against 78 098).
  auto ffd = [](const std::vector<int> &sz, int cap, int maxn, std::vector<int> &bin) {
    const int n = (int)sz.size();
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return sz[x] > sz[y]; });
    std::vector<int> used, cnt;
    bin.assign(n, -1);
    for (int x : ord) {
      int b = 0;
      while (b < (int)used.size() && (used[b] + sz[x] > cap || cnt[b] >= maxn)) ++b;
      if (b == (int)used.size()) {
        used.push_back(0);
        cnt.push_back(0);
      }
      used[b] += sz[x];
      cnt[b] += 1;
      bin[x] = b;
    }
    return (int)used.size();
  };
  // B panels (op(B) block rows) packed into N-tiles
  std::vector<PNTile> nt;
  std::vector<int4> blist;
  std::vector<int2> bwhere((size_t)nbk, make_int2(-1, -1));
  std::vector<int32_t> kv0((size_t)K, 0), knN((size_t)K, 0);
  int64_t bimg = 0;
  std::vector<int> sz, bin;
  for (int32_t k = 0; k < K; ++k) {
    kv0[k] = (int32_t)nt.size();
    const int nq = (acs[k] + 15) / 16;
    if (kcnt[k + 1] == kcnt[k]) continue;  // no op(A) block in this panel
    const int32_t e0 = vb.rowptr[k], ne = vb.rowptr[k + 1] - e0;
    if (ne == 0) continue;
    sz.resize(ne);
    for (int x = 0; x < ne; ++x) sz[x] = bcs[vb.col[e0 + x]];
    const int nbins = ffd(sz, kTN, kMaxBB, bin);
    int cum = 0;
    for (int b = 0; b < nbins; ++b) {
      PNTile V{};
      V.b_img = bimg;
      V.bb0 = (int)blist.size();
      V.cum = cum;
      V.nq = nq;
      int used = 0;
      for (int x = 0; x < ne; ++x) {
        if (bin[x] != b) continue;
        const int32_t e = e0 + x;
        bwhere[(size_t)vb.blk[e]] = make_int2((int)nt.size(), V.nbb);
        blist.push_back(make_int4(vb.blk[e], used, sz[x], 0));
        used += sz[x];
        ++V.nbb;
      }
      cum += V.nbb;
      bimg += (int64_t)kDig * nq * kBStep;
      nt.push_back(V);
    }
    knN[k] = (int32_t)nt.size() - kv0[k];
  }
  // A tiles: units (k, tile) of panels with op(B) blocks, packed the same way
  struct HU {
    PUnit U;
    double cost;
    std::vector<int32_t> blocks;
  };
  std::vector<HU> hu;
  double tiles_mac = 0.0;
  for (int32_t k = 0; k < K; ++k) {
    if (knN[k] == 0) continue;
    const int nq = (acs[k] + 15) / 16;
    const int64_t e0 = kcnt[k];
    const int ne = (int)(kcnt[k + 1] - e0);
    sz.resize(ne);
    for (int x = 0; x < ne; ++x) sz[x] = ars[arowi[e0 + x]];
    const int nbins = ffd(sz, kTM, kMaxAB, bin);
    for (int b = 0; b < nbins; ++b) {
      HU h{};
      h.U.v0 = kv0[k];
      h.U.nN = knN[k];
      h.U.nq = nq;
      for (int x = 0; x < ne; ++x)
        if (bin[x] == b) h.blocks.push_back((int32_t)(e0 + x));
      h.U.nab = (int)h.blocks.size();
      h.cost = (double)h.U.nN * (2.0 + nq);
      tiles_mac += (double)h.U.nN * kTM * kTN * 16 * nq;
      hu.push_back(std::move(h));
    }
  }
  if (hu.empty()) return;
  PS.fill = p->stats.flops / (2.0 * tiles_mac);
  std::stable_sort(hu.begin(), hu.end(), [](const HU &x, const HU &y) { return x.cost > y.cost; });
  std::vector<PUnit> units(hu.size());
  std::vector<int4> alist;
  std::vector<int2> awhere((size_t)na, make_int2(-1, -1));
  int64_t aimg = 0, pb = 0;
  for (size_t u = 0; u < hu.size(); ++u) {
    PUnit U = hu[u].U;
    U.a_img = aimg;
    U.ab0 = (int)alist.size();
    U.pb = pb;
    int ro = 0;
    for (int x = 0; x < U.nab; ++x) {
      const int64_t e = hu[u].blocks[(size_t)x];
      const int m = ars[arowi[e]];
      awhere[(size_t)apan[e]] = make_int2((int)u, x);
      alist.push_back(make_int4(apan[e], ro, m, 0));
      ro += m;
    }
    int64_t nbb = 0;
    for (int v = U.v0; v < U.v0 + U.nN; ++v) nbb += nt[(size_t)v].nbb;
    pb += (int64_t)U.nab * nbb;
    aimg += (int64_t)kDig * U.nq * kAStep;
    units[u] = U;
  }
  BST_REQUIRE(pb < INT32_MAX, BST_ERR_UNSUPPORTED, "panel schedule above 2^31 pairs");
  PS.nunits = (int64_t)units.size();
  PS.nntiles = (int64_t)nt.size();
  PS.npairs = pb;
  PS.a_img_bytes = aimg;
  PS.b_img_bytes = bimg;
  double tf = 0.0;
  for (const PUnit &U : units) tf += (double)U.nN * U.nq * 21.0 * 2.0 * kTM * kTN * 16;
  PS.tensor_flops = tf;
  // epilogue records: per unit its A blocks {row offset, m, exponent, stored block}, per
  // N-tile {nbb}, the column table ((B block << 8) | column in it, or -256) and its B
  // blocks {column offset, n, exponent, ceil(2^20 / n)} (the last for the division-free
  // row of an element: e / n = (e * ceil(2^20 / n)) >> 20 for e < 4096, n <= 32, checked
  // exhaustively); exponents are filled per execute
  std::vector<int4> urec(units.size() * kURec, make_int4(0, 0, 0, 0));
  for (size_t u = 0; u < units.size(); ++u)
    for (int x = 0; x < units[u].nab; ++x) {
      const int4 e = alist[(size_t)units[u].ab0 + x];
      urec[u * kURec + x] = make_int4(e.y, e.z, 0, e.x);
    }
  std::vector<int4> ntrec(nt.size() * kNTRec, make_int4(0, 0, 0, 0));
  for (size_t v = 0; v < nt.size(); ++v) {
    int4 *r = &ntrec[v * kNTRec];
    r[0] = make_int4(nt[v].nbb, ((1 << 16) + nt[v].nbb - 1) / nt[v].nbb, 0, 0);
    int *col = reinterpret_cast<int *>(r + 1);
    for (int c = 0; c < kTN; ++c) col[c] = -256;
    for (int j = 0; j < nt[v].nbb; ++j) {
      const int4 e = blist[(size_t)nt[v].bb0 + j];
      r[9 + j] = make_int4(e.y, e.z, 0, ((1 << 20) + e.z - 1) / e.z);  // ceil(2^20 / n)
      for (int q = 0; q < e.z; ++q) col[e.y + q] = (j << 8) | q;
    }
  }
  Arena &ar = PS.ar;
  {
    Upload up(p->ctx, s);
    PS.units = up.add_vector(ar, units);
    PS.ntiles = up.add_vector(ar, nt);
    PS.alist = up.add_vector(ar, alist);
    PS.blist = up.add_vector(ar, blist);
    PS.a_where = up.add_vector(ar, awhere);
    PS.b_where = up.add_vector(ar, bwhere);
    PS.urec = up.add_vector(ar, urec);
    PS.ntrec = up.add_vector(ar, ntrec);
    up.done();
  }
  PS.a_img = static_cast<char *>(ar.alloc((size_t)std::max<int64_t>(aimg, 16)));
  PS.b_img = static_cast<char *>(ar.alloc((size_t)std::max<int64_t>(bimg, 16)));
  // padding rows and inner positions never written by a block stay zero
  BST_CUDA(cudaMemsetAsync(PS.a_img, 0, (size_t)aimg, s));
  BST_CUDA(cudaMemsetAsync(PS.b_img, 0, (size_t)bimg, s));
  PS.pairs = ar.alloc_n<int4>((size_t)std::max<int64_t>(pb, 1));
  BST_CUDA(cudaMemsetAsync(PS.pairs, 0xff, 16 * (size_t)pb, s));  // dst -1: filtered
  // C blocks: products per block, the reduced ones, their slots
  Arena scratch;
  scratch.ctx = static_cast<Ctx *>(p->ctx);
  scratch.stream = s;
  int32_t *cnt = scratch.alloc_n<int32_t>((size_t)nc);
  int32_t *flag = scratch.alloc_n<int32_t>((size_t)nc);
  int64_t *ssz = scratch.alloc_n<int64_t>((size_t)nc);
  int32_t *rpos = ar.alloc_n<int32_t>((size_t)nc + 1);
  PS.cbeg = ar.alloc_n<int64_t>((size_t)nc + 1);
  PS.slot_base = ar.alloc_n<int64_t>((size_t)nc + 1);
  PS.pair_pos = ar.alloc_n<int32_t>((size_t)p->T);
  PS.c_scale = ar.alloc_n<int32_t>((size_t)nc);
  const bst_matrix *C = p->C;
  k_pan_count<<<nblk(nc, 256), 256, 0, s>>>(nc, p->Dk, p->run_len, cnt);
  BST_CHECK_LAUNCH();
  exscan_i32_i64(cnt, PS.cbeg, nc, scratch, s);
  k_pan_red_flags<<<nblk(nc, 256), 256, 0, s>>>(nc, cnt, p->c_cin, C->row, C->col, C->rsz, C->csz,
                                                 flag, ssz);
  BST_CHECK_LAUNCH();
  exscan_i64(ssz, PS.slot_base, nc, scratch, s);
  exscan_i32(flag, rpos, nc, scratch, s);
  int64_t totals[2] = {0, 0};
  int32_t nred = 0;
  {
    ReadBack rb(p->ctx, s);
    rb.add(&totals[0], PS.slot_base + nc, 8);
    rb.add(&nred, rpos + nc, 4);
    rb.done();
  }
  PS.slot_elems = totals[0];
  PS.nred = nred;
  PS.red = ar.alloc_n<int32_t>((size_t)std::max<int32_t>(nred, 1));
  k_pan_compact<<<nblk(nc, 256), 256, 0, s>>>(nc, flag, rpos, PS.red);
  BST_CHECK_LAUNCH();
  PS.red_desc = ar.alloc_n<int4>(2 * (size_t)std::max<int32_t>(nred, 1));
  if (nred > 0) {
    k_pan_red_desc<<<nblk(nred, 256), 256, 0, s>>>(nred, PS.red, cnt, p->c_cin, C->row, C->col,
                                                    C->rsz, C->csz, PS.slot_base, C->off,
                                                    PS.red_desc);
    BST_CHECK_LAUNCH();
  }

  PS.slots = ar.alloc_n<int64_t>((size_t)std::max<int64_t>(PS.slot_elems, 1));
  PairArgs pa{};
  pa.nc = nc;
  pa.Dk = p->Dk;
  pa.run_start = p->run_start;
  pa.run_len = p->run_len;
  pa.s_ab = p->s_ab;
  pa.s_bb = p->s_bb;
  pa.flag = flag;
  pa.crow = C->row;
  pa.ccol = C->col;
  pa.rsz = C->rsz;
  pa.csz = C->csz;
  pa.c_off = C->off;
  pa.cbeg = PS.cbeg;
  pa.slot_base = PS.slot_base;
  pa.units = PS.units;
  pa.ntiles = PS.ntiles;
  pa.a_where = PS.a_where;
  pa.b_where = PS.b_where;
  pa.pairs = PS.pairs;
  pa.pair_pos = PS.pair_pos;
  k_pan_pairs<<<nblk(nc, 256), 256, 0, s>>>(pa);
  BST_CHECK_LAUNCH();
  PS.a_exp = ar.alloc_n<int32_t>((size_t)std::max<int64_t>(na, 1));
  PS.b_exp = ar.alloc_n<int32_t>((size_t)std::max<int64_t>(nbk, 1));
  PS.err = ar.alloc_n<int>(1);
  BST_CUDA(cudaMemsetAsync(PS.err, 0, sizeof(int), s));
  BST_CUDA(cudaStreamSynchronize(s));
  scratch.release_all();
  PS.eligible = true;
}

static PanelState &panel_state(bst_plan *p, cudaStream_t s) {
  if (!p->panel) {
    p->panel = new PanelState();
    p->panel->ar.ctx = static_cast<Ctx *>(p->ctx);
    p->panel->ar.stream = s;
  }
  PanelState &PS = *p->panel;
  if (!PS.built) panel_build(p, PS, s);
  return PS;
}

// By default (BST_TUNE_EMU_PANEL = 1) a plan's first emulated execute runs the C-block
// kernel and the panel schedule is built at its second one: building it costs host work
// and a few synchronisations of the order of the kernel time it saves, so a plan run
// once (a step of a chain of fresh products) never pays for it.
// An execute captured into a CUDA graph never builds the schedule (that synchronises):
// it runs the C-block kernel, whose state the plan's first emulated execute built.
bool panel_usable(bst_plan *p, cudaStream_t s, bool count) {
  const int mode = p->ctx->tune_emu_panel;
  if (!mode || p->C->nblocks == 0) return false;
  if (mode == 1 && !p->panel) {
    const int n = p->emu_executes + 1;  // the execute this call is about
    if (count) p->emu_executes = n;
    if (n < 2) return false;
  }
  if (!p->panel || !p->panel->built) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BST_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return false;
  }
  const PanelState &PS = panel_state(p, s);
  return PS.eligible;
}

void panel_state_free(bst_plan *p) {
  delete p->panel;
  p->panel = nullptr;
}

void panel_costs(bst_plan *p, cudaStream_t s, double *out) {
  PanelState &PS = panel_state(p, s);
  out[0] = PS.tensor_flops;
  // FP64 operands read by the exponent and digit passes, digit images written and read
  // once, C written, the schedule's pair table read
  out[1] = 16.0 * (double)(p->A->nelem + p->B->nelem) +
           2.0 * (double)(PS.a_img_bytes + PS.b_img_bytes) + 8.0 * (double)p->C->nelem +
           16.0 * (double)PS.npairs;
  // int64 partial products of the C blocks with several products (written and read)
  out[2] = 16.0 * (double)PS.slot_elems;
}

int panel_error(bst_plan *p) {
  if (!p->panel || !p->panel->err) return 0;
  int e = 0;
  BST_CUDA(cudaMemcpy(&e, p->panel->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) BST_CUDA(cudaMemset(p->panel->err, 0, sizeof(int)));
  return e;
}

namespace {

PanPlan pan_plan(const PanelState &PS, const NumArgs &a) {
  PanPlan Q{};
  Q.units = PS.units;
  Q.ntiles = PS.ntiles;
  Q.a_img = PS.a_img;
  Q.b_img = PS.b_img;
  Q.urec = PS.urec;
  Q.ntrec = PS.ntrec;
  Q.pairs = PS.pairs;
  Q.C = a.C;
  Q.slots = reinterpret_cast<long long *>(PS.slots);
  Q.alpha = a.alpha;
  Q.alpha_one = a.alpha == 1.0;
  return Q;
}

void launch_pan_mma(const PanArgs &P, int num_sms, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    BST_CUDA(cudaFuncSetAttribute(k_pan_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemBytes));
    attr_set = true;
  }
  if (P.nunits == 0) return;
  const int grid = (int)std::min<int64_t>(num_sms, P.nunits);
  k_pan_mma<<<grid, 576, kSmemBytes, s>>>(P);
  BST_CHECK_LAUNCH();
}

}  // namespace

// slicing of the current operand data, record exponents and slot shifts (launches only)
void panel_prepare(bst_plan *p, const NumArgs &a, cudaStream_t s) {
  PanelState &PS = panel_state(p, s);
  const int wpb = 8;
  for (int side = 0; side < 2; ++side) {
    const bst_matrix *X = side ? p->B : p->A;
    if (X->nblocks == 0) continue;
    SideP S = side_p(X, side ? p->tb : p->ta, side == 1, side ? a.B : a.A);
    S.bexp = side ? PS.b_exp : PS.a_exp;
    S.where = side ? PS.b_where : PS.a_where;
    S.units = PS.units;
    S.ntiles = PS.ntiles;
    S.list = side ? PS.blist : PS.alist;
    S.img = side ? PS.b_img : PS.a_img;
    k_pan_digits<<<nblk(X->nblocks, wpb), 32 * wpb, 0, s>>>(S);
    BST_CHECK_LAUNCH();
  }
  {
    const int64_t n = PS.nunits * kURec + PS.nntiles * kMaxBB;
    k_pan_recexp<<<nblk(n, 256), 256, 0, s>>>(PS.nunits, PS.nntiles, PS.urec, PS.ntrec, PS.ntiles,
                                              PS.blist, PS.a_exp, PS.b_exp);
    BST_CHECK_LAUNCH();
  }
  if (PS.nred > 0) {
    ShiftArgs sh{};
    sh.nred = PS.nred;
    sh.Dk = p->Dk;
    sh.red = PS.red;
    sh.run_start = p->run_start;
    sh.run_len = p->run_len;
    sh.s_ab = p->s_ab;
    sh.s_bb = p->s_bb;
    sh.pair_pos = PS.pair_pos;
    sh.cbeg = PS.cbeg;
    sh.a_exp = PS.a_exp;
    sh.b_exp = PS.b_exp;
    sh.pairs = PS.pairs;
    sh.desc = PS.red_desc;
    sh.c_scale = PS.c_scale;
    k_pan_shift<<<nblk(PS.nred, 256), 256, 0, s>>>(sh);
    BST_CHECK_LAUNCH();
  }
}

// the C blocks summed from slots (launch only)
void panel_finish(bst_plan *p, const NumArgs &a, cudaStream_t s) {
  PanelState &PS = *p->panel;
  if (PS.nred == 0) return;
  RedArgs R{};
  R.nred = PS.nred;
  R.red = PS.red;
  R.desc = PS.red_desc;
  R.crow = p->C->row;
  R.ccol = p->C->col;
  R.rsz = p->C->rsz;
  R.csz = p->C->csz;
  R.c_cin = p->c_cin;
  R.cbeg = PS.cbeg;
  R.slot_base = PS.slot_base;
  R.c_off = p->C->off;
  R.cin_off = p->Cin ? p->Cin->off : nullptr;
  R.c_scale = PS.c_scale;
  R.slots = reinterpret_cast<const long long *>(PS.slots);
  R.Cin = a.Cin;
  R.C = a.C;
  R.alpha = a.alpha;
  R.beta = a.beta;
  R.alpha_one = a.alpha == 1.0;
  R.has_beta = a.beta != 0.0 && a.Cin != nullptr;
  const int wpb = 8;
  k_pan_reduce<<<nblk(PS.nred, wpb), 32 * wpb, 0, s>>>(R);
  BST_CHECK_LAUNCH();
}

void execute_emu_panel(bst_plan *p, const NumArgs &a, cudaStream_t s) {
  PanelState &PS = panel_state(p, s);
  panel_prepare(p, a, s);
  PanArgs P{};
  P.one = pan_plan(PS, a);
  P.plans = nullptr;
  P.ulist = nullptr;
  P.nunits = PS.nunits;
  P.err = PS.err;
  launch_pan_mma(P, p->ctx->num_sms, s);
  panel_finish(p, a, s);
}

// ---- batches -------------------------------------------------------------------

// whether a batch runs this plan's emulated products on the panel kernel (the schedule is
// built now, whatever the plan's execute count: batch executes must not synchronise)
bool panel_batch_eligible(bst_plan *p, cudaStream_t s) {
  const int mode = p->ctx->tune_emu_panel;
  if (!mode || p->C->nblocks == 0) return false;
  const PanelState &PS = panel_state(p, s);
  return PS.eligible;
}

size_t panel_plan_bytes() { return sizeof(PanPlan); }

void panel_fill_plan(bst_plan *p, const NumArgs &a, void *out) {
  const PanPlan Q = pan_plan(*p->panel, a);
  std::memcpy(out, &Q, sizeof(Q));
}

// the (plan, unit) list of a batch: every unit of the given plans, by decreasing cost
int64_t panel_batch_units(const std::vector<bst_plan *> &plans, Arena &ar, int2 **out,
                          cudaStream_t s) {
  std::vector<std::pair<double, int2>> all;
  for (size_t q = 0; q < plans.size(); ++q) {
    const PanelState &PS = *plans[q]->panel;
    std::vector<PUnit> u((size_t)PS.nunits);
    {
      ReadBack rb(plans[q]->ctx, s);
      rb.add(u.data(), PS.units, sizeof(PUnit) * u.size());
      rb.done();
    }
    for (size_t x = 0; x < u.size(); ++x)
      all.push_back({(double)u[x].nN * (2.0 + u[x].nq), make_int2((int)q, (int)x)});
  }
  std::stable_sort(all.begin(), all.end(),
                   [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) {
                     return x.first > y.first;
                   });
  std::vector<int2> list(all.size());
  for (size_t i = 0; i < all.size(); ++i) list[i] = all[i].second;
  if (list.empty()) list.push_back(make_int2(0, 0));
  Upload up(plans.empty() ? nullptr : plans[0]->ctx, s);
  *out = up.add_vector(ar, list);
  up.done();
  return (int64_t)all.size();
}

void launch_panel_batch(const void *d_plans, const int2 *ulist, int64_t n, int *err, int num_sms,
                        cudaStream_t s) {
  PanArgs P{};
  P.plans = static_cast<const PanPlan *>(d_plans);
  P.ulist = ulist;
  P.nunits = n;
  P.err = err;
  launch_pan_mma(P, num_sms, s);
}

int *panel_err_flag(bst_plan *p) { return p->panel ? p->panel->err : nullptr; }

}  // namespace bst

extern "C" bst_status bst_debug_wait_probe(bst_ctx *ctx, int64_t bound_ns, void *stream) {
  API_BEGIN
  BST_REQUIRE(ctx, BST_ERR_INVALID_ARG, "NULL context");
  BST_REQUIRE(bound_ns >= 1000 && bound_ns <= 1000000000, BST_ERR_INVALID_ARG,
              "bound_ns outside [1e3, 1e9]");
  int cur = -1;
  BST_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bst::Arena scratch;
  scratch.ctx = static_cast<bst::Ctx *>(ctx);
  scratch.stream = s;
  int *err = scratch.alloc_n<int>(1);
  BST_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  bst::k_pan_wait_probe<<<1, 32, 0, s>>>(err, (unsigned long long)bound_ns);
  BST_CHECK_LAUNCH();
  int e = 0;
  BST_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  scratch.release_all();
  if (cur != ctx->device) BST_CUDA(cudaSetDevice(cur));
  BST_REQUIRE(e == 0, BST_ERR_TIMEOUT, "a bounded device wait gave up");
  API_END
}
