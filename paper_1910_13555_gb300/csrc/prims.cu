// Device primitives of the symbolic phase: exclusive scans, a stable counting sort
// (partition by a small integer key) and an LSD radix sort built on it.
//
// All of them are deterministic: the counting sort is stable because every warp
// owns one contiguous segment of the input and emits it in order, with the ranks of
// equal keys inside a 32-element batch taken from __match_any_sync.
#include <algorithm>
#include <cstring>

#include "bst_internal.h"

namespace bst {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) >= d) v += o;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the exclusive prefix,
// *total gets the block sum.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
  constexpr int NW = kScanThreads / 32;
  __shared__ T warp_sums[NW];
  __shared__ T tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < NW ? warp_sums[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < NW) warp_sums[lane] = wi - w;
    if (lane == NW - 1) tot = wi;
  }
  __syncthreads();
  T excl = inc - v + warp_sums[wid];
  *total = tot;
  __syncthreads();  // the shared slots are reused by the next call
  return excl;
}

template <class TI, class TO>
__global__ void k_tile_sums(const TI *__restrict__ in, int64_t n, TO *__restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  TO acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
    if (i < n) acc += (TO)in[i];
  }
  TO total;
  block_excl_scan<TO>(acc, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single-CTA exclusive scan of the tile sums (in place), carry across chunks
template <class TO>
__global__ void k_scan_sums(TO *sums, int64_t nt) {
  TO carry = 0;
  for (int64_t c0 = 0; c0 < nt; c0 += kScanThreads) {
    int64_t i = c0 + threadIdx.x;
    TO v = i < nt ? sums[i] : TO(0);
    TO total;
    TO ex = block_excl_scan<TO>(v, &total);
    if (i < nt) sums[i] = ex + carry;
    carry += total;
  }
}

template <class TI, class TO>
__global__ void k_tile_scan(const TI *__restrict__ in, int64_t n, const TO *__restrict__ sums,
                            TO *__restrict__ out) {
  // each thread takes kScanItems consecutive elements
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = base + r;
    v[r] = i < n ? (TO)in[i] : TO(0);
    acc += v[r];
  }
  TO total;
  TO ex = block_excl_scan<TO>(acc, &total) + sums[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = base + r;
    if (i < n) out[i] = ex;
    ex += v[r];
  }
  // the grand total goes to out[n]
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = ex;
}

template <class TI, class TO>
void exscan_impl(const TI *in, TO *out, int64_t n, Arena &ar, cudaStream_t s) {
  if (n == 0) {
    BST_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
    return;
  }
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  TO *sums = ar.alloc_n<TO>((size_t)nt);
  k_tile_sums<TI, TO><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, sums);
  BST_CHECK_LAUNCH();
  k_scan_sums<TO><<<1, kScanThreads, 0, s>>>(sums, nt);
  BST_CHECK_LAUNCH();
  k_tile_scan<TI, TO><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, sums, out);
  BST_CHECK_LAUNCH();
}

// ---- stable counting sort ------------------------------------------------------

__global__ void k_part_hist(const int32_t *__restrict__ keys, int64_t n, int64_t L, int64_t G,
                            int32_t *__restrict__ hist) {
  const int lane = threadIdx.x & 31;
  int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= G) return;
  int64_t p0 = g * L, p1 = min(n, p0 + L);
  for (int64_t b = p0; b < p1; b += 32) {
    int64_t p = b + lane;
    unsigned act = __ballot_sync(0xffffffffu, p < p1);
    if (p < p1) {
      int32_t key = keys[p];
      unsigned peers = __match_any_sync(act, key);
      if ((int)(__ffs(peers) - 1) == lane) atomicAdd(&hist[(int64_t)key * G + g], __popc(peers));
    }
  }
}

__global__ void k_part_keyptr(const int32_t *__restrict__ base, int32_t nkeys, int64_t G,
                              int32_t *__restrict__ key_ptr) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= nkeys) key_ptr[k] = base[k * G];
}

__global__ void k_part_scatter(const int32_t *__restrict__ keys, int64_t n, int64_t L, int64_t G,
                               int32_t *__restrict__ base, int32_t *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= G) return;
  int64_t p0 = g * L, p1 = min(n, p0 + L);
  for (int64_t b = p0; b < p1; b += 32) {
    int64_t p = b + lane;
    unsigned act = __ballot_sync(0xffffffffu, p < p1);
    int32_t key = 0;
    unsigned peers = 0;
    int32_t pos = 0;
    if (p < p1) {
      key = keys[p];
      peers = __match_any_sync(act, key);
      unsigned lt = peers & ((1u << lane) - 1u);
      pos = base[(int64_t)key * G + g] + __popc(lt);
      perm[pos] = (int32_t)p;
    }
    __syncwarp();
    if (p < p1 && (int)(__ffs(peers) - 1) == lane) base[(int64_t)key * G + g] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_iota(int32_t *p, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

__global__ void k_fill(int32_t *p, int32_t v, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_gather(const int32_t *__restrict__ src, const int32_t *__restrict__ idx,
                         int32_t *__restrict__ dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_digits(const uint64_t *__restrict__ keys, const int32_t *__restrict__ perm,
                         int64_t n, int shift, int32_t *__restrict__ dig) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dig[i] = (int32_t)((keys[perm[i]] >> shift) & 0xffu);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void exscan_i32_i64(const int32_t *in, int64_t *out, int64_t n, Arena &ar, cudaStream_t s) {
  exscan_impl<int32_t, int64_t>(in, out, n, ar, s);
}
void exscan_i64(const int64_t *in, int64_t *out, int64_t n, Arena &ar, cudaStream_t s) {
  exscan_impl<int64_t, int64_t>(in, out, n, ar, s);
}
void exscan_i32(const int32_t *in, int32_t *out, int64_t n, Arena &ar, cudaStream_t s) {
  exscan_impl<int32_t, int32_t>(in, out, n, ar, s);
}

void iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_iota<<<nblk(n, 256), 256, 0, s>>>(p, n);
  BST_CHECK_LAUNCH();
}
__global__ void k_copy_bytes(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src,
                             int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// n bytes, both ends 16-byte aligned: 16-byte words, then the tail byte by byte
__global__ void k_copy_aligned(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src,
                               int64_t n) {
  const int64_t nw = n >> 4, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = i0; i < nw; i += stride)
    reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
  for (int64_t i = (nw << 4) + i0; i < n; i += stride) dst[i] = src[i];
}

ReadBack::ReadBack(bst_ctx *c, cudaStream_t st) : ctx(c), s(st) {
  ctx->rb_mutex.lock();
  locked = true;
}

ReadBack::~ReadBack() {
  if (locked) {
    // an exception left copies in flight: let them land before the buffer is reused
    if (!items.empty()) (void)cudaStreamSynchronize(s);
    ctx->rb_mutex.unlock();
  }
}

void ReadBack::done() {
  finish();
  if (locked) {
    locked = false;
    ctx->rb_mutex.unlock();
  }
}

void ReadBack::add(void *host_dst, const void *dev_src, size_t bytes) {
  if (bytes == 0) return;
  const size_t off = (used + 15) & ~(size_t)15;
  if (off + bytes > ctx->rb_cap) {
    // grow (geometrically, never shrinking: freeing pinned memory synchronises the whole
    // device): earlier items of this ReadBack are still pending, so finish them first
    if (!items.empty()) finish();
    const size_t cap = std::max<size_t>({(size_t)1 << 20, 2 * ctx->rb_cap, 2 * (off + bytes)});
    BST_CUDA(cudaStreamSynchronize(s));
    if (ctx->rb_host) BST_CUDA(cudaFreeHost(ctx->rb_host));
    ctx->rb_host = nullptr;
    ctx->rb_cap = 0;
    BST_CUDA(cudaHostAlloc(&ctx->rb_host, cap, cudaHostAllocMapped));
    ctx->rb_cap = cap;
    return add(host_dst, dev_src, bytes);
  }
  void *dev_view = nullptr;
  BST_CUDA(cudaHostGetDevicePointer(&dev_view, ctx->rb_host, 0));
  const int64_t n = (int64_t)bytes;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  k_copy_bytes<<<blocks, 256, 0, s>>>(static_cast<unsigned char *>(dev_view) + off,
                                      static_cast<const unsigned char *>(dev_src), n);
  BST_CHECK_LAUNCH();
  items.push_back({host_dst, off, bytes});
  used = off + bytes;
}

void ReadBack::finish() {
  BST_CUDA(cudaStreamSynchronize(s));
  for (const Item &it : items)
    std::memcpy(it.dst, static_cast<const char *>(ctx->rb_host) + it.off, it.bytes);
  items.clear();
  used = 0;
}

Upload::Upload(bst_ctx *c, cudaStream_t st) : ctx(c), s(st) {
  ctx->up_mutex.lock();
  locked = true;
}

Upload::~Upload() {
  if (locked) {
    // an exception left copies in flight: let them land before the buffer is reused
    if (!items.empty() || used) (void)cudaStreamSynchronize(s);
    ctx->up_mutex.unlock();
  }
}

void Upload::done() {
  flush();
  if (locked) {
    locked = false;
    ctx->up_mutex.unlock();
  }
}

void Upload::done_async() {
  if (!items.empty()) {
    launch();
    if (!ctx->up_event) BST_CUDA(cudaEventCreateWithFlags(&ctx->up_event, cudaEventDisableTiming));
    BST_CUDA(cudaEventRecord(ctx->up_event, s));
    ctx->up_pending = true;
    items.clear();
    used = 0;
  }
  if (locked) {
    locked = false;
    ctx->up_mutex.unlock();
  }
}

void Upload::add(void *dev_dst, const void *host_src, size_t bytes) {
  if (bytes == 0) return;
  if (ctx->up_pending) {  // an earlier Upload's copies may still read the buffer
    BST_CUDA(cudaEventSynchronize(ctx->up_event));
    ctx->up_pending = false;
  }
  const size_t off = (used + 15) & ~(size_t)15;
  if (off + bytes > ctx->up_cap) {
    // grow (geometrically, never shrinking: freeing pinned memory synchronises the whole
    // device): the items staged so far are copied out first
    flush();
    const size_t cap = std::max<size_t>({(size_t)1 << 20, 2 * ctx->up_cap, 2 * (off + bytes)});
    if (ctx->up_host) BST_CUDA(cudaFreeHost(ctx->up_host));
    ctx->up_host = nullptr;
    ctx->up_cap = 0;
    BST_CUDA(cudaHostAlloc(&ctx->up_host, cap, cudaHostAllocMapped));
    ctx->up_cap = cap;
    return add(dev_dst, host_src, bytes);
  }
  std::memcpy(static_cast<char *>(ctx->up_host) + off, host_src, bytes);
  items.push_back({dev_dst, off, bytes});
  used = off + bytes;
}

void Upload::flush() {
  if (items.empty()) return;
  launch();
  BST_CUDA(cudaStreamSynchronize(s));
  items.clear();
  used = 0;
}

void Upload::launch() {
  void *dev_view = nullptr;
  BST_CUDA(cudaHostGetDevicePointer(&dev_view, ctx->up_host, 0));
  for (const Item &it : items) {
    const int64_t n = (int64_t)it.bytes;
    unsigned char *dst = static_cast<unsigned char *>(it.dst);
    const unsigned char *src = static_cast<const unsigned char *>(dev_view) + it.off;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      const unsigned blocks = (unsigned)std::min<int64_t>((n / 16 + 255) / 256 + 1, 1024);
      k_copy_aligned<<<blocks, 256, 0, s>>>(dst, src, n);
    } else {
      const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
      k_copy_bytes<<<blocks, 256, 0, s>>>(dst, src, n);
    }
    BST_CHECK_LAUNCH();
  }
}

void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<<<nblk(n, 256), 256, 0, s>>>(p, v, n);
  BST_CHECK_LAUNCH();
}
void gather_i32(const int32_t *src, const int32_t *idx, int32_t *dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_gather<<<nblk(n, 256), 256, 0, s>>>(src, idx, dst, n);
  BST_CHECK_LAUNCH();
}

void stable_partition(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                      int32_t *key_ptr, Arena &ar, cudaStream_t s) {
  BST_REQUIRE(nkeys >= 1, BST_ERR_INVALID_ARG, "stable_partition: nkeys < 1");
  if (n == 0) {
    BST_CUDA(cudaMemsetAsync(key_ptr, 0, sizeof(int32_t) * ((size_t)nkeys + 1), s));
    return;
  }
  // segment length: at least 256 items per warp, and at most 2^24 histogram cells
  int64_t L = 256;
  const int64_t max_cells = int64_t(1) << 24;
  while ((int64_t)nkeys * ((n + L - 1) / L) > max_cells) L *= 2;
  int64_t G = (n + L - 1) / L;
  int64_t cells = (int64_t)nkeys * G;
  int32_t *hist = ar.alloc_n<int32_t>((size_t)cells);
  int32_t *base = ar.alloc_n<int32_t>((size_t)cells + 1);
  BST_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)cells, s));
  const int wpb = 8;
  k_part_hist<<<nblk(G, wpb), 32 * wpb, 0, s>>>(keys, n, L, G, hist);
  BST_CHECK_LAUNCH();
  exscan_i32(hist, base, cells, ar, s);
  // key_ptr[k] = base[k * G]; the entry for k = nkeys reads base[cells] = n
  k_part_keyptr<<<nblk((int64_t)nkeys + 1, 256), 256, 0, s>>>(base, nkeys, G, key_ptr);
  BST_CHECK_LAUNCH();
  k_part_scatter<<<nblk(G, wpb), 32 * wpb, 0, s>>>(keys, n, L, G, base, perm);
  BST_CHECK_LAUNCH();
}

void radix_sort_perm(const uint64_t *keys, int64_t n, int bits, int32_t *perm, Arena &ar,
                     cudaStream_t s) {
  iota_i32(perm, n, s);
  if (n <= 1 || bits <= 0) return;
  int32_t *dig = ar.alloc_n<int32_t>((size_t)n);
  int32_t *p2 = ar.alloc_n<int32_t>((size_t)n);
  int32_t *cur = ar.alloc_n<int32_t>((size_t)n);
  int32_t *kp = ar.alloc_n<int32_t>(257);
  for (int shift = 0; shift < bits; shift += 8) {
    k_digits<<<nblk(n, 256), 256, 0, s>>>(keys, perm, n, shift, dig);
    BST_CHECK_LAUNCH();
    stable_partition(dig, n, 256, p2, kp, ar, s);
    // new perm[i] = perm[p2[i]]
    gather_i32(perm, p2, cur, n, s);
    BST_CUDA(cudaMemcpyAsync(perm, cur, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace bst
