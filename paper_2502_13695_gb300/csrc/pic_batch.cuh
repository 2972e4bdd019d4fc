// Batch launches: one launch per phase of a step covering every member of a
// batch (the fluence scan's uneven instances), instead of one per member.
//   fixed grids (field, window, ionisation, flux, scan kernels): member m
//     owns the flat blocks [start[m], start[m + 1]), laid out x fastest over
//     its own gx[m] x gy[m] grid; a block finds its member by binary search;
//   particle and Keldysh loops: each member's items (slots in use, queued
//     cells; read on the device) are cut into chunks; blocks of a resident
//     grid take chunk after chunk from one counter, so the work spreads over
//     the GPU in proportion to what each member holds at that step.
// Every member's Ctx lives in device memory (two copies: the pool halves as
// at the start of a graph period, and swapped); a block copies its member's
// into shared memory before running the same body as a member's own launch.
#pragma once
#include "pic_kernels.cuh"

namespace pg {

constexpr int kMaxBatch = 1024;

struct FlatGrid {
  const int *start;  // n + 1 flat block offsets
  const int *gx;     // n: blocks along x of each member's grid
  int n;
};

// Per-member buffers of the pool sort (outside the Ctx).
struct SortBufs {
  unsigned int *cnt;            // ncell counts, then cell or frame ends
  unsigned int *bsum;           // nb_scan block sums
  unsigned long long *total;    // slots after the sort
  long long ncell;
  int nb_scan;
  int pad_;
};

// Counters of the chunked loops, zeroed at the start of every step.
enum { kCntPush = 0, kCntKeldysh = 1, kCntHist = 2, kCntScatter = 3, kCntN = 4 };

__device__ __forceinline__ int flat_member(const FlatGrid &G, int b) {
  int lo = 0, hi = G.n - 1;  // the largest m with start[m] <= b (members with
  while (lo < hi) {          // no blocks share their successor's start)
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(G.start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ Blk flat_blk(const FlatGrid &G, int &m) {
  const int b = (int)blockIdx.x;
  m = flat_member(G, b);
  const int local = b - __ldg(G.start + m), gx = __ldg(G.gx + m);
  const int gy = (__ldg(G.start + m + 1) - __ldg(G.start + m)) / gx;
  return Blk{local % gx, local / gx, gx, gy};
}

// The member's Ctx copied into shared memory in 8-byte words (one copy per
// block; the caller separates reuses with a barrier).
template <class R>
__device__ __forceinline__ const Ctx<R> &member_ctx(const Ctx<R> *ctx, int m) {
  static_assert(sizeof(Ctx<R>) % 8 == 0, "Ctx is copied in 8-byte words");
  __shared__ unsigned long long buf[sizeof(Ctx<R>) / 8];
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(ctx + m);
  for (int w = threadIdx.x; w < (int)(sizeof(Ctx<R>) / 8); w += blockDim.x) buf[w] = src[w];
  __syncthreads();
  return *reinterpret_cast<const Ctx<R> *>(buf);
}

// Chunk counts of every member's items, prefix-summed into pref[0..n] by the
// first warp (each block computes the same table from the same counts).
template <class R, class Count>
__device__ __forceinline__ void chunk_prefix(const Ctx<R> *ctx, int n, long long chunk,
                                             Count count, unsigned int *pref) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned int run = 0;
    if (lane == 0) pref[0] = 0;
    for (int base = 0; base < n; base += 32) {
      const int m = base + lane;
      unsigned int c = 0;
      if (m < n) {
        const long long items = count(ctx[m]);
        c = (unsigned int)((items + chunk - 1) / chunk);
      }
      unsigned int incl = c;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl += v;
      }
      if (m < n) pref[m + 1] = run + incl;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();
}

// The next chunk for this block: false when none is left; else its member m
// and chunk index c (items [c chunk, (c + 1) chunk) of that member).
__device__ __forceinline__ bool next_chunk(unsigned int *counter, const unsigned int *pref, int n,
                                           int &m, long long &c) {
  __shared__ unsigned int task;
  __syncthreads();  // the block is done with the previous chunk
  if (threadIdx.x == 0) task = atomicAdd(counter, 1u);
  __syncthreads();
  const unsigned int t = task;
  if (t >= pref[n]) return false;
  int lo = 0, hi = n - 1;  // the largest m with pref[m] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  m = lo;
  c = (long long)(t - pref[lo]);
  return true;
}

template <class R>
struct SlotsInUse {
  __device__ long long operator()(const Ctx<R> &X) const {
    return (long long)min(*X.d.nslots, X.d.cap);
  }
};
template <class R>
struct QueuedCells {
  __device__ long long operator()(const Ctx<R> &X) const { return (long long)*X.work_n; }
};

// Chunk sizes (items per block task); the push's chunk and grid are chosen
// per batch by measurement (pic_api.cu, batch_tune).
constexpr long long kKeldyshChunk = 256 * 4, kSortChunk = 256 * 8;

// Start of a step: zero the chunk counters and every member's Keldysh queue.
template <class R>
__global__ void k_batch_prep(const Ctx<R> *ctx, int n, unsigned int *counters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kCntN) counters[t] = 0u;
  if (t < n) *ctx[t].work_n = 0;
}

template <class R>
__global__ void __launch_bounds__(256, PushOcc<R>::v)
    k_push_batch(const Ctx<R> *ctx, int n, unsigned int *counters, long long chunk) {
  __shared__ unsigned int pref[kMaxBatch + 1];
  chunk_prefix(ctx, n, chunk, SlotsInUse<R>(), pref);
  int m;
  long long c;
  while (next_chunk(counters + kCntPush, pref, n, m, c)) {
    const Ctx<R> &X = member_ctx(ctx, m);
    const double pushed = push_items(X, (unsigned long long)(c * chunk),
                                     (unsigned long long)((c + 1) * chunk),
                                     (unsigned long long)blockDim.x);
    const double tot = block_sum<R>(pushed);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(X.d.acc + 4, tot);
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_keldysh_batch(const Ctx<R> *ctx, int n,
                                                       unsigned int *counters) {
  __shared__ unsigned int pref[kMaxBatch + 1];
  chunk_prefix(ctx, n, kKeldyshChunk, QueuedCells<R>(), pref);
  int m;
  long long c;
  while (next_chunk(counters + kCntKeldysh, pref, n, m, c)) {
    const Ctx<R> &X = member_ctx(ctx, m);
    keldysh_items(X, (int)(c * kKeldyshChunk), min((int)((c + 1) * kKeldyshChunk), *X.work_n),
                  blockDim.x);
  }
}

template <int V, class R, bool kLay>
__global__ void __launch_bounds__(256, 3) k_efull_batch(const Ctx<R> *ctx, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  efull_body<V, kLay>(member_ctx(ctx, m), bk);
}

template <int V, class R, bool kLay>
__global__ void __launch_bounds__(256) k_bstep_batch(const Ctx<R> *ctx, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  bstep_body<V, kFullRecord, kLay>(member_ctx(ctx, m).d, bk);
}

template <int V, class R>
__global__ void __launch_bounds__(256) k_window_batch(const Ctx<R> *ctx, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  window_body<V>(member_ctx(ctx, m), bk);
}

template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 3)
    k_ionize_batch(const Ctx<R> *ctx, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  ionize_body(member_ctx(ctx, m), bk);
}

template <class R>
__global__ void __launch_bounds__(256) k_flux_advance_batch(const Ctx<R> *ctx, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  flux_advance_body(member_ctx(ctx, m).d, bk);
}

// ---- pool sort by deposit-frame base, every member at once ----------------
// zero the counts: member m's ncell counts over its flat blocks
__global__ void __launch_bounds__(256) k_zero_cnt_batch(const SortBufs *sb, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  const long long q = (long long)bk.x * blockDim.x + threadIdx.x;
  const SortBufs S = sb[m];
  if (q < S.ncell) S.cnt[q] = 0u;
}

template <class R>
__global__ void k_hist_batch(const Ctx<R> *ctx, const SortBufs *sb, int n, unsigned int *counters) {
  __shared__ unsigned int pref[kMaxBatch + 1];
  chunk_prefix(ctx, n, kSortChunk, SlotsInUse<R>(), pref);
  int m;
  long long c;
  while (next_chunk(counters + kCntHist, pref, n, m, c)) {
    const Ctx<R> &X = member_ctx(ctx, m);
    hist_items<true>(X.d, sb[m].cnt, (unsigned long long)(c * kSortChunk),
                     (unsigned long long)((c + 1) * kSortChunk), (unsigned long long)blockDim.x);
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce_batch(const SortBufs *sb, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  const SortBufs S = sb[m];
  scan_reduce_body(S.cnt, S.ncell, S.bsum, bk.x);
}

// one block per member
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks_batch(const SortBufs *sb) {
  const SortBufs S = sb[blockIdx.x];
  unsigned int carry = 0;
  for (int base = 0; base < S.nb_scan; base += kScanThreads) {
    const int idx = base + threadIdx.x;
    const unsigned int v = idx < S.nb_scan ? S.bsum[idx] : 0u;
    unsigned int tot;
    const unsigned int ex = block_excl_scan(v, tot);
    if (idx < S.nb_scan) S.bsum[idx] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *S.total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final_batch(const SortBufs *sb, FlatGrid G) {
  int m;
  const Blk bk = flat_blk(G, m);
  const SortBufs S = sb[m];
  scan_final_body(S.cnt, S.ncell, S.bsum, bk.x);
}

// scatter from one pool half (ctx) into the other, then the slot counts
template <class R>
__global__ void __launch_bounds__(256) k_scatter_batch(const Ctx<R> *ctx, const SortBufs *sb, int n,
                                                       unsigned int *counters) {
  __shared__ unsigned int pref[kMaxBatch + 1];
  chunk_prefix(ctx, n, kSortChunk, SlotsInUse<R>(), pref);
  int m;
  long long c;
  while (next_chunk(counters + kCntScatter, pref, n, m, c)) {
    const Ctx<R> &X = member_ctx(ctx, m);
    scatter_items<true>(X, sb[m].cnt, (unsigned long long)(c * kSortChunk),
                        (unsigned long long)((c + 1) * kSortChunk), (unsigned long long)blockDim.x);
  }
}

template <class R>
__global__ void k_set_slots_batch(const Ctx<R> *ctx, const SortBufs *sb, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) *ctx[t].d.nslots = *sb[t].total;
}

}  // namespace pg
