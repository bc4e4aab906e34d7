// CSR / degree-normalization builder (Sec. 2: L = D - A and
// I - D^{-1/2} A D^{-1/2}).
//
// Pipeline, all on the device:
//   1. validate ids; emit both orientations of every non-loop edge as 64-bit
//      keys (row << cs | col), with the weight as payload; in a batch the
//      column field holds the graph-local id (its graph follows from the
//      row), which saves sort bits;
//   2. stable LSD radix sort of the keys (8-bit digits, reduce-then-scan,
//      tiles reordered by digit in shared memory before the scatter);
//   3. merge duplicates (largest weight kept), rowptr from the sorted rows;
//   4. degrees, optional removal of isolated nodes with order-preserving
//      renumbering, scales s_i = 1/sqrt(d_i) and off-diagonal values;
//   5. an execution copy with nodes renumbered by descending degree;
//   6. the SpMM schedule that splits rows of more than `heavy_degree`
//      entries into chunks.
// The result is canonical (sorted columns, merged duplicates), so it equals
// any correct builder's bit for bit.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace slaq {
namespace {

// ------------------------------------------------------------- block scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_inclusive_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's prefix and writes the block total to *total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_tot[33];   // [0, 32): warp prefixes, [32]: total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  int64_t inc = warp_inclusive_scan(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nwarps ? warp_tot[lane] : 0;
    int64_t wi = warp_inclusive_scan(w);
    if (lane < nwarps) warp_tot[lane] = wi - w;
    if (lane == 31) warp_tot[32] = wi;  // lanes past nwarps add zeros
  }
  __syncthreads();
  int64_t res = warp_tot[warp] + inc - v;
  if (total) *total = warp_tot[32];
  __syncthreads();
  return res;
}

template <typename TI>
__global__ void k_scan_tile_sums(const TI *in, int64_t n, int64_t *bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
#pragma unroll
  for (int it = 0; it < kScanItems; ++it) {
    int64_t i = base + (int64_t)it * kScanThreads + threadIdx.x;
    if (i < n) acc += (int64_t)in[i];
  }
  int64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block scans the tile sums in place (exclusive) and stores the grand
// total in *total.
__global__ void k_scan_tile_prefix(int64_t *bsum, int64_t nb, int64_t *total) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <typename TI>
__global__ void k_scan_apply(const TI *in, int64_t n, const int64_t *bsum, int64_t *out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t vals[kScanItems];
  int64_t acc = 0;
#pragma unroll
  for (int it = 0; it < kScanItems; ++it) {
    int64_t i = base + it;
    vals[it] = i < n ? (int64_t)in[i] : 0;
    acc += vals[it];
  }
  int64_t ex = block_exclusive_scan(acc, nullptr) + bsum[blockIdx.x];
#pragma unroll
  for (int it = 0; it < kScanItems; ++it) {
    int64_t i = base + it;
    if (i < n) out[i] = ex;
    ex += vals[it];
  }
}

// out[0..n) = exclusive prefix sums of in; *total_dev = sum (device int64).
template <typename TI>
int exclusive_scan(const TI *in, int64_t n, int64_t *out, int64_t *total_dev, cudaStream_t st) {
  int64_t nb = std::max<int64_t>(1, ceil_div(n, kScanTile));
  int64_t *bsum = nullptr;
  SLAQ_TRY(dalloc_t(&bsum, nb, st));
  struct Free {
    int64_t *p;
    cudaStream_t st;
    ~Free() { dfree(p, st); }
  } free_bsum{bsum, st};
  if (n > 0) {
    ++tl_launches;
    k_scan_tile_sums<TI><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum);
  } else {
    SLAQ_CHECK_CUDA(cudaMemsetAsync(bsum, 0, sizeof(int64_t), st));
  }
  ++tl_launches;
  k_scan_tile_prefix<<<1, 1024, 0, st>>>(bsum, nb, total_dev);
  if (n > 0) {
    // the apply kernel walks kScanItems consecutive items per thread
    ++tl_launches;
    k_scan_apply<TI><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum, out);
  }
  SLAQ_CHECK_LAUNCH("exclusive_scan");
  return SLAQ_OK;
}

// ------------------------------------------------------------- radix sort
constexpr int kRsThreads = 512;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 8;                        // 32-key rounds per warp
constexpr int kRsTile = kRsThreads * kRsRounds;     // 4096 keys per block
constexpr int kRsHistThreads = 256;

__global__ void __launch_bounds__(kRsHistThreads)
    k_radix_hist(const uint64_t *keys, int64_t n, int shift, uint32_t *counts, int64_t ntiles) {
  __shared__ uint32_t hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int it = 0; it < kRsTile / kRsHistThreads; ++it) {
    int64_t i = base + (int64_t)it * kRsHistThreads + threadIdx.x;
    if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns keys [tile + 256 w, tile + 256 (w+1))
// and ranks them round by round (32 keys per round, lane order), so equal
// digits keep their input order inside the warp; warps are ordered by a
// per-digit prefix over warps.  The tile is first reordered by digit in
// shared memory, then written out run by run, so that consecutive threads
// store consecutive addresses of one digit's run; tiles are ordered by the
// digit-major global scan of the per-tile counts.
template <bool PAYLOAD>
__global__ void __launch_bounds__(kRsThreads, 3)
    k_radix_scatter(const uint64_t *__restrict__ kin, const double *__restrict__ pin,
                    uint64_t *__restrict__ kout, double *__restrict__ pout, int64_t n, int shift,
                    const int64_t *__restrict__ offsets, int64_t ntiles) {
  __shared__ uint32_t whist[kRsWarps][256];
  __shared__ uint32_t dstart[256];  // first slot of each digit in the reordered tile
  __shared__ int64_t gbase[256];    // first output slot of each digit of this tile
  __shared__ uint32_t wsum[8];
  extern __shared__ __align__(16) unsigned char rs_dyn[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(rs_dyn);      // [kRsTile]
  double *spay = reinterpret_cast<double *>(skey + kRsTile);  // [kRsTile] (PAYLOAD)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  const int64_t seg = tile0 + (int64_t)warp * (32 * kRsRounds);
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t key[kRsRounds];
  uint32_t local[kRsRounds / 2];  // ranks within the warp (< 512), two per word
  // all loads first: the ranking below synchronizes the warp every round
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = seg + r * 32 + lane;
    key[r] = i < n ? kin[i] : 0ull;
  }
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = seg + r * 32 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? (uint32_t)((key[r] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    uint32_t before = d < 256u ? whist[warp][d] : 0u;
    __syncwarp();
    if (d < 256u && rank == 0) whist[warp][d] = before + __popc(peers);
    __syncwarp();
    if (r & 1) local[r >> 1] |= (before + rank) << 16;
    else local[r >> 1] = before + rank;
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;  // one digit per thread: prefix over warps
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
    gbase[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
    // exclusive scan of the digit totals over the 256 threads (8 warps)
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    dstart[d] = inc - run;  // within the warp; warp offsets added below
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += wsum[w];
    dstart[threadIdx.x] += add;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = seg + r * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)((key[r] >> shift) & 255u);
      const uint32_t slot = dstart[d] + whist[warp][d] + ((local[r >> 1] >> (16 * (r & 1))) & 0xffffu);
      skey[slot] = key[r];
      if (PAYLOAD) spay[slot] = pin[i];
    }
  }
  __syncthreads();
  const int count = (int)min((int64_t)kRsTile, n - tile0);
  for (int q = threadIdx.x; q < count; q += kRsThreads) {
    const uint64_t k = skey[q];
    const uint32_t d = (uint32_t)((k >> shift) & 255u);
    const int64_t pos = gbase[d] + (q - (int)dstart[d]);
    kout[pos] = k;
    if (PAYLOAD) pout[pos] = spay[q];
  }
}

inline size_t rs_smem(bool payload) {
  return (size_t)kRsTile * (sizeof(uint64_t) + (payload ? sizeof(double) : 0));
}

// Sorts n keys on their low `bits` bits.  Result in *keys (buffers swapped
// as needed; both buffers hold n entries).
int radix_sort(uint64_t **keys, uint64_t **keys_alt, double **pay, double **pay_alt, int64_t n,
               int bits, cudaStream_t st) {
  if (n <= 1) return SLAQ_OK;
  const int64_t ntiles = ceil_div(n, kRsTile);
  uint32_t *counts = nullptr;
  int64_t *offsets = nullptr, *total = nullptr;
  struct Free {
    uint32_t **c;
    int64_t **o, **t;
    cudaStream_t st;
    ~Free() {
      dfree(*c, st);
      dfree(*o, st);
      dfree(*t, st);
    }
  } free_tmp{&counts, &offsets, &total, st};
  SLAQ_TRY(dalloc_t(&counts, 256 * ntiles, st));
  SLAQ_TRY(dalloc_t(&offsets, 256 * ntiles, st));
  SLAQ_TRY(dalloc_t(&total, 1, st));
  const bool with_pay = pay && *pay;
  // once per process (a thread-safe static initialization)
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rs_smem(true));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_radix_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rs_smem(false));
    return e;
  }();
  SLAQ_CHECK_CUDA(attr);
  for (int shift = 0; shift < bits; shift += 8) {
    ++tl_launches;
    k_radix_hist<<<(unsigned)ntiles, kRsHistThreads, 0, st>>>(*keys, n, shift, counts, ntiles);
    SLAQ_CHECK_LAUNCH("radix_hist");
    SLAQ_TRY(exclusive_scan(counts, 256 * ntiles, offsets, total, st));
    if (with_pay) {
      ++tl_launches;
      k_radix_scatter<true><<<(unsigned)ntiles, kRsThreads, rs_smem(true), st>>>(
          *keys, *pay, *keys_alt, *pay_alt, n, shift, offsets, ntiles);
      std::swap(*pay, *pay_alt);
    } else {
      ++tl_launches;
      k_radix_scatter<false><<<(unsigned)ntiles, kRsThreads, rs_smem(false), st>>>(
          *keys, nullptr, *keys_alt, nullptr, n, shift, offsets, ntiles);
    }
    SLAQ_CHECK_LAUNCH("radix_scatter");
    std::swap(*keys, *keys_alt);
  }
  return SLAQ_OK;
}

// ---------------------------------------------------------- CSR kernels
// Adds a warp's self-loop count to *loops (no atomic when it is zero, so
// loop-free inputs cost nothing).
__device__ __forceinline__ void add_loops(unsigned cnt, unsigned long long *loops) {
  const unsigned tot = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(loops, (unsigned long long)tot);
}

__global__ void k_validate(const int32_t *src, const int32_t *dst, const double *w, int64_t m,
                           int64_t n, int32_t *bad, unsigned long long *loops) {
  unsigned cnt = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = src[e], b = dst[e];
    if (a < 0 || b < 0 || a >= n || b >= n) atomicOr(bad, 1);
    if (w && !(w[e] > 0.0)) atomicOr(bad, 2);
    cnt += a == b;
  }
  add_loops(cnt, loops);
}

// Batches: edge e of graph g (edge_off[g] <= e < edge_off[g+1]) has local
// ids in [0, n_g); write union ids (node_off[g] + local) and flag bad ids.
__device__ __forceinline__ int find_segment(const int64_t *off, int G, int64_t x) {
  int lo = 0, hi = G;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// A batch's edges by chunks of one graph: edges [e0, e0 + len) of graph g.
struct EdgeChunk {
  int64_t e0;
  int32_t g, len;
};
constexpr int kEdgeChunk = 8192;

// One block per chunk (the graph of its edges is known, no search): local
// ids checked against the graph's node count and shifted to union ids.
__global__ void k_union_ids(const int32_t *src, const int32_t *dst, const double *w,
                            const EdgeChunk *chunks, const int64_t *node_off, int32_t *usrc,
                            int32_t *udst, int32_t *bad, unsigned long long *loops) {
  const EdgeChunk c = chunks[blockIdx.x];
  const int64_t base = node_off[c.g], ng = node_off[c.g + 1] - base;
  unsigned cnt = 0;
  for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
    const int64_t e = c.e0 + i;
    const int32_t a = src[e], b = dst[e];
    if (a < 0 || b < 0 || a >= ng || b >= ng) atomicOr(bad, 1);
    if (w && !(w[e] > 0.0)) atomicOr(bad, 2);
    usrc[e] = (int32_t)(base + (a < 0 ? 0 : a));
    udst[e] = (int32_t)(base + (b < 0 ? 0 : b));
    cnt += a == b;
  }
  add_loops(cnt, loops);
}

// Graph of every kept node (canonical order), its id within its graph, and
// per-graph statistics: kept nodes, non-isolated nodes, integer degree sum,
// largest degree (non-negative doubles order like their bit patterns).  One
// thread per node; a warp whose nodes share one graph adds its sums once.
__global__ void k_node_graph(const int64_t *old_id, const double *deg, const int64_t *rowptr,
                             int64_t n, const int64_t *node_off, int G, int32_t *gid,
                             int64_t *local, unsigned long long *kept,
                             unsigned long long *nonisol, unsigned long long *degsum,
                             unsigned long long *maxdeg, unsigned long long *entries) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = i < n;
  int g = -1;
  unsigned long long c_kept = 0, c_non = 0, c_sum = 0, c_max = 0, c_ent = 0;
  if (valid) {
    g = find_segment(node_off, G, old_id[i]);
    gid[i] = g;
    local[i] = old_id[i] - node_off[g];
    const double d = deg[i];
    c_kept = 1;
    c_non = d > 0.0 ? 1 : 0;
    c_sum = (unsigned long long)d;
    c_max = (unsigned long long)__double_as_longlong(d);
    c_ent = (unsigned long long)(rowptr[i + 1] - rowptr[i]);
  }
  const int g0 = __shfl_sync(0xffffffffu, g, 0);
  const bool uniform = __all_sync(0xffffffffu, !valid || g == g0) && g0 >= 0;
  if (uniform) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c_kept += __shfl_down_sync(0xffffffffu, c_kept, o);
      c_non += __shfl_down_sync(0xffffffffu, c_non, o);
      c_sum += __shfl_down_sync(0xffffffffu, c_sum, o);
      c_ent += __shfl_down_sync(0xffffffffu, c_ent, o);
      const unsigned long long other = __shfl_down_sync(0xffffffffu, c_max, o);
      c_max = other > c_max ? other : c_max;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(kept + g0, c_kept);
      if (c_non) atomicAdd(nonisol + g0, c_non);
      atomicAdd(degsum + g0, c_sum);
      atomicMax(maxdeg + g0, c_max);
      atomicAdd(entries + g0, c_ent);
    }
  } else if (valid) {
    atomicAdd(kept + g, c_kept);
    if (c_non) atomicAdd(nonisol + g, c_non);
    atomicAdd(degsum + g, c_sum);
    atomicMax(maxdeg + g, c_max);
    atomicAdd(entries + g, c_ent);
  }
}

// Both orientations of every non-loop edge; slots taken with one atomic per
// warp, so the emission order is arbitrary (the sort removes it).
__global__ void k_emit(const int32_t *src, const int32_t *dst, const int32_t *csrc,
                       const int32_t *cdst, const double *w, int64_t m, int cs, uint64_t *keys,
                       double *pay, unsigned long long *counter) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < m; e0 += stride) {
    const int64_t e = e0 + threadIdx.x;
    bool emit = false;
    uint64_t a = 0, b = 0, ca = 0, cbv = 0;
    if (e < m) {
      a = (uint32_t)src[e];
      b = (uint32_t)dst[e];
      emit = a != b;
      ca = (uint32_t)csrc[e];
      cbv = (uint32_t)cdst[e];
    }
    const unsigned mask = __ballot_sync(0xffffffffu, emit);
    if (mask == 0) continue;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, 2ull * __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (emit) {
      const unsigned long long pos = base + 2ull * __popc(mask & ((1u << lane) - 1u));
      keys[pos] = (a << cs) | cbv;
      keys[pos + 1] = (b << cs) | ca;
      if (pay) {
        pay[pos] = w[e];
        pay[pos + 1] = w[e];
      }
    }
  }
}

// Loop-free input: edge e gives keys 2e and 2e+1.
__global__ void k_emit_direct(const int32_t *src, const int32_t *dst, const int32_t *csrc,
                              const int32_t *cdst, const double *w, int64_t m, int cs,
                              uint64_t *keys, double *pay) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = (uint32_t)src[e], b = (uint32_t)dst[e];
    const uint64_t ca = (uint32_t)csrc[e], cbv = (uint32_t)cdst[e];
    reinterpret_cast<ulonglong2 *>(keys)[e] = make_ulonglong2((a << cs) | cbv, (b << cs) | ca);
    if (pay) reinterpret_cast<double2 *>(pay)[e] = make_double2(w[e], w[e]);
  }
}

// Merging duplicates is a stream compaction of the sorted keys: key i starts a
// run if i = 0 or it differs from key i-1.  k_unique_count counts run starts
// per scan tile; after the tiles' exclusive scan, k_unique_compact finds the
// starts again (warp ballots over coalesced rounds), scans their counts
// within the tile and writes each run's key, and its largest weight, to the
// run's slot.  No per-key flag or position array.
__global__ void __launch_bounds__(kScanThreads)
    k_unique_count(const uint64_t *__restrict__ k, int64_t m, int64_t *__restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
#pragma unroll
  for (int it = 0; it < kScanItems; ++it) {
    const int64_t i = base + (int64_t)it * kScanThreads + threadIdx.x;
    if (i < m) acc += (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
  }
  int64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads)
    k_unique_compact(const uint64_t *__restrict__ k, const double *__restrict__ pay, int64_t m,
                     const int64_t *__restrict__ bsum, uint64_t *__restrict__ ukey,
                     double *__restrict__ uw) {
  // round r covers items t0 + r * kScanThreads + threadIdx.x (coalesced); in
  // key order the items run round by round, warp by warp, lane by lane, so
  // the run starts of (round, warp) pairs are counted by ballots, scanned in
  // that order, and placed within a warp by the lanes below
  constexpr int kW = kScanThreads / 32;
  constexpr int kCnt = kScanItems * kW;  // (round, warp) counts, a multiple of 32
  static_assert(kCnt % 32 == 0, "count table must split evenly over a warp");
  __shared__ int64_t cnt[kCnt];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  uint32_t ball[kScanItems];
  uint64_t key[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t i = t0 + (int64_t)r * kScanThreads + threadIdx.x;
    const uint64_t kv = i < m ? k[i] : 0;
    uint64_t prev = __shfl_up_sync(0xffffffffu, kv, 1);
    if (lane == 0 && i > 0 && i < m) prev = k[i - 1];
    ball[r] = __ballot_sync(0xffffffffu, i < m && (i == 0 || kv != prev));
    key[r] = kv;
    if (lane == 0) cnt[r * kW + warp] = __popc(ball[r]);
  }
  __syncthreads();
  if (warp == 0) {
    constexpr int per = kCnt / 32;
    int64_t v[per], sum = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      v[q] = cnt[lane * per + q];
      sum += v[q];
    }
    int64_t ex = warp_inclusive_scan(sum) - sum + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < per; ++q) {
      cnt[lane * per + q] = ex;
      ex += v[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    if (!((ball[r] >> lane) & 1u)) continue;
    const int64_t pos = cnt[r * kW + warp] + __popc(ball[r] & ((1u << lane) - 1u));
    ukey[pos] = key[r];
    if (pay) {
      const int64_t i = t0 + (int64_t)r * kScanThreads + threadIdx.x;
      double mx = pay[i];
      for (int64_t j = i + 1; j < m && k[j] == key[r]; ++j) mx = fmax(mx, pay[j]);
      uw[pos] = mx;
    }
  }
}

// rowptr[r] = index of the first key with row >= r (rows = key >> shift).
__global__ void k_rowptr(const uint64_t *ukey, int64_t nnz, int shift, int64_t n,
                         int64_t *rowptr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r_prev = i == 0 ? -1 : (int64_t)(ukey[i - 1] >> shift);
    const int64_t r_cur = i == nnz ? n : (int64_t)(ukey[i] >> shift);
    for (int64_t r = r_prev + 1; r <= r_cur; ++r) rowptr[r] = i;
  }
}

// Degrees: entry counts, or weights summed left to right in column order.
__global__ void k_degree(const int64_t *rowptr, const double *uw, int64_t n, double *deg,
                         uint8_t *keep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    double d;
    if (uw) {
      d = 0.0;
      for (int64_t j = b; j < e; ++j) d += uw[j];
    } else {
      d = (double)(e - b);
    }
    deg[i] = d;
    keep[i] = e > b ? 1 : 0;
  }
}

// Compacted node arrays (old ids, degrees, row starts).  With drop == 0
// newid is the identity and every node is kept.
__global__ void k_compact_nodes(const int64_t *rowptr, const double *deg, const uint8_t *keep,
                                const int64_t *newid, int64_t n, int drop, int64_t nnz,
                                int64_t n_out, int64_t *rowptr_out, double *deg_out,
                                int64_t *old_id) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (drop && !keep[i]) continue;
    const int64_t j = drop ? newid[i] : i;
    rowptr_out[j] = rowptr[i];
    deg_out[j] = deg[i];
    old_id[j] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rowptr_out[n_out] = nnz;
}

__global__ void k_scale(const double *deg, int64_t n, int kind, double *scale, double *diag,
                        float *scale32, float *diag32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = deg[i];
    double s, g;
    if (kind == SLAQ_NORMALIZED) {
      s = d > 0.0 ? 1.0 / sqrt(d) : 0.0;   // IEEE round-to-nearest sqrt and divide
      g = d > 0.0 ? 1.0 : 0.0;
    } else {
      s = 1.0;
      g = d;
    }
    scale[i] = s;
    diag[i] = g;
    scale32[i] = (float)s;
    diag32[i] = (float)g;
  }
}

// tr(L_g^2) = sum_ij (L_g)_ij^2 of every graph, in two deterministic levels.
// A graph's rows are contiguous, so its diagonal (n_g values) and its stored
// off-diagonal entries (E_g values) are two contiguous ranges.  Level 1 cuts
// both ranges into chunks of kSqChunk values, one block per chunk: each
// thread sums the squares of a fixed strided subset of 32 values with FP64
// FMAs (relative error <= 32 eps; a compensated add per value would make the
// kernel FP64-ALU-bound) and the threads combine in a fixed tree order.
// Level 2: one block per graph adds its chunks' partials, Neumaier-compensated
// per thread, in a fixed tree.  The result depends on neither the scheduling
// nor the number of SMs, and chunks of equal size balance graphs with a few
// very long rows.
constexpr int kSqThreads = 256;
constexpr int kSqChunk = 8192;
struct Neumaier {
  double sm = 0.0, cp = 0.0;
  __device__ void add(double x) {
    const double t = sm + x;
    cp += fabs(sm) >= fabs(x) ? (sm - t) + x : (x - t) + sm;
    sm = t;
  }
};
__device__ double block_tree_sum(Neumaier acc, double *ssum, double *scmp) {
  ssum[threadIdx.x] = acc.sm;
  scmp[threadIdx.x] = acc.cp;
  __syncthreads();
  for (int w = kSqThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ssum[threadIdx.x] += ssum[threadIdx.x + w];
      scmp[threadIdx.x] += scmp[threadIdx.x + w];
    }
    __syncthreads();
  }
  return ssum[0] + scmp[0];
}
// Graph q owns blocks coff[q] .. coff[q+1]-1: first its diagonal chunks, then
// its entry chunks (graphs without rows own none).  goff / eoff: first row /
// first stored entry of every graph.
__global__ void __launch_bounds__(kSqThreads)
    k_graph_sq_chunks(const double *vals, const double *diag, const int64_t *goff,
                      const int64_t *eoff, const int64_t *coff, int G, double *partial) {
  __shared__ double ssum[kSqThreads], scmp[kSqThreads];
  const int64_t b = blockIdx.x;
  const int q = find_segment(coff, G, b);
  const int64_t j = b - coff[q];
  const int64_t n_diag = (goff[q + 1] - goff[q] + kSqChunk - 1) / kSqChunk;
  const double *x;
  int64_t lo, hi;
  if (j < n_diag) {
    x = diag;
    lo = goff[q] + j * kSqChunk;
    hi = min(lo + kSqChunk, goff[q + 1]);
  } else {
    x = vals;
    lo = eoff[q] + (j - n_diag) * kSqChunk;
    hi = min(lo + kSqChunk, eoff[q + 1]);
  }
  double sq = 0.0;
  for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += 4 * kSqThreads) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + (int64_t)u * kSqThreads;
      v[u] = i < hi ? x[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sq = fma(v[u], v[u], sq);
  }
  Neumaier acc;
  acc.sm = sq;
  const double v = block_tree_sum(acc, ssum, scmp);
  if (threadIdx.x == 0) partial[b] = v;
}
__global__ void __launch_bounds__(kSqThreads)
    k_graph_sq_sum(const double *partial, const int64_t *coff, double *out) {
  __shared__ double ssum[kSqThreads], scmp[kSqThreads];
  const int q = blockIdx.x;
  Neumaier acc;
  for (int64_t c = coff[q] + threadIdx.x; c < coff[q + 1]; c += kSqThreads) acc.add(partial[c]);
  const double v = block_tree_sum(acc, ssum, scmp);
  if (threadIdx.x == 0) out[q] = v;
}

// Batches: first union id of the graph of every input node (keys carry
// graph-local column ids).
__global__ void k_row_base(const int64_t *node_off, int G, int64_t n, int64_t *rowbase) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = G;  // node_off[lo] <= i < node_off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (node_off[mid] <= i) lo = mid;
      else hi = mid;
    }
    rowbase[i] = node_off[lo];
  }
}

__global__ void k_values(const uint64_t *ukey, const double *uw, const int64_t *newid, int drop,
                         int cs, const int64_t *rowbase, int64_t nnz, int kind,
                         const double *scale, int32_t *colidx, double *vals, float *vals32) {
  const uint64_t cmask = (1ull << cs) - 1ull;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = ukey[j];
    const int64_t r_old = (int64_t)(key >> cs);
    const int64_t c_old = (rowbase ? rowbase[r_old] : 0) + (int64_t)(key & cmask);
    const int64_t r = drop ? newid[r_old] : r_old;
    const int64_t c = drop ? newid[c_old] : c_old;
    const double a = uw ? uw[j] : 1.0;
    double v;
    if (kind == SLAQ_NORMALIZED) v = -((a * scale[r]) * scale[c]);
    else v = -a;
    colidx[j] = (int32_t)c;
    vals[j] = v;
    if (vals32) vals32[j] = (float)v;
  }
}

__global__ void k_heavy_flags(const int64_t *rowptr, int64_t n, int64_t heavy_degree,
                              int32_t *is_heavy, int64_t *nchunk) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    const bool h = d > heavy_degree;
    is_heavy[i] = h ? 1 : 0;
    nchunk[i] = h ? (d + kHeavyChunk - 1) / kHeavyChunk : 0;
  }
}

__global__ void k_heavy_table(const int32_t *is_heavy, const int64_t *slot_of,
                              const int64_t *chunk_of, const int64_t *nchunk, int64_t n,
                              int64_t n_heavy, int64_t n_chunks, int32_t *heavy_row,
                              int64_t *heavy_first, int32_t *chunk_slot) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!is_heavy[i]) continue;
    const int64_t slot = slot_of[i];
    heavy_row[slot] = (int32_t)i;
    heavy_first[slot] = chunk_of[i];
    for (int64_t c = 0; c < nchunk[i]; ++c) chunk_slot[chunk_of[i] + c] = (int32_t)slot;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) heavy_first[n_heavy] = n_chunks;
}

// Sort key of the execution order: graph, then descending entry count,
// then id (graph | n - count | id, from high bits to low).
__global__ void k_perm_keys(const int64_t *rowptr, const int32_t *gid, int64_t n, int cb, int db,
                            uint64_t *key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t cnt = (uint64_t)(rowptr[i + 1] - rowptr[i]);
    key[i] = ((((uint64_t)gid[i] << db) | ((uint64_t)n - cnt)) << cb) | (uint64_t)i;
  }
}

__global__ void k_perm_index(const uint64_t *key, const int64_t *rowptr, int64_t n, int cb,
                             int64_t *perm, int64_t *inv, int64_t *xcnt) {
  const uint64_t mask = (1ull << cb) - 1ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(key[r] & mask);
    perm[r] = i;
    inv[i] = r;
    xcnt[r] = rowptr[i + 1] - rowptr[i];
  }
}

// Execution row r is canonical row perm[r]; columns are renamed through inv.
// One thread per canonical entry (its row comes from the sorted key).
__global__ void k_perm_entries(const uint64_t *ukey, const int64_t *newid, int drop, int shift,
                               const int64_t *rowptr, const int32_t *colidx, const double *vals,
                               const float *vals32, const int64_t *inv, int64_t nnz,
                               const int64_t *xrowptr, int32_t *xcol, double *xvals,
                               float *xvals32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r_old = (int64_t)(ukey[e] >> shift);
    const int64_t i = drop ? newid[r_old] : r_old;
    const int64_t x = xrowptr[inv[i]] + (e - rowptr[i]);
    xcol[x] = (int32_t)inv[colidx[e]];
    if (xvals) xvals[x] = vals[e];
    if (xvals32) xvals32[x] = vals32[e];
  }
}

__global__ void k_perm_nodes(const double *diag, const double *scale, const int64_t *local,
                             const int32_t *gid, const int64_t *perm, int64_t n, double *xdiag,
                             double *xscale, float *xdiag32, float *xscale32, int64_t *xold,
                             int32_t *xgraph) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[r];
    xdiag[r] = diag[i];
    xscale[r] = scale[i];
    xdiag32[r] = (float)diag[i];
    xscale32[r] = (float)scale[i];
    xold[r] = local[i];
    xgraph[r] = gid[i];
  }
}

inline unsigned grid_for(int64_t n, int threads) {
  int64_t b = ceil_div(std::max<int64_t>(n, 1), threads);
  return (unsigned)std::min<int64_t>(b, 65535LL * 8);
}

template <typename T>
int to_host(T *host, const T *dev, size_t count, cudaStream_t st) {
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  return SLAQ_OK;
}

int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && (1ll << b) < n) ++b;
  return b;
}

}  // namespace

namespace {
std::mutex g_live_mutex;
std::unordered_map<slaq_graph, uint64_t> g_live;  // handles not yet freed -> uid
uint64_t g_next_uid = 1;
}  // namespace

void graph_register(slaq_graph g) {
  std::lock_guard<std::mutex> lk(g_live_mutex);
  g->uid = g_next_uid++;
  g_live[g] = g->uid;
}

bool graph_alive(slaq_graph g, uint64_t uid) {
  std::lock_guard<std::mutex> lk(g_live_mutex);
  const auto it = g_live.find(g);
  return it != g_live.end() && it->second == uid;
}

void graph_free(slaq_graph g, cudaStream_t st) {
  if (!g) return;
  {
    std::lock_guard<std::mutex> lk(g_live_mutex);
    g_live.erase(g);
  }
  void *ptrs[] = {g->rowptr, g->colidx, g->vals, g->vals32, g->diag, g->scale, g->diag32,
                  g->scale32, g->old_id, g->heavy_row, g->heavy_first, g->chunk_slot,
                  g->x_rowptr, g->x_colidx, g->x_vals, g->x_vals32, g->x_diag, g->x_scale,
                  g->x_diag32, g->x_scale32, g->x_old_id, g->goff_dev, g->gn_dev,
                  g->gtrace_dev, g->gbound_dev, g->x_graph, g->gtrace2_dev};
  for (void *p : ptrs) dfree(p, st);
  delete g;
}

namespace {
// Temporaries released on every exit path (stream-ordered frees).
struct Temps {
  cudaStream_t st;
  std::vector<void *> ptrs;
  explicit Temps(cudaStream_t s) : st(s) {}
  template <typename T>
  int get(T **p, size_t count) {
    int r = dalloc_t(p, std::max<size_t>(count, 1), st);
    if (r == SLAQ_OK) ptrs.push_back(*p);
    return r;
  }
  ~Temps() {
    for (void *p : ptrs) dfree(p, st);
  }
};

template <typename T>
int persistent(T **p, size_t count, cudaStream_t st) {
  // stream-ordered, from the device pool that keeps freed blocks cached: a
  // build of the same size reuses the last build's memory without a driver
  // allocation (graph_free returns it the same way)
  return dalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T), st);
}
}  // namespace

// SpMM schedule for rows of the execution copy with more than heavy_degree
// entries: each is split into chunks of kHeavyChunk entries.
static int heavy_schedule(slaq_graph g, Temps &tmp, cudaStream_t st) {
  int64_t *d_total = nullptr;
  SLAQ_TRY(tmp.get(&d_total, 1));
  g->heavy_degree = 4 * kHeavyChunk;
  if (g->n > 0) {
    int32_t *is_heavy = nullptr;
    int64_t *nchunk = nullptr, *slot_of = nullptr, *chunk_of = nullptr;
    SLAQ_TRY(tmp.get(&is_heavy, g->n));
    SLAQ_TRY(tmp.get(&nchunk, g->n));
    SLAQ_TRY(tmp.get(&slot_of, g->n));
    SLAQ_TRY(tmp.get(&chunk_of, g->n));
    ++tl_launches;
    k_heavy_flags<<<grid_for(g->n, 256), 256, 0, st>>>(g->x_rowptr, g->n, g->heavy_degree,
                                                        is_heavy, nchunk);
    SLAQ_CHECK_LAUNCH("heavy_flags");
    SLAQ_TRY(exclusive_scan(is_heavy, g->n, slot_of, d_total, st));
    SLAQ_TRY(to_host(&g->n_heavy, d_total, 1, st));
    SLAQ_TRY(exclusive_scan(nchunk, g->n, chunk_of, d_total, st));
    SLAQ_TRY(to_host(&g->n_chunks, d_total, 1, st));
    if (g->n_heavy > 0) {
      SLAQ_TRY(persistent(&g->heavy_row, g->n_heavy, st));
      SLAQ_TRY(persistent(&g->heavy_first, g->n_heavy + 1, st));
      SLAQ_TRY(persistent(&g->chunk_slot, g->n_chunks, st));
      ++tl_launches;
      k_heavy_table<<<grid_for(g->n, 256), 256, 0, st>>>(is_heavy, slot_of, chunk_of, nchunk,
                                                          g->n, g->n_heavy, g->n_chunks,
                                                          g->heavy_row, g->heavy_first,
                                                          g->chunk_slot);
      SLAQ_CHECK_LAUNCH("heavy_table");
    }
  }
  return SLAQ_OK;
}

int build_laplacian(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                    const double *weights, int kind, int flags, cudaStream_t st,
                    slaq_graph *out, int n_graphs, const int64_t *edge_off_host,
                    const int64_t *node_off_host) {
  if (!out) return set_error(SLAQ_EINVAL, "out is NULL");
  const bool batch = n_graphs > 1 || edge_off_host || node_off_host;
  std::vector<int64_t> node_off{0, n};
  if (batch) {
    // 65535: per-graph launches put the graph on a grid's y or z axis
    if (n_graphs < 1 || n_graphs > 65535 || !edge_off_host || !node_off_host)
      return set_error(SLAQ_EINVAL, "a batch needs 1..65535 graphs and both offset arrays");
    if (edge_off_host[0] != 0 || node_off_host[0] != 0)
      return set_error(SLAQ_EINVAL, "offsets must start at 0");
    for (int g = 0; g < n_graphs; ++g) {
      if (edge_off_host[g + 1] < edge_off_host[g] || node_off_host[g + 1] <= node_off_host[g])
        return set_error(SLAQ_EINVAL, "graph %d: offsets must increase (every graph needs a node)", g);
    }
    m = edge_off_host[n_graphs];
    n = node_off_host[n_graphs];
    node_off.assign(node_off_host, node_off_host + n_graphs + 1);
  }
  const int G = batch ? n_graphs : 1;
  *out = nullptr;
  if (n < 0 || m < 0) return set_error(SLAQ_EINVAL, "negative n_nodes or n_edges");
  if (kind != SLAQ_NORMALIZED && kind != SLAQ_COMBINATORIAL)
    return set_error(SLAQ_EINVAL, "unknown Laplacian kind %d", kind);
  if (flags & ~SLAQ_DROP_ISOLATED) return set_error(SLAQ_EINVAL, "unknown flags 0x%x", flags);
  if (n > 0x7fffffffLL) return set_error(SLAQ_EUNSUPPORTED, "n_nodes must be < 2^31");
  if (m > 0 && (!src || !dst)) return set_error(SLAQ_EINVAL, "src/dst is NULL");
  if (m > (1ll << 34)) return set_error(SLAQ_EUNSUPPORTED, "too many edges");
  const bool drop = (flags & SLAQ_DROP_ISOLATED) != 0;
  const bool weighted = weights != nullptr;
  ProfScope prof(SLAQ_PROF_BUILD, st);
  Temps tmp(st);

  // 1. validate (batches: local ids per graph, converted to union ids)
  int64_t *d_node_off = nullptr;
  SLAQ_TRY(tmp.get(&d_node_off, G + 1));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(d_node_off, node_off.data(), (G + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, st));
  unsigned long long n_loops = 0;
  // keys are row << cs | column, with graph-local columns in a batch (fewer
  // sort bits); csrc / cdst hold the ids that go into the column field
  const int32_t *csrc = src, *cdst = dst;
  if (m > 0) {
    int32_t *bad = nullptr;
    unsigned long long *loops = nullptr;
    SLAQ_TRY(tmp.get(&bad, 1));
    SLAQ_TRY(tmp.get(&loops, 1));
    SLAQ_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    SLAQ_CHECK_CUDA(cudaMemsetAsync(loops, 0, sizeof(unsigned long long), st));
    if (batch) {
      std::vector<EdgeChunk> chunks;
      for (int g = 0; g < G; ++g)
        for (int64_t e = edge_off_host[g]; e < edge_off_host[g + 1]; e += kEdgeChunk)
          chunks.push_back({e, (int32_t)g,
                            (int32_t)std::min<int64_t>(kEdgeChunk, edge_off_host[g + 1] - e)});
      EdgeChunk *d_chunks = nullptr;
      int32_t *usrc = nullptr, *udst = nullptr;
      SLAQ_TRY(tmp.get(&d_chunks, std::max<int64_t>(1, (int64_t)chunks.size())));
      SLAQ_TRY(tmp.get(&usrc, m));
      SLAQ_TRY(tmp.get(&udst, m));
      // pageable source: staged before the call returns
      SLAQ_CHECK_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(EdgeChunk),
                                      cudaMemcpyHostToDevice, st));
      ++tl_launches;
      k_union_ids<<<(unsigned)chunks.size(), 256, 0, st>>>(src, dst, weights, d_chunks, d_node_off,
                                                          usrc, udst, bad, loops);
      src = usrc;
      dst = udst;  // csrc / cdst keep the local ids
    } else {
      ++tl_launches;
      k_validate<<<grid_for(m, 256), 256, 0, st>>>(src, dst, weights, m, n, bad, loops);
    }
    SLAQ_CHECK_LAUNCH("validate");
    int32_t hbad = 0;
    SLAQ_TRY(to_host(&hbad, bad, 1, st));
    if (hbad & 1) return set_error(SLAQ_EINVAL, "edge endpoint outside [0, n_nodes)");
    if (hbad & 2) return set_error(SLAQ_EINVAL, "edge weights must be positive");
    SLAQ_TRY(to_host(&n_loops, loops, 1, st));
  }

  // 2. emit and sort
  const int cb = bits_for(n);
  int cs = cb;
  int64_t *rowbase = nullptr;
  if (batch) {
    int64_t gmax = 1;
    for (int g = 0; g < G; ++g) gmax = std::max(gmax, node_off[g + 1] - node_off[g]);
    cs = bits_for(gmax);
    SLAQ_TRY(tmp.get(&rowbase, n));
    ++tl_launches;
    k_row_base<<<grid_for(n, 256), 256, 0, st>>>(d_node_off, G, n, rowbase);
    SLAQ_CHECK_LAUNCH("row_base");
  }
  uint64_t *k0 = nullptr, *k1 = nullptr;
  double *p0 = nullptr, *p1 = nullptr;
  unsigned long long *counter = nullptr;
  SLAQ_TRY(tmp.get(&k0, 2 * m));
  SLAQ_TRY(tmp.get(&k1, 2 * m));
  if (weighted) {
    SLAQ_TRY(tmp.get(&p0, 2 * m));
    SLAQ_TRY(tmp.get(&p1, 2 * m));
  }
  SLAQ_TRY(tmp.get(&counter, 1));
  SLAQ_CHECK_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  if (m > 0 && n_loops == 0) {
    ++tl_launches;
    k_emit_direct<<<grid_for(m, 256), 256, 0, st>>>(src, dst, csrc, cdst, weights, m, cs, k0, p0);
    SLAQ_CHECK_LAUNCH("emit");
  } else if (m > 0) {
    ++tl_launches;
    k_emit<<<grid_for(m, 256), 256, 0, st>>>(src, dst, csrc, cdst, weights, m, cs, k0, p0, counter);
    SLAQ_CHECK_LAUNCH("emit");
  }
  const int64_t m2 = 2 * (m - (int64_t)n_loops);
  {
    uint64_t *ka = k0, *kb = k1;
    double *pa = p0, *pb = p1;
    SLAQ_TRY(radix_sort(&ka, &kb, weighted ? &pa : nullptr, &pb, m2, cb + cs, st));
    k0 = ka;
    k1 = kb;
    p0 = pa;
    p1 = pb;
  }

  // 3. merge duplicates, rows
  const int64_t nut = std::max<int64_t>(1, ceil_div(m2, kScanTile));
  int64_t *ubsum = nullptr, *d_total = nullptr;
  SLAQ_TRY(tmp.get(&ubsum, nut));
  SLAQ_TRY(tmp.get(&d_total, 1));
  if (m2 > 0) {
    ++tl_launches;
    k_unique_count<<<(unsigned)nut, kScanThreads, 0, st>>>(k0, m2, ubsum);
  } else {
    SLAQ_CHECK_CUDA(cudaMemsetAsync(ubsum, 0, sizeof(int64_t), st));
  }
  ++tl_launches;
  k_scan_tile_prefix<<<1, 1024, 0, st>>>(ubsum, nut, d_total);
  SLAQ_CHECK_LAUNCH("unique_count");
  int64_t nnz = 0;
  SLAQ_TRY(to_host(&nnz, d_total, 1, st));
  uint64_t *ukey = k1;  // the sort's spare buffer
  double *uw = weighted ? p1 : nullptr;
  if (m2 > 0) {
    ++tl_launches;
    k_unique_compact<<<(unsigned)nut, kScanThreads, 0, st>>>(k0, weighted ? p0 : nullptr, m2,
                                                              ubsum, ukey, uw);
    SLAQ_CHECK_LAUNCH("unique");
  }
  int64_t *rowptr_full = nullptr;
  double *deg_full = nullptr;
  uint8_t *keep = nullptr;
  SLAQ_TRY(tmp.get(&rowptr_full, n + 1));
  SLAQ_TRY(tmp.get(&deg_full, n));
  SLAQ_TRY(tmp.get(&keep, n));
  ++tl_launches;
  k_rowptr<<<grid_for(nnz + 1, 256), 256, 0, st>>>(ukey, nnz, cs, n, rowptr_full);
  SLAQ_CHECK_LAUNCH("rowptr");
  if (n > 0) {
    ++tl_launches;
    k_degree<<<grid_for(n, 256), 256, 0, st>>>(rowptr_full, uw, n, deg_full, keep);
    SLAQ_CHECK_LAUNCH("degree");
  }

  // 4. isolated nodes, renumbering
  int64_t *newid = nullptr;
  SLAQ_TRY(tmp.get(&newid, n));
  SLAQ_TRY(exclusive_scan(keep, n, newid, d_total, st));
  int64_t n_nonisolated = 0;
  SLAQ_TRY(to_host(&n_nonisolated, d_total, 1, st));
  const int64_t n_out = drop ? n_nonisolated : n;

  slaq_graph g = new slaq_graph_s();
  graph_register(g);
  struct Guard {
    slaq_graph *g;
    cudaStream_t st;
    ~Guard() {
      if (*g) graph_free(*g, st);
    }
  } guard{&g, st};
  SLAQ_CHECK_CUDA(cudaGetDevice(&g->device));
  g->n_input = n;
  g->n = n_out;
  g->nnz = nnz;
  g->kind = kind;
  g->flags = flags;
  g->weighted = weighted;
  SLAQ_TRY(persistent(&g->rowptr, n_out + 1, st));
  SLAQ_TRY(persistent(&g->colidx, nnz, st));
  SLAQ_TRY(persistent(&g->vals, nnz, st));
  if (weighted) SLAQ_TRY(persistent(&g->vals32, nnz, st));
  SLAQ_TRY(persistent(&g->diag, n_out, st));
  SLAQ_TRY(persistent(&g->scale, n_out, st));
  SLAQ_TRY(persistent(&g->diag32, n_out, st));
  SLAQ_TRY(persistent(&g->scale32, n_out, st));
  SLAQ_TRY(persistent(&g->old_id, n_out, st));
  double *deg = nullptr;
  SLAQ_TRY(tmp.get(&deg, n_out));
  ++tl_launches;
  k_compact_nodes<<<grid_for(n, 256), 256, 0, st>>>(rowptr_full, deg_full, keep, newid, n,
                                                    drop ? 1 : 0, nnz, n_out, g->rowptr, deg,
                                                    g->old_id);
  SLAQ_CHECK_LAUNCH("compact_nodes");
  if (n_out > 0) {
    ++tl_launches;
    k_scale<<<grid_for(n_out, 256), 256, 0, st>>>(deg, n_out, kind, g->scale, g->diag,
                                                  g->scale32, g->diag32);
    SLAQ_CHECK_LAUNCH("scale");
    ++tl_launches;
    k_values<<<grid_for(nnz, 256), 256, 0, st>>>(ukey, uw, newid, drop ? 1 : 0, cs, rowbase, nnz,
                                                 kind, g->scale, g->colidx, g->vals, g->vals32);
    SLAQ_CHECK_LAUNCH("values");
  }

  // per-graph bookkeeping: graph of each kept node, kept counts, traces, bounds
  int32_t *gid = nullptr;
  int64_t *local = nullptr;
  // [5][G]: kept, non-isolated, degree sum, max degree, stored entries
  unsigned long long *stats = nullptr;
  SLAQ_TRY(tmp.get(&gid, n_out));
  SLAQ_TRY(tmp.get(&local, n_out));
  SLAQ_TRY(tmp.get(&stats, 5 * (size_t)G));
  SLAQ_CHECK_CUDA(cudaMemsetAsync(stats, 0, 5 * (size_t)G * sizeof(unsigned long long), st));
  if (n_out > 0) {
    ++tl_launches;
    k_node_graph<<<(unsigned)ceil_div(n_out, 256), 256, 0, st>>>(
        g->old_id, deg, g->rowptr, n_out, d_node_off, G, gid, local, stats, stats + G,
        stats + 2 * G, stats + 3 * G, stats + 4 * G);
    SLAQ_CHECK_LAUNCH("node_graph");
  }
  std::vector<unsigned long long> hst(5 * (size_t)G);
  SLAQ_TRY(to_host(hst.data(), stats, 5 * (size_t)G, st));
  g->n_graphs = G;
  g->goff.assign(G + 1, 0);
  g->gtrace.assign(G, 0.0);
  g->gbound.assign(G, 0.0);
  for (int q = 0; q < G; ++q) {
    g->goff[q + 1] = g->goff[q] + (int64_t)hst[q];
    const double mx = __builtin_bit_cast(double, (long long)hst[3 * G + q]);
    if (kind == SLAQ_NORMALIZED) {
      g->gtrace[q] = (double)hst[G + q];
      g->gbound[q] = 2.0;
    } else {
      g->gtrace[q] = (double)hst[2 * G + q];  // integer degrees: exact
      g->gbound[q] = 2.0 * mx;
    }
  }
  if (kind == SLAQ_COMBINATORIAL && weighted) {
    // weighted degrees: Neumaier-compensated sums on the host, graph by graph
    std::vector<double> hdeg(n_out);
    if (n_out > 0) SLAQ_TRY(to_host(hdeg.data(), deg, n_out, st));
    for (int q = 0; q < G; ++q) {
      double sm = 0.0, c = 0.0;
      for (int64_t i = g->goff[q]; i < g->goff[q + 1]; ++i) {
        const double d = hdeg[i];
        const double t = sm + d;
        c += std::fabs(sm) >= std::fabs(d) ? (sm - t) + d : (d - t) + sm;
        sm = t;
      }
      g->gtrace[q] = sm + c;
    }
  }
  g->trace = g->gtrace[0];
  g->bound = *std::max_element(g->gbound.begin(), g->gbound.end());
  {
    std::vector<double> gn(G);
    for (int q = 0; q < G; ++q) gn[q] = (double)(g->goff[q + 1] - g->goff[q]);
    SLAQ_TRY(persistent(&g->goff_dev, G + 1, st));
    SLAQ_TRY(persistent(&g->gn_dev, G, st));
    SLAQ_TRY(persistent(&g->gtrace_dev, G, st));
    SLAQ_TRY(persistent(&g->gbound_dev, G, st));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->goff_dev, g->goff.data(), (G + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gn_dev, gn.data(), G * sizeof(double), cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gtrace_dev, g->gtrace.data(), G * sizeof(double),
                               cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gbound_dev, g->gbound.data(), G * sizeof(double),
                               cudaMemcpyHostToDevice));
    // tr(L_g^2) for the polynomial control variate of the heat trace
    SLAQ_TRY(persistent(&g->gtrace2_dev, G, st));
    // offs = [coff | eoff]: first chunk and first stored entry of every graph
    std::vector<int64_t> offs(2 * ((size_t)G + 1), 0);
    int64_t *coff = offs.data(), *eoff = coff + G + 1;
    for (int q = 0; q < G; ++q) {
      const int64_t e = (int64_t)hst[4 * (size_t)G + q];
      eoff[q + 1] = eoff[q] + e;
      coff[q + 1] = coff[q] + ceil_div(g->goff[q + 1] - g->goff[q], kSqChunk) + ceil_div(e, kSqChunk);
    }
    if (eoff[G] != nnz)
      return set_error(SLAQ_EINVAL, "internal: stored entries per graph sum to %lld, not %lld",
                       (long long)eoff[G], (long long)nnz);
    const int64_t n_chunks = coff[G];
    int64_t *d_offs = nullptr;
    double *partial = nullptr;
    SLAQ_TRY(tmp.get(&d_offs, offs.size()));
    SLAQ_TRY(tmp.get(&partial, std::max<int64_t>(n_chunks, 1)));
    SLAQ_CHECK_CUDA(cudaMemcpy(d_offs, offs.data(), offs.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice));
    if (n_chunks > 0) {
      ++tl_launches;
      k_graph_sq_chunks<<<(unsigned)n_chunks, kSqThreads, 0, st>>>(
          g->vals, g->diag, g->goff_dev, d_offs + G + 1, d_offs, G, partial);
      SLAQ_CHECK_LAUNCH("graph_sq_chunks");
    }
    ++tl_launches;
    k_graph_sq_sum<<<(unsigned)G, kSqThreads, 0, st>>>(partial, d_offs, g->gtrace2_dev);
    SLAQ_CHECK_LAUNCH("graph_sq_sum");
    g->gtrace2.assign(G, 0.0);
    SLAQ_TRY(to_host(g->gtrace2.data(), g->gtrace2_dev, G, st));
  }

  // 5. execution copy: graph-major, then descending degree, then id
  SLAQ_TRY(persistent(&g->x_rowptr, n_out + 1, st));
  SLAQ_TRY(persistent(&g->x_colidx, nnz, st));
  // the SpMM reads values only in the weighted form; unweighted graphs run the
  // pattern form from the scales, so their execution copy keeps no values
  if (weighted) SLAQ_TRY(persistent(&g->x_vals, nnz, st));
  if (weighted) SLAQ_TRY(persistent(&g->x_vals32, nnz, st));
  SLAQ_TRY(persistent(&g->x_diag, n_out, st));
  SLAQ_TRY(persistent(&g->x_scale, n_out, st));
  SLAQ_TRY(persistent(&g->x_diag32, n_out, st));
  SLAQ_TRY(persistent(&g->x_scale32, n_out, st));
  SLAQ_TRY(persistent(&g->x_old_id, n_out, st));
  SLAQ_TRY(persistent(&g->x_graph, n_out, st));
  if (n_out > 0) {
    const int pcb = bits_for(n_out);
    const int pdb = bits_for(n_out + 1);
    const int pgb = G > 1 ? bits_for(G) : 0;
    if (pcb + pdb + pgb > 64) return set_error(SLAQ_EUNSUPPORTED, "batch too large to order");
    uint64_t *pk0 = nullptr, *pk1 = nullptr;
    int64_t *perm = nullptr, *inv = nullptr, *xcnt = nullptr;
    SLAQ_TRY(tmp.get(&pk0, n_out));
    SLAQ_TRY(tmp.get(&pk1, n_out));
    SLAQ_TRY(tmp.get(&perm, n_out));
    SLAQ_TRY(tmp.get(&inv, n_out));
    SLAQ_TRY(tmp.get(&xcnt, n_out));
    ++tl_launches;
    k_perm_keys<<<grid_for(n_out, 256), 256, 0, st>>>(g->rowptr, gid, n_out, pcb, pdb, pk0);
    SLAQ_CHECK_LAUNCH("perm_keys");
    SLAQ_TRY(radix_sort(&pk0, &pk1, nullptr, nullptr, n_out, pcb + pdb + pgb, st));
    ++tl_launches;
    k_perm_index<<<grid_for(n_out, 256), 256, 0, st>>>(pk0, g->rowptr, n_out, pcb, perm, inv, xcnt);
    SLAQ_CHECK_LAUNCH("perm_index");
    SLAQ_TRY(exclusive_scan(xcnt, n_out, g->x_rowptr, d_total, st));
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(g->x_rowptr + n_out, d_total, sizeof(int64_t),
                                    cudaMemcpyDeviceToDevice, st));
    if (nnz > 0) {
      ++tl_launches;
      k_perm_entries<<<grid_for(nnz, 256), 256, 0, st>>>(
          ukey, newid, drop ? 1 : 0, cs, g->rowptr, g->colidx, g->vals, g->vals32, inv, nnz,
          g->x_rowptr, g->x_colidx, g->x_vals, g->x_vals32);
    }
    ++tl_launches;
    k_perm_nodes<<<grid_for(n_out, 256), 256, 0, st>>>(g->diag, g->scale, local, gid, perm, n_out,
                                                       g->x_diag, g->x_scale, g->x_diag32,
                                                       g->x_scale32, g->x_old_id, g->x_graph);
    SLAQ_CHECK_LAUNCH("perm");
  } else {
    SLAQ_CHECK_CUDA(cudaMemsetAsync(g->x_rowptr, 0, sizeof(int64_t), st));
  }

  // 6. SpMM schedule for heavy rows (execution order)
  SLAQ_TRY(heavy_schedule(g, tmp, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  *out = g;
  g = nullptr;  // ownership passed to the caller
  return SLAQ_OK;
}


// --------------------------------------------------------------- unions
namespace {
// One block per chunk of one part: dst[dst0 + i] = src[part][src0 + i] + add
// for i < len (coalesced copies, no search for the part).
struct ConcatChunk {
  int64_t src0, dst0;
  int32_t part, len;
};
constexpr int kConcatChunk = 8192;

template <typename T>
__global__ void k_concat(const T *const *src, const ConcatChunk *chunks, const T *add, T *dst) {
  const ConcatChunk c = chunks[blockIdx.x];
  const T *s = src[c.part] + c.src0;
  const T a = add ? add[c.part] : T(0);
  T *d = dst + c.dst0;
  for (int i = threadIdx.x; i < c.len; i += blockDim.x) d[i] = s[i] + a;
}

// Concatenates one array over the parts: part h contributes count[h]
// elements of srcs[h], each plus add[h] (no addend if add is empty).
template <typename T>
int concat(Temps &tmp, const std::vector<const T *> &srcs, const std::vector<int64_t> &count,
           const std::vector<T> &add, T *dst, cudaStream_t st) {
  const int parts = (int)srcs.size();
  std::vector<ConcatChunk> chunks;
  int64_t off = 0;
  for (int h = 0; h < parts; ++h) {
    for (int64_t q = 0; q < count[h]; q += kConcatChunk)
      chunks.push_back({q, off + q, (int32_t)h, (int32_t)std::min<int64_t>(kConcatChunk, count[h] - q)});
    off += count[h];
  }
  if (chunks.empty()) return SLAQ_OK;
  if (chunks.size() > 0x7fffffffu) return set_error(SLAQ_EUNSUPPORTED, "batch too large to concatenate");
  const T **d_src = nullptr;
  ConcatChunk *d_chunks = nullptr;
  T *d_add = nullptr;
  SLAQ_TRY(tmp.get(&d_src, parts));
  SLAQ_TRY(tmp.get(&d_chunks, (int64_t)chunks.size()));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(d_src, srcs.data(), parts * sizeof(T *), cudaMemcpyHostToDevice, st));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(ConcatChunk),
                                  cudaMemcpyHostToDevice, st));
  if (!add.empty()) {
    SLAQ_TRY(tmp.get(&d_add, parts));
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(d_add, add.data(), parts * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  ++tl_launches;
  k_concat<T><<<(unsigned)chunks.size(), 256, 0, st>>>(d_src, d_chunks, d_add, dst);
  SLAQ_CHECK_LAUNCH("concat");
  // the host vectors are staged before the copies from pageable memory return
  return SLAQ_OK;
}
}  // namespace

int union_graphs(const slaq_graph *gs, int count, cudaStream_t st, slaq_graph *out) {
  if (!out) return set_error(SLAQ_EINVAL, "out is NULL");
  *out = nullptr;
  if (!gs || count < 1) return set_error(SLAQ_EINVAL, "need at least one graph");
  int dev = 0;
  SLAQ_CHECK_CUDA(cudaGetDevice(&dev));
  int64_t G = 0;
  for (int h = 0; h < count; ++h) {
    const slaq_graph a = gs[h];
    if (!a) return set_error(SLAQ_EINVAL, "graph %d is NULL", h);
    if (a->device != dev) return set_error(SLAQ_EINVAL, "graph %d lives on another device", h);
    if (a->kind != gs[0]->kind || a->weighted != gs[0]->weighted)
      return set_error(SLAQ_EINVAL, "graph %d: all graphs need one Laplacian kind and all or "
                       "none weighted", h);
    G += a->n_graphs;
  }
  if (G > 65535) return set_error(SLAQ_EINVAL, "a batch holds at most 65535 graphs");
  Temps tmp(st);
  slaq_graph g = new slaq_graph_s();
  graph_register(g);
  struct Guard {
    slaq_graph *g;
    cudaStream_t st;
    ~Guard() {
      if (*g) graph_free(*g, st);
    }
  } guard{&g, st};
  g->device = dev;
  g->kind = gs[0]->kind;
  g->flags = gs[0]->flags;
  g->weighted = gs[0]->weighted;
  g->n_graphs = (int)G;
  g->goff.assign(1, 0);
  std::vector<int64_t> n_of(count), nnz_of(count), np1_of(count);
  std::vector<int64_t> entry_add(count);
  std::vector<int32_t> col_add(count), graph_add(count);
  int64_t n = 0, nnz = 0, n_in = 0;
  int32_t gfirst = 0;
  for (int h = 0; h < count; ++h) {
    const slaq_graph a = gs[h];
    n_of[h] = a->n;
    nnz_of[h] = a->nnz;
    np1_of[h] = a->n;  // rowptr: the first n entries of each part, the end appended
    col_add[h] = (int32_t)n;
    entry_add[h] = nnz;
    graph_add[h] = gfirst;
    for (int q = 0; q < a->n_graphs; ++q) {
      g->goff.push_back(n + a->goff[q + 1]);
      g->gtrace.push_back(a->gtrace[q]);
      g->gtrace2.push_back(a->gtrace2[q]);
      g->gbound.push_back(a->gbound[q]);
    }
    n += a->n;
    nnz += a->nnz;
    n_in += a->n_input;
    gfirst += a->n_graphs;
  }
  if (n > 0x7fffffffLL) return set_error(SLAQ_EUNSUPPORTED, "more than 2^31 - 1 nodes in a batch");
  g->n = n;
  g->nnz = nnz;
  g->n_input = n_in;
  g->trace = g->gtrace[0];
  g->bound = *std::max_element(g->gbound.begin(), g->gbound.end());
  const bool w = g->weighted;
  // The union lives inside slaq_lanczos_batched's Krylov handle and is never
  // exported: it carries the execution copy and the per-graph scalars only,
  // not the canonical CSR.
  SLAQ_TRY(persistent(&g->x_rowptr, n + 1, st));
  SLAQ_TRY(persistent(&g->x_colidx, nnz, st));
  if (w) SLAQ_TRY(persistent(&g->x_vals, nnz, st));
  if (w) SLAQ_TRY(persistent(&g->x_vals32, nnz, st));
  SLAQ_TRY(persistent(&g->x_diag, n, st));
  SLAQ_TRY(persistent(&g->x_scale, n, st));
  SLAQ_TRY(persistent(&g->x_diag32, n, st));
  SLAQ_TRY(persistent(&g->x_scale32, n, st));
  SLAQ_TRY(persistent(&g->x_old_id, n, st));
  SLAQ_TRY(persistent(&g->x_graph, n, st));
  auto ptrs = [&](auto field) {
    using T = std::remove_pointer_t<std::remove_reference_t<decltype(gs[0]->*field)>>;
    std::vector<const T *> v(count);
    for (int h = 0; h < count; ++h) v[h] = gs[h]->*field;
    return v;
  };
  const std::vector<double> no_d;
  const std::vector<float> no_f;
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_rowptr), np1_of, entry_add, g->x_rowptr, st));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(g->x_rowptr + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_colidx), nnz_of, col_add, g->x_colidx, st));
  if (w) SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_vals), nnz_of, no_d, g->x_vals, st));
  if (w) SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_vals32), nnz_of, no_f, g->x_vals32, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_diag), n_of, no_d, g->x_diag, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_scale), n_of, no_d, g->x_scale, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_diag32), n_of, no_f, g->x_diag32, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_scale32), n_of, no_f, g->x_scale32, st));
  // execution ids stay local to their graph (the probe signs), graph numbers
  // are shifted
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_old_id), n_of, std::vector<int64_t>(), g->x_old_id, st));
  SLAQ_TRY(concat(tmp, ptrs(&slaq_graph_s::x_graph), n_of, graph_add, g->x_graph, st));
  {
    std::vector<double> gn(G);
    for (int64_t q = 0; q < G; ++q) gn[q] = (double)(g->goff[q + 1] - g->goff[q]);
    SLAQ_TRY(persistent(&g->goff_dev, G + 1, st));
    SLAQ_TRY(persistent(&g->gn_dev, G, st));
    SLAQ_TRY(persistent(&g->gtrace_dev, G, st));
    SLAQ_TRY(persistent(&g->gbound_dev, G, st));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->goff_dev, g->goff.data(), (G + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gn_dev, gn.data(), G * sizeof(double), cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gtrace_dev, g->gtrace.data(), G * sizeof(double),
                               cudaMemcpyHostToDevice));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gbound_dev, g->gbound.data(), G * sizeof(double),
                               cudaMemcpyHostToDevice));
    SLAQ_TRY(persistent(&g->gtrace2_dev, G, st));
    SLAQ_CHECK_CUDA(cudaMemcpy(g->gtrace2_dev, g->gtrace2.data(), G * sizeof(double),
                               cudaMemcpyHostToDevice));
  }
  SLAQ_TRY(heavy_schedule(g, tmp, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  *out = g;
  g = nullptr;
  return SLAQ_OK;
}

}  // namespace slaq
