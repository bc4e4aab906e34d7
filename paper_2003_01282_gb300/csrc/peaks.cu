// Gather ceiling of this GPU for the SpMM's access pattern (profiling only;
// not part of the method).
//
// Every stored entry of L makes the SpMM gather one whole basis row (nv
// values) from L2: the rows are too many for shared memory and are reused by
// other rows only through L2.  So the SpMM is bound by how fast the L2 can
// serve row gathers to the SMs, far above the bytes that reach HBM.  This
// probe measures that ceiling directly: random gathers of row_bytes-wide rows
// from an L2-resident table (64 MiB, below the L2 capacity) through a stream
// of row ids read four at a time, one 16-byte vector per lane, the way the
// SpMM's light rows gather, summed so that no load is dead.  It is the
// denominator the SpMM's gathered bytes are set against, beside the HBM
// roofline of its algorithmic bytes.
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace slaq {
namespace {

constexpr int64_t kPeakTableBytes = 64ll << 20;
constexpr int64_t kPeakEntries = 32ll << 20;

// Row ids of the entry stream, uniform over [0, rows): the murmur3 32-bit
// finalizer (published constants) of the entry index, scaled by rows with a
// multiply-high.  Written once, read as the SpMM reads its column ids.
__global__ void k_peak_ids(int32_t *__restrict__ ids, int64_t count, uint32_t rows) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)e;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    ids[e] = (int32_t)__umulhi(h, rows);
  }
}

// A team of Vp lanes (V = row_bytes / 16 rounded up to a power of two, the
// SpMM's packed row teams) sums the rows of its entries [team * per,
// (team + 1) * per), four ids per 16-byte load (streamed past L2), one
// 16-byte vector of each row per lane; lanes >= V of a team idle.
__global__ void __launch_bounds__(256) k_gather_peak(const float4 *__restrict__ table,
                                                     const int32_t *__restrict__ ids, int V, int Vp,
                                                     int64_t per, int64_t nteams,
                                                     float *__restrict__ sink) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t team = tid / Vp;
  const int lane = (int)(tid - team * Vp);
  if (team >= nteams || lane >= V) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int32_t *ix = ids + team * per;
  for (int64_t e = 0; e < per; e += 4) {
    const int4 c = __ldcs(reinterpret_cast<const int4 *>(ix + e));
    const float4 v0 = __ldg(table + (int64_t)c.x * V + lane);
    const float4 v1 = __ldg(table + (int64_t)c.y * V + lane);
    const float4 v2 = __ldg(table + (int64_t)c.z * V + lane);
    const float4 v3 = __ldg(table + (int64_t)c.w * V + lane);
    acc.x += (v0.x + v1.x) + (v2.x + v3.x);
    acc.y += (v0.y + v1.y) + (v2.y + v3.y);
    acc.z += (v0.z + v1.z) + (v2.z + v3.z);
    acc.w += (v0.w + v1.w) + (v2.w + v3.w);
  }
  if (acc.x == 1.234567f) sink[0] = acc.y + acc.z + acc.w;  // keeps the loads live
}

}  // namespace

int profile_gather_peak(int row_bytes, double *tbps) {
  if (row_bytes < 16 || row_bytes > 512 || row_bytes % 16)
    return set_error(SLAQ_EINVAL, "row_bytes must be a multiple of 16 in [16, 512]");
  const int V = row_bytes / 16;
  int Vp = 1;
  while (Vp < V) Vp *= 2;
  const int64_t rows = kPeakTableBytes / row_bytes;
  const int64_t threads = (int64_t)num_sms() * 64 * 32;  // full occupancy of 256-thread blocks
  const int64_t nteams = threads / Vp;
  const int64_t per = std::max<int64_t>(4, kPeakEntries / nteams / 4 * 4);
  cudaStream_t st = nullptr;
  void *table = nullptr, *sink = nullptr, *ids = nullptr;
  SLAQ_TRY(dmalloc(&table, (size_t)kPeakTableBytes));
  struct Free {
    void **a, **b, **c;
    ~Free() {
      dmfree(*a);
      dmfree(*b);
      dmfree(*c);
    }
  } fr{&table, &sink, &ids};
  SLAQ_TRY(dmalloc(&sink, 16));
  SLAQ_TRY(dmalloc(&ids, (size_t)(per * nteams) * sizeof(int32_t)));
  SLAQ_CHECK_CUDA(cudaMemsetAsync(table, 0, (size_t)kPeakTableBytes, st));
  ++tl_launches;
  k_peak_ids<<<(unsigned)(num_sms() * 16), 256, 0, st>>>(static_cast<int32_t *>(ids), per * nteams,
                                                         (uint32_t)rows);
  SLAQ_CHECK_LAUNCH("peak_ids");
  cudaEvent_t a = nullptr, b = nullptr;
  SLAQ_CHECK_CUDA(cudaEventCreate(&a));
  SLAQ_CHECK_CUDA(cudaEventCreate(&b));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{a, b};
  const unsigned blocks = (unsigned)(threads / 256);
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {  // the first run warms the L2
    SLAQ_CHECK_CUDA(cudaEventRecord(a, st));
    ++tl_launches;
    k_gather_peak<<<blocks, 256, 0, st>>>(static_cast<const float4 *>(table),
                                          static_cast<const int32_t *>(ids), V, Vp, per, nteams,
                                          static_cast<float *>(sink));
    SLAQ_CHECK_LAUNCH("gather_peak");
    SLAQ_CHECK_CUDA(cudaEventRecord(b, st));
    SLAQ_CHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    SLAQ_CHECK_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0) best = rep == 1 ? ms : std::min(best, ms);
  }
  *tbps = (double)(per * nteams) * row_bytes / (best * 1e-3) / 1e12;
  return SLAQ_OK;
}

}  // namespace slaq
