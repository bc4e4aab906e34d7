// Gather ceiling of this GPU for the SpMM's access pattern (profiling only;
// not part of the method).
//
// Every stored entry of L makes the SpMM gather one whole basis row (nv
// values) from L2: the rows are too many for shared memory and are reused by
// other rows only through L2.  So the SpMM is bound by how fast the L2 can
// serve row gathers to the SMs, far above the bytes that reach HBM.  This
// probe measures that ceiling directly: random gathers of row_bytes-wide rows
// from an L2-resident table (64 MiB, below the L2 capacity), one 16-byte
// vector per lane, the way the SpMM's light rows gather, summed so that no
// load is dead.  It is the denominator the SpMM's gathered bytes are set
// against, beside the HBM roofline of its algorithmic bytes.
#include <algorithm>

#include "common.cuh"

namespace slaq {
namespace {

constexpr int64_t kPeakTableBytes = 64ll << 20;
constexpr int64_t kPeakEntries = 32ll << 20;

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
  // SplitMix64 finalizer, low word (published mixing constants)
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)(x ^ (x >> 31));
}

// Warp w sums the rows of entries [w * per, (w + 1) * per); entry e gathers
// row mix32(e) % rows.  Lanes >= V (row_bytes / 16) idle.
__global__ void __launch_bounds__(256) k_gather_peak(const float4 *__restrict__ table, int64_t rows,
                                                     int V, int64_t per, int64_t nwarps,
                                                     float *__restrict__ sink) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nwarps || lane >= V) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t e0 = w * per;
  for (int64_t e = e0; e < e0 + per; e += 4) {
    float4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = mix32((uint64_t)(e + q)) % (uint64_t)rows;
      v[q] = __ldg(table + r * V + lane);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc.x += v[q].x;
      acc.y += v[q].y;
      acc.z += v[q].z;
      acc.w += v[q].w;
    }
  }
  if (acc.x == 1.234567f) sink[0] = acc.y + acc.z + acc.w;  // keeps the loads live
}

}  // namespace

int profile_gather_peak(int row_bytes, double *tbps) {
  if (row_bytes < 16 || row_bytes > 512 || row_bytes % 16)
    return set_error(SLAQ_EINVAL, "row_bytes must be a multiple of 16 in [16, 512]");
  const int V = row_bytes / 16;
  const int64_t rows = kPeakTableBytes / row_bytes;
  const int64_t nwarps = (int64_t)num_sms() * 64;  // full occupancy of 256-thread blocks
  const int64_t per = std::max<int64_t>(4, kPeakEntries / nwarps / 4 * 4);
  cudaStream_t st = nullptr;
  void *table = nullptr, *sink = nullptr;
  SLAQ_TRY(dmalloc(&table, (size_t)kPeakTableBytes));
  struct Free {
    void **a, **b;
    ~Free() {
      dmfree(*a);
      dmfree(*b);
    }
  } fr{&table, &sink};
  SLAQ_TRY(dmalloc(&sink, 16));
  SLAQ_CHECK_CUDA(cudaMemsetAsync(table, 0, (size_t)kPeakTableBytes, st));
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
  const unsigned blocks = (unsigned)(nwarps * 32 / 256);
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {  // the first run warms the L2
    SLAQ_CHECK_CUDA(cudaEventRecord(a, st));
    ++tl_launches;
    k_gather_peak<<<blocks, 256, 0, st>>>(static_cast<const float4 *>(table), rows, V, per, nwarps,
                                          static_cast<float *>(sink));
    SLAQ_CHECK_LAUNCH("gather_peak");
    SLAQ_CHECK_CUDA(cudaEventRecord(b, st));
    SLAQ_CHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    SLAQ_CHECK_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0) best = rep == 1 ? ms : std::min(best, ms);
  }
  *tbps = (double)(per * nwarps) * row_bytes / (best * 1e-3) / 1e12;
  return SLAQ_OK;
}

}  // namespace slaq
