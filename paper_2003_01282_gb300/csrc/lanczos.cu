// s-step Lanczos over a block of nv probes (Sec. 3.1, Algorithm 1 `lanczos`)
// with full reorthogonalization.
//
// Every probe runs its own Lanczos process; all probes share one sparse
// matrix product per step.  Layout in HBM: the basis is U[j][i][p] (step j,
// node i, probe p innermost, row stride ld), so the gather of neighbour j in
// the SpMM reads one contiguous row of nv values.
//
// The basis is kept UNNORMALIZED (u_0 is the +-1 probe itself); q_j =
// u_j / ||u_j||.  Step k, for every probe:
//     z       = L u_k                                          (SpMM)
//     d_j     = u_j^T z,  G_jk = u_j^T u_k      j = 0..k       (dots)
//     x       = G^{-1} d  over the Gram matrix G of u_0..u_k    (solve)
//     alpha_k = d_k / G_kk = q_k^T L q_k,  beta_{k-1} = ||u_k|| = sqrt(G_kk)
//     u_{k+1} = (z - sum_j x_j u_j) / ||u_k||                  (update)
// u_{k+1} is beta_k q_{k+1}, the vector that "three-term recurrence, then
// Gram-Schmidt against q_0..q_k" produces before its normalization: both
// remove the projection of L q_k on span{q_0..q_k}.  Solving with the Gram
// matrix (accumulated in the dots pass, which reads u_k anyway) makes that
// projection exact for the stored, rounded basis, so orthogonality does not
// decay step by step (one classical Gram-Schmidt pass would lose it by a
// factor (alpha+beta)/beta per step).  Leaving the factor beta_k in the
// stored vector saves one pass over the basis per step, and dividing by
// ||u_k|| keeps the norms at beta (they would otherwise shrink or grow
// geometrically and leave the FP32 range within a few dozen steps).
#include <algorithm>
#include <atomic>
#include <limits>
#include <cmath>
#include <cstdlib>
#include <type_traits>

#include <cudaTypedefs.h>

#include "common.cuh"

namespace slaq {
namespace {

// ------------------------------------------------------------ form traits
template <int P>
struct Form;
template <>
struct Form<SLAQ_FP64> {
  using TB = double;
  using TW = double;
  static constexpr int VE = 2;  // probe columns per 16-byte basis vector
};
template <>
struct Form<SLAQ_FP32> {
  using TB = float;
  using TW = float;
  static constexpr int VE = 4;
};
template <>
struct Form<SLAQ_FP32_BF16BASIS> {
  using TB = __nv_bfloat16;
  using TW = float;
  static constexpr int VE = 8;
};

// Column slicing of a block of vectors [n][ld] (probe columns innermost):
// stored as consecutive [n][width_s] blocks, slice s holding columns
// [s*w, s*w + width_s), width_s = min(w, ld - s*w).  A slice of the basis is
// then contiguous, so the SpMM's gathers of one slice stay within an
// L2-sized footprint.  Offsets are in elements.
struct Slc {
  int64_t n;
  int ld, w;
  __host__ __device__ __forceinline__ int64_t base(int col, int &stride) const {
    const int sl = col / w;
    const int c0 = sl * w;
    stride = min(w, ld - c0);
    return (int64_t)sl * n * w + (col - c0);
  }
  __host__ __device__ __forceinline__ int nslices() const { return (ld + w - 1) / w; }
};

// 16-byte basis loads (read-only path) and stores, widened to TW.
__device__ __forceinline__ void ldb(const double *p, double (&v)[2]) {
  double2 t = __ldg(reinterpret_cast<const double2 *>(p));
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ldb(const float *p, float (&v)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void unpack_bf16x8(const uint4 &t, float (&v)[8]) {
  const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ void ldb(const __nv_bfloat16 *p, float (&v)[8]) {
  unpack_bf16x8(__ldg(reinterpret_cast<const uint4 *>(p)), v);
}
// coherent loads, for rows this kernel also writes (in-place second pass)
__device__ __forceinline__ void ldb_rw(const double *p, double (&v)[2]) {
  double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ldb_rw(const float *p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ldb_rw(const __nv_bfloat16 *p, float (&v)[8]) {
  uint4 t = *reinterpret_cast<const uint4 *>(p);
  const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
// round to the basis type; r receives the rounded values
__device__ __forceinline__ void stb(double *p, const double (&v)[2], double (&r)[2]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  r[0] = v[0];
  r[1] = v[1];
}
__device__ __forceinline__ void stb(float *p, const float (&v)[4], float (&r)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] = v[i];
}
__device__ __forceinline__ void stb(__nv_bfloat16 *p, const float (&v)[8], float (&r)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * i]);
    __nv_bfloat16 hi = __float2bfloat16_rn(v[2 * i + 1]);
    uint32_t l = __bfloat16_as_ushort(lo), h = __bfloat16_as_ushort(hi);
    w[i] = l | (h << 16);
    r[2 * i] = __uint_as_float(l << 16);
    r[2 * i + 1] = __uint_as_float(h << 16);
  }
  *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
// the 16-byte basis vector at p as raw bits (read-only path)
__device__ __forceinline__ uint4 ldraw(const void *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ void unpack(const uint4 &t, double (&v)[2]) {
  v[0] = __hiloint2double((int)t.y, (int)t.x);
  v[1] = __hiloint2double((int)t.w, (int)t.z);
}
__device__ __forceinline__ void unpack(const uint4 &t, float (&v)[4]) {
  v[0] = __uint_as_float(t.x);
  v[1] = __uint_as_float(t.y);
  v[2] = __uint_as_float(t.z);
  v[3] = __uint_as_float(t.w);
}
__device__ __forceinline__ void unpack(const uint4 &t, float (&v)[8]) { unpack_bf16x8(t, v); }

// work vectors (TW) of VE elements
template <typename TW, int VE>
__device__ __forceinline__ void ldw(const TW *p, TW (&v)[VE]) {
  static_assert(sizeof(TW) * VE % 16 == 0, "work vector must be whole 16-byte words");
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TW) * VE / 16); ++i) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
    reinterpret_cast<float4 *>(v)[i] = t;
  }
}
template <typename TW, int VE>
__device__ __forceinline__ void ldw_cg(const TW *p, TW (&v)[VE]) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TW) * VE / 16); ++i) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(p) + i);
    reinterpret_cast<float4 *>(v)[i] = t;
  }
}
template <typename TW, int VE>
__device__ __forceinline__ void stw(TW *p, const TW (&v)[VE]) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TW) * VE / 16); ++i)
    reinterpret_cast<float4 *>(p)[i] = reinterpret_cast<const float4 *>(v)[i];
}
// streaming (evict-first) store: the SpMM output must not push the gathered
// basis out of L2
template <typename TW, int VE>
__device__ __forceinline__ void stw_cs(TW *p, const TW (&v)[VE]) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(TW) * VE / 16); ++i)
    __stcs(reinterpret_cast<float4 *>(p) + i, reinterpret_cast<const float4 *>(v)[i]);
}

// ------------------------------------------------------------ probe init
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Column p of the block is generator probe probe0 + p (probe ranges split one
// seed's probes over several runs, e.g. one per GPU).
template <int P>
__global__ void k_probe_init(typename Form<P>::TB *U0, const int64_t *old_id,
                             const int32_t *xgraph, Slc S, int nv, const uint64_t *seed_p,
                             uint64_t graph_id, uint64_t probe0, const float *yscale, float *Y0) {
  using TB = typename Form<P>::TB;
  const uint64_t seed = *seed_p;  // in device memory, so that a captured run can be replayed
                                  // with another seed
  const int64_t n = S.n;
  const int ld = S.ld;
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ld;
    const int p = (int)(idx - i * ld);
    int stride;
    const int64_t cbase = S.base(p, stride);
    const int64_t off = cbase + i * stride;
    float v = 0.0f;
    if (p < nv) {
      const uint64_t gfield = (graph_id + (uint64_t)xgraph[i]) & 0xffffull;
      const uint64_t c = (gfield << 48) | (((uint64_t)p + probe0) << 32) | (uint64_t)old_id[i];
      const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * (c + 1ull));
      v = (z >> 63) ? -1.0f : 1.0f;
    }
    U0[off] = (TB)v;
    if (Y0) Y0[off] = yscale[i] * v;
  }
}

__global__ void k_probe_export(double *out, const int64_t *old_id, int64_t n, int nv,
                               uint64_t seed, uint64_t graph_id) {
  const int64_t total = n * nv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nv;
    const int p = (int)(idx - i * nv);
    const uint64_t c = (graph_id << 48) | ((uint64_t)p << 32) | (uint64_t)old_id[i];
    const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * (c + 1ull));
    out[idx] = (z >> 63) ? -1.0 : 1.0;
  }
}

// m = s for every (graph, probe), except m = 0 for a graph of a batch that
// kept no nodes (all isolated and dropped): its Krylov space is empty, and
// its traces and entropy come out 0.
__global__ void k_init_scalars(double *alpha, double *beta, int32_t *m, int64_t nvs, int64_t nvt,
                               int s, int nv, const double *gn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvs;
       i += (int64_t)gridDim.x * blockDim.x) {
    alpha[i] = 0.0;
    beta[i] = 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvt;
       i += (int64_t)gridDim.x * blockDim.x)
    m[i] = gn[i / nv] > 0.0 ? s : 0;
}

// ------------------------------------------------------------------ SpMM
// MODE 0: normalized, unweighted   z_i = diag_i u_i - s_i sum_j s_j u_j
// MODE 1: combinatorial, unweighted z_i = d_i u_i - sum_j u_j
// MODE 2: weighted                  z_i = diag_i u_i + sum_j val_ij u_j
// MODE 3: normalized, unweighted, with the gathered rows pre-scaled:
//         z_i = diag_i u_i - s_i sum_j y_j, y_j = s_j u_j written by the kernel
//         that produced u_k (FP32 form: saves the per-entry gather of s_j)
// s += w x, or Kahan-compensated (c carries the lost low part; true sum s - c)
template <bool COMP, typename T>
__device__ __forceinline__ void acc_add(T &s, T &c, T w, T x) {
  if (COMP) {
    const T y = fma(w, x, -c);
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s = fma(w, x, s);
  }
}

// COMP: compensated sums, for the split rows of the reduced forms (a row of
// thousands of entries whose sum nearly cancels, such as a hub's row against
// the null vector, otherwise loses about sqrt(entries) units of FP32 rounding)
// Every gather is loaded as raw 16 bytes and widened only when it is summed,
// so that four rows in flight per thread cost 16 registers whatever the form.
template <int P, int MODE, bool COMP = false>
__device__ __forceinline__ void gather_rows(const int32_t *__restrict__ col,
                                            const typename Form<P>::TW *__restrict__ vals,
                                            const typename Form<P>::TW *__restrict__ scale,
                                            const typename Form<P>::TB *__restrict__ Ul, int stride,
                                            int64_t b, int64_t e,
                                            typename Form<P>::TW (&acc)[Form<P>::VE]) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  TW cmp[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) cmp[v] = TW(0);
  auto row_ptr = [&](int c) { return (const void *)(Ul + (int64_t)c * stride); };
  int64_t j = b;
  // FP32: single entries up to a 16-byte boundary of col, then 4 indices per
  // load (measured faster for FP32, slower for the BF16 basis)
  constexpr bool kVecIdx = P == SLAQ_FP32;
  for (; kVecIdx && j < e && (j & 3); ++j) {
    const int c = __ldcs(col + j);
    const TW w = MODE == 0 ? __ldg(scale + c) : (MODE == 2 ? __ldcs(vals + j) : TW(1));
    TW x[VE];
    unpack(ldraw(row_ptr(c)), x);
#pragma unroll
    for (int v = 0; v < VE; ++v) acc_add<COMP>(acc[v], cmp[v], w, x[v]);
  }
  for (; j + 4 <= e; j += 4) {
    int c[4];
    if constexpr (kVecIdx) {
      const int4 c4 = __ldcs(reinterpret_cast<const int4 *>(col + j));  // streamed: keep L2 for the basis
      c[0] = c4.x;
      c[1] = c4.y;
      c[2] = c4.z;
      c[3] = c4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = __ldcs(col + j + q);
    }
    TW w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = MODE == 0 ? __ldg(scale + c[q]) : (MODE == 2 ? __ldcs(vals + j + q) : TW(1));
    uint4 raw[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) raw[q] = ldraw(row_ptr(c[q]));
    if (COMP) {
      // the group's four products summed plainly, then one compensated add
      TW x[4][VE];
#pragma unroll
      for (int q = 0; q < 4; ++q) unpack(raw[q], x[q]);
#pragma unroll
      for (int v = 0; v < VE; ++v) {
        TW g = w[0] * x[0][v];
#pragma unroll
        for (int q = 1; q < 4; ++q) g = fma(w[q], x[q][v], g);
        acc_add<true>(acc[v], cmp[v], TW(1), g);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        TW x[VE];
        unpack(raw[q], x);
#pragma unroll
        for (int v = 0; v < VE; ++v) acc_add<false>(acc[v], cmp[v], w[q], x[v]);
      }
    }
  }
  for (; j < e; ++j) {
    const int c = __ldcs(col + j);
    const TW w = MODE == 0 ? __ldg(scale + c) : (MODE == 2 ? __ldcs(vals + j) : TW(1));
    TW x[VE];
    unpack(ldraw(row_ptr(c)), x);
#pragma unroll
    for (int v = 0; v < VE; ++v) acc_add<COMP>(acc[v], cmp[v], w, x[v]);
  }
  if (COMP) {
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] -= cmp[v];
  }
}

template <int P, int MODE>
__device__ __forceinline__ void finish_row(int64_t row, const typename Form<P>::TW *diag,
                                           const typename Form<P>::TW *scale,
                                           const typename Form<P>::TB *Ul, int stride,
                                           typename Form<P>::TW (&acc)[Form<P>::VE],
                                           typename Form<P>::TW *zrow) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  TW y[VE];
  ldb(Ul + row * stride, y);
  const TW g = diag[row];
  const TW sr = (MODE == 0 || MODE == 3) ? scale[row] : TW(1);
  TW z[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v)
    z[v] = MODE == 2 ? fma(g, y[v], acc[v]) : fma(g, y[v], -sr * acc[v]);
  stw_cs<TW, VE>(zrow, z);
}

// Probe slice sl = blockIdx.x / bps, rows (blockIdx.x % bps) * R + team:
// a team of Tw threads per row, Vt = w / VE of them active, each owning VE
// probe columns.  Tw is Vt, or Vt rounded up to a power of two (whole warps
// above 32) so that no row is split between two warps, which saves the extra
// L1 wavefront of the 128-byte line both warps would touch; the host picks
// by row width (measured).  Blocks run slice-major, so one slice of u_k is
// gathered at a time.  The kernel is bound by gather latency (no memory unit
// near its peak, long-scoreboard stalls dominate), so occupancy is what keeps
// gathers in flight: the FP32 form runs at 32 registers per thread (full
// occupancy), the BF16 basis at 40 (three blocks of 512 per SM; its eight
// columns per thread need more), FP64 (bound by its FP64 arithmetic) unbounded.
template <int P>
constexpr int spmm_min_blocks() {
  return P == SLAQ_FP32 ? 4 : (P == SLAQ_FP32_BF16BASIS ? 3 : 1);
}
template <int P, int MODE>
__global__ void __launch_bounds__(512, spmm_min_blocks<P>())
    k_spmm_light(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                 const typename Form<P>::TW *__restrict__ vals,
                 const typename Form<P>::TW *__restrict__ diag,
                 const typename Form<P>::TW *__restrict__ scale,
                 const typename Form<P>::TB *__restrict__ U, typename Form<P>::TW *__restrict__ Z,
                 const typename Form<P>::TB *__restrict__ Yg, Slc S, int Vt, int Tw, int R,
                 int64_t bps, int64_t heavy_degree) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  const int sl = (int)(blockIdx.x / bps);
  const int64_t rb = blockIdx.x - (int64_t)sl * bps;
  const int team = threadIdx.x / Tw, lane = threadIdx.x - team * Tw;
  if (team >= R || lane >= Vt) return;
  const int c = sl * S.w + lane * VE;
  if (c >= S.ld) return;  // narrower last slice
  const int64_t row = rb * R + team;
  if (row >= S.n) return;
  const int64_t b = rowptr[row], e = rowptr[row + 1];
  if (e - b > heavy_degree) return;  // split rows: k_spmm_heavy
  int stride;
  const int64_t off = S.base(c, stride);
  const auto *Ul = U + off;
  TW acc[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) acc[v] = TW(0);
  gather_rows<P, MODE>(col, vals, scale, MODE == 3 ? Yg + off : Ul, stride, b, e, acc);
  finish_row<P, MODE>(row, diag, scale, Ul, stride, acc, Z + off + row * stride);
}

// One (slice, chunk of a split row) per block, slice-major; the last block to
// finish a row's slice sums the chunk partials in chunk order
// (deterministic) and writes that slice of the row.
template <int P, int MODE>
__global__ void __launch_bounds__(256)
    k_spmm_heavy(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                 const typename Form<P>::TW *__restrict__ vals,
                 const typename Form<P>::TW *__restrict__ diag,
                 const typename Form<P>::TW *__restrict__ scale,
                 const typename Form<P>::TB *__restrict__ U, typename Form<P>::TW *__restrict__ Z,
                 typename Form<P>::TW *__restrict__ part, const int32_t *__restrict__ heavy_row,
                 const int64_t *__restrict__ heavy_first, const int32_t *__restrict__ chunk_slot,
                 uint32_t *__restrict__ heavy_count, const typename Form<P>::TB *__restrict__ Yg,
                 Slc S, int Vt, int64_t n_chunks) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  __shared__ int is_last;
  const int sl = (int)(blockIdx.x / n_chunks);
  const int64_t q = blockIdx.x - (int64_t)sl * n_chunks;
  const int slot = chunk_slot[q];
  const int64_t row = heavy_row[slot];
  const int64_t first = heavy_first[slot];
  const int64_t nch = heavy_first[slot + 1] - first;
  const int64_t c = q - first;
  const int64_t rb = rowptr[row], re = rowptr[row + 1];
  const int64_t b = rb + c * kHeavyChunk;
  const int64_t e = min(b + (int64_t)kHeavyChunk, re);
  const int lane = threadIdx.x;
  const int cc0 = sl * S.w + lane * VE;
  const bool active = lane < Vt && cc0 < S.ld;
  int stride = 1;
  const int64_t off = active ? S.base(cc0, stride) : 0;
  const auto *Ul = U + off;
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    gather_rows<P, MODE, P != SLAQ_FP64>(col, vals, scale, MODE == 3 ? Yg + off : Ul, stride, b,
                                          e, acc);
    stw<TW, VE>(part + q * S.ld + cc0, acc);
  }
  __threadfence();
  __syncthreads();
  uint32_t *counter = heavy_count + (int64_t)slot * S.nslices() + sl;
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == (unsigned)(nch - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    for (int64_t ch = 0; ch < nch; ++ch) {
      TW x[VE];
      ldw_cg<TW, VE>(part + (first + ch) * S.ld + cc0, x);
#pragma unroll
      for (int v = 0; v < VE; ++v) acc[v] += x[v];
    }
    finish_row<P, MODE>(row, diag, scale, Ul, stride, acc, Z + off + row * stride);
  }
  if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
}

// Split rows with rows of at most 32 active threads (Vt <= 32): one chunk
// per warp, kHeavyWarps chunks per block, so that more than one warp per
// block is resident (a 32-thread block per chunk caps the SM at 32 warps).
// The last warp to finish a row's slice sums the chunk partials in chunk
// order, as in k_spmm_heavy.
constexpr int kHeavyWarps = 4;

template <int P, int MODE>
__global__ void __launch_bounds__(32 * kHeavyWarps)
    k_spmm_heavy_warps(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                       const typename Form<P>::TW *__restrict__ vals,
                       const typename Form<P>::TW *__restrict__ diag,
                       const typename Form<P>::TW *__restrict__ scale,
                       const typename Form<P>::TB *__restrict__ U,
                       typename Form<P>::TW *__restrict__ Z, typename Form<P>::TW *__restrict__ part,
                       const int32_t *__restrict__ heavy_row,
                       const int64_t *__restrict__ heavy_first,
                       const int32_t *__restrict__ chunk_slot, uint32_t *__restrict__ heavy_count,
                       const typename Form<P>::TB *__restrict__ Yg, Slc S, int Vt,
                       int64_t n_chunks) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  const int64_t bpc = (n_chunks + kHeavyWarps - 1) / kHeavyWarps;  // blocks per slice
  const int sl = (int)(blockIdx.x / bpc);
  const int64_t q = (blockIdx.x - (int64_t)sl * bpc) * kHeavyWarps + (threadIdx.x >> 5);
  if (q >= n_chunks) return;  // whole warp; no block barrier below
  const int lane = threadIdx.x & 31;
  const int slot = chunk_slot[q];
  const int64_t row = heavy_row[slot];
  const int64_t first = heavy_first[slot];
  const int64_t nch = heavy_first[slot + 1] - first;
  const int64_t c = q - first;
  const int64_t rb = rowptr[row], re = rowptr[row + 1];
  const int64_t b = rb + c * kHeavyChunk;
  const int64_t e = min(b + (int64_t)kHeavyChunk, re);
  const int cc0 = sl * S.w + lane * VE;
  const bool active = lane < Vt && cc0 < S.ld;
  int stride = 1;
  const int64_t off = active ? S.base(cc0, stride) : 0;
  const auto *Ul = U + off;
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    gather_rows<P, MODE, P != SLAQ_FP64>(col, vals, scale, MODE == 3 ? Yg + off : Ul, stride, b,
                                          e, acc);
    stw<TW, VE>(part + q * S.ld + cc0, acc);
  }
  __threadfence();
  __syncwarp();
  uint32_t *counter = heavy_count + (int64_t)slot * S.nslices() + sl;
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(counter, 1u);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != (unsigned)(nch - 1)) return;
  __threadfence();
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    for (int64_t ch = 0; ch < nch; ++ch) {
      TW x[VE];
      ldw_cg<TW, VE>(part + (first + ch) * S.ld + cc0, x);
#pragma unroll
      for (int v = 0; v < VE; ++v) acc[v] += x[v];
    }
    finish_row<P, MODE>(row, diag, scale, Ul, stride, acc, Z + off + row * stride);
  }
  if (lane == 0) *counter = 0u;  // ready for the next launch
}

// ------------------------------------------- light rows through TMA gathers
// The light rows again, with the row gathers done by the tensor memory
// accelerator: each warp streams the entries of its rows, and one lane turns
// every four of them into a cp.async.bulk.tensor tile::gather4 load that
// copies the four gathered rows of u_k (or y) into shared memory, completing
// on an mbarrier.  A warp keeps NS stages of eight rows in flight, and
// unlike the load path the rows in flight hold no registers.  The lanes then
// sum the staged rows: with rows of more than 16 lanes the whole warp takes
// each entry; narrower rows split the warp into G groups that take every
// G-th entry and add their sums at the end of the row.
//
// Work items are ranges of kTmaTaskEntries entries: an item owns the rows
// that start in its range (a row that starts there and runs past it is
// still the item's), found once per run by a binary search of the row
// pointers.  Split rows (more than heavy_degree entries) are skipped; the
// split-row kernels write them.  The tensor map spans the whole stored basis
// (or y), and gathers are addressed as row0 + j.  Waits are bounded: a wait
// that gives up sets err and the kernel drains its copies in flight before
// it returns.
//
// Measured on GB300 it is slower than the load path on every workload tried
// (R-MAT 2^20 FP32: 61 against 21 ms of SpMM per run; BF16 basis at 2^24:
// 525 against 326 ms): a warp serializes its rows' control work (row ends,
// the row's own values, the next row's pointers) behind one stage pipeline,
// while the load path overlaps that work across 64 warps per SM, and most
// light rows hold only a few entries.  It is kept as an opt-in
// (slaq_set_spmm_gathers), tested against the load path.
constexpr int kTmaWarps = 8;                  // warps per block
constexpr int kTmaG4 = 2;                     // gather4 loads per stage
constexpr int kTmaStage = 4 * kTmaG4;         // entries per stage
constexpr int64_t kTmaTaskEntries = 2048;     // entries per work item
constexpr int kTmaSpinLimit = 1 << 17;        // mbarrier polls before giving up (each
                                              // suspends up to 20 us: about 2.6 s in all)

// shared memory of one gather4 load (four rows), 128-byte aligned
__host__ __device__ inline int tma_slot_bytes(int row_bytes) {
  return (4 * row_bytes + 127) / 128 * 128;
}
// one warp: NS stages, then NS mbarriers, NS x 8 weights and NS entry counts
__host__ __device__ inline int tma_warp_bytes(int row_bytes, int ns) {
  const int tail = ns * 8 + ns * kTmaStage * 4 + ns * 4;
  return ns * kTmaG4 * tma_slot_bytes(row_bytes) + (tail + 127) / 128 * 128;
}
inline size_t tma_block_smem(int row_bytes, int ns) {
  return (size_t)kTmaWarps * tma_warp_bytes(row_bytes, ns) + 128;  // + alignment slack
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kTmaSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(20000)
        : "memory");
    if (done) return true;
  }
  return false;
}

// A walk over the light rows of a work item: row r, next entry j, row end e.
struct TmaCursor {
  int64_t r, j, e;
};
// Moves c to the first light row at or after r (r1 when none is left).
__device__ __forceinline__ void tma_seek(TmaCursor &c, int64_t r, int64_t r1,
                                         const int64_t *__restrict__ rowptr, int64_t heavy) {
  int64_t b = 0, e = 0;
  for (; r < r1; ++r) {
    b = __ldg(rowptr + r);
    e = __ldg(rowptr + r + 1);
    if (e - b <= heavy) break;
  }
  c.r = r;
  c.j = b;
  c.e = e;
}

// task_row[t] = first row that starts at or after entry t * per (n if none),
// t = 0 .. ntasks; task t owns rows [task_row[t], task_row[t + 1]).
__global__ void k_tma_tasks(const int64_t *__restrict__ rowptr, int64_t n, int64_t per,
                            int64_t ntasks, int64_t *__restrict__ task_row) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntasks;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t == ntasks) {
      task_row[t] = n;
      continue;
    }
    const int64_t target = t * per;
    int64_t lo = 0, hi = n;  // first r in [0, n) with rowptr[r] >= target, else n
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (rowptr[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    task_row[t] = lo;
  }
}

template <int P, int MODE, int G, int NS>
__global__ void __launch_bounds__(32 * kTmaWarps, G == 4 ? 3 : 2)
    k_spmm_tma(const __grid_constant__ CUtensorMap map, int row0,
               const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
               const typename Form<P>::TW *__restrict__ vals,
               const typename Form<P>::TW *__restrict__ diag,
               const typename Form<P>::TW *__restrict__ scale,
               const typename Form<P>::TB *__restrict__ U, typename Form<P>::TW *__restrict__ Z,
               int ld, int64_t heavy_degree, const int64_t *__restrict__ task_row, int64_t ntasks,
               int32_t *__restrict__ err, int giveup) {
  using TW = typename Form<P>::TW;
  using TB = typename Form<P>::TB;
  constexpr int VE = Form<P>::VE;
  constexpr int LPG = 32 / G;  // lanes per group
  static_assert(G == 1 || G == 2 || G == 4, "one, two or four row groups per warp");
  extern __shared__ unsigned char tma_smem[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / LPG, li = lane - grp * LPG;
  const bool act = li < ld / VE;
  const int rowb = ld * (int)sizeof(TB);
  const int slotb = tma_slot_bytes(rowb);
  const int stageb = kTmaG4 * slotb;
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tma_smem) + 127) &
                                        ~(uintptr_t)127) +
      (size_t)wib * tma_warp_bytes(rowb, NS);
  uint64_t *bar = reinterpret_cast<uint64_t *>(base + NS * stageb);
  TW *wst = reinterpret_cast<TW *>(bar + NS);                  // [NS][kTmaStage]
  int *cnt = reinterpret_cast<int *>(wst + NS * kTmaStage);  // [NS]
  if (lane == 0)
    for (int s = 0; s < NS; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + s)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();

  const int64_t nw = (int64_t)gridDim.x * kTmaWarps;
  uint32_t pc = 0, cc = 0;  // stages issued and consumed by this warp (phases follow)
  bool ok = true;
  TW acc[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) acc[v] = TW(0);
  for (int64_t t = (int64_t)blockIdx.x * kTmaWarps + wib; t < ntasks && ok; t += nw) {
    const int64_t r1 = task_row[t + 1];
    TmaCursor pcur, ccur;
    tma_seek(pcur, task_row[t], r1, rowptr, heavy_degree);
    ccur = pcur;
    bool pdone = false;
    // The producer prepares stages three deep in registers, so that no load
    // latency sits on the issue path: stage C has its column loads in
    // flight, B its weight loads (scale of the column, which needs the
    // column first), A is complete and is the next to issue.  Lane q holds
    // entry q of a stage.
    struct Pre {
      int c, filled;
      TW w;
    };
    Pre A{0, 0, TW(1)}, B{0, 0, TW(1)}, C{0, 0, TW(1)};
    auto prepare = [&](Pre &x) {
      int64_t jq = 0;
      int filled = 0;
      if (pcur.r < r1 && pcur.e - pcur.j >= kTmaStage) {  // the stage lies in one row
        jq = pcur.j + lane;
        filled = kTmaStage;
        pcur.j += kTmaStage;
      } else {
        while (filled < kTmaStage) {
          while (pcur.r < r1 && pcur.j == pcur.e)
            tma_seek(pcur, pcur.r + 1, r1, rowptr, heavy_degree);
          if (pcur.r >= r1) break;
          const int take = (int)::min((int64_t)(kTmaStage - filled), pcur.e - pcur.j);
          if (lane >= filled && lane < filled + take) jq = pcur.j + (lane - filled);
          filled += take;
          pcur.j += take;
        }
      }
      x.filled = filled;
      if (lane < filled) {
        x.c = __ldcs(col + jq);
        if (MODE == 2) x.w = __ldcs(vals + jq);
      }
    };
    auto weigh = [&](Pre &x) {
      if (MODE == 0 && lane < x.filled) x.w = __ldg(scale + x.c);
    };
    prepare(A);
    weigh(A);
    prepare(B);
    weigh(B);
    prepare(C);
    // issues stage A into the next slot, then shifts the pipeline
    auto issue = [&]() {
      const int filled = A.filled;
      if (filled == 0) {
        pdone = true;
        return;
      }
      const int slot = (int)(pc % NS);
      int c = A.c;
      if ((MODE == 0 || MODE == 2) && lane < filled) wst[slot * kTmaStage + lane] = A.w;
      // unused slots of the last gather4 repeat the stage's last row (never summed)
      if (filled < kTmaStage) {
        const int clast = __shfl_sync(0xffffffffu, c, filled - 1);
        if (lane >= filled) c = clast;
      }
      c += row0;
      // lanes 0 and 4 issue the two gather4 loads, each with its own four rows
      const int c1 = __shfl_down_sync(0xffffffffu, c, 1);
      const int c2 = __shfl_down_sync(0xffffffffu, c, 2);
      const int c3 = __shfl_down_sync(0xffffffffu, c, 3);
      const uint32_t b = smem_u32(bar + slot);
      const int nblk = (filled + 3) >> 2;
      if (lane == 0) {
        cnt[slot] = filled;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                     "r"(nblk * 4 * rowb)
                     : "memory");
      }
      __syncwarp();  // weights and count stored, the stage armed, before its loads
      if ((lane & 3) == 0 && (lane >> 2) < nblk)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::"
            "bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(
                smem_u32(base + (size_t)slot * stageb + (size_t)(lane >> 2) * slotb)),
            "l"(reinterpret_cast<uint64_t>(&map)), "r"(0), "r"(c), "r"(c1), "r"(c2), "r"(c3),
            "r"(b)
            : "memory");
      ++pc;
      A = B;
      B = C;
      weigh(B);
      prepare(C);
    };
    // The consumer's current row: its own basis values, diagonal and scale,
    // loaded when the row becomes current and used when it is written.
    uint4 ru = make_uint4(0, 0, 0, 0);
    TW rdiag = TW(0), rscale = TW(1);
    auto load_row = [&]() {
      if (ccur.r < r1 && grp == 0 && act) {
        ru = ldraw(U + ccur.r * ld + li * VE);
        rdiag = __ldg(diag + ccur.r);
        if (MODE == 0 || MODE == 3) rscale = __ldg(scale + ccur.r);
      }
    };
    // the end of row r: add the groups' sums, write z_r, clear
    auto flush = [&](int64_t row) {
      if (G > 1) {
#pragma unroll
        for (int v = 0; v < VE; ++v)
#pragma unroll
          for (int o = LPG; o < 32; o <<= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
      }
      if (grp == 0 && act) {
        TW y[VE], z[VE];
        unpack(ru, y);
#pragma unroll
        for (int v = 0; v < VE; ++v)
          z[v] = MODE == 2 ? fma(rdiag, y[v], acc[v]) : fma(rdiag, y[v], -rscale * acc[v]);
        stw_cs<TW, VE>(Z + row * ld + li * VE, z);
      }
#pragma unroll
      for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    };
    // rows without entries at the consumer's position are written at once
    auto settle = [&]() {
      while (ccur.r < r1 && ccur.j == ccur.e) {
        flush(ccur.r);
        tma_seek(ccur, ccur.r + 1, r1, rowptr, heavy_degree);
        load_row();
      }
    };
    while (pc - cc < (uint32_t)NS && !pdone) issue();
    __syncwarp();
    load_row();
    settle();
    while (ccur.r < r1) {
      if (cc == pc) {  // the walks disagree: cannot happen
        ok = false;
        break;
      }
      const int slot = (int)(cc % NS);
      // giveup (a test hook): the warp's first wait gives up at once, as a
      // wait that ran out of polls would
      if ((giveup && cc == 0) || !mbar_wait(smem_u32(bar + slot), (cc / NS) & 1u)) {
        ok = false;
        break;
      }
      const int filled = cnt[slot];
      const unsigned char *stg = base + (size_t)slot * stageb;
      int q0 = 0;
      if (filled == kTmaStage && ccur.e - ccur.j >= kTmaStage) {
        // the whole stage lies in the current row: this group's entries,
        // unrolled
        if (act) {
#pragma unroll
          for (int i = 0; i < kTmaStage / G; ++i) {
            const int q = grp + G * i;
            const TW w = (MODE == 0 || MODE == 2) ? wst[slot * kTmaStage + q] : TW(1);
            const uint4 raw = *reinterpret_cast<const uint4 *>(stg + (q >> 2) * slotb +
                                                               (q & 3) * rowb + li * 16);
            TW x[VE];
            unpack(raw, x);
#pragma unroll
            for (int v = 0; v < VE; ++v) acc[v] = fma(w, x[v], acc[v]);
          }
        }
        q0 = kTmaStage;
        ccur.j += kTmaStage;
        if (ccur.j == ccur.e) {
          flush(ccur.r);
          tma_seek(ccur, ccur.r + 1, r1, rowptr, heavy_degree);
          load_row();
          settle();
        }
      }
      while (q0 < filled) {
        const int take = (int)::min((int64_t)(filled - q0), ccur.e - ccur.j);
        if (ccur.r >= r1 || take <= 0) {  // the walks disagree: cannot happen
          ok = false;
          break;
        }
        for (int q = q0; q < q0 + take; ++q) {
          if ((q & (G - 1)) != grp || !act) continue;
          const TW w = (MODE == 0 || MODE == 2) ? wst[slot * kTmaStage + q] : TW(1);
          const uint4 raw =
              *reinterpret_cast<const uint4 *>(stg + (q >> 2) * slotb + (q & 3) * rowb + li * 16);
          TW x[VE];
          unpack(raw, x);
#pragma unroll
          for (int v = 0; v < VE; ++v) acc[v] = fma(w, x[v], acc[v]);
        }
        q0 += take;
        ccur.j += take;
        if (ccur.j == ccur.e) {
          flush(ccur.r);
          tma_seek(ccur, ccur.r + 1, r1, rowptr, heavy_degree);
          load_row();
          settle();
        }
      }
      __syncwarp();  // every lane has read the stage before it is refilled
      ++cc;
      if (!ok) break;
      if (!pdone) issue();
      __syncwarp();
    }
    if (ok && cc != pc) ok = false;
  }
  if (!ok) {
    if (lane == 0) atomicOr(err, 1);
    for (; cc < pc; ++cc)  // copies still in flight land before the block exits
      if (!mbar_wait(smem_u32(bar + cc % NS), (cc / NS) & 1u)) break;
  }
}

}  // namespace

std::atomic<int> g_tma_giveup{0};

int debug_tma_giveup(int on) {
  g_tma_giveup.store(on ? 1 : 0);
  return SLAQ_OK;
}

namespace {

// ------------------------------------------------------ compensated sums
// Per-thread running sums of chunk sums.  FP64 form: plain FP64.  FP32
// forms: Kahan summation in FP32 (sum, c); the true value is sum - c.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
struct PlainD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
struct PlainF {
  float s = 0.f;
  __device__ __forceinline__ void add(float x) { s += x; }
  __device__ __forceinline__ double value() const { return (double)s; }
};
// FP64: plain FP64; FP32: Kahan; BF16 basis: plain FP32 (the basis's own
// 2^-9 rounding dominates; saves the registers the wider vectors need).
template <int P>
struct Acc;
template <>
struct Acc<SLAQ_FP64> {
  using type = PlainD;
};
template <>
struct Acc<SLAQ_FP32> {
  using type = KahanF;
};
template <>
struct Acc<SLAQ_FP32_BF16BASIS> {
  using type = PlainF;
};

// Neumaier-compensated FP64 pair sum.
struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// ------------------------------------------------------------------ dots
// Thread (x, y) of block (g, c) owns probe columns [x*VE, x*VE + VE) of basis
// vector j = jfirst + c*Jb + y over the rows of row block g and accumulates
//   d_j = u_j^T x          (x = z = L u_k, or u_{k+1} in the second pass)
//   g_j = u_j^T u_k        (Gram column of the newest vector; WITH_G only)
// Every (j, column) has a single owner, so no reduction inside the block.
// The rows of x and u_k, which every y of a column needs, are staged tile by
// tile in shared memory (cp.async, double buffered); only the u_j stream
// comes from HBM per thread.  Sums are plain over a tile of tile_rows rows
// (kTile, fewer for rows so wide that two tiles would not fit shared memory) and
// compensated across tiles.
constexpr int kTile = 32;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// smem element loads of VE columns (16 or 32 bytes)
__device__ __forceinline__ void lds(const double *p, double (&v)[2]) {
  const double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void lds(const float *p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void lds(const float *p, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0];
  const float4 b = reinterpret_cast<const float4 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void lds(const __nv_bfloat16 *p, float (&v)[8]) {
  const uint4 t = *reinterpret_cast<const uint4 *>(p);
  const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// Copy rows [row0, row0 + nr) of a sliced [n][ld] block (element type T) to
// shared memory as a dense [nr][ld] tile, 16 bytes per cp.async.
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, const T *src, const Slc &S, int64_t row0, int nr,
                                           int tid, int nthr) {
  constexpr int E = 16 / sizeof(T);
  const int per_row = S.ld / E;
  for (int q = tid; q < nr * per_row; q += nthr) {
    const int r = q / per_row;
    const int col = (q - r * per_row) * E;
    int stride;
    const int64_t cb = S.base(col, stride);
    cp_async16(dst + r * S.ld + col, src + cb + (row0 + r) * stride);
  }
}

template <int P, bool X_IS_BASIS, bool WITH_G>
__global__ void __launch_bounds__(512, 2)
    k_dots(const typename Form<P>::TB *__restrict__ U, const void *__restrict__ Xv,
           const typename Form<P>::TB *__restrict__ Uk, Slc S, const int64_t *__restrict__ crow0,
           const int32_t *__restrict__ crows, int sub, int64_t ustride, int jfirst, int jlast,
           int Jb, double *__restrict__ part, int s, int tile_rows) {
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  using TX = typename std::conditional<X_IS_BASIS, TB, TW>::type;
  constexpr int VE = Form<P>::VE;
  using A = typename Acc<P>::type;
  extern __shared__ __align__(16) unsigned char dyn[];
  const int ld = S.ld;
  TX *xs = reinterpret_cast<TX *>(dyn);                 // [2][tile_rows][ld]
  TB *us = reinterpret_cast<TB *>(xs + 2 * tile_rows * ld);  // [2][tile_rows][ld]
  const TX *X = static_cast<const TX *>(Xv);
  // z = row phase: narrow probe blocks (few column vectors) split the rows of
  // a tile over blockDim.z groups and add the groups' sums at the end
  const int RZ = blockDim.z, rz = threadIdx.z;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int g = blockIdx.x;
  const int j = jfirst + (int)blockIdx.y * Jb + (int)threadIdx.y;
  const bool active = j <= jlast;  // idle threads still stage and synchronize
  const int col = threadIdx.x * VE;
  // block g covers part (g % sub) of chunk (g / sub); partials are indexed by g
  const int chunk = g / sub, piece = g - chunk * sub;
  const int64_t cr = crows[chunk];
  const int64_t per = (cr + sub - 1) / sub;
  const int64_t r0 = crow0[chunk] + min(cr, per * piece);
  const int64_t r1 = crow0[chunk] + min(cr, per * (piece + 1));
  const int ntile = (int)((r1 - r0 + tile_rows - 1) / tile_rows);
  int stride;
  const int64_t off = S.base(col, stride);
  const TB *Uj = U + (int64_t)(active ? j : jfirst) * ustride + off;
  A d[VE], gg[VE];
  auto stage = [&](int t) {
    const int64_t row0 = r0 + (int64_t)t * tile_rows;
    const int nr = (int)min((int64_t)tile_rows, r1 - row0);
    const int buf = t & 1;
    stage_rows<TX>(xs + buf * tile_rows * ld, X, S, row0, nr, tid, nthr);
    if (WITH_G) stage_rows<TB>(us + buf * tile_rows * ld, Uk, S, row0, nr, tid, nthr);
  };
  if (ntile > 0) stage(0);
  cp_async_commit();
  for (int t = 0; t < ntile; ++t) {
    if (t + 1 < ntile) stage(t + 1);
    cp_async_commit();
    cp_async_wait1();  // tile t has landed
    __syncthreads();
    if (active) {
      const int64_t row0 = r0 + (int64_t)t * tile_rows;
      const int nr = (int)min((int64_t)tile_rows, r1 - row0);
      const TX *xt = xs + (t & 1) * tile_rows * ld + col;
      const TB *ut = us + (t & 1) * tile_rows * ld + col;
      TW dc[VE], gc[VE];
#pragma unroll
      for (int v = 0; v < VE; ++v) {
        dc[v] = TW(0);
        gc[v] = TW(0);
      }
      constexpr int UNR = VE >= 8 ? 2 : 4;  // rows in flight per thread (register budget)
      int r = rz;
      if constexpr (P == SLAQ_FP32_BF16BASIS) {
        // BF16: four rows in flight as packed 16-byte words, unpacked one at
        // a time (eight floats per row would not fit the register budget)
        for (; r + 3 * RZ < nr; r += 4 * RZ) {
          uint4 raw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            raw[q] = __ldg(reinterpret_cast<const uint4 *>(Uj + (row0 + r + q * RZ) * stride));
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            TW u[VE], x[VE];
            unpack_bf16x8(raw[q], u);
            lds(xt + (r + q * RZ) * ld, x);
#pragma unroll
            for (int v = 0; v < VE; ++v) dc[v] = fma(u[v], x[v], dc[v]);
            if (WITH_G) {
              TW w[VE];
              lds(ut + (r + q * RZ) * ld, w);
#pragma unroll
              for (int v = 0; v < VE; ++v) gc[v] = fma(u[v], w[v], gc[v]);
            }
          }
        }
      }
      for (; r + (UNR - 1) * RZ < nr; r += UNR * RZ) {
        TW u[UNR][VE];
#pragma unroll
        for (int q = 0; q < UNR; ++q) ldb(Uj + (row0 + r + q * RZ) * stride, u[q]);
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          TW x[VE];
          lds(xt + (r + q * RZ) * ld, x);
#pragma unroll
          for (int v = 0; v < VE; ++v) dc[v] = fma(u[q][v], x[v], dc[v]);
          if (WITH_G) {
            TW w[VE];
            lds(ut + (r + q * RZ) * ld, w);
#pragma unroll
            for (int v = 0; v < VE; ++v) gc[v] = fma(u[q][v], w[v], gc[v]);
          }
        }
      }
      for (; r < nr; r += RZ) {
        TW u[VE], x[VE];
        ldb(Uj + (row0 + r) * stride, u);
        lds(xt + r * ld, x);
#pragma unroll
        for (int v = 0; v < VE; ++v) dc[v] = fma(u[v], x[v], dc[v]);
        if (WITH_G) {
          TW w[VE];
          lds(ut + r * ld, w);
#pragma unroll
          for (int v = 0; v < VE; ++v) gc[v] = fma(u[v], w[v], gc[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < VE; ++v) {
        d[v].add(dc[v]);
        if (WITH_G) gg[v].add(gc[v]);
      }
    }
    __syncthreads();  // buffer t&1 is restaged at t+2
  }
  // sum the row phases in a fixed order; the staging buffers are free now
  double *red = reinterpret_cast<double *>(dyn);  // [RZ][Jb][ld][2]
  const int slot = ((rz * blockDim.y + threadIdx.y) * ld + col) * 2;
  if (RZ > 1) {
#pragma unroll
    for (int v = 0; v < VE; ++v) {
      red[slot + 2 * v] = d[v].value();
      red[slot + 2 * v + 1] = WITH_G ? gg[v].value() : 0.0;
    }
    __syncthreads();
  }
  if (!active || rz != 0) return;
  double *pd = part + (((int64_t)g * 2 + 0) * s + j) * ld + col;
  double *pg = part + (((int64_t)g * 2 + 1) * s + j) * ld + col;
#pragma unroll
  for (int v = 0; v < VE; ++v) {
    double dv = d[v].value(), gv = WITH_G ? gg[v].value() : 0.0;
    for (int q = 1; q < RZ; ++q) {
      const int sl = ((q * blockDim.y + threadIdx.y) * ld + col) * 2;
      dv += red[sl + 2 * v];
      gv += red[sl + 2 * v + 1];
    }
    pd[v] = dv;
    if (WITH_G) pg[v] = gv;
  }
}

// row phases of a dots block: narrow blocks (few column vectors and basis
// vectors) grow along threadIdx.z up to `target` threads
inline int dots_phases(int V, int Jb, int target) {
  return std::max(1, std::min(8, target / (V * Jb)));
}

// dynamic shared memory of a dots block: staging tiles, reused at the end
// for the row-phase sums ([rz][Jb][ld][2] doubles)
constexpr size_t kDotsSmemMax = 200 * 1024;  // the kernels' dynamic shared memory limit

// rows per staged tile: kTile, or fewer so that two tiles of the widest rows
// (nv = 512 in FP64: 8 KiB per row and tile pair) fit
inline int dots_tile_rows(int precision, int ld, bool x_is_basis) {
  const int bx = x_is_basis ? basis_bytes(precision) : work_bytes(precision);
  const size_t per_row = (size_t)2 * ld * (bx + basis_bytes(precision));
  return (int)std::max<size_t>(1, std::min<size_t>(kTile, kDotsSmemMax / per_row));
}

inline size_t dots_smem(int precision, int ld, bool x_is_basis, int Jb = 0, int RZ = 1) {
  const int bx = x_is_basis ? basis_bytes(precision) : work_bytes(precision);
  const size_t tiles =
      (size_t)2 * dots_tile_rows(precision, ld, x_is_basis) * ld * (bx + basis_bytes(precision));
  const size_t red = RZ > 1 ? (size_t)RZ * Jb * ld * 2 * sizeof(double) : 0;
  return std::max(tiles, red);
}

// Sum the partials of graph g's chunks [goff[g], goff[g+1]) of d_j and, with_g,
// of the Gram column, for j in [jfirst, jfirst + jcount): d to dsum[g][j][p];
// g_j is the Gram entry (j, k), stored in gram[g][j][k][p] and gram[g][k][j][p].
// proj (reduced forms, first pass only): d_j = u_j^T L u_k is also entry
// (j, k) of the projected matrix, stored like the Gram entries.
// Block (32, kRedY): x = column, y strides over the chunks; grid
// (columns / 32, 1 or 2, G).
constexpr int kRedY = 32;
__global__ void k_dot_reduce(const double *__restrict__ part, const int32_t *__restrict__ goff,
                             int sub, int s, int ld, int jfirst, int jcount, int k,
                             double *__restrict__ dsum, double *__restrict__ gram,
                             double *__restrict__ proj) {
  __shared__ double ss[kRedY][33];
  const int ncol = jcount * ld;
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int which = blockIdx.y;  // 0: d, 1: g
  const int gr = blockIdx.z;
  const bool valid = col < ncol;
  const int j = jfirst + (valid ? col / ld : 0);
  const int p = valid ? col % ld : 0;
  // plain FP64 sums of the strided partials (few terms; FP64 is scarce on
  // this chip), compensated combination of the kRedY sums
  double acc = 0.0;
  if (valid)
    for (int c = goff[gr] * sub + threadIdx.y; c < goff[gr + 1] * sub; c += kRedY)
      acc += part[(((int64_t)c * 2 + which) * s + j) * ld + p];
  ss[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && valid) {
    Neumaier tot;
    for (int y = 0; y < kRedY; ++y) tot.add(ss[y][threadIdx.x]);
    const double v = tot.value();
    const int64_t gs = (int64_t)gr * s;
    if (which == 0) {
      dsum[(gs + j) * ld + p] = v;
      if (proj) {
        double *pm = proj + (int64_t)gr * s * s * ld;
        pm[((int64_t)j * s + k) * ld + p] = v;
        pm[((int64_t)k * s + j) * ld + p] = v;
      }
    } else {
      double *gm = gram + (int64_t)gr * s * s * ld;
      gm[((int64_t)j * s + k) * ld + p] = v;
      gm[((int64_t)k * s + j) * ld + p] = v;
    }
  }
}

// Same sums, one thread per output (graph, which, column): for batches whose
// graphs have few partials each.
__global__ void k_dot_reduce_narrow(const double *__restrict__ part, const int32_t *__restrict__ goff,
                                    int sub, int s, int ld, int jfirst, int jcount, int k, int G,
                                    int with_g, double *__restrict__ dsum,
                                    double *__restrict__ gram, double *__restrict__ proj) {
  const int ncol = jcount * ld;
  const int64_t total = (int64_t)G * (with_g ? 2 : 1) * ncol;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(o % ncol);
    const int which = (int)((o / ncol) % (with_g ? 2 : 1));
    const int gr = (int)(o / ((int64_t)ncol * (with_g ? 2 : 1)));
    const int j = jfirst + col / ld, p = col % ld;
    Neumaier acc;
    for (int c = goff[gr] * sub; c < goff[gr + 1] * sub; ++c)
      acc.add(part[(((int64_t)c * 2 + which) * s + j) * ld + p]);
    const double v = acc.value();
    const int64_t gs = (int64_t)gr * s;
    if (which == 0) {
      dsum[(gs + j) * ld + p] = v;
      if (proj) {
        double *pm = proj + (int64_t)gr * s * s * ld;
        pm[((int64_t)j * s + k) * ld + p] = v;
        pm[((int64_t)k * s + j) * ld + p] = v;
      }
    } else {
      double *gm = gram + (int64_t)gr * s * s * ld;
      gm[((int64_t)j * s + k) * ld + p] = v;
      gm[((int64_t)k * s + j) * ld + p] = v;
    }
  }
}

// ---------------------------------------------------------------- solve
// One warp per (graph, probe) problem.  With G the Gram matrix of the
// stored basis u_0..u_k and d_j = u_j^T z, the coefficients of the projection
// of z on span(u_0..u_k) are x = G^{-1} d (Cholesky of the unit-diagonal
// scaling of G).  With an exactly orthogonal basis x_j = d_j / ||u_j||^2,
// which is classical Gram-Schmidt; solving with G keeps the new vector
// orthogonal to the stored basis to working precision even when the stored
// vectors are rounded (BF16), like a second Gram-Schmidt pass.
// first_pass: also records beta_{k-1} = ||u_k|| = sqrt(G_kk) (stopping the
// probe with m = k if beta_{k-1} <= tol_abs) and alpha_k = d_k / G_kk, and
// writes the update's scale 1/||u_k|| to row s-1 of the coefficients (a row
// no step's coefficients use: they fill rows 0..k <= s-2); 1 in the second
// pass.  need_coef == 0 on the last step.
// Partial reorthogonalization (Simon, Math. Comp. 42, 1984; not in the
// paper).  full == nullptr: every step projects against all previous vectors.
// Otherwise step k of graph g projects against all of them if full[g][k]
// (stride s + 2), else against u_{k-1} and u_k only; omega[g][p][k % 3][j]
// holds the estimate omega_{k,j} ~ q_k^T q_j of the last three steps (with
// omega_{k,k} = 1); eps is the unit roundoff of the basis arithmetic.
struct ProArgs {
  int32_t *full;
  int32_t *any;
  double *omega;
  double eps;
};

// first basis vector step k of graph g projects against
__device__ __forceinline__ int pro_first(const ProArgs &P, int g, int k, int s) {
  return (P.full && !P.full[(int64_t)g * (s + 2) + k]) ? max(0, k - 1) : 0;
}

// Row k of the orthogonality estimates of problem (g, p), entries j = j_begin,
// j_begin + j_step, ... < k; returns their largest |omega_{k,j}| over j <= k-2.
// Steps whose Gram column covers every j (measured) take omega_{k,j} =
// G_jk / sqrt(G_jj G_kk); the others take the recurrence that q_k^T L q_j =
// q_j^T L q_k imposes,
//   beta_{k-1} omega_{k,j} = beta_j omega_{k-1,j+1} + (alpha_j - alpha_{k-1}) omega_{k-1,j}
//                            + beta_{j-1} omega_{k-1,j-1} - beta_{k-2} omega_{k-2,j}
// plus eps (beta_{k-1} + beta_j) in the direction that grows |omega|, with
// omega_{k,k-1} = eps (the local projection leaves u_k orthogonal to u_{k-1}
// to rounding).  alpha, beta: this problem's rows (beta_{k-1} already set).
__device__ double omega_row(const ProArgs &P, int64_t prob, int k, int s, bool measured,
                            const double *alpha, const double *beta, const double *gram, int ld,
                            int p, int j_begin, int j_step) {
  double *om = P.omega + prob * 3 * s;
  double *rk = om + (k % 3) * s;
  const double *r1 = om + ((k + 2) % 3) * s;  // row k-1
  const double *r2 = om + ((k + 1) % 3) * s;  // row k-2
  const double bk1 = beta[k - 1];
  double mx = 0.0;
  for (int j = j_begin; j < k; j += j_step) {
    double w;
    if (measured) {
      w = gram[((int64_t)j * s + k) * ld + p] *
          rsqrt(gram[((int64_t)j * s + j) * ld + p] * gram[((int64_t)k * s + k) * ld + p]);
    } else if (j == k - 1) {
      w = P.eps;
    } else {
      double t = beta[j] * r1[j + 1] + (alpha[j] - alpha[k - 1]) * r1[j];
      if (j > 0) t += beta[j - 1] * r1[j - 1];
      if (k >= 2) t -= beta[k - 2] * r2[j];
      t += copysign(P.eps * (bk1 + beta[j]), t);
      w = t / bk1;
    }
    rk[j] = w;
    if (j <= k - 2) mx = fmax(mx, fabs(w));
  }
  return mx;
}

// the next two steps of graph g project against all previous vectors
__device__ __forceinline__ void pro_flag_next(const ProArgs &P, int g, int k, int s) {
  int32_t *f = P.full + (int64_t)g * (s + 2);
  f[k + 1] = 1;
  f[k + 2] = 1;
  P.any[k + 1] = 1;
  P.any[k + 2] = 1;
}

__global__ void k_solve(const double *__restrict__ dsum_all, double *__restrict__ gram_all,
                        int k, int s, int ld, int nv, int first_pass, int need_coef, double tol,
                        const double *__restrict__ gbound, int32_t *__restrict__ m_all,
                        double *__restrict__ alpha_all, double *__restrict__ beta_all,
                        double *__restrict__ coef_all, ProArgs P, int jl) {
  extern __shared__ double sol_smem[];  // A [K1*K1], y [K1], sc [K1]
  __shared__ int run_flag;
  const int p = blockIdx.x;
  const int gr = blockIdx.y;
  const int lane = threadIdx.x;
  double *gram = gram_all + (int64_t)gr * s * s * ld;
  const double *dsum = dsum_all + (int64_t)gr * s * ld;
  double *coef = coef_all + (int64_t)gr * s * ld;
  int32_t *m = m_all + (int64_t)gr * nv;
  double *alpha = alpha_all + (int64_t)gr * nv * s;
  double *beta = beta_all + (int64_t)gr * nv * s;
  const double tol_abs = tol * gbound[gr];
  if (lane == 0) {
    bool running = p < nv && m[p] > k;
    if (running && first_pass) {
      const double nk = gram[((int64_t)k * s + k) * ld + p];
      if (k > 0) {
        const double b = sqrt(nk);  // ||u_k|| = beta_{k-1} (rescaled basis)
        if (b <= tol_abs) {
          m[p] = k;
          running = false;
        } else {
          beta[p * s + k - 1] = b;
        }
      }
      if (running) alpha[p * s + k] = dsum[k * ld + p] / nk;
    }
    run_flag = running ? 1 : 0;
  }
  __syncthreads();
  // partial reorthogonalization: this step projects on u_j, j >= j0, and
  // knows the Gram entries (j, k) for j >= j1 (the rest are zeroed: unknown)
  const int j0 = pro_first(P, gr, k, s);
  const int j1 = max(j0, jl);
  if (P.full && first_pass && p < nv) {
    if (run_flag && k >= 1 && need_coef) {
      double mx = omega_row(P, (int64_t)gr * nv + p, k, s, j1 == 0, alpha + (int64_t)p * s,
                            beta + (int64_t)p * s, gram, ld, p, lane, 32);
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > sqrt(P.eps)) pro_flag_next(P, gr, k, s);
    }
    if (run_flag && lane == 0) P.omega[(((int64_t)gr * nv + p) * 3 + k % 3) * s + k] = 1.0;
    for (int j = lane; j < j1; j += 32) {
      gram[((int64_t)j * s + k) * ld + p] = 0.0;
      gram[((int64_t)k * s + j) * ld + p] = 0.0;
    }
  }
  if (!need_coef) return;
  const int K1 = k + 1 - j0;  // the projection's basis vectors j0 .. k
  double *A = sol_smem;
  double *y = A + K1 * K1;
  double *sc = y + K1;
  if (!run_flag) {
    for (int j = lane; j <= k; j += blockDim.x) coef[j * ld + p] = 0.0;
    return;
  }
  for (int j = lane; j < j0; j += blockDim.x) coef[j * ld + p] = 0.0;
  for (int j = lane; j < K1; j += blockDim.x) {
    sc[j] = rsqrt(gram[((int64_t)(j0 + j) * s + j0 + j) * ld + p]);
    y[j] = dsum[(j0 + j) * ld + p];
  }
  __syncthreads();
  for (int e = lane; e < K1 * K1; e += blockDim.x) {
    const int i = e / K1, j = e - i * K1;
    if (j <= i) A[i * K1 + j] = gram[((int64_t)(j0 + i) * s + j0 + j) * ld + p] * sc[i] * sc[j];
  }
  __syncthreads();
  // partial reorthogonalization: the Gram entries no step measured are zero
  // in the solve, which is accurate while the basis is semi-orthogonal (the
  // scaled pivots stay near 1).  A pivot below 1/2 means a near-breakdown
  // has left it too far from orthogonal for that: the probe's Krylov space is
  // numerically exhausted, and it stops as at a breakdown.
  const bool pro = P.full != nullptr;
  bool degenerate = false;
  // Cholesky of Ghat = D^-1/2 G D^-1/2 (unit diagonal), in place, right-looking:
  // the diagonal keeps the inverse pivot 1/L_cc, column c is scaled by it,
  // then the trailing block is updated by all lanes of the warp.
  for (int c = 0; c < K1; ++c) {
    degenerate = degenerate || (pro && A[c * K1 + c] < 0.5);
    __syncwarp();
    if (lane == 0) A[c * K1 + c] = rsqrt(fmax(A[c * K1 + c], 1e-300));
    __syncwarp();
    const double ipiv = A[c * K1 + c];
    for (int i = c + 1 + lane; i < K1; i += 32) A[i * K1 + c] *= ipiv;
    __syncwarp();
    const int rem = K1 - c - 1;  // trailing rows c+1..K1-1, lower triangle
    for (int e = lane; e < rem * rem; e += 32) {
      const int i = c + 1 + e / rem, q = c + 1 + e % rem;
      if (q <= i) A[i * K1 + q] -= A[i * K1 + c] * A[q * K1 + c];
    }
    __syncwarp();
  }
  // Ghat xhat = D^-1/2 d (column-oriented substitutions), x = D^-1/2 xhat
  for (int i = lane; i < K1; i += 32) y[i] *= sc[i];
  __syncwarp();
  for (int c = 0; c < K1; ++c) {
    if (lane == 0) y[c] *= A[c * K1 + c];
    __syncwarp();
    for (int i = c + 1 + lane; i < K1; i += 32) y[i] -= A[i * K1 + c] * y[c];
    __syncwarp();
  }
  for (int c = K1 - 1; c >= 0; --c) {
    if (lane == 0) y[c] *= A[c * K1 + c];
    __syncwarp();
    for (int i = lane; i < c; i += 32) y[i] -= A[c * K1 + i] * y[c];
    __syncwarp();
  }
  if (pro) {
    bool finite = !degenerate;
    for (int j = lane; j < K1; j += 32) finite = finite && isfinite(y[j] * sc[j]);
    if (!__all_sync(0xffffffffu, finite)) {  // numerically exhausted: stop as at a breakdown
      if (lane == 0) {
        m[p] = k + 1;  // alpha_k stands; u_{k+1} is written as zero
        coef[(s - 1) * ld + p] = 0.0;
      }
      for (int j = lane; j <= k; j += 32) coef[j * ld + p] = 0.0;
      return;
    }
  }
  for (int j = lane; j < K1; j += blockDim.x) coef[(j0 + j) * ld + p] = y[j] * sc[j];
  // the update divides by ||u_k|| (first pass), so ||u_{k+1}|| = beta_k
  if (lane == 0)
    coef[(s - 1) * ld + p] = first_pass ? rsqrt(gram[((int64_t)k * s + k) * ld + p]) : 1.0;
}

// The same step for many problems at once (batches of graphs): one thread per
// (graph, probe), all steps of the solve serial in that thread, so that every
// lane of a warp does useful work -- on GB300's narrow FP64 pipe an
// instruction costs the same with 1 or 32 active lanes.  Each thread keeps the
// packed lower triangle of Ghat, y and D^-1/2 in shared memory, entry-major
// with stride kSolveLanes, so a warp's accesses are consecutive words.  T is
// the arithmetic of the solve: double for the FP64 form, float for the reduced
// forms, whose update applies the coefficients in FP32 anyway.
constexpr int kSolveLanes = 32;

constexpr int64_t kSolveLanesMin = 4096;            // problems per launch
constexpr size_t kSolveLanesSmemMax = 160 * 1024;   // bytes per block

inline size_t solve_lanes_smem(int K1, int tbytes) {
  return (size_t)kSolveLanes * ((size_t)K1 * (K1 + 1) / 2 + 2 * K1) * tbytes;
}

template <typename T>
__device__ __forceinline__ T rsq(T x) {
  return rsqrt(x);
}
template <>
__device__ __forceinline__ float rsq<float>(float x) {
  return rsqrtf(x);
}

template <typename T>
__global__ void __launch_bounds__(kSolveLanes)
    k_solve_lanes(const double *__restrict__ dsum_all, double *__restrict__ gram_all, int k,
                  int s, int ld, int nv, int n_graphs, int first_pass, int need_coef, double tol,
                  const double *__restrict__ gbound, int32_t *__restrict__ m_all,
                  double *__restrict__ alpha_all, double *__restrict__ beta_all,
                  double *__restrict__ coef_all, ProArgs P, int jl) {
  extern __shared__ __align__(16) unsigned char sl_dyn[];
  const int64_t t = (int64_t)blockIdx.x * kSolveLanes + threadIdx.x;
  if (t >= (int64_t)n_graphs * nv) return;  // no block-wide barrier below
  const int gr = (int)(t / nv), p = (int)(t - (int64_t)gr * nv);
  double *gram = gram_all + (int64_t)gr * s * s * ld;
  const double *dsum = dsum_all + (int64_t)gr * s * ld;
  double *coef = coef_all + (int64_t)gr * s * ld;
  int32_t *m = m_all + (int64_t)gr * nv;
  bool running = m[p] > k;
  if (running && first_pass) {
    const double nk = gram[((int64_t)k * s + k) * ld + p];
    if (k > 0) {
      const double b = sqrt(nk);  // ||u_k|| = beta_{k-1} (rescaled basis)
      if (b <= tol * gbound[gr]) {
        m[p] = k;
        running = false;
      } else {
        beta_all[((int64_t)gr * nv + p) * s + k - 1] = b;
      }
    }
    if (running) alpha_all[((int64_t)gr * nv + p) * s + k] = dsum[k * ld + p] / nk;
  }
  // partial reorthogonalization (see k_solve)
  const int j0 = pro_first(P, gr, k, s);
  const int j1 = max(j0, jl);
  if (P.full && first_pass) {
    const int64_t prob = (int64_t)gr * nv + p;
    if (running && k >= 1 && need_coef &&
        omega_row(P, prob, k, s, j1 == 0, alpha_all + prob * s, beta_all + prob * s, gram, ld, p,
                  0, 1) > sqrt(P.eps))
      pro_flag_next(P, gr, k, s);
    if (running) P.omega[(prob * 3 + k % 3) * s + k] = 1.0;
    for (int j = 0; j < j1; ++j) {
      gram[((int64_t)j * s + k) * ld + p] = 0.0;
      gram[((int64_t)k * s + j) * ld + p] = 0.0;
    }
  }
  if (!need_coef) return;
  if (!running) {
    for (int j = 0; j <= k; ++j) coef[j * ld + p] = 0.0;
    return;
  }
  for (int j = 0; j < j0; ++j) coef[j * ld + p] = 0.0;
  const int K1 = k + 1 - j0;  // the projection's basis vectors j0 .. k
  T *A = reinterpret_cast<T *>(sl_dyn) + threadIdx.x;  // packed (i, j <= i)
  T *y = A + (size_t)kSolveLanes * (K1 * (K1 + 1) / 2);
  T *sc = y + (size_t)kSolveLanes * K1;
#define SLAQ_A(i, j) A[(((i) * ((i) + 1)) / 2 + (j)) * kSolveLanes]
  for (int i = 0; i < K1; ++i) {
    sc[i * kSolveLanes] = (T)rsqrt(gram[((int64_t)(j0 + i) * s + j0 + i) * ld + p]);
    y[i * kSolveLanes] = (T)dsum[(j0 + i) * ld + p] * sc[i * kSolveLanes];
  }
  for (int i = 0; i < K1; ++i) {
    const T si = sc[i * kSolveLanes];
    for (int j = 0; j <= i; ++j)
      SLAQ_A(i, j) = (T)gram[((int64_t)(j0 + i) * s + j0 + j) * ld + p] * si * sc[j * kSolveLanes];
  }
  // partial reorthogonalization: a scaled pivot below 1/2 stops the probe (see k_solve)
  const bool pro = P.full != nullptr;
  bool degenerate = false;
  // right-looking Cholesky, inverse pivots on the diagonal
  for (int c = 0; c < K1; ++c) {
    degenerate = degenerate || (pro && SLAQ_A(c, c) < T(0.5));
    const T ip = rsq<T>(fmax(SLAQ_A(c, c), std::numeric_limits<T>::min()));
    SLAQ_A(c, c) = ip;
    for (int i = c + 1; i < K1; ++i) SLAQ_A(i, c) *= ip;
    for (int i = c + 1; i < K1; ++i) {
      const T lic = SLAQ_A(i, c);
      for (int q = c + 1; q <= i; ++q) SLAQ_A(i, q) -= lic * SLAQ_A(q, c);
    }
  }
  for (int c = 0; c < K1; ++c) {  // L w = D^-1/2 d
    const T wc = y[c * kSolveLanes] * SLAQ_A(c, c);
    y[c * kSolveLanes] = wc;
    for (int i = c + 1; i < K1; ++i) y[i * kSolveLanes] -= SLAQ_A(i, c) * wc;
  }
  for (int c = K1 - 1; c >= 0; --c) {  // L^T xhat = w
    const T xc = y[c * kSolveLanes] * SLAQ_A(c, c);
    y[c * kSolveLanes] = xc;
    for (int i = 0; i < c; ++i) y[i * kSolveLanes] -= SLAQ_A(c, i) * xc;
  }
#undef SLAQ_A
  bool finite = !degenerate;
  for (int j = 0; j < K1; ++j) finite = finite && isfinite(y[j * kSolveLanes] * sc[j * kSolveLanes]);
  if (pro && !finite) {  // numerically exhausted: stop the probe as at a breakdown
    m[p] = k + 1;         // alpha_k stands; u_{k+1} is written as zero
    for (int j = 0; j <= k; ++j) coef[j * ld + p] = 0.0;
    coef[(s - 1) * ld + p] = 0.0;
    return;
  }
  for (int j = 0; j < K1; ++j)
    coef[(j0 + j) * ld + p] = (double)(y[j * kSolveLanes] * sc[j * kSolveLanes]);
  coef[(s - 1) * ld + p] = first_pass ? rsqrt(gram[((int64_t)k * s + k) * ld + p]) : 1.0;
}

// ---------------------------------------------------------------- update
// u_{k+1} = zs (x - sum_{j<=k} coef_j u_j) with x = z and zs = 1/||u_k||
// (first pass), or x = the stored u_{k+1} and zs = 1 (second pass, in
// place), rounded to the basis type; stopped probes and padding columns get
// 0.  A pure streaming pass over the basis.
template <int P, bool SECOND, bool PARTIAL = false>
__global__ void __launch_bounds__(512)
    k_update(const typename Form<P>::TB *__restrict__ U, const typename Form<P>::TW *__restrict__ Z,
             typename Form<P>::TB *Unext, Slc S, const int64_t *__restrict__ crow0,
             const int32_t *__restrict__ crows, const int32_t *__restrict__ cgraph, int V, int R,
             int64_t ustride, int k, int s, const double *__restrict__ coef_all,
             const int32_t *__restrict__ m_all, int nv, const typename Form<P>::TW *__restrict__ yscale,
             typename Form<P>::TW *Ynext, const int32_t *__restrict__ pro_full) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  extern __shared__ __align__(16) unsigned char dyn[];
  const int ld = S.ld;
  const int gr = cgraph[blockIdx.x];
  const double *coef = coef_all + (int64_t)gr * s * ld;
  const int32_t *m = m_all + (int64_t)gr * nv;
  // coefficients, then the step's scale zs = 1/||u_k|| (row s-1 of coef;
  // 1 in the second pass): u_{k+1} = zs (x - sum_j c_j u_j)
  TW *cf = reinterpret_cast<TW *>(dyn);  // [(k+2) * ld]
  for (int i = threadIdx.x; i < (k + 1) * ld; i += blockDim.x) cf[i] = (TW)coef[i];
  for (int i = threadIdx.x; i < ld; i += blockDim.x)
    cf[(k + 1) * ld + i] = (TW)coef[(int64_t)(s - 1) * ld + i];
  __syncthreads();
  const int team = threadIdx.x / V, lane = threadIdx.x - team * V;
  if (team >= R) return;
  bool keep[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) {
    const int p = lane * VE + v;
    keep[v] = p < nv && m[p] > k;
  }
  const int64_t r0 = crow0[blockIdx.x];
  const int64_t r1 = r0 + crows[blockIdx.x];
  // partial reorthogonalization: only u_{k-1} and u_k unless the graph's step is full
  int j0 = 0;
  if constexpr (PARTIAL) j0 = pro_full[(int64_t)gr * (s + 2) + k] ? 0 : max(0, k - 1);
  int stride;
  const int64_t off = S.base(lane * VE, stride);
  for (int64_t row = r0 + team; row < r1; row += R) {
    const int64_t o = off + row * stride;
    TW x[VE];
    if (SECOND) ldb_rw(Unext + o, x);
    else ldw<TW, VE>(Z + o, x);
    int j = 0;
    if (PARTIAL && j0 > 0) {  // partial reorthogonalization step: u_{k-1} and u_k only
      TW u0[VE], u1[VE];
      ldb(U + (int64_t)(k - 1) * ustride + o, u0);
      ldb(U + (int64_t)k * ustride + o, u1);
      const TW *c0 = cf + (k - 1) * ld + lane * VE;
      const TW *c1 = c0 + ld;
#pragma unroll
      for (int v = 0; v < VE; ++v) {
        x[v] = fma(-c0[v], u0[v], x[v]);
        x[v] = fma(-c1[v], u1[v], x[v]);
      }
      j = k + 1;
    }
    for (; j + 2 <= k + 1; j += 2) {
      TW u0[VE], u1[VE];
      ldb(U + (int64_t)j * ustride + o, u0);
      ldb(U + (int64_t)(j + 1) * ustride + o, u1);
      const TW *c0 = cf + j * ld + lane * VE;
      const TW *c1 = c0 + ld;
#pragma unroll
      for (int v = 0; v < VE; ++v) {
        x[v] = fma(-c0[v], u0[v], x[v]);
        x[v] = fma(-c1[v], u1[v], x[v]);
      }
    }
    for (; j <= k; ++j) {
      TW u0[VE];
      ldb(U + (int64_t)j * ustride + o, u0);
      const TW *c0 = cf + j * ld + lane * VE;
#pragma unroll
      for (int v = 0; v < VE; ++v) x[v] = fma(-c0[v], u0[v], x[v]);
    }
    {
      const TW *zv = cf + (k + 1) * ld + lane * VE;
#pragma unroll
      for (int v = 0; v < VE; ++v) x[v] = keep[v] ? x[v] * zv[v] : TW(0);
    }
    TW r[VE];
    stb(Unext + o, x, r);
    if (Ynext) {  // pre-scaled copy for the next SpMM (MODE 3)
      const TW sc = yscale[row];
#pragma unroll
      for (int v = 0; v < VE; ++v) r[v] *= sc;
      stw<TW, VE>(Ynext + o, r);
    }
  }
}

// ------------------------------------------------------------ host side
constexpr int kMaxSub = 16;  // most pieces a dots chunk is split into
// Batches: dots chunks of about a quarter of a wave's rows, so that a large
// graph's chunks do not run on after the small graphs' blocks have finished
// (measured on 5000 SBM graphs: 7.9 -> 6.3 ms per FP32 run, 12.7 -> 9.0 with
// the BF16 basis; eight waves gained nothing more, nor did finer update
// chunks).  One graph: one wave of equal chunks.
constexpr int kBatchDotsWaves = 4;

struct Geometry {
  int V, R, threads;      // teams of V threads, R rows per pass (update)
  Slc S;                  // probe slicing of the basis and work vectors
  int Vt, Tw, Rt, tthreads;  // SpMM: Vt active of Tw threads per row and slice, Rt rows per block
  int sms;
  int Jb;                 // basis vectors per dots block
  int dots_threads;       // row phases fill narrow dots blocks up to this
};

// Slice width in elements: whole rows unless the tuning asks for slices of
// slice_bytes (rounded down to whole 32-byte sectors).  Measured on R-MAT
// 2^20, unsliced gathers are the fastest, so that is the default.
int slice_width(int precision, int ld, int slice_bytes) {
  if (slice_bytes <= 0) return ld;
  const int b = basis_bytes(precision);
  const int w = std::max(32 / b, slice_bytes / 32 * 32 / b);
  return std::min(w, ld);
}

Geometry geometry(int precision, int ld, int64_t n, int sms, const slaq_tuning &t) {
  Geometry g;
  g.sms = sms;
  g.S.n = n;
  g.S.ld = ld;
  g.S.w = slice_width(precision, ld, t.slice_bytes);
  g.Vt = g.S.w / vec_elems(precision);
  g.Tw = g.Vt;
  // measured: whole-warp teams win for wide rows (R-MAT, nv = 100 FP32: 26 of
  // 32 lanes), packed teams for narrow ones (BF16 nv = 100: 13 lanes; SBM
  // batches, nv = 20 FP32: 6 lanes)
  const bool align = t.spmm_align < 0 ? g.Vt > 16 : t.spmm_align != 0;
  if (align) {
    g.Tw = 1;
    while (g.Tw < g.Vt && g.Tw < 32) g.Tw *= 2;
    if (g.Vt > 32) g.Tw = (g.Vt + 31) / 32 * 32;
  }
  g.Rt = std::max(1, std::min(t.spmm_threads, 512) / g.Tw);
  g.tthreads = g.Tw * g.Rt;
  g.V = ld / vec_elems(precision);
  g.R = std::max(1, std::min(t.upd_threads, 512) / g.V);
  g.threads = g.V * g.R;
  const int dt = t.dots_threads > 0 ? t.dots_threads : (precision == SLAQ_FP32_BF16BASIS ? 256 : 128);
  g.dots_threads = std::max(32, std::min(dt, 512));
  g.Jb = std::max(1, std::min(64, 512 / g.V));
  return g;
}

// Row chunks of about `rows` rows that never cross a graph boundary; every
// graph gets at least one.  first[g] (optional) is graph g's first chunk.
void make_chunks(const std::vector<int64_t> &goff, int64_t rows, std::vector<int64_t> &row0,
                 std::vector<int32_t> &nr, std::vector<int32_t> &graph,
                 std::vector<int32_t> *first) {
  const int G = (int)goff.size() - 1;
  row0.clear();
  nr.clear();
  graph.clear();
  if (first) first->assign(G + 1, 0);
  rows = std::max<int64_t>(1, rows);
  for (int q = 0; q < G; ++q) {
    const int64_t a = goff[q], b = goff[q + 1];
    if (first) (*first)[q] = (int32_t)row0.size();
    const int64_t nch = std::max<int64_t>(1, ceil_div(b - a, rows));
    const int64_t per = std::max<int64_t>(1, ceil_div(b - a, nch));
    for (int64_t r = a; r < b; r += per) {
      row0.push_back(r);
      nr.push_back((int32_t)std::min(per, b - r));
      graph.push_back(q);
    }
  }
  if (first) (*first)[G] = (int32_t)row0.size();
}

template <typename Kern>
int blocks_per_sm(Kern kern, int threads, size_t smem) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm;
}

template <typename T>
int grow(T **p, size_t count);

template <typename T>
int upload(T **dev, int64_t *cap, const std::vector<T> &host, cudaStream_t st) {
  if ((int64_t)host.size() > *cap) {
    SLAQ_TRY(grow(dev, host.size()));
    *cap = (int64_t)host.size();
  }
  if (!host.empty())
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(*dev, host.data(), host.size() * sizeof(T),
                                    cudaMemcpyHostToDevice, st));
  return SLAQ_OK;
}

// ---------------------------------------------------- TMA light-row path
// Stages in flight per warp: 8 for rows of at most 128 bytes (the BF16
// basis with nv <= 64: three blocks of 8 warps still fit an SM), else 4.
inline int tma_stages(int row_bytes) { return row_bytes <= 128 ? 8 : 4; }

std::atomic<int> g_spmm_gathers{-1};

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                        &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// Decides the light-row path of this run and, for TMA, encodes the tensor
// map (rows of ld elements over the stored basis, or over y) and builds the
// work items.  Ineligible shapes keep the load path: sliced rows, rows wider
// than a TMA box (256 elements) or a warp, or more rows than an int32
// coordinate holds.
template <int P>
int tma_setup(slaq_graph gr, slaq_krylov K, const Geometry &geo, cudaStream_t st) {
  K->tma = false;
  if constexpr (P == SLAQ_FP64) {
    return SLAQ_OK;
  } else {
    using TB = typename Form<P>::TB;
    const int forced = g_spmm_gathers.load();
    const bool want = forced >= 0 ? forced != 0 : K->tune.spmm_tma > 0;
    if (!want || gr->n < 1) return SLAQ_OK;
    const int ld = K->ld;
    const int64_t rows = K->ymode ? gr->n : (int64_t)K->s * gr->n;
    const int rowb = ld * (int)sizeof(TB);
    if (geo.S.w != ld || ld > 256 || ld / Form<P>::VE > 32 || rows > INT32_MAX ||
        tma_block_smem(rowb, tma_stages(rowb)) > (size_t)227 * 1024)
      return SLAQ_OK;
    EncodeTiled enc = encode_tiled();
    if (!enc) return SLAQ_OK;
    void *gbase = K->ymode ? static_cast<void *>(K->Y) : K->U;
    const cuuint64_t gdim[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)rowb};
    const cuuint32_t box[2] = {(cuuint32_t)ld, 1};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult cr =
        enc(&K->tma_map,
            P == SLAQ_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            gbase, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return SLAQ_OK;
    const int64_t ntasks = gr->nnz / kTmaTaskEntries + 1;
    if (ntasks + 1 > K->tma_task_cap) {
      K->tma_task_cap = 0;
      SLAQ_TRY(grow(&K->tma_task, (size_t)(ntasks + 1)));
      K->tma_task_cap = ntasks + 1;
    }
    ++tl_launches;
    k_tma_tasks<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ntasks + 1, 256), 4096)),
                  256, 0, st>>>(gr->x_rowptr, gr->n, kTmaTaskEntries, ntasks, K->tma_task);
    SLAQ_CHECK_LAUNCH("tma_tasks");
    K->tma_ntasks = ntasks;
    K->tma = true;
    return SLAQ_OK;
  }
}

template <int P, int MODE, int G, int NS>
int launch_tma(slaq_graph gr, slaq_krylov K, int row0, const typename Form<P>::TW *vals,
               const typename Form<P>::TW *diag, const typename Form<P>::TW *scale,
               const typename Form<P>::TB *Uk, typename Form<P>::TW *Z, cudaStream_t st) {
  using TB = typename Form<P>::TB;
  auto kern = k_spmm_tma<P, MODE, G, NS>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  SLAQ_CHECK_CUDA(attr);
  const size_t smem = tma_block_smem(K->ld * (int)sizeof(TB), NS);
  const int per_sm = blocks_per_sm(kern, 32 * kTmaWarps, smem);
  const int64_t blocks = std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(K->tma_ntasks, kTmaWarps), (int64_t)per_sm * num_sms()));
  ++tl_launches;
  kern<<<(unsigned)blocks, 32 * kTmaWarps, smem, st>>>(K->tma_map, row0, gr->x_rowptr,
                                                      gr->x_colidx, vals, diag, scale, Uk, Z, K->ld,
                                                      gr->heavy_degree, K->tma_task, K->tma_ntasks,
                                                      K->status + 1, g_tma_giveup.load());
  return SLAQ_OK;
}

template <int P, int MODE>
int spmm_tma(slaq_graph gr, slaq_krylov K, int row0, const typename Form<P>::TW *vals,
             const typename Form<P>::TW *diag, const typename Form<P>::TW *scale,
             const typename Form<P>::TB *Uk, typename Form<P>::TW *Z, cudaStream_t st) {
  // one, two or four rows per warp; rows of at most 8 lanes (128 bytes)
  // take four rows per warp and 8 stages (tma_stages)
  const int V = K->ld / Form<P>::VE;
  if (V > 16) return launch_tma<P, MODE, 1, 4>(gr, K, row0, vals, diag, scale, Uk, Z, st);
  if (V > 8) return launch_tma<P, MODE, 2, 4>(gr, K, row0, vals, diag, scale, Uk, Z, st);
  return launch_tma<P, MODE, 4, 8>(gr, K, row0, vals, diag, scale, Uk, Z, st);
}

template <int P>
int spmm(slaq_graph gr, slaq_krylov K, const Geometry &geo, int k, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_SPMM, st);
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  const int64_t n = gr->n;
  const TB *Uk = static_cast<const TB *>(K->U) + (int64_t)k * n * K->ld;
  TW *Z = static_cast<TW *>(K->Z);
  const TW *vals, *diag, *scale;
  if constexpr (P == SLAQ_FP64) {
    vals = gr->x_vals;
    diag = gr->x_diag;
    scale = gr->x_scale;
  } else {
    vals = gr->x_vals32;
    diag = gr->x_diag32;
    scale = gr->x_scale32;
  }
  const int mode =
      gr->weighted ? 2 : (gr->kind == SLAQ_NORMALIZED ? (K->ymode ? 3 : 0) : 1);
  const TB *Yg = nullptr;
  if constexpr (P == SLAQ_FP32) Yg = K->Y;
  const int ns = geo.S.nslices();
  const int64_t bps = ceil_div(n, geo.Rt);
  const unsigned blocks = (unsigned)(ns * bps);
  const unsigned hblocks = (unsigned)(ns * gr->n_chunks);
  const int hthreads = (int)ceil_div(geo.Vt, 32) * 32;
  const unsigned hwblocks = (unsigned)(ns * ceil_div(gr->n_chunks, (int64_t)kHeavyWarps));
#define SLAQ_SPMM_CASE(MODE)                                                                    \
  if (gr->n_chunks > 0 && hthreads == 32) {                                                     \
    ++tl_launches;                                                                              \
    k_spmm_heavy_warps<P, MODE><<<hwblocks, 32 * kHeavyWarps, 0, K->side>>>(                    \
        gr->x_rowptr, gr->x_colidx, vals, diag, scale, Uk, Z, static_cast<TW *>(K->P),          \
        gr->heavy_row, gr->heavy_first, gr->chunk_slot, K->hcount, Yg, geo.S, geo.Vt,           \
        gr->n_chunks);                                                                          \
  } else if (gr->n_chunks > 0) {                                                                \
    ++tl_launches;                                                                              \
    k_spmm_heavy<P, MODE><<<hblocks, hthreads, 0, K->side>>>(                                   \
        gr->x_rowptr, gr->x_colidx, vals, diag, scale, Uk, Z, static_cast<TW *>(K->P),          \
        gr->heavy_row, gr->heavy_first, gr->chunk_slot, K->hcount, Yg, geo.S, geo.Vt,           \
        gr->n_chunks);                                                                          \
  }                                                                                             \
  if (K->tma) {                                                                                 \
    if constexpr (P != SLAQ_FP64)                                                               \
      SLAQ_TRY((spmm_tma<P, MODE>(gr, K, MODE == 3 ? 0 : (int)((int64_t)k * n), vals, diag,      \
                                  scale, Uk, Z, st)));                                          \
  } else {                                                                                      \
    ++tl_launches;                                                                              \
    k_spmm_light<P, MODE><<<blocks, geo.tthreads, 0, st>>>(                                     \
        gr->x_rowptr, gr->x_colidx, vals, diag, scale, Uk, Z, Yg, geo.S, geo.Vt, geo.Tw,        \
        geo.Rt, bps, gr->heavy_degree);                                                         \
  }
  // split rows on the side stream, concurrently with the light rows (the two
  // write disjoint rows of z)
  if (gr->n_chunks > 0) {
    SLAQ_CHECK_CUDA(cudaEventRecord(K->ev_fork, st));
    SLAQ_CHECK_CUDA(cudaStreamWaitEvent(K->side, K->ev_fork, 0));
  }
  if (mode == 0) {
    SLAQ_SPMM_CASE(0)
  } else if (mode == 1) {
    SLAQ_SPMM_CASE(1)
  } else if (mode == 2) {
    SLAQ_SPMM_CASE(2)
  } else {
    if constexpr (P == SLAQ_FP32) { SLAQ_SPMM_CASE(3) }
  }
  if (gr->n_chunks > 0) {
    SLAQ_CHECK_CUDA(cudaEventRecord(K->ev_join, K->side));
    SLAQ_CHECK_CUDA(cudaStreamWaitEvent(st, K->ev_join, 0));
  }
#undef SLAQ_SPMM_CASE
  SLAQ_CHECK_LAUNCH("spmm");
  return SLAQ_OK;
}

// Dot products of basis vectors jfirst..jlast with X (z, or u_{k+1} when
// x_is_basis), plus the Gram column of u_k when with_g; one block per dots
// chunk and group of Jb basis vectors.
template <int P>
int dots(slaq_krylov K, const Geometry &geo, int64_t n, int k, int jfirst, int jlast,
         bool x_is_basis, bool with_g, const void *X, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_DOTS, st);
  using TB = typename Form<P>::TB;
  const int jcount = jlast - jfirst + 1;
  const int Jb = std::min(jcount, geo.Jb);
  const int RZ = dots_phases(geo.V, Jb, geo.dots_threads);
  const size_t smem = dots_smem(P, K->ld, x_is_basis, Jb, RZ);
  const int tr = dots_tile_rows(P, K->ld, x_is_basis);
  const int threads = geo.V * Jb * RZ;
  // split every chunk so that small blocks (few basis vectors) still fill the SMs
  int per_sm;
  if (x_is_basis) per_sm = blocks_per_sm(k_dots<P, true, false>, threads, smem);
  else if (with_g) per_sm = blocks_per_sm(k_dots<P, false, true>, threads, smem);
  else per_sm = blocks_per_sm(k_dots<P, false, false>, threads, smem);
  const int64_t want = (int64_t)geo.sms * per_sm;
  const int sub = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)kMaxSub, want / std::max(1, K->n_dchunks),
                            (int64_t)K->G / std::max(1, K->n_dchunks)}));
  K->dsub = sub;
  const dim3 grid(K->n_dchunks * sub, (unsigned)ceil_div(jcount, Jb));
  const dim3 block(geo.V, Jb, RZ);
  const TB *U = static_cast<const TB *>(K->U);
  const TB *Uk = U + (int64_t)k * n * K->ld;
  const int64_t ustride = n * K->ld;
  ++tl_launches;
  if (x_is_basis)
    k_dots<P, true, false><<<grid, block, smem, st>>>(U, X, Uk, geo.S, K->d_row0, K->d_rows, sub,
                                                      ustride, jfirst, jlast, Jb, K->part, K->s, tr);
  else if (with_g)
    k_dots<P, false, true><<<grid, block, smem, st>>>(U, X, Uk, geo.S, K->d_row0, K->d_rows, sub,
                                                      ustride, jfirst, jlast, Jb, K->part, K->s, tr);
  else
    k_dots<P, false, false><<<grid, block, smem, st>>>(U, X, Uk, geo.S, K->d_row0, K->d_rows, sub,
                                                       ustride, jfirst, jlast, Jb, K->part, K->s, tr);
  SLAQ_CHECK_LAUNCH("dots");
  return SLAQ_OK;
}

ProArgs pro_args(slaq_krylov K) {
  ProArgs P{nullptr, nullptr, nullptr, 0.0};
  if (K->reorth == 0) {
    P.full = K->pro_full;
    P.any = K->pro_any;
    P.omega = K->omega;
    P.eps = K->precision == SLAQ_FP64 ? 0x1p-53 : 0x1p-24;
  }
  return P;
}

int reduce_and_solve(slaq_krylov K, int k, int jfirst, int jcount, bool with_g, bool first_pass,
                     bool need_coef, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_REDUCE, st);
  // the projected matrix feeds the reduced forms' Rayleigh-Ritz step, which
  // partial reorthogonalization does not use (null for the FP64 form too)
  double *pj = (with_g && K->reorth != 0) ? K->proj : nullptr;
  const ProArgs P = pro_args(K);
  ++tl_launches;
  // a block per graph and column group pays off for few graphs with many
  // partials each (one large graph); thousands of graphs take one thread per
  // output (a block per graph there cost 29 ms against 1.4 on 5000 graphs)
  if (K->max_chunks_per_graph * K->dsub >= 8 && K->n_graphs <= 256) {
    const dim3 grid((unsigned)ceil_div((int64_t)jcount * K->ld, 32), with_g ? 2 : 1,
                    (unsigned)K->n_graphs);
    k_dot_reduce<<<grid, dim3(32, kRedY), 0, st>>>(K->part, K->d_goff, K->dsub, K->s, K->ld, jfirst,
                                                   jcount, k, K->dsum, K->gram, pj);
  } else {
    const int64_t total = (int64_t)K->n_graphs * (with_g ? 2 : 1) * jcount * K->ld;
    k_dot_reduce_narrow<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 65535LL * 16), 256, 0,
                          st>>>(K->part, K->d_goff, K->dsub, K->s, K->ld, jfirst, jcount, k,
                                K->n_graphs, with_g ? 1 : 0, K->dsum, K->gram, pj);
  }
  const int K1 = k + 1;
  const int64_t problems = (int64_t)K->n_graphs * K->nv;
  const int tbytes = K->precision == SLAQ_FP64 ? 8 : 4;
  ++tl_launches;
  if (problems >= kSolveLanesMin && solve_lanes_smem(K1, tbytes) <= kSolveLanesSmemMax) {
    // many small problems: thread per problem
    const unsigned blocks = (unsigned)ceil_div(problems, kSolveLanes);
    const size_t smem = solve_lanes_smem(K1, tbytes);
    if (tbytes == 8)
      k_solve_lanes<double><<<blocks, kSolveLanes, smem, st>>>(
          K->dsum, K->gram, k, K->s, K->ld, K->nv, K->n_graphs, first_pass ? 1 : 0,
          need_coef ? 1 : 0, K->tol, K->gbound, K->m, K->alpha, K->beta, K->coef, P, jfirst);
    else
      k_solve_lanes<float><<<blocks, kSolveLanes, smem, st>>>(
          K->dsum, K->gram, k, K->s, K->ld, K->nv, K->n_graphs, first_pass ? 1 : 0,
          need_coef ? 1 : 0, K->tol, K->gbound, K->m, K->alpha, K->beta, K->coef, P, jfirst);
  } else {
    // few problems: a warp per problem spreads them over the SMs
    const size_t smem = (size_t)(K1 * K1 + 2 * K1) * sizeof(double);
    k_solve<<<dim3(K->nv, K->n_graphs), 32, smem, st>>>(
        K->dsum, K->gram, k, K->s, K->ld, K->nv, first_pass ? 1 : 0, need_coef ? 1 : 0, K->tol,
        K->gbound, K->m, K->alpha, K->beta, K->coef, P, jfirst);
  }
  SLAQ_CHECK_LAUNCH("reduce_and_solve");
  return SLAQ_OK;
}

template <int P>
int update(slaq_krylov K, const Geometry &geo, int64_t n, int k, bool second, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_UPDATE, st);
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  const TB *U = static_cast<const TB *>(K->U);
  TB *Unext = static_cast<TB *>(K->U) + (int64_t)(k + 1) * n * K->ld;
  const int64_t ustride = n * K->ld;
  // the FP32 form also writes y = s * u_{k+1} for the next SpMM (MODE 3)
  const TW *yscale = nullptr;
  TW *Ynext = nullptr;
  if constexpr (P == SLAQ_FP32) {
    if (K->ymode) {
      yscale = K->yscale;
      Ynext = K->Y;
    }
  }
  const size_t smem = (size_t)(k + 2) * K->ld * sizeof(TW);
  const TW *Z = static_cast<const TW *>(K->Z);
  ++tl_launches;
  if (second)
    k_update<P, true><<<K->n_uchunks, geo.threads, smem, st>>>(
        U, Z, Unext, geo.S, K->u_row0, K->u_rows, K->u_graph, geo.V, geo.R, ustride, k, K->s,
        K->coef, K->m, K->nv, yscale, Ynext, nullptr);
  else if (K->reorth == 0)
    k_update<P, false, true><<<K->n_uchunks, geo.threads, smem, st>>>(
        U, Z, Unext, geo.S, K->u_row0, K->u_rows, K->u_graph, geo.V, geo.R, ustride, k, K->s,
        K->coef, K->m, K->nv, yscale, Ynext, K->pro_full);
  else
    k_update<P, false><<<K->n_uchunks, geo.threads, smem, st>>>(
        U, Z, Unext, geo.S, K->u_row0, K->u_rows, K->u_graph, geo.V, geo.R, ustride, k, K->s,
        K->coef, K->m, K->nv, yscale, Ynext, nullptr);
  SLAQ_CHECK_LAUNCH("update");
  return SLAQ_OK;
}

// launch_only: the chunk tables and buffers of this graph are in place (a
// replay capture); only the run's launches are issued.
template <int P>
int lanczos_form(slaq_graph gr, slaq_krylov K, cudaStream_t st, bool launch_only) {
  using TB = typename Form<P>::TB;
  const int64_t n = gr->n;
  K->ymode = P == SLAQ_FP32 && !gr->weighted && gr->kind == SLAQ_NORMALIZED && K->Y;
  K->yscale = gr->x_scale32;
  const Geometry geo = geometry(P, K->ld, n, num_sms(), K->tune);
  // once per process and form (a thread-safe static initialization)
  static const cudaError_t attr = [] {
    const void *fs[] = {(const void *)k_update<P, false>, (const void *)k_update<P, true>,
                        (const void *)k_update<P, false, true>,
                        (const void *)k_dots<P, false, true>, (const void *)k_dots<P, false, false>,
                        (const void *)k_dots<P, true, false>};
    for (const void *f : fs) {
      const cudaError_t e =
          cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDotsSmemMax);
      if (e != cudaSuccess) return e;
    }
    const void *gs[] = {(const void *)k_solve_lanes<double>, (const void *)k_solve_lanes<float>};
    for (const void *f : gs) {
      const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSolveLanesSmemMax);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }();
  SLAQ_CHECK_CUDA(attr);
  // chunk tables: dots chunks fill one wave; update chunks are smaller
  if (!launch_only) {
    const int Jb = std::min(K->s, geo.Jb);
    const int RZ = dots_phases(geo.V, Jb, geo.dots_threads);
    const int per_sm = blocks_per_sm(k_dots<P, false, true>, geo.V * Jb * RZ,
                                     dots_smem(P, K->ld, false, Jb, RZ));
    const int64_t want_d = (int64_t)geo.sms * per_sm;
    const int64_t waves_d = gr->n_graphs > 1 ? kBatchDotsWaves : 1;
    const int64_t rows_d = std::max<int64_t>(64, ceil_div(n, want_d * waves_d));
    make_chunks(gr->goff, rows_d, K->hd_row0, K->hd_rows, K->hd_graph, &K->hd_goff);
    const int64_t want_u = std::min<int64_t>(std::max<int64_t>(1, ceil_div(n, 8LL * geo.R)),
                                             16LL * geo.sms);
    const int64_t rows_u = std::max<int64_t>(1, ceil_div(n, want_u));
    make_chunks(gr->goff, rows_u, K->hu_row0, K->hu_rows, K->hu_graph, nullptr);
    K->n_dchunks = (int)K->hd_row0.size();
    K->n_uchunks = (int)K->hu_row0.size();
    K->max_chunks_per_graph = 1;
    for (size_t q = 0; q + 1 < K->hd_goff.size(); ++q)
      K->max_chunks_per_graph = std::max(K->max_chunks_per_graph, K->hd_goff[q + 1] - K->hd_goff[q]);
    int64_t c0 = K->dcap, c1 = K->dcap, c2 = K->dcap;
    K->dcap = 0;  // until the three tables below are in place
    SLAQ_TRY(upload(&K->d_row0, &c0, K->hd_row0, st));
    SLAQ_TRY(upload(&K->d_rows, &c1, K->hd_rows, st));
    SLAQ_TRY(upload(&K->d_goff, &c2, K->hd_goff, st));
    K->dcap = std::min({c0, c1, c2});
    int64_t u0 = K->ucap, u1 = K->ucap, u2 = K->ucap;
    K->ucap = 0;
    SLAQ_TRY(upload(&K->u_row0, &u0, K->hu_row0, st));
    SLAQ_TRY(upload(&K->u_rows, &u1, K->hu_rows, st));
    SLAQ_TRY(upload(&K->u_graph, &u2, K->hu_graph, st));
    K->ucap = std::min({u0, u1, u2});
    // partial rows: chunks x pieces, where dots() splits chunks into at most
    // kMaxSub pieces and only while fewer than sms * 32 blocks (the most an
    // SM holds) would result
    const int64_t pieces = std::max<int64_t>(
        1, std::min<int64_t>(kMaxSub, (int64_t)geo.sms * 32 / std::max(1, K->n_dchunks)));
    if ((int64_t)K->n_dchunks * pieces > K->G) {
      K->G = 0;
      SLAQ_TRY(grow(&K->part, (size_t)K->n_dchunks * pieces * 2 * K->s * K->ld));
      K->G = (int)(K->n_dchunks * pieces);
    }
  }
  if (!launch_only) SLAQ_TRY(tma_setup<P>(gr, K, geo, st));
  SLAQ_CHECK_CUDA(cudaMemsetAsync(K->status + 1, 0, sizeof(int32_t), st));
  {
    ProfScope prof(SLAQ_PROF_PROBES, st);
    const int64_t nvt = (int64_t)K->n_graphs * K->nv;
    ++tl_launches;
    k_init_scalars<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nvt * K->s, 256), 1024)),
                     256, 0, st>>>(K->alpha, K->beta, K->m, nvt * K->s, nvt, K->s, K->nv, K->gn);
    ++tl_launches;
    k_probe_init<P><<<(unsigned)std::min<int64_t>(ceil_div(n * K->ld, 256), 152LL * 64), 256, 0,
                      st>>>(static_cast<TB *>(K->U), gr->x_old_id, gr->x_graph, geo.S, K->nv,
                            K->seed_dev, (uint64_t)K->graph_id, (uint64_t)K->probe0,
                            K->ymode ? K->yscale : nullptr,
                            K->ymode ? K->Y : nullptr);
  }
  SLAQ_CHECK_LAUNCH("probe_init");
  const bool pro = K->reorth == 0;
  if (pro) {
    SLAQ_CHECK_CUDA(cudaMemsetAsync(K->pro_full, 0, (size_t)K->n_graphs * (K->s + 2) * 4, st));
    SLAQ_CHECK_CUDA(cudaMemsetAsync(K->pro_any, 0, (size_t)(K->s + 2) * 4, st));
  }
  for (int k = 0; k < K->s; ++k) {
    SLAQ_TRY(spmm<P>(gr, K, geo, k, st));
    const bool last = (k == K->s - 1);
    // last step: only alpha_k = d_k / G_kk and the Gram diagonal entry, except
    // for the reduced forms, whose Rayleigh-Ritz step needs the whole column
    // of the projected matrix
    int jfirst = (last && (P == SLAQ_FP64 || pro)) ? k : 0;
    if (pro && !last && k >= 2) {
      // partial reorthogonalization: project on all vectors only if some
      // graph's flag for this step is set (decided by step k-1's solve; the
      // update of step k-1 and this SpMM run on the device meanwhile)
      SLAQ_CHECK_CUDA(cudaEventSynchronize(K->ev_flag));
      if (!K->pro_any_host[k]) jfirst = k - 1;
    }
    SLAQ_TRY(dots<P>(K, geo, n, k, jfirst, k, false, true, K->Z, st));
    SLAQ_TRY(reduce_and_solve(K, k, jfirst, k - jfirst + 1, true, true, !last, st));
    if (pro && k >= 1 && k + 1 < K->s - 1) {
      SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->pro_any_host + k + 1, K->pro_any + k + 1, sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, st));
      SLAQ_CHECK_CUDA(cudaEventRecord(K->ev_flag, st));
    }
    if (last) break;
    SLAQ_TRY(update<P>(K, geo, n, k, false, st));
    if (K->reorth == 2) {
      const TB *Unext = static_cast<const TB *>(K->U) + (int64_t)(k + 1) * n * K->ld;
      SLAQ_TRY(dots<P>(K, geo, n, k, 0, k, true, false, Unext, st));
      SLAQ_TRY(reduce_and_solve(K, k, 0, k + 1, false, false, true, st));
      SLAQ_TRY(update<P>(K, geo, n, k, true, st));
    }
  }
  return SLAQ_OK;
}

double default_tol(int precision) {
  // the BF16 form takes the FP32 bar: its new vectors are formed in FP32
  // (only the stored copy is rounded to BF16), so beta is as accurate as in
  // the FP32 form, and a looser bar truncates legitimately small betas
  // (a 2600-node star's beta_0 is 0.029)
  return precision == SLAQ_FP64 ? 1e-10 : 1e-4;
}

// Replaces *p by a new allocation of count elements (the old contents are
// dropped).  On failure *p is NULL: callers reset the capacity that covers
// *p before growing, so a later call on the handle grows it again instead of
// launching a kernel on NULL.
template <typename T>
int grow(T **p, size_t count) {
  dmfree(*p);
  *p = nullptr;
  return dmalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

namespace {
// out[g][k] = 1 if step k of graph g formed u_{k+1} by projecting against
// all previous vectors (k < min(max_p m_gp, s - 1); with partial
// reorthogonalization only steps 0, 1 and the flagged ones)
__global__ void k_full_steps(const int32_t *pro_full, const int32_t *m_all, int G, int nv, int s,
                             int32_t *out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)G * s) return;
  const int g = (int)(i / s), k = (int)(i - (int64_t)g * s);
  int mx = 0;
  for (int p = 0; p < nv; ++p) mx = max(mx, m_all[(int64_t)g * nv + p]);
  const bool formed = k < min(mx, s - 1);
  const bool full = !pro_full || k <= 1 || pro_full[(int64_t)g * (s + 2) + k];
  out[i] = formed && full ? 1 : 0;
}
}  // namespace

int full_steps(slaq_krylov K, int32_t *out, cudaStream_t st) {
  if (!K || !out) return set_error(SLAQ_EINVAL, "NULL Krylov handle or output");
  const int64_t total = (int64_t)K->n_graphs * K->s;
  ++tl_launches;
  k_full_steps<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(
      K->reorth == 0 ? K->pro_full : nullptr, K->m, K->n_graphs, K->nv, K->s, out);
  SLAQ_CHECK_LAUNCH("full_steps");
  return SLAQ_OK;
}

int probes(slaq_graph g, int nv, uint64_t seed, int graph_id, double *out, cudaStream_t st) {
  if (!g || !out) return set_error(SLAQ_EINVAL, "NULL graph or output");
  if (nv < 1 || graph_id < 0 || graph_id > 0xffff) return set_error(SLAQ_EINVAL, "bad nv or graph_id");
  if (g->n_graphs != 1) return set_error(SLAQ_EUNSUPPORTED, "probe export is for single graphs");
  if (g->n == 0) return SLAQ_OK;
  ProfScope prof(SLAQ_PROF_PROBES, st);
  ++tl_launches;
  k_probe_export<<<(unsigned)std::min<int64_t>(ceil_div(g->n * nv, 256), 152LL * 64), 256, 0, st>>>(
      out, g->old_id, g->n, nv, seed, (uint64_t)graph_id);
  SLAQ_CHECK_LAUNCH("probes");
  return SLAQ_OK;
}

void krylov_free(slaq_krylov k) {
  if (!k) return;
  void *ptrs[] = {k->U, k->Z, k->Y, k->P, k->part, k->dsum, k->coef, k->gram, k->proj, k->rscratch,
                  k->alpha, k->beta,
                  k->m, k->theta, k->tau2, k->status, k->hcount, k->gn, k->gtrace, k->gtrace2,
                  k->gbound,
                  k->d_row0, k->d_rows, k->d_goff, k->u_row0, k->u_rows, k->u_graph,
                  k->pro_full, k->pro_any, k->omega, k->tma_task};
  for (void *p : ptrs) dmfree(p);
  hmfree(k->pro_any_host);
  if (k->ev_flag) cudaEventDestroy(k->ev_flag);
  dmfree(k->seed_dev);
  if (k->gexec) cudaGraphExecDestroy(k->gexec);
  if (k->cap) cudaStreamDestroy(k->cap);
  if (k->ev_fork) cudaEventDestroy(k->ev_fork);
  if (k->ev_join) cudaEventDestroy(k->ev_join);
  if (k->side) cudaStreamDestroy(k->side);
  graph_free(k->owned, 0);  // callers have synchronized the device or k's stream
  delete k;
}

int run_lanczos(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision,
                int reorth, cudaStream_t st, slaq_krylov *inout, const slaq_tuning *tune,
                int probe0) {
  if (!g || !inout) return set_error(SLAQ_EINVAL, "NULL graph or output handle");
  if (nv < 1 || nv > 512) return set_error(SLAQ_EINVAL, "nv must be in [1, 512]");
  if (probe0 < 0 || (int64_t)probe0 + nv > 65536)
    return set_error(SLAQ_EINVAL, "probes probe0 .. probe0 + nv - 1 must lie in [0, 65536)");
  if (s < 1 || s > 64) return set_error(SLAQ_EINVAL, "s must be in [1, 64]");
  if (graph_id < 0 || graph_id > 0xffff) return set_error(SLAQ_EINVAL, "graph_id must be < 65536");
  if (precision != SLAQ_FP64 && precision != SLAQ_FP32 && precision != SLAQ_FP32_BF16BASIS)
    return set_error(SLAQ_EINVAL, "unknown precision %d", precision);
  if (reorth != 0 && reorth != 1 && reorth != 2)
    return set_error(SLAQ_EINVAL, "reorth_passes must be 0 (partial), 1 or 2");
  if (reorth == 0 && precision == SLAQ_FP32_BF16BASIS)
    return set_error(SLAQ_EUNSUPPORTED,
                     "partial reorthogonalization needs an FP64 or FP32 basis (BF16 storage "
                     "rounds above the semi-orthogonality level)");
  if (g->n < 1) return set_error(SLAQ_EINVAL, "graph has no nodes");
  if (g->n > (1LL << 31)) return set_error(SLAQ_EUNSUPPORTED, "too many nodes");
  const int ld = row_ld(nv, precision);
  if ((size_t)s * ld * work_bytes(precision) > kDotsSmemMax)
    return set_error(SLAQ_EUNSUPPORTED, "s * nv too large for the update kernel's coefficient table");
  slaq_krylov K = *inout;
  const bool fresh = (K == nullptr);
  if (!fresh && (K->nv != nv || K->s != s || K->precision != precision))
    return set_error(SLAQ_EINVAL, "reused Krylov handle has a different nv, s or precision");
  if (fresh) {
    K = new slaq_krylov_s();
    K->nv = nv;
    K->s = s;
    K->precision = precision;
    K->ld = ld;
    SLAQ_CHECK_CUDA(cudaGetDevice(&K->device));
    SLAQ_CHECK_CUDA(cudaStreamCreateWithFlags(&K->side, cudaStreamNonBlocking));
    SLAQ_CHECK_CUDA(cudaEventCreateWithFlags(&K->ev_fork, cudaEventDisableTiming));
    SLAQ_CHECK_CUDA(cudaEventCreateWithFlags(&K->ev_join, cudaEventDisableTiming));
  }
  struct Guard {
    slaq_krylov *K;
    bool fresh;
    ~Guard() {
      if (fresh && *K) {
        cudaDeviceSynchronize();  // launches of the failed run may still read its buffers
        krylov_free(*K);
      }
    }
  } guard{&K, fresh};
  if (graph_id + g->n_graphs - 1 > 0xffff)
    return set_error(SLAQ_EINVAL, "graph_id + n_graphs - 1 must be < 65536");
  K->ready = false;  // until this run has completed
  K->tune = tune ? *tune : slaq_tuning();
  const int64_t n = g->n;
  const int G = g->n_graphs;
  const Geometry geo = geometry(precision, ld, n, num_sms(), K->tune);
  if (n > K->n_cap) {
    K->n_cap = 0;  // until every buffer below is grown
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->U), (size_t)s * n * ld * basis_bytes(precision)));
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->Z), (size_t)n * ld * work_bytes(precision)));
    if (precision == SLAQ_FP32) SLAQ_TRY(grow(&K->Y, (size_t)n * ld));
    K->n_cap = n;
  }
  if (g->n_chunks > K->chunk_cap || !K->P) {
    const int64_t cap = std::max<int64_t>(g->n_chunks, 1);
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->P), (size_t)cap * ld * work_bytes(precision)));
    K->chunk_cap = cap;
  }
  {
    const int64_t need = std::max<int64_t>(1, g->n_heavy * geo.S.nslices());
    if (need > K->hcount_cap) {
      K->hcount_cap = 0;
      SLAQ_TRY(grow(&K->hcount, (size_t)need));
      SLAQ_CHECK_CUDA(cudaMemsetAsync(K->hcount, 0, need * sizeof(uint32_t), st));
      K->hcount_cap = need;
    }
  }
  if (G > K->gcap) {
    K->gcap = 0;  // until every per-graph array below is grown
    const size_t ns = (size_t)G * nv * s;
    SLAQ_TRY(grow(&K->dsum, (size_t)G * s * ld));
    SLAQ_TRY(grow(&K->coef, (size_t)G * s * ld));
    // padding columns of the coefficients are never written: keep them zero
    SLAQ_CHECK_CUDA(cudaMemsetAsync(K->coef, 0, (size_t)G * s * ld * sizeof(double), st));
    SLAQ_TRY(grow(&K->gram, (size_t)G * s * s * ld));
    if (precision != SLAQ_FP64) SLAQ_TRY(grow(&K->proj, (size_t)G * s * s * ld));
    SLAQ_TRY(grow(&K->alpha, ns));
    SLAQ_TRY(grow(&K->beta, ns));
    SLAQ_TRY(grow(&K->m, (size_t)G * nv));
    SLAQ_TRY(grow(&K->theta, ns));
    SLAQ_TRY(grow(&K->tau2, ns));
    SLAQ_TRY(grow(&K->gn, (size_t)G));
    SLAQ_TRY(grow(&K->gtrace, (size_t)G));
    SLAQ_TRY(grow(&K->gtrace2, (size_t)G));
    SLAQ_TRY(grow(&K->gbound, (size_t)G));
    K->gcap = G;
  }
  // status word (int32 [0]), then two 64-bit words at byte 8 for the monitor
  if (!K->status) SLAQ_TRY(grow(&K->status, 8));
  if (reorth == 0 && G > K->pro_gcap) {
    K->pro_gcap = 0;
    SLAQ_TRY(grow(&K->pro_full, (size_t)G * (s + 2)));
    SLAQ_TRY(grow(&K->omega, (size_t)G * nv * 3 * s));
    K->pro_gcap = G;
  }
  if (reorth == 0) {
    if (!K->pro_any) SLAQ_TRY(grow(&K->pro_any, (size_t)s + 2));
    if (!K->pro_any_host)
      SLAQ_TRY(hmalloc(reinterpret_cast<void **>(&K->pro_any_host), (size_t)(s + 2) * sizeof(int32_t)));
    if (!K->ev_flag) SLAQ_CHECK_CUDA(cudaEventCreateWithFlags(&K->ev_flag, cudaEventDisableTiming));
  }
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->gn, g->gn_dev, G * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->gtrace2, g->gtrace2_dev, G * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->gtrace, g->gtrace_dev, G * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->gbound, g->gbound_dev, G * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
  K->seed = seed;
  if (!K->seed_dev) SLAQ_TRY(grow(&K->seed_dev, 1));
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->seed_dev, &K->seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  // a replay graph of an earlier run no longer matches
  if (K->gexec) cudaGraphExecDestroy(K->gexec);
  K->gexec = nullptr;
  K->last_g = g;
  K->last_uid = g->uid;
  K->graph_id = graph_id;
  K->probe0 = probe0;
  K->reorth = reorth;
  K->n = n;
  K->n_graphs = G;
  K->kind = g->kind;
  K->trace = g->trace;
  K->bound = g->bound;
  K->tol = default_tol(precision);
  int r;
  if (precision == SLAQ_FP64) r = lanczos_form<SLAQ_FP64>(g, K, st, false);
  else if (precision == SLAQ_FP32) r = lanczos_form<SLAQ_FP32>(g, K, st, false);
  else r = lanczos_form<SLAQ_FP32_BF16BASIS>(g, K, st, false);
  if (r != SLAQ_OK) return r;
  SLAQ_TRY(run_ritz(K, st));
  K->ready = true;
  *inout = K;
  guard.fresh = false;  // the caller owns it now
  return SLAQ_OK;
}

int set_spmm_gathers(int mode) {
  if (mode < -1 || mode > 1) return set_error(SLAQ_EINVAL, "gather path must be -1, 0 or 1");
  g_spmm_gathers.store(mode);
  return SLAQ_OK;
}

int krylov_ready(slaq_krylov K) {
  if (!K) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  if (!K->ready)
    return set_error(SLAQ_EINVAL, "the Krylov handle's last run did not complete; run it again");
  return SLAQ_OK;
}

// Replays the last run's launches (probe init, s Lanczos steps, Gauss rules)
// with a new seed.  The first call captures them into a CUDA graph on a
// private stream (capture needs a stream other than the legacy default one);
// later calls only copy the seed and launch the graph.  Partial
// reorthogonalization decides on the host between steps and is not replayed.
int lanczos_rerun(slaq_krylov K, uint64_t seed, cudaStream_t st) {
  if (!K || !K->last_g) return set_error(SLAQ_EINVAL, "Krylov handle has no run to replay");
  SLAQ_TRY(krylov_ready(K));
  if (!graph_alive(K->last_g, K->last_uid))
    return set_error(SLAQ_EINVAL, "the graph of the run to replay has been destroyed");
  if (K->reorth == 0)
    return set_error(SLAQ_EUNSUPPORTED, "partial reorthogonalization is not replayed");
  if (!K->gexec) {
    if (!K->cap) SLAQ_CHECK_CUDA(cudaStreamCreateWithFlags(&K->cap, cudaStreamNonBlocking));
    // the capture stream starts after the work already on st
    SLAQ_CHECK_CUDA(cudaEventRecord(K->ev_fork, st));
    SLAQ_CHECK_CUDA(cudaStreamWaitEvent(K->cap, K->ev_fork, 0));
    SLAQ_CHECK_CUDA(cudaStreamBeginCapture(K->cap, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = tl_launches;
    int r;
    {
      ProfPause pause;  // no profiling events inside the capture
      if (K->precision == SLAQ_FP64) r = lanczos_form<SLAQ_FP64>(K->last_g, K, K->cap, true);
      else if (K->precision == SLAQ_FP32) r = lanczos_form<SLAQ_FP32>(K->last_g, K, K->cap, true);
      else r = lanczos_form<SLAQ_FP32_BF16BASIS>(K->last_g, K, K->cap, true);
      if (r == SLAQ_OK) r = run_ritz(K, K->cap);
    }
    tl_launches = l0;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(K->cap, &graph);
    if (r != SLAQ_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    SLAQ_CHECK_CUDA(e);
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    const cudaError_t ei = cudaGraphInstantiate(&K->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) K->gexec = nullptr;
    SLAQ_CHECK_CUDA(ei);
    K->graph_nodes = (int64_t)nodes;
  }
  K->seed = seed;
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(K->seed_dev, &K->seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  SLAQ_CHECK_CUDA(cudaGraphLaunch(K->gexec, st));
  tl_launches += K->graph_nodes;
  return SLAQ_OK;
}

}  // namespace slaq
