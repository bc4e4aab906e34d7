// s-step Lanczos over a block of nv probes (Sec. 3.1, Algorithm 1 `lanczos`)
// with full reorthogonalization.
//
// Every probe runs its own Lanczos process; all probes share one sparse
// matrix product per step.  Layout in HBM: the basis is U[j][i][p] (step j,
// node i, probe p innermost, row stride ld), so the gather of neighbour j in
// the SpMM reads one contiguous row of nv values.
//
// The basis is kept UNNORMALIZED (u_0 is the +-1 probe itself) with the
// squared norms nu_j^2 = ||u_j||^2 tracked per probe; q_j = u_j / nu_j.
// Step k, for every probe:
//     z       = L u_k                                        (SpMM)
//     d_j     = u_j^T z                    j = 0..k          (dots)
//     alpha_k = d_k / nu_k^2  (= q_k^T L q_k)
//     u_{k+1} = z - sum_j (d_j / nu_j^2) u_j                 (update)
//     nu_{k+1}^2 = ||u_{k+1}||^2,  beta_k = nu_{k+1} / nu_k
// u_{k+1} is nu_k times the vector the textbook order "three-term recurrence,
// then one classical Gram-Schmidt pass over q_0..q_k" produces: both remove
// the projection of L q_k on span{q_0..q_k}; they differ only by rounding.
// Deferring the normalization saves one pass over the basis per step.
#include <algorithm>
#include <cmath>

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
  static constexpr int VE = 2;
  static constexpr int J = 8;  // basis vectors per dots block
};
template <>
struct Form<SLAQ_FP32> {
  using TB = float;
  using TW = float;
  static constexpr int VE = 4;
  static constexpr int J = 8;
};
template <>
struct Form<SLAQ_FP32_BF16BASIS> {
  using TB = __nv_bfloat16;
  using TW = float;
  static constexpr int VE = 8;
  static constexpr int J = 4;
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
__device__ __forceinline__ void ldb(const __nv_bfloat16 *p, float (&v)[8]) {
  uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
  const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
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

// ------------------------------------------------------------ probe init
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int P>
__global__ void k_probe_init(typename Form<P>::TB *U0, const int64_t *old_id, int64_t n, int ld,
                             int nv, uint64_t seed, uint64_t graph_id) {
  using TB = typename Form<P>::TB;
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ld;
    const int p = (int)(idx - i * ld);
    float v = 0.0f;
    if (p < nv) {
      const uint64_t c = (graph_id << 48) | ((uint64_t)p << 32) | (uint64_t)old_id[i];
      const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * (c + 1ull));
      v = (z >> 63) ? -1.0f : 1.0f;
    }
    U0[idx] = (TB)v;
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

__global__ void k_init_scalars(double *nu2, double *alpha, double *beta, int32_t *m, int nv, int s,
                               int ld, double n) {
  for (int i = threadIdx.x; i < s * ld; i += blockDim.x) nu2[i] = (i < nv) ? n : 0.0;
  for (int i = threadIdx.x; i < nv * s; i += blockDim.x) {
    alpha[i] = 0.0;
    beta[i] = 0.0;
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) m[i] = s;
}

// ------------------------------------------------------------------ SpMM
// MODE 0: normalized, unweighted   z_i = diag_i u_i - s_i sum_j s_j u_j
// MODE 1: combinatorial, unweighted z_i = d_i u_i - sum_j u_j
// MODE 2: weighted                  z_i = diag_i u_i + sum_j val_ij u_j
template <int P, int MODE>
__device__ __forceinline__ void gather_rows(const int32_t *__restrict__ col,
                                            const typename Form<P>::TW *__restrict__ vals,
                                            const typename Form<P>::TW *__restrict__ scale,
                                            const typename Form<P>::TB *__restrict__ Ul, int ld,
                                            int64_t b, int64_t e,
                                            typename Form<P>::TW (&acc)[Form<P>::VE]) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  int64_t j = b;
  for (; j + 4 <= e; j += 4) {
    int c[4];
    TW w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = __ldg(col + j + q);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = MODE == 0 ? __ldg(scale + c[q]) : (MODE == 2 ? __ldg(vals + j + q) : TW(1));
    TW x[4][VE];
#pragma unroll
    for (int q = 0; q < 4; ++q) ldb(Ul + (int64_t)c[q] * ld, x[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int v = 0; v < VE; ++v) acc[v] = fma(w[q], x[q][v], acc[v]);
  }
  for (; j < e; ++j) {
    const int c = __ldg(col + j);
    const TW w = MODE == 0 ? __ldg(scale + c) : (MODE == 2 ? __ldg(vals + j) : TW(1));
    TW x[VE];
    ldb(Ul + (int64_t)c * ld, x);
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = fma(w, x[v], acc[v]);
  }
}

template <int P, int MODE>
__device__ __forceinline__ void finish_row(int64_t row, const typename Form<P>::TW *diag,
                                           const typename Form<P>::TW *scale,
                                           const typename Form<P>::TB *Ul, int ld,
                                           typename Form<P>::TW (&acc)[Form<P>::VE],
                                           typename Form<P>::TW *zrow) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  TW y[VE];
  ldb(Ul + row * ld, y);
  const TW g = diag[row];
  const TW sr = MODE == 0 ? scale[row] : TW(1);
  TW z[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v)
    z[v] = MODE == 2 ? fma(g, y[v], acc[v]) : fma(g, y[v], -sr * acc[v]);
  stw<TW, VE>(zrow, z);
}

template <int P, int MODE>
__global__ void __launch_bounds__(256)
    k_spmm_light(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                 const typename Form<P>::TW *__restrict__ vals,
                 const typename Form<P>::TW *__restrict__ diag,
                 const typename Form<P>::TW *__restrict__ scale,
                 const typename Form<P>::TB *__restrict__ U, typename Form<P>::TW *__restrict__ Z,
                 int64_t n, int V, int R, int ld, int64_t heavy_degree) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  const int team = threadIdx.x / V, lane = threadIdx.x - team * V;
  if (team >= R) return;
  const int64_t row = (int64_t)blockIdx.x * R + team;
  if (row >= n) return;
  const int64_t b = rowptr[row], e = rowptr[row + 1];
  if (e - b > heavy_degree) return;  // split rows: k_spmm_heavy
  const auto *Ul = U + lane * VE;
  TW acc[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) acc[v] = TW(0);
  gather_rows<P, MODE>(col, vals, scale, Ul, ld, b, e, acc);
  finish_row<P, MODE>(row, diag, scale, Ul, ld, acc, Z + row * ld + lane * VE);
}

// One chunk of a split row per block; the last block to finish a row sums
// the chunk partials in chunk order (deterministic) and writes the row.
template <int P, int MODE>
__global__ void __launch_bounds__(256)
    k_spmm_heavy(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                 const typename Form<P>::TW *__restrict__ vals,
                 const typename Form<P>::TW *__restrict__ diag,
                 const typename Form<P>::TW *__restrict__ scale,
                 const typename Form<P>::TB *__restrict__ U, typename Form<P>::TW *__restrict__ Z,
                 typename Form<P>::TW *__restrict__ part, const int32_t *__restrict__ heavy_row,
                 const int64_t *__restrict__ heavy_first, const int32_t *__restrict__ chunk_slot,
                 uint32_t *__restrict__ heavy_count, int V, int ld) {
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  __shared__ int is_last;
  const int64_t q = blockIdx.x;
  const int slot = chunk_slot[q];
  const int64_t row = heavy_row[slot];
  const int64_t first = heavy_first[slot];
  const int64_t nch = heavy_first[slot + 1] - first;
  const int64_t c = q - first;
  const int64_t rb = rowptr[row], re = rowptr[row + 1];
  const int64_t b = rb + c * kHeavyChunk;
  const int64_t e = min(b + (int64_t)kHeavyChunk, re);
  const int lane = threadIdx.x;
  const bool active = lane < V;
  const auto *Ul = U + lane * VE;
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    gather_rows<P, MODE>(col, vals, scale, Ul, ld, b, e, acc);
    stw<TW, VE>(part + q * ld + lane * VE, acc);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(heavy_count + slot, 1u);
    is_last = (prev == (unsigned)(nch - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (active) {
    TW acc[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v] = TW(0);
    for (int64_t cc = 0; cc < nch; ++cc) {
      TW x[VE];
      ldw_cg<TW, VE>(part + (first + cc) * ld + lane * VE, x);
#pragma unroll
      for (int v = 0; v < VE; ++v) acc[v] += x[v];
    }
    finish_row<P, MODE>(row, diag, scale, Ul, ld, acc, Z + row * ld + lane * VE);
  }
  if (threadIdx.x == 0) heavy_count[slot] = 0u;  // ready for the next launch
}

// ------------------------------------------------------ compensated sums
// FP64 form: plain FP64 accumulation per thread.  FP32 forms: Kahan
// summation in FP32 per thread (sum, c); the true value is sum - c.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float y = fmaf(a, b, -c);
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
struct PlainD {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <typename TW>
struct Acc;
template <>
struct Acc<double> {
  using type = PlainD;
};
template <>
struct Acc<float> {
  using type = KahanF;
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

// Reduce one double per (team, column) over the block's teams, in team
// order, and store it to out[col] for the block's VE columns of each lane.
__device__ __forceinline__ void block_team_sum(double *sm, int V, int R, int VE, int team, int lane,
                                               const double *mine, double *out) {
  const int width = V * VE;
  for (int v = 0; v < VE; ++v) sm[team * width + lane * VE + v] = mine[v];
  __syncthreads();
  if (team == 0) {
    for (int v = 0; v < VE; ++v) {
      Neumaier acc;
      for (int t = 0; t < R; ++t) acc.add(sm[t * width + lane * VE + v]);
      out[lane * VE + v] = acc.value();
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ dots
// part[g][j][ld] = sum over the rows of block g of u_j[i][p] * x[i][p] for
// j in [j0, j0 + J) with j <= jlast, where x is the work vector z (TW) or,
// for the second Gram-Schmidt pass, the stored basis vector u_{k+1} (TB).
template <int P, bool X_IS_BASIS>
__global__ void __launch_bounds__(256)
    k_dots(const typename Form<P>::TB *__restrict__ U, const void *__restrict__ Xv, int64_t n,
           int64_t rows_per_block, int V, int R, int ld, int64_t ustride, int jfirst, int jlast,
           int JC, double *__restrict__ part, int s) {
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  constexpr int J = Form<P>::J;
  using A = typename Acc<TW>::type;
  __shared__ double sm[256 * VE];
  const int g = blockIdx.x / JC, jc = blockIdx.x - g * JC;
  const int j0 = jfirst + jc * J;
  const int team = threadIdx.x / V, lane = threadIdx.x - team * V;
  const bool in_team = team < R;
  A acc[J][VE];
  if (in_team) {
    const int64_t r0 = (int64_t)g * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    for (int64_t row = r0 + team; row < r1; row += R) {
      TW x[VE];
      if (X_IS_BASIS) ldb(static_cast<const TB *>(Xv) + row * ld + lane * VE, x);
      else ldw<TW, VE>(static_cast<const TW *>(Xv) + row * ld + lane * VE, x);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) {
        if (j0 + jj <= jlast) {
          TW u[VE];
          ldb(U + (int64_t)(j0 + jj) * ustride + row * ld + lane * VE, u);
#pragma unroll
          for (int v = 0; v < VE; ++v) acc[jj][v].add_prod(u[v], x[v]);
        }
      }
    }
  }
  const int t = in_team ? team : 0;
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    if (j0 + jj > jlast) break;  // uniform over the block
    double mine[VE];
#pragma unroll
    for (int v = 0; v < VE; ++v) mine[v] = in_team ? acc[jj][v].value() : 0.0;
    // threads outside the teams (blockDim = V*R exactly, so none) never write
    block_team_sum(sm, V, R, VE, t, lane, mine,
                   part + ((int64_t)g * s + (j0 + jj)) * ld);
  }
}

// Sum the G block partials of rows [jfirst, jfirst + jcount) of the dot
// products; turn them into Gram-Schmidt coefficients c_j = d_j / nu_j^2 for
// probes still running at step k (0 for stopped probes and padding), and
// alpha_k = c_k.  Block (32, 8): x = column, y strides over blocks.
__global__ void k_dot_reduce(const double *__restrict__ part, int G, int s, int ld, int jfirst,
                             int jcount, int k, const double *__restrict__ nu2,
                             const int32_t *__restrict__ m, int nv, double *__restrict__ coef,
                             double *__restrict__ alpha, int write_alpha) {
  __shared__ double ss[8][33], sc[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool valid = col < jcount * ld;
  const int j = jfirst + (valid ? col / ld : 0);
  const int p = valid ? col % ld : 0;
  Neumaier acc;
  if (valid)
    for (int g = threadIdx.y; g < G; g += 8) acc.add(part[((int64_t)g * s + j) * ld + p]);
  ss[threadIdx.y][threadIdx.x] = acc.s;
  sc[threadIdx.y][threadIdx.x] = acc.c;
  __syncthreads();
  if (threadIdx.y == 0 && valid) {
    Neumaier tot;
    for (int y = 0; y < 8; ++y) {
      tot.add(ss[y][threadIdx.x]);
      tot.add(sc[y][threadIdx.x]);
    }
    const double d = tot.value();
    const bool running = p < nv && m[p] > k;
    const double c = running ? d / nu2[j * ld + p] : 0.0;
    coef[j * ld + p] = c;
    if (write_alpha && j == k && running) alpha[p * s + k] = c;
  }
}

// ---------------------------------------------------------------- update
// u_{k+1} = x - sum_{j<=k} coef_j * u_j, with x = z (first pass) or the
// stored u_{k+1} (second pass, in place); stopped probes get 0.  Also the
// per-block partial sums of u_{k+1}^2 of the rounded stored values.
template <int P, bool SECOND>
__global__ void __launch_bounds__(256)
    k_update(const typename Form<P>::TB *__restrict__ U, const typename Form<P>::TW *__restrict__ Z,
             typename Form<P>::TB *Unext, int64_t n, int64_t rows_per_block, int V, int R, int ld,
             int64_t ustride, int k, const double *__restrict__ coef,
             const int32_t *__restrict__ m, int nv, double *__restrict__ part, int s) {
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  using A = typename Acc<TW>::type;
  extern __shared__ __align__(16) unsigned char dyn[];
  TW *cf = reinterpret_cast<TW *>(dyn);                         // [(k+1) * ld]
  double *sm = reinterpret_cast<double *>(cf + (k + 1) * ld);   // [V*R*VE]
  for (int i = threadIdx.x; i < (k + 1) * ld; i += blockDim.x) {
    const int p = i % ld;
    const bool running = p < nv && m[p] > k;
    cf[i] = running ? (TW)coef[i] : TW(0);
  }
  __syncthreads();
  const int g = blockIdx.x;
  const int team = threadIdx.x / V, lane = threadIdx.x - team * V;
  bool keep[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) {
    const int p = lane * VE + v;
    keep[v] = p < nv && m[p] > k;
  }
  A acc[VE];
  const int64_t r0 = (int64_t)g * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  for (int64_t row = r0 + team; row < r1; row += R) {
    TW x[VE];
    if (SECOND) ldb_rw(Unext + row * ld + lane * VE, x);
    else ldw<TW, VE>(Z + row * ld + lane * VE, x);
    int j = 0;
    for (; j + 2 <= k + 1; j += 2) {
      TW u0[VE], u1[VE];
      ldb(U + (int64_t)j * ustride + row * ld + lane * VE, u0);
      ldb(U + (int64_t)(j + 1) * ustride + row * ld + lane * VE, u1);
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
      ldb(U + (int64_t)j * ustride + row * ld + lane * VE, u0);
      const TW *c0 = cf + j * ld + lane * VE;
#pragma unroll
      for (int v = 0; v < VE; ++v) x[v] = fma(-c0[v], u0[v], x[v]);
    }
#pragma unroll
    for (int v = 0; v < VE; ++v)
      if (!keep[v]) x[v] = TW(0);
    TW r[VE];
    stb(Unext + row * ld + lane * VE, x, r);
#pragma unroll
    for (int v = 0; v < VE; ++v) acc[v].add_prod(r[v], r[v]);
  }
  double mine[VE];
#pragma unroll
  for (int v = 0; v < VE; ++v) mine[v] = acc[v].value();
  block_team_sum(sm, V, R, VE, team, lane, mine, part + (int64_t)g * s * ld);
}

// nu_{k+1}^2 from the block partials; beta_k = nu_{k+1} / nu_k; a probe
// whose beta_k <= tol * bound stops with m = k + 1.
__global__ void k_norm_reduce(const double *__restrict__ part, int G, int s, int ld, int k,
                              double *__restrict__ nu2, int32_t *__restrict__ m, int nv,
                              double *__restrict__ beta, double tol_abs) {
  __shared__ double ss[8][33], sc[8][33];
  const int p = blockIdx.x * 32 + threadIdx.x;
  const bool valid = p < ld;
  Neumaier acc;
  if (valid)
    for (int g = threadIdx.y; g < G; g += 8) acc.add(part[(int64_t)g * s * ld + p]);
  ss[threadIdx.y][threadIdx.x] = acc.s;
  sc[threadIdx.y][threadIdx.x] = acc.c;
  __syncthreads();
  if (threadIdx.y == 0 && valid) {
    Neumaier tot;
    for (int y = 0; y < 8; ++y) {
      tot.add(ss[y][threadIdx.x]);
      tot.add(sc[y][threadIdx.x]);
    }
    const double nn = tot.value();
    double keep_nu2 = 0.0;
    if (p < nv && m[p] > k) {
      const double b = sqrt(nn) / sqrt(nu2[k * ld + p]);
      if (b <= tol_abs) {
        m[p] = k + 1;
      } else {
        beta[p * s + k] = b;
        keep_nu2 = nn;
      }
    }
    nu2[(k + 1) * ld + p] = keep_nu2;
  }
}

// ------------------------------------------------------------ host side
struct Geometry {
  int V, R, threads;
  int64_t rows_per_block;
  int G;
};

Geometry geometry(int precision, int ld, int64_t n, int sms) {
  Geometry g;
  g.V = ld / vec_elems(precision);
  g.R = std::max(1, 256 / g.V);
  g.threads = g.V * g.R;
  int64_t G = std::min<int64_t>(std::max<int64_t>(1, ceil_div(n, 1024)), 4LL * sms);
  g.rows_per_block = std::max<int64_t>(1, ceil_div(n, G));
  g.G = (int)std::max<int64_t>(1, ceil_div(n, g.rows_per_block));
  return g;
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
    vals = gr->vals;
    diag = gr->diag;
    scale = gr->scale;
  } else {
    vals = gr->vals32;
    diag = gr->diag32;
    scale = gr->scale32;
  }
  const int mode = gr->weighted ? 2 : (gr->kind == SLAQ_NORMALIZED ? 0 : 1);
  const unsigned blocks = (unsigned)ceil_div(n, geo.R);
  const int hthreads = (int)ceil_div(geo.V, 32) * 32;
#define SLAQ_SPMM_CASE(MODE)                                                                  \
  ++tl_launches;                                                                              \
  k_spmm_light<P, MODE><<<blocks, geo.threads, 0, st>>>(gr->rowptr, gr->colidx, vals, diag,   \
                                                        scale, Uk, Z, n, geo.V, geo.R, K->ld, \
                                                        gr->heavy_degree);                    \
  if (gr->n_chunks > 0) ++tl_launches;                                                        \
  if (gr->n_chunks > 0)                                                                       \
    k_spmm_heavy<P, MODE><<<(unsigned)gr->n_chunks, hthreads, 0, st>>>(                       \
        gr->rowptr, gr->colidx, vals, diag, scale, Uk, Z, static_cast<TW *>(K->P),            \
        gr->heavy_row, gr->heavy_first, gr->chunk_slot, gr->heavy_count, geo.V, K->ld);
  if (mode == 0) {
    SLAQ_SPMM_CASE(0)
  } else if (mode == 1) {
    SLAQ_SPMM_CASE(1)
  } else {
    SLAQ_SPMM_CASE(2)
  }
#undef SLAQ_SPMM_CASE
  SLAQ_CHECK_LAUNCH("spmm");
  return SLAQ_OK;
}

template <int P>
int dots(slaq_krylov K, const Geometry &geo, int64_t n, int jfirst, int jlast, bool x_is_basis,
         const void *X, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_DOTS, st);
  using TB = typename Form<P>::TB;
  constexpr int J = Form<P>::J;
  const int JC = (int)ceil_div(jlast - jfirst + 1, J);
  const unsigned blocks = (unsigned)(geo.G * JC);
  const TB *U = static_cast<const TB *>(K->U);
  const int64_t ustride = n * K->ld;
  ++tl_launches;
  if (x_is_basis)
    k_dots<P, true><<<blocks, geo.threads, 0, st>>>(U, X, n, geo.rows_per_block, geo.V, geo.R,
                                                    K->ld, ustride, jfirst, jlast, JC, K->part,
                                                    K->s);
  else
    k_dots<P, false><<<blocks, geo.threads, 0, st>>>(U, X, n, geo.rows_per_block, geo.V, geo.R,
                                                     K->ld, ustride, jfirst, jlast, JC, K->part,
                                                     K->s);
  SLAQ_CHECK_LAUNCH("dots");
  return SLAQ_OK;
}

template <int P>
int update(slaq_krylov K, const Geometry &geo, int64_t n, int k, bool second, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_UPDATE, st);
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  constexpr int VE = Form<P>::VE;
  const TB *U = static_cast<const TB *>(K->U);
  TB *Unext = static_cast<TB *>(K->U) + (int64_t)(k + 1) * n * K->ld;
  const int64_t ustride = n * K->ld;
  const size_t smem = (size_t)(k + 1) * K->ld * sizeof(TW) + (size_t)geo.threads * VE * sizeof(double);
  ++tl_launches;
  if (second)
    k_update<P, true><<<geo.G, geo.threads, smem, st>>>(U, static_cast<const TW *>(K->Z), Unext, n,
                                                        geo.rows_per_block, geo.V, geo.R, K->ld,
                                                        ustride, k, K->coef, K->m, K->nv, K->part,
                                                        K->s);
  else
    k_update<P, false><<<geo.G, geo.threads, smem, st>>>(U, static_cast<const TW *>(K->Z), Unext,
                                                         n, geo.rows_per_block, geo.V, geo.R,
                                                         K->ld, ustride, k, K->coef, K->m, K->nv,
                                                         K->part, K->s);
  SLAQ_CHECK_LAUNCH("update");
  return SLAQ_OK;
}

int dot_reduce(slaq_krylov K, const Geometry &geo, int jfirst, int jcount, int k, bool write_alpha,
               cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_REDUCE, st);
  const unsigned blocks = (unsigned)ceil_div((int64_t)jcount * K->ld, 32);
  ++tl_launches;
  k_dot_reduce<<<blocks, dim3(32, 8), 0, st>>>(K->part, geo.G, K->s, K->ld, jfirst, jcount, k,
                                               K->nu2, K->m, K->nv, K->coef, K->alpha,
                                               write_alpha ? 1 : 0);
  SLAQ_CHECK_LAUNCH("dot_reduce");
  return SLAQ_OK;
}

template <int P>
int lanczos_form(slaq_graph gr, slaq_krylov K, cudaStream_t st) {
  using TB = typename Form<P>::TB;
  using TW = typename Form<P>::TW;
  const int64_t n = gr->n;
  const Geometry geo = geometry(P, K->ld, n, num_sms());
  if (geo.G > K->G) return set_error(SLAQ_EINVAL, "internal: reduction workspace too small");
  static bool attr_set = false;
  if (!attr_set) {
    SLAQ_CHECK_CUDA(cudaFuncSetAttribute(k_update<P, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    SLAQ_CHECK_CUDA(cudaFuncSetAttribute(k_update<P, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  {
    ProfScope prof(SLAQ_PROF_PROBES, st);
    ++tl_launches;
    k_init_scalars<<<1, 256, 0, st>>>(K->nu2, K->alpha, K->beta, K->m, K->nv, K->s, K->ld,
                                      (double)n);
    ++tl_launches;
    k_probe_init<P><<<(unsigned)std::min<int64_t>(ceil_div(n * K->ld, 256), 152LL * 64), 256, 0,
                      st>>>(static_cast<TB *>(K->U), gr->old_id, n, K->ld, K->nv, K->seed,
                            (uint64_t)K->graph_id);
  }
  SLAQ_CHECK_LAUNCH("probe_init");
  const double tol_abs = K->tol * gr->bound;
  for (int k = 0; k < K->s; ++k) {
    SLAQ_TRY(spmm<P>(gr, K, geo, k, st));
    const bool last = (k == K->s - 1);
    const int jfirst = last ? k : 0;
    SLAQ_TRY(dots<P>(K, geo, n, jfirst, k, false, K->Z, st));
    SLAQ_TRY(dot_reduce(K, geo, jfirst, k - jfirst + 1, k, true, st));
    if (last) break;
    SLAQ_TRY(update<P>(K, geo, n, k, false, st));
    if (K->reorth == 2) {
      const TB *Unext = static_cast<const TB *>(K->U) + (int64_t)(k + 1) * n * K->ld;
      SLAQ_TRY(dots<P>(K, geo, n, 0, k, true, Unext, st));
      SLAQ_TRY(dot_reduce(K, geo, 0, k + 1, k, false, st));
      SLAQ_TRY(update<P>(K, geo, n, k, true, st));
    }
    ProfScope prof(SLAQ_PROF_REDUCE, st);
    ++tl_launches;
    k_norm_reduce<<<(unsigned)ceil_div(K->ld, 32), dim3(32, 8), 0, st>>>(
        K->part, geo.G, K->s, K->ld, k, K->nu2, K->m, K->nv, K->beta, tol_abs);
    SLAQ_CHECK_LAUNCH("norm_reduce");
  }
  (void)sizeof(TW);
  return SLAQ_OK;
}

double default_tol(int precision) {
  return precision == SLAQ_FP64 ? 1e-10 : (precision == SLAQ_FP32 ? 1e-4 : 3e-2);
}

template <typename T>
int grow(T **p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(SLAQ_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                     cudaGetErrorString(e));
  }
  return SLAQ_OK;
}

}  // namespace

int probes(slaq_graph g, int nv, uint64_t seed, int graph_id, double *out, cudaStream_t st) {
  if (!g || !out) return set_error(SLAQ_EINVAL, "NULL graph or output");
  if (nv < 1 || graph_id < 0 || graph_id > 0xffff) return set_error(SLAQ_EINVAL, "bad nv or graph_id");
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
  void *ptrs[] = {k->U, k->Z, k->P, k->part, k->dsum, k->coef, k->nu2, k->alpha, k->beta,
                  k->m, k->theta, k->tau2, k->status};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete k;
}

int run_lanczos(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision,
                int reorth, cudaStream_t st, slaq_krylov *inout) {
  if (!g || !inout) return set_error(SLAQ_EINVAL, "NULL graph or output handle");
  if (nv < 1 || nv > 512) return set_error(SLAQ_EINVAL, "nv must be in [1, 512]");
  if (s < 1 || s > 64) return set_error(SLAQ_EINVAL, "s must be in [1, 64]");
  if (graph_id < 0 || graph_id > 0xffff) return set_error(SLAQ_EINVAL, "graph_id must be < 65536");
  if (precision != SLAQ_FP64 && precision != SLAQ_FP32 && precision != SLAQ_FP32_BF16BASIS)
    return set_error(SLAQ_EINVAL, "unknown precision %d", precision);
  if (reorth != 1 && reorth != 2) return set_error(SLAQ_EINVAL, "reorth_passes must be 1 or 2");
  if (g->n < 1) return set_error(SLAQ_EINVAL, "graph has no nodes");
  if (g->n > (1LL << 31)) return set_error(SLAQ_EUNSUPPORTED, "too many nodes");
  const int ld = row_ld(nv, precision);
  if ((size_t)s * ld * work_bytes(precision) + 256 * 8 * 8 > 200 * 1024)
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
  }
  struct Guard {
    slaq_krylov *K;
    bool fresh;
    ~Guard() {
      if (fresh && *K) krylov_free(*K);
    }
  } guard{&K, fresh};
  const int64_t n = g->n;
  const Geometry geo = geometry(precision, ld, n, num_sms());
  if (n > K->n_cap) {
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->U), (size_t)s * n * ld * basis_bytes(precision)));
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->Z), (size_t)n * ld * work_bytes(precision)));
    K->n_cap = n;
  }
  if (g->n_chunks > K->chunk_cap || !K->P) {
    const int64_t cap = std::max<int64_t>(g->n_chunks, 1);
    SLAQ_TRY(grow(reinterpret_cast<unsigned char **>(&K->P), (size_t)cap * ld * work_bytes(precision)));
    K->chunk_cap = cap;
  }
  if (geo.G > K->G) {
    SLAQ_TRY(grow(&K->part, (size_t)geo.G * s * ld));
    K->G = geo.G;
  }
  if (fresh) {
    SLAQ_TRY(grow(&K->dsum, (size_t)s * ld));
    SLAQ_TRY(grow(&K->coef, (size_t)s * ld));
    SLAQ_TRY(grow(&K->nu2, (size_t)(s + 1) * ld));
    SLAQ_TRY(grow(&K->alpha, (size_t)nv * s));
    SLAQ_TRY(grow(&K->beta, (size_t)nv * s));
    SLAQ_TRY(grow(&K->m, (size_t)nv));
    SLAQ_TRY(grow(&K->theta, (size_t)nv * s));
    SLAQ_TRY(grow(&K->tau2, (size_t)nv * s));
    SLAQ_TRY(grow(&K->status, 1));
  }
  K->seed = seed;
  K->graph_id = graph_id;
  K->reorth = reorth;
  K->n = n;
  K->kind = g->kind;
  K->trace = g->trace;
  K->bound = g->bound;
  K->tol = default_tol(precision);
  int r;
  if (precision == SLAQ_FP64) r = lanczos_form<SLAQ_FP64>(g, K, st);
  else if (precision == SLAQ_FP32) r = lanczos_form<SLAQ_FP32>(g, K, st);
  else r = lanczos_form<SLAQ_FP32_BF16BASIS>(g, K, st);
  if (r != SLAQ_OK) return r;
  SLAQ_TRY(run_ritz(K, st));
  *inout = K;
  guard.fresh = false;  // the caller owns it now
  return SLAQ_OK;
}

}  // namespace slaq
