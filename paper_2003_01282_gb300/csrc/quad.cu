// Gauss rule per probe and the Hutchinson estimate of Eq. slq for the heat
// trace (Eq. heat-trace), the wave trace and the VNGE (Definition 1,
// Sec. 2.1); spectral distances between descriptors (Sec. 4.2).
// Eigensolves and sums are FP64; the FP32 and BF16 forms evaluate exp, cos
// and sin in FP32 (see fval).  Probe sums run in a fixed order, so results
// are deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tridiag.cuh"

namespace slaq {
namespace {

constexpr int kMaxS = 64;
constexpr int kMaxNv = 512;

// One thread per (graph, probe) problem; problems are rows of [total][s].
// The rule size m[p] is clamped to [0, s] (s <= kMaxS): a value outside that
// range, possible only where the caller supplies m, sets bit 2 of *status;
// m_out (or NULL) receives the clamped sizes for the quadrature that follows.
__global__ void k_ritz(const double *__restrict__ alpha, const double *__restrict__ beta,
                       const int32_t *__restrict__ mm, int nv, int s, double *__restrict__ theta,
                       double *__restrict__ tau2, int32_t *status, int32_t *__restrict__ m_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;  // nv = number of problems
  if (p >= nv) return;
  double d[kMaxS], e[kMaxS], w[kMaxS];
  const int m_in = mm[p];
  const int m = min(max(m_in, 0), min(s, kMaxS));
  if (m != m_in) atomicOr(status, 2);
  if (m_out) m_out[p] = m;
  for (int i = 0; i < m; ++i) d[i] = alpha[p * s + i];
  for (int i = 0; i + 1 < m; ++i) e[i] = beta[p * s + i];
  if (tridiag_gauss(d, e, w, m) != 0) atomicOr(status, 1);
  for (int i = 0; i < s; ++i) {
    theta[p * s + i] = i < m ? d[i] : 0.0;
    tau2[p * s + i] = i < m ? w[i] : 0.0;
  }
}

// Rayleigh-Ritz on the stored basis, for the reduced forms.  With a basis
// rounded to FP32 or BF16 the recurrence's T (alpha_k = d_k / G_kk, beta from
// norm ratios, entries beyond the tridiagonal dropped) carries first-order
// rounding errors of the stored vectors: with BF16 that is 1e-2 on the heat
// trace at large t.  The projected pencil (M, G), M = U^T L U and G = U^T U
// of the stored vectors u_0..u_{m-1}, is exact for the subspace they span,
// and its Ritz pairs are accurate to second order in those errors.  With
// G = C C^T (after scaling G to unit diagonal), A = C^{-1} M C^{-T} is the
// projection of L on the orthonormal basis U C^{-T}, whose first vector is
// u_0 / ||u_0||: so the Gauss rule of the start vector is that of A's first
// unit vector.  A is reduced to tridiagonal form by Householder reflections
// that fix the first unit vector (Golub & Van Loan, Sec. 8.3.1), and that
// tridiagonal goes through the same Gauss-rule solver as the FP64 form; it
// replaces alpha and beta, so exports and traces use the corrected rule.  In
// exact arithmetic A equals the recurrence's T.  One thread per problem; the
// dense matrices live in global scratch, entry-major over the problems, so
// a warp's accesses are consecutive words.
__global__ void k_ritz_pencil(const double *__restrict__ gram_all,
                              const double *__restrict__ proj_all, const int32_t *__restrict__ mm,
                              int nv, int s, int ld, int total, double *__restrict__ scr,
                              double *__restrict__ alpha, double *__restrict__ beta,
                              double *__restrict__ theta, double *__restrict__ tau2,
                              int32_t *status) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int gr = q / nv, pp = q - gr * nv;
  const double *Gm = gram_all + (int64_t)gr * s * s * ld;
  const double *Mm = proj_all + (int64_t)gr * s * s * ld;
  const int m = mm[q];
  const int64_t P = total;
  double *Ab = scr;                                   // [s][s] full
  double *Cb = scr + (int64_t)s * s * P;              // packed lower triangle
  double *Vb = Cb + (int64_t)(s * (s + 1) / 2) * P;   // [2][s] vectors
#define RA(i, j) Ab[((int64_t)(i) * s + (j)) * P + q]
#define RC(i, j) Cb[((int64_t)((i) * ((i) + 1) / 2 + (j))) * P + q]
#define RV(i) Vb[(int64_t)(i) * P + q]
#define RW(i) Vb[(int64_t)(s + (i)) * P + q]
#define GE(i, j) Gm[((int64_t)(i) * s + (j)) * ld + pp]
#define ME(i, j) Mm[((int64_t)(i) * s + (j)) * ld + pp]
  int bad = 0;
  // unit-diagonal scaling D = diag(G)^{-1/2}, kept in RV
  for (int i = 0; i < m; ++i) RV(i) = rsqrt(GE(i, i));
  // Cholesky of D G D; ic holds the reciprocal pivots, so that the solves
  // below multiply (an FP64 division costs several FMAs on the FP64 pipe this
  // kernel is bound by)
  double ic[kMaxS];
  for (int j = 0; j < m; ++j) {
    double dj = GE(j, j) * RV(j) * RV(j);
    for (int k = 0; k < j; ++k) dj -= RC(j, k) * RC(j, k);
    if (!(dj > 0.0)) {
      bad = 1;
      dj = 1e-300;
    }
    const double cjj = sqrt(dj), icjj = 1.0 / cjj;
    RC(j, j) = cjj;
    ic[j] = icjj;
    for (int i = j + 1; i < m; ++i) {
      double x = GE(i, j) * RV(i) * RV(j);
      for (int k = 0; k < j; ++k) x -= RC(i, k) * RC(j, k);
      RC(i, j) = x * icjj;
    }
  }
  // B = C^{-1} (D M D): forward substitution down the columns
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      double x = ME(i, j) * RV(i) * RV(j);
      for (int k = 0; k < i; ++k) x -= RC(i, k) * RA(k, j);
      RA(i, j) = x * ic[i];
    }
  // A = B C^{-T}, symmetric: only its lower triangle is formed (entry (i, l)
  // needs B's row i up to column l) and used below
  for (int i = 0; i < m; ++i)
    for (int l = 0; l <= i; ++l) {
      double y = RA(i, l);
      for (int k = 0; k < l; ++k) y -= RC(l, k) * RA(i, k);
      RA(i, l) = y * ic[l];
    }
  // Householder tridiagonalization on the lower triangle; reflector k acts
  // on indices k+1..m-1
  double d[kMaxS], e[kMaxS], w[kMaxS];
  for (int k = 0; k + 2 < m; ++k) {
    double xn2 = 0.0;
    for (int i = k + 1; i < m; ++i) xn2 += RA(i, k) * RA(i, k);
    const double xn = sqrt(xn2);
    const double x0 = RA(k + 1, k);
    if (xn == 0.0) {
      e[k] = 0.0;
      continue;
    }
    const double sg = x0 >= 0.0 ? 1.0 : -1.0;
    e[k] = -sg * xn;
    // v = x + sg ||x|| e_1 (in RV), b = 2 / v^T v
    RV(k + 1) = x0 + sg * xn;
    for (int i = k + 2; i < m; ++i) RV(i) = RA(i, k);
    const double vtv = xn2 + 2.0 * sg * xn * x0 + xn2;  // |x|^2 + 2 sg |x| x0 + |x|^2
    const double b = 2.0 / vtv;
    // p = b A22 v (in RW), then w = p - (b/2)(p^T v) v
    double pv = 0.0;
    for (int i = k + 1; i < m; ++i) {
      double x = 0.0;
      for (int j = k + 1; j <= i; ++j) x += RA(i, j) * RV(j);
      for (int j = i + 1; j < m; ++j) x += RA(j, i) * RV(j);
      x *= b;
      RW(i) = x;
      pv += x * RV(i);
    }
    const double hw = 0.5 * b * pv;
    for (int i = k + 1; i < m; ++i) RW(i) -= hw * RV(i);
    for (int i = k + 1; i < m; ++i)
      for (int j = k + 1; j <= i; ++j) RA(i, j) -= RV(i) * RW(j) + RW(i) * RV(j);
  }
  for (int i = 0; i < m; ++i) d[i] = RA(i, i);
  if (m >= 2) e[m - 2] = RA(m - 1, m - 2);
  for (int i = 0; i + 1 < m; ++i) e[i] = fabs(e[i]);
#undef RA
#undef RC
#undef RV
#undef RW
#undef GE
#undef ME
  for (int i = 0; i < s; ++i) {
    alpha[(int64_t)q * s + i] = i < m ? d[i] : 0.0;
    beta[(int64_t)q * s + i] = i + 1 < m ? e[i] : 0.0;
  }
  if (bad || tridiag_gauss(d, e, w, m) != 0) atomicOr(status, 1);
  for (int i = 0; i < s; ++i) {
    theta[(int64_t)q * s + i] = i < m ? d[i] : 0.0;
    tau2[(int64_t)q * s + i] = i < m ? w[i] : 0.0;
  }
}

// The same Rayleigh-Ritz step with one warp per problem, for runs with few
// problems (one graph): the lanes share the dense work (Cholesky, the two
// triangular solves, the Householder products and rank-2 updates) in shared
// memory, and lane 0 runs the tridiagonal Gauss rule.
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

inline size_t ritz_warp_smem(int s) { return ((size_t)2 * s * s + 3 * s) * sizeof(double); }

__global__ void __launch_bounds__(32)
    k_ritz_pencil_warp(const double *__restrict__ gram_all, const double *__restrict__ proj_all,
                       const int32_t *__restrict__ mm, int nv, int s, int ld,
                       double *__restrict__ alpha, double *__restrict__ beta,
                       double *__restrict__ theta, double *__restrict__ tau2, int32_t *status) {
  extern __shared__ double rw_smem[];
  double *A = rw_smem;           // [s][s]
  double *C = A + s * s;         // [s][s], lower triangle
  double *V = C + s * s;         // [s] Householder vector
  double *W = V + s;             // [s]
  double *D = W + s;             // [s] unit-diagonal scaling
  const int q = blockIdx.x, lane = threadIdx.x;
  const int gr = q / nv, pp = q - gr * nv;
  const double *Gm = gram_all + (int64_t)gr * s * s * ld;
  const double *Mm = proj_all + (int64_t)gr * s * s * ld;
  const int m = mm[q];
  for (int i = lane; i < m; i += 32) D[i] = rsqrt(Gm[((int64_t)i * s + i) * ld + pp]);
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    const int i = e / m, j = e - i * m;
    const double sij = D[i] * D[j];
    A[i * s + j] = Mm[((int64_t)i * s + j) * ld + pp] * sij;
    if (j <= i) C[i * s + j] = Gm[((int64_t)i * s + j) * ld + pp] * sij;
  }
  __syncwarp();
  int bad = 0;
  for (int j = 0; j < m; ++j) {  // right-looking Cholesky
    const double cjj = C[j * s + j];
    if (!(cjj > 0.0)) bad = 1;
    const double r = sqrt(cjj > 0.0 ? cjj : 1e-300);
    __syncwarp();
    if (lane == 0) C[j * s + j] = r;
    for (int i = j + 1 + lane; i < m; i += 32) C[i * s + j] /= r;
    __syncwarp();
    const int rem = m - j - 1;
    for (int e = lane; e < rem * rem; e += 32) {
      const int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) C[i * s + k] -= C[i * s + j] * C[k * s + j];
    }
    __syncwarp();
  }
  for (int i = 0; i < m; ++i) {  // A := C^{-1} A, row by row
    const double cii = C[i * s + i];
    for (int j = lane; j < m; j += 32) A[i * s + j] /= cii;
    __syncwarp();
    const int rem = m - i - 1;
    for (int e = lane; e < rem * m; e += 32) {
      const int r = i + 1 + e / m, j = e % m;
      A[r * s + j] -= C[r * s + i] * A[i * s + j];
    }
    __syncwarp();
  }
  for (int l = 0; l < m; ++l) {  // A := A C^{-T}, column by column
    const double cll = C[l * s + l];
    for (int i = lane; i < m; i += 32) A[i * s + l] /= cll;
    __syncwarp();
    const int rem = m - l - 1;
    for (int e = lane; e < rem * m; e += 32) {
      const int i = e / rem, r = l + 1 + e % rem;
      A[i * s + r] -= C[r * s + l] * A[i * s + l];
    }
    __syncwarp();
  }
  for (int e = lane; e < m * m; e += 32) {  // symmetrize
    const int i = e / m, j = e - i * m;
    if (j < i) {
      const double a = 0.5 * (A[i * s + j] + A[j * s + i]);
      A[i * s + j] = a;
      A[j * s + i] = a;
    }
  }
  __syncwarp();
  // Householder reduction; e_k goes to C[k] (row 0 of C, free after the solves)
  for (int k = 0; k + 2 < m; ++k) {
    double part = 0.0;
    for (int i = k + 1 + lane; i < m; i += 32) part += A[i * s + k] * A[i * s + k];
    const double xn2 = warp_sum(part);
    const double xn = sqrt(xn2);
    const double x0 = A[(k + 1) * s + k];
    __syncwarp();
    if (xn == 0.0) {
      if (lane == 0) C[k] = 0.0;
      __syncwarp();
      continue;
    }
    const double sg = x0 >= 0.0 ? 1.0 : -1.0;
    if (lane == 0) C[k] = -sg * xn;
    for (int i = k + 1 + lane; i < m; i += 32) V[i] = (i == k + 1) ? x0 + sg * xn : A[i * s + k];
    __syncwarp();
    const double b = 2.0 / (2.0 * xn2 + 2.0 * sg * xn * x0);
    double pv_part = 0.0;
    for (int i = k + 1 + lane; i < m; i += 32) {
      double x = 0.0;
      for (int j = k + 1; j < m; ++j) x += A[i * s + j] * V[j];
      x *= b;
      W[i] = x;
      pv_part += x * V[i];
    }
    const double hw = 0.5 * b * warp_sum(pv_part);
    __syncwarp();
    for (int i = k + 1 + lane; i < m; i += 32) W[i] -= hw * V[i];
    __syncwarp();
    const int rem = m - k - 1;
    for (int e = lane; e < rem * rem; e += 32) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      A[i * s + j] -= V[i] * W[j] + W[i] * V[j];
    }
    __syncwarp();
  }
  if (lane == 0) {
    double d[kMaxS], e[kMaxS], w[kMaxS];
    for (int i = 0; i < m; ++i) d[i] = A[i * s + i];
    for (int i = 0; i + 2 < m; ++i) e[i] = fabs(C[i]);
    if (m >= 2) e[m - 2] = fabs(A[(m - 1) * s + (m - 2)]);
    for (int i = 0; i < s; ++i) {
      alpha[(int64_t)q * s + i] = i < m ? d[i] : 0.0;
      beta[(int64_t)q * s + i] = i + 1 < m ? e[i] : 0.0;
    }
    if (bad || tridiag_gauss(d, e, w, m) != 0) atomicOr(status, 1);
    for (int i = 0; i < s; ++i) {
      theta[(int64_t)q * s + i] = i < m ? d[i] : 0.0;
      tau2[(int64_t)q * s + i] = i < m ? w[i] : 0.0;
    }
  }
}

struct NeumaierD {
  double s = 0.0, c = 0.0;
  __device__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ double value() const { return s + c; }
};

// mean and standard error over nv values held in shared memory (thread 0)
__device__ void mean_se(const double *g, int nv, double *mean_out, double *se_out) {
  NeumaierD acc;
  for (int p = 0; p < nv; ++p) acc.add(g[p]);
  const double mean = acc.value() / nv;
  double se = nan("");
  if (nv > 1) {
    NeumaierD sq;
    for (int p = 0; p < nv; ++p) {
      const double dv = g[p] - mean;
      sq.add(dv * dv);
    }
    se = sqrt(sq.value() / (nv - 1) / nv);
  }
  *mean_out = mean;
  if (se_out) *se_out = se;
}

// FUN 0: exp(-t theta); FUN 1: cos(t theta); FUN 2: -sin(t theta).
// F32: the product t * theta is formed in FP64 (and reduced modulo 2 pi in
// FP64 for cos / sin), the function is evaluated in FP32; used by the FP32
// forms, whose Ritz values carry FP32-level errors anyway.  FP64 is scarce on
// this chip and these evaluations dominate batched quadratures.
template <int FUN>
__device__ __forceinline__ float fval32(double t, double th) {
  const double x = t * th;
  if (FUN == 0) return expf((float)(-x));
  const double two_pi = 6.283185307179586, inv_two_pi = 0.15915494309189535;
  const double r = x - two_pi * rint(x * inv_two_pi);
  if (FUN == 1) return cosf((float)r);
  return -sinf((float)r);
}
template <int FUN, bool F32>
__device__ __forceinline__ double fval(double t, double th) {
  if (F32) return (double)fval32<FUN>(t, th);
  const double x = t * th;
  if (FUN == 0) return exp(-x);
  if (FUN == 1) return cos(x);
  return -sin(x);
}

// Block (chunk of kTT time values, graph gr); thread (tt, pg) evaluates
// g_p = n_g sum_k tau2 f(t theta_k) for probes p = pg, pg + kPG, ... of the
// graph, keeping a Welford mean and squared deviation; the kPG partial states
// are combined in a fixed order (Chan et al.), so results are deterministic.
// out[gr][t] = mean over probes, se[gr][t] = sample std / sqrt(nv).
constexpr int kTT = 32, kPG = 4;
template <int FUN, bool F32>
__global__ void __launch_bounds__(kTT * kPG)
    k_trace_t(const double *__restrict__ theta, const double *__restrict__ tau2,
              const int32_t *__restrict__ mm, int nv, int s, const double *__restrict__ gn,
              double n0, const double *__restrict__ t, int nt, double *out, double *se,
              double *per_probe) {
  __shared__ double sh_mean[kPG][kTT], sh_m2[kPG][kTT];
  __shared__ int sh_cnt[kPG][kTT];
  const int tt = threadIdx.x % kTT, pg = threadIdx.x / kTT;
  const int ti = blockIdx.x * kTT + tt;
  const int gr = blockIdx.y;
  double mean = 0.0, m2 = 0.0;
  int cnt = 0;
  if (ti < nt) {
    const double tv = t[ti];
    const double n = gn ? gn[gr] : n0;
    for (int p = pg; p < nv; p += kPG) {
      const int64_t q = (int64_t)gr * nv + p;
      double acc = 0.0;
      const int m = mm[q];
      if (F32) {
        // FP32 values summed in FP32 (m <= 64 terms of weights summing to 1):
        // the sum's rounding is of the size of the values' own
        float af = 0.0f;
        for (int k = 0; k < m; ++k)
          af = fmaf((float)tau2[q * s + k], fval32<FUN>(tv, theta[q * s + k]), af);
        acc = (double)af;
      } else {
        for (int k = 0; k < m; ++k) acc += tau2[q * s + k] * fval<FUN, false>(tv, theta[q * s + k]);
      }
      const double x = n * acc;
      if (per_probe) per_probe[q * nt + ti] = x;
      ++cnt;
      const double d = x - mean;
      mean += d / cnt;
      m2 += d * (x - mean);
    }
  }
  sh_mean[pg][tt] = mean;
  sh_m2[pg][tt] = m2;
  sh_cnt[pg][tt] = cnt;
  __syncthreads();
  if (pg == 0 && ti < nt) {
    double M = sh_mean[0][tt], S2 = sh_m2[0][tt];
    int N = sh_cnt[0][tt];
    for (int h = 1; h < kPG; ++h) {
      const int nb = sh_cnt[h][tt];
      if (nb == 0) continue;
      const double delta = sh_mean[h][tt] - M;
      const int nn = N + nb;
      M += delta * nb / nn;
      S2 += sh_m2[h][tt] + delta * delta * ((double)N * nb / nn);
      N = nn;
    }
    if (out) out[(int64_t)gr * nt + ti] = M;
    if (se) se[(int64_t)gr * nt + ti] = nv > 1 ? sqrt(S2 / (nv - 1) / nv) : nan("");
  }
}

// Heat trace with the polynomial control variate (Sec. 3.1, "2-term
// polynomial" variance reduction; reading: Chebyshev interpolant of degree
// DEG of f_t(x) = exp(-t x) on [0, bound_g]).  The Gauss rule of every probe
// is exact for p_t, so subtracting sum_k tau2 p_t(theta_k) from each probe's
// estimate and adding the exact c0 n + c1 tr L + c2 tr L^2 leaves the mean
// unbiased and removes the part of its variance p_t explains.  Same block
// layout and fixed-order Welford/Chan combination as k_trace_t.
template <bool F32>
__global__ void __launch_bounds__(kTT * kPG)
    k_trace_cv(const double *__restrict__ theta, const double *__restrict__ tau2,
               const int32_t *__restrict__ mm, int nv, int s, const double *__restrict__ gn,
               const double *__restrict__ gtrace, const double *__restrict__ gtrace2,
               const double *__restrict__ gbound, int degree, const double *__restrict__ t,
               int nt, double *out, double *se, double *per_probe) {
  __shared__ double sh_mean[kPG][kTT], sh_m2[kPG][kTT];
  __shared__ int sh_cnt[kPG][kTT];
  const int tt = threadIdx.x % kTT, pg = threadIdx.x / kTT;
  const int ti = blockIdx.x * kTT + tt;
  const int gr = blockIdx.y;
  double mean = 0.0, m2 = 0.0, exact_part = 0.0;
  int cnt = 0;
  if (ti < nt) {
    const double tv = t[ti];
    const double n = gn[gr], b = gbound[gr];
    // Chebyshev nodes of [0, b] and Newton divided differences of f there
    const double pi = 3.141592653589793;
    double c0, c1, c2 = 0.0;
    if (degree == 1) {
      const double x0 = 0.5 * b * (1.0 + cos(0.25 * pi)), x1 = 0.5 * b * (1.0 + cos(0.75 * pi));
      const double f0 = exp(-tv * x0), f1 = exp(-tv * x1);
      c1 = (f1 - f0) / (x1 - x0);
      c0 = f0 - c1 * x0;
    } else {
      const double x0 = 0.5 * b * (1.0 + cos(pi / 6.0)), x1 = 0.5 * b,
                   x2 = 0.5 * b * (1.0 + cos(5.0 * pi / 6.0));
      const double f0 = exp(-tv * x0), f1 = exp(-tv * x1), f2 = exp(-tv * x2);
      const double d01 = (f1 - f0) / (x1 - x0), d12 = (f2 - f1) / (x2 - x1);
      const double d012 = (d12 - d01) / (x2 - x0);
      c2 = d012;
      c1 = d01 - d012 * (x0 + x1);
      c0 = f0 - d01 * x0 + d012 * x0 * x1;
    }
    exact_part = c0 * n + c1 * gtrace[gr] + c2 * gtrace2[gr];
    for (int p = pg; p < nv; p += kPG) {
      const int64_t q = (int64_t)gr * nv + p;
      double acc = 0.0;
      const int m = mm[q];
      for (int k = 0; k < m; ++k) {
        const double th = theta[q * s + k];
        acc += tau2[q * s + k] * (fval<0, F32>(tv, th) - (c0 + th * (c1 + th * c2)));
      }
      const double x = n * acc;
      if (per_probe) per_probe[q * nt + ti] = x + exact_part;
      ++cnt;
      const double d = x - mean;
      mean += d / cnt;
      m2 += d * (x - mean);
    }
  }
  sh_mean[pg][tt] = mean;
  sh_m2[pg][tt] = m2;
  sh_cnt[pg][tt] = cnt;
  __syncthreads();
  if (pg == 0 && ti < nt) {
    double M = sh_mean[0][tt], S2 = sh_m2[0][tt];
    int N = sh_cnt[0][tt];
    for (int h = 1; h < kPG; ++h) {
      const int nb = sh_cnt[h][tt];
      if (nb == 0) continue;
      const double delta = sh_mean[h][tt] - M;
      const int nn = N + nb;
      M += delta * nb / nn;
      S2 += sh_m2[h][tt] + delta * delta * ((double)N * nb / nn);
      N = nn;
    }
    out[(int64_t)gr * nt + ti] = M + exact_part;
    if (se) se[(int64_t)gr * nt + ti] = nv > 1 ? sqrt(S2 / (nv - 1) / nv) : nan("");
  }
}

// VNGE of graph blockIdx.x: f(theta) = -(theta/c) ln(theta/c) for theta > 0,
// else 0, with c = tr(L_g).
__global__ void k_vnge(const double *__restrict__ theta, const double *__restrict__ tau2,
                       const int32_t *__restrict__ mm, int nv, int s,
                       const double *__restrict__ gn, const double *__restrict__ gtrace,
                       double *out, double *se, double *per_probe) {
  __shared__ double g[kMaxNv];
  const int gr = blockIdx.x;
  const double n = gn[gr], c = gtrace[gr];
  for (int p = threadIdx.x; p < nv; p += blockDim.x) {
    const int64_t q = (int64_t)gr * nv + p;
    double acc = 0.0;
    const int m = mm[q];
    for (int k = 0; k < m; ++k) {
      const double th = theta[q * s + k];
      if (th > 0.0 && c > 0.0) {
        const double x = th / c;
        acc += tau2[q * s + k] * (-x * log(x));
      }
    }
    g[p] = n * acc;
    if (per_probe) per_probe[q] = n * acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) mean_se(g, nv, out + gr, se ? se + gr : nullptr);
}

// The paper's O(m) comparators (Sec. 2.3) for graph blockIdx.x, from the
// traces the builder computed: the Taylor heat trace of Eq. hks-taylor,
// n - t tr L + (t^2/2) tr L^2, at every t; the quadratic VNGE approximation
// Q = 1 - tr(L^2) / tr(L)^2 (the two-term expansion x (1 - x) of -x ln x over
// the eigenvalues of P = L / tr L; both printed forms are garbled); FINGER's
// -Q ln(bound / tr L) with the Gershgorin bound of the spectrum, and
// -Q ln(lambda_max / tr L) with lambda_max the largest Ritz value of the
// graph's probes (the extreme Ritz values converge first).
__global__ void k_comparators(const double *__restrict__ theta, const int32_t *__restrict__ mm, int nv,
                              int s, const double *__restrict__ gn, const double *__restrict__ gtrace,
                              const double *__restrict__ gtrace2, const double *__restrict__ gbound,
                              const double *__restrict__ t, int nt, double *taylor, double *q_out,
                              double *bar_out, double *hat_out) {
  __shared__ double red[256];
  const int gr = blockIdx.x;
  const double n = gn[gr], tr = gtrace[gr], tr2 = gtrace2[gr];
  if (taylor)
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      const double tv = t[i];
      taylor[(int64_t)gr * nt + i] = n - tv * tr + 0.5 * tv * tv * tr2;
    }
  double mx = 0.0;
  for (int p = threadIdx.x; p < nv; p += blockDim.x) {
    const int64_t q = (int64_t)gr * nv + p;
    const int m = mm[q];
    if (m > 0) mx = fmax(mx, theta[q * s + m - 1]);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = 1; i < (int)blockDim.x; ++i) mx = fmax(mx, red[i]);
  const double q = tr > 0.0 ? 1.0 - tr2 / (tr * tr) : 0.0;
  if (q_out) q_out[gr] = q;
  if (bar_out) bar_out[gr] = tr > 0.0 ? -q * log(gbound[gr] / tr) : 0.0;
  if (hat_out) hat_out[gr] = (tr > 0.0 && mx > 0.0) ? -q * log(mx / tr) : 0.0;
}

// Orthogonality monitor of problem q = (graph, probe): the largest
// |u_j^T u_k| / (||u_j|| ||u_k||), j < k < min(m, kcap), over the measured
// Gram entries of the stored basis, and the smallest beta_k, k < m - 1.
// Both are non-negative, so their bit patterns order like the values and
// atomicMax / atomicMin on the 64-bit words combine the problems.
__global__ void k_monitor(const double *__restrict__ gram_all, const double *__restrict__ beta,
                          const int32_t *__restrict__ mm, int nv, int s, int ld, int total, int kcap,
                          unsigned long long *ortho_bits, unsigned long long *beta_bits) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int gr = q / nv, p = q - gr * nv;
  const double *G = gram_all + (int64_t)gr * s * s * ld;
  const int m = min(mm[q], s);
  const int kend = min(m, kcap);
  double mx = 0.0;
  for (int k = 1; k < kend; ++k) {
    const double gkk = G[((int64_t)k * s + k) * ld + p];
    for (int j = 0; j < k; ++j) {
      const double gjj = G[((int64_t)j * s + j) * ld + p];
      const double r = fabs(G[((int64_t)j * s + k) * ld + p]) * rsqrt(gjj * gkk);
      if (r == r) mx = fmax(mx, r);
    }
  }
  double mb = INFINITY;
  for (int k = 0; k + 1 < m; ++k) mb = fmin(mb, beta[(int64_t)q * s + k]);
  atomicMax(ortho_bits, (unsigned long long)__double_as_longlong(mx));
  if (m >= 2) atomicMin(beta_bits, (unsigned long long)__double_as_longlong(mb));
}

__global__ void k_distance(const double *a, const double *b, int len, int absdiff, double *out) {
  __shared__ double ps[256], pc[256];
  NeumaierD acc;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double d = a[i] - b[i];
    acc.add(d * d);
  }
  ps[threadIdx.x] = acc.s;
  pc[threadIdx.x] = acc.c;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (absdiff) {
      out[0] = fabs(a[0] - b[0]);
    } else {
      NeumaierD tot;
      for (int i = 0; i < (int)blockDim.x; ++i) {
        tot.add(ps[i]);
        tot.add(pc[i]);
      }
      out[0] = sqrt(tot.value());
    }
  }
}

}  // namespace

int run_ritz(slaq_krylov K, cudaStream_t st) {
  ProfScope prof(SLAQ_PROF_RITZ, st);
  SLAQ_CHECK_CUDA(cudaMemsetAsync(K->status, 0, sizeof(int32_t), st));
  ++tl_launches;
  const int total = K->n_graphs * K->nv;
  // the solver is latency-bound: few problems go one per block, over many SMs
  const int tpb = std::max(1, std::min(32, total / std::max(1, num_sms())));
  // partial reorthogonalization keeps the recurrence's T in every form (no
  // projected matrix is formed); full reorthogonalization in the reduced
  // forms takes the Rayleigh-Ritz matrix of the stored basis
  const bool pencil = K->precision != SLAQ_FP64 && K->reorth != 0;
  if (pencil && total < 4096) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_ritz_pencil_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ritz_warp_smem(kMaxS));
    SLAQ_CHECK_CUDA(attr);
    k_ritz_pencil_warp<<<(unsigned)total, 32, ritz_warp_smem(K->s), st>>>(
        K->gram, K->proj, K->m, K->nv, K->s, K->ld, K->alpha, K->beta, K->theta, K->tau2,
        K->status);
  } else if (pencil) {
    const int64_t need = (int64_t)total * ((int64_t)K->s * K->s + K->s * (K->s + 1) / 2 + 2 * K->s);
    if (need > K->rscratch_cap) {
      dmfree(K->rscratch);
      K->rscratch = nullptr;
      K->rscratch_cap = 0;
      SLAQ_TRY(dmalloc(reinterpret_cast<void **>(&K->rscratch), need * sizeof(double)));
      K->rscratch_cap = need;
    }
    k_ritz_pencil<<<(unsigned)ceil_div(total, tpb), tpb, 0, st>>>(
        K->gram, K->proj, K->m, K->nv, K->s, K->ld, total, K->rscratch, K->alpha, K->beta,
        K->theta, K->tau2, K->status);
  } else {
    k_ritz<<<(unsigned)ceil_div(total, tpb), tpb, 0, st>>>(K->alpha, K->beta, K->m, total, K->s,
                                                            K->theta, K->tau2, K->status, nullptr);
  }
  SLAQ_CHECK_LAUNCH("ritz");
  return SLAQ_OK;
}

namespace {
// Heat trace of the reduced forms with no FP64 work per term (FP64 is the
// narrow pipe of GB300).  The block stages its graph's rules once: theta as
// two floats (hi = fl(theta), lo = fl(theta - hi)) and tau2 as a float.  The
// product t theta is formed as p = fl(t_hi theta_hi) plus its residual
// c = fma(t_hi, theta_hi, -p) + t_hi theta_lo + t_lo theta_hi, with
// |c| <= 3 * 2^-24 |p|, so that e^{-t theta} = e^{-p} (1 - c) up to c^2 / 2
// (below 2e-10 wherever e^{-p} is a normal float).  Rounding t theta itself
// to a float, as a plain FP32 evaluation does, would cost |t theta| 2^-24
// relative instead.  Same layout, probe order, Welford updates and
// combination as k_trace_t, so slaq_pool_probes_host reproduces the mean and
// standard error from the per-probe values to the last bit.  The Welford
// division d / c takes Markstein's correction instead of a division (an
// FP64 division is a long sequence on the FP64 pipe): with r = 1/c correctly
// rounded (staged), q = fl(d r) and fl(q + fl(d - q c) r), the residual
// formed exactly by an FMA, is the correctly rounded quotient (P. Markstein,
// IBM J. Res. Dev. 34, 1990; tests/test_markstein_cpu.py checks it against
// IEEE division for c = 1..512).
inline size_t heat_f32_smem(int nv, int s) {
  const size_t per = (size_t)nv * s;
  const size_t nrcp = (size_t)(nv + kPG - 1) / kPG + 1;
  return nrcp * sizeof(double) + per * 3 * sizeof(float) + (size_t)nv * sizeof(int32_t);
}
constexpr size_t kHeatF32SmemMax = 48 * 1024;

__global__ void __launch_bounds__(kTT * kPG)
    k_heat_f32(const double *__restrict__ theta, const double *__restrict__ tau2,
               const int32_t *__restrict__ mm, int nv, int s, const double *__restrict__ gn,
               const double *__restrict__ t, int nt, double *out, double *se, double *per_probe) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int nrcp = (nv + kPG - 1) / kPG + 1;
  double *rcp = reinterpret_cast<double *>(dyn);         // rcp[c] = 1 / c
  float *th_hi = reinterpret_cast<float *>(rcp + nrcp);  // [nv][s] of this graph
  float *th_lo = th_hi + nv * s;
  float *wt = th_lo + nv * s;
  int32_t *ms = reinterpret_cast<int32_t *>(wt + nv * s);
  __shared__ double sh_mean[kPG][kTT], sh_m2[kPG][kTT];
  __shared__ int sh_cnt[kPG][kTT];
  const int gr = blockIdx.y;
  const int64_t base = (int64_t)gr * nv * s;
  for (int i = threadIdx.x; i < nv * s; i += blockDim.x) {
    const double th = theta[base + i];
    const float hi = (float)th;
    th_hi[i] = hi;
    th_lo[i] = (float)(th - (double)hi);
    wt[i] = (float)tau2[base + i];
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) ms[i] = mm[(int64_t)gr * nv + i];
  for (int i = threadIdx.x; i < nrcp; i += blockDim.x) rcp[i] = i > 0 ? 1.0 / i : 0.0;
  __syncthreads();
  const int tt = threadIdx.x % kTT, pg = threadIdx.x / kTT;
  const int ti = blockIdx.x * kTT + tt;
  double mean = 0.0, m2 = 0.0;
  int cnt = 0;
  if (ti < nt) {
    const double tv = t[ti];
    const float t_hi = (float)tv, t_lo = (float)(tv - (double)t_hi);
    const double n = gn[gr];
    for (int p = pg; p < nv; p += kPG) {
      const int m = min(ms[p], s);
      const float *h = th_hi + p * s, *l = th_lo + p * s, *w = wt + p * s;
      float af = 0.0f;
      for (int k = 0; k < m; ++k) {
        const float pr = t_hi * h[k];
        const float c = fmaf(t_hi, h[k], -pr) + fmaf(t_hi, l[k], t_lo * h[k]);
        af = fmaf(w[k], expf(-pr) * (1.0f - c), af);
      }
      const double x = n * (double)af;
      const int64_t q = (int64_t)gr * nv + p;
      if (per_probe) per_probe[q * nt + ti] = x;
      ++cnt;
      const double d = x - mean;
      const double r = rcp[cnt], qd = __dmul_rn(d, r);
      mean += fma(fma(-qd, (double)cnt, d), r, qd);  // d / cnt, correctly rounded
      m2 += d * (x - mean);
    }
  }
  sh_mean[pg][tt] = mean;
  sh_m2[pg][tt] = m2;
  sh_cnt[pg][tt] = cnt;
  __syncthreads();
  if (pg == 0 && ti < nt) {
    double M = sh_mean[0][tt], S2 = sh_m2[0][tt];
    int N = sh_cnt[0][tt];
    for (int h = 1; h < kPG; ++h) {
      const int nb = sh_cnt[h][tt];
      if (nb == 0) continue;
      const double delta = sh_mean[h][tt] - M;
      const int nn = N + nb;
      M += delta * nb / nn;
      S2 += sh_m2[h][tt] + delta * delta * ((double)N * nb / nn);
      N = nn;
    }
    if (out) out[(int64_t)gr * nt + ti] = M;
    if (se) se[(int64_t)gr * nt + ti] = nv > 1 ? sqrt(S2 / (nv - 1) / nv) : nan("");
  }
}
}  // namespace

int check_reduced_t(slaq_krylov K, const double *t, int nt, const char *what, cudaStream_t st);

int trace_heat(slaq_krylov K, const double *t, int nt, double *out, double *se, double *per_probe,
               cudaStream_t st) {
  if (nt < 1 || !t || !out) return set_error(SLAQ_EINVAL, "heat trace needs t, nt >= 1 and out");
  SLAQ_TRY(check_reduced_t(K, t, nt, "heat trace", st));
  ProfScope prof(SLAQ_PROF_TRACE, st);
  ++tl_launches;
  const dim3 grid((unsigned)ceil_div(nt, kTT), K->n_graphs);
  if (K->precision == SLAQ_FP64)
    k_trace_t<0, false><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                     t, nt, out, se, per_probe);
  else if (heat_f32_smem(K->nv, K->s) <= kHeatF32SmemMax)
    k_heat_f32<<<grid, kTT * kPG, heat_f32_smem(K->nv, K->s), st>>>(
        K->theta, K->tau2, K->m, K->nv, K->s, K->gn, t, nt, out, se, per_probe);
  else
    k_trace_t<0, true><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                    t, nt, out, se, per_probe);
  SLAQ_CHECK_LAUNCH("trace_heat");
  return SLAQ_OK;
}

int trace_heat_cv(slaq_krylov K, const double *t, int nt, int degree, double *out, double *se,
                  double *per_probe, cudaStream_t st) {
  if (nt < 1 || !t || !out) return set_error(SLAQ_EINVAL, "heat trace needs t, nt >= 1 and out");
  if (degree != 1 && degree != 2) return set_error(SLAQ_EINVAL, "control-variate degree must be 1 or 2");
  SLAQ_TRY(check_reduced_t(K, t, nt, "heat trace", st));
  ProfScope prof(SLAQ_PROF_TRACE, st);
  ++tl_launches;
  const dim3 grid((unsigned)ceil_div(nt, kTT), K->n_graphs);
  if (K->precision == SLAQ_FP64)
    k_trace_cv<false><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn,
                                                   K->gtrace, K->gtrace2, K->gbound, degree, t, nt,
                                                   out, se, per_probe);
  else
    k_trace_cv<true><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn,
                                                  K->gtrace, K->gtrace2, K->gbound, degree, t, nt,
                                                  out, se, per_probe);
  SLAQ_CHECK_LAUNCH("trace_heat_cv");
  return SLAQ_OK;
}

// The reduced forms serve heat and wave traces for |t| * bound <= a limit
// of their own (bound: 2 on a normalized Laplacian, 2 max d on L = D - A).
// The stored basis is rounded (2^-9 for BF16, 2^-24 for FP32), which moves
// the Ritz values that are not yet converged at first order, by about the
// rounding times bound; exp(-t theta) and cos(t theta) turn that into errors
// that grow with t * bound.  Measured against the FP64 form (nv 24 and 64,
// s 16 and 20):
// * BF16 basis, limit 20: within 2.3e-5 relative (heat) and 1e-5 of max
//   |Re| (wave) up to t * bound = 20 on every graph tried (R-MAT, BA, ER, SBM
//   batches, trees, cycles, paths, grids, weighted and not, both Laplacians);
//   beyond it the first failures of the 1e-4 bars came at t * bound = 58
//   (heat) and 40 (wave) on normalized small-eigenvalue graphs, 82 and 69 on
//   weighted cycles and paths with L = D - A;
// * FP32, limit 2000: within 4.4e-7 (heat) up to t * bound = 1000 on BA,
//   ER, R-MAT, cycles and paths with L = D - A; the heat bar first failed at
//   t * bound = 22,000 (a weighted BA graph), the wave's beyond 287,000.
//   (On a normalized Laplacian the limit is t <= 1000.)
constexpr double kBf16TB = 20.0;
constexpr double kFp32TB = 2000.0;

// SLAQ_OK, or SLAQ_EUNSUPPORTED if some t is beyond the reduced form's
// limit (copies t to the host and synchronizes st for the reduced forms).
int check_reduced_t(slaq_krylov K, const double *t, int nt, const char *what, cudaStream_t st) {
  if (K->precision == SLAQ_FP64) return SLAQ_OK;
  const bool bf16 = K->precision == SLAQ_FP32_BF16BASIS;
  const double limit = bf16 ? kBf16TB : kFp32TB;
  std::vector<double> th(nt);
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(th.data(), t, nt * sizeof(double), cudaMemcpyDeviceToHost, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < nt; ++i)
    if (!(std::fabs(th[i]) * K->bound <= limit))
      return set_error(SLAQ_EUNSUPPORTED,
                       "the %s form serves the %s for |t| * bound <= %g only (t = %g, bound %g): "
                       "beyond it the basis rounding moves the trace by more than 1e-4; use %s",
                       bf16 ? "BF16-basis" : "FP32", what, limit, th[i], K->bound,
                       bf16 ? "SLAQ_FP32 or SLAQ_FP64" : "SLAQ_FP64");
  return SLAQ_OK;
}

// re/im (means) may be NULL when only the per-probe values pp_re/pp_im
// ([G][nv][nt]) are wanted (slaq_trace_wave_per_probe).
int trace_wave(slaq_krylov K, const double *t, int nt, double *re, double *im, double *se_re,
               double *se_im, cudaStream_t st, double *pp_re, double *pp_im) {
  if (nt < 1 || !t || ((!re || !im) && (!pp_re || !pp_im)))
    return set_error(SLAQ_EINVAL, "wave trace needs t, nt, and re, im or per-probe outputs");
  SLAQ_TRY(check_reduced_t(K, t, nt, "wave trace", st));
  ProfScope prof(SLAQ_PROF_TRACE, st);
  ++tl_launches;
  const dim3 grid((unsigned)ceil_div(nt, kTT), K->n_graphs);
  const bool f32 = K->precision != SLAQ_FP64;
  if (f32)
    k_trace_t<1, true><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                    t, nt, re, se_re, pp_re);
  else
    k_trace_t<1, false><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                     t, nt, re, se_re, pp_re);
  ++tl_launches;
  if (f32)
    k_trace_t<2, true><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                    t, nt, im, se_im, pp_im);
  else
    k_trace_t<2, false><<<grid, kTT * kPG, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, 0.0,
                                                     t, nt, im, se_im, pp_im);
  SLAQ_CHECK_LAUNCH("trace_wave");
  return SLAQ_OK;
}

int trace_vnge(slaq_krylov K, double *out, double *se, double *per_probe, cudaStream_t st) {
  if (!out) return set_error(SLAQ_EINVAL, "vnge needs out");
  ProfScope prof(SLAQ_PROF_TRACE, st);
  ++tl_launches;
  k_vnge<<<K->n_graphs, 128, 0, st>>>(K->theta, K->tau2, K->m, K->nv, K->s, K->gn, K->gtrace, out,
                                       se, per_probe);
  SLAQ_CHECK_LAUNCH("trace_vnge");
  return SLAQ_OK;
}

int comparators(slaq_krylov K, const double *t, int nt, double *taylor, double *q, double *bar,
                double *hat, cudaStream_t st) {
  if (taylor && (!t || nt < 1)) return set_error(SLAQ_EINVAL, "the Taylor heat trace needs t and nt >= 1");
  ProfScope prof(SLAQ_PROF_TRACE, st);
  ++tl_launches;
  k_comparators<<<K->n_graphs, 256, 0, st>>>(K->theta, K->m, K->nv, K->s, K->gn, K->gtrace, K->gtrace2,
                                              K->gbound, t, taylor ? nt : 0, taylor, q, bar, hat);
  SLAQ_CHECK_LAUNCH("comparators");
  return SLAQ_OK;
}

int krylov_monitor(slaq_krylov K, double *ortho, double *min_beta, cudaStream_t st) {
  // the Gram column of the newest vector is formed on every step except the
  // last step of the FP64 form and of partial reorthogonalization (only its
  // diagonal entry): there the last vector is left out
  const int kcap = (K->precision == SLAQ_FP64 || K->reorth == 0) ? K->s - 1 : K->s;
  const int total = K->n_graphs * K->nv;
  unsigned long long *bits = reinterpret_cast<unsigned long long *>(K->status) + 1;
  const unsigned long long init[2] = {0ull, (unsigned long long)0x7ff0000000000000ull};  // 0, +inf
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(bits, init, sizeof(init), cudaMemcpyHostToDevice, st));
  ++tl_launches;
  k_monitor<<<(unsigned)ceil_div(total, 128), 128, 0, st>>>(K->gram, K->beta, K->m, K->nv, K->s,
                                                            K->ld, total, kcap, bits, bits + 1);
  SLAQ_CHECK_LAUNCH("krylov_monitor");
  unsigned long long h[2];
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(h, bits, sizeof(h), cudaMemcpyDeviceToHost, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  double v[2];
  std::memcpy(v, h, sizeof(v));
  if (ortho) *ortho = v[0];
  if (min_beta) *min_beta = v[1];
  return SLAQ_OK;
}

int distance(const double *a, const double *b, int nt, int kind, double *out, cudaStream_t st) {
  if (!a || !b || !out) return set_error(SLAQ_EINVAL, "distance needs a, b and out");
  int len;
  if (kind == SLAQ_DIST_HEAT) len = nt;
  else if (kind == SLAQ_DIST_WAVE) len = 2 * nt;
  else if (kind == SLAQ_DIST_VNGE) len = 1;
  else return set_error(SLAQ_EINVAL, "unknown distance kind %d", kind);
  if (len < 1) return set_error(SLAQ_EINVAL, "nt must be >= 1");
  ProfScope prof(SLAQ_PROF_DIST, st);
  ++tl_launches;
  k_distance<<<1, 256, 0, st>>>(a, b, len, kind == SLAQ_DIST_VNGE ? 1 : 0, out);
  SLAQ_CHECK_LAUNCH("distance");
  return SLAQ_OK;
}

// --------------------------------------------------- no-allocation variant
// Gauss nodes and weights of the allocation-free heat trace live in this
// file-scope device array (every device that loads the library holds it until
// the process exits).  Host code must not pass the symbol itself to a kernel:
// in host code it names a host-side stand-in, not device memory.  Its device
// address is obtained once per device with cudaGetSymbolAddress.
constexpr int kStaticMaxNvS = kMaxNv * kMaxS;  // 512 probes x 64 steps
static __device__ __align__(256) double g_static_gauss[2 * kStaticMaxNvS];
static __device__ __align__(256) int32_t g_static_status[8];
static __device__ __align__(256) int32_t g_static_m[kMaxNv];  // rule sizes clamped to [0, s]

namespace {
struct StaticScratch {
  double *gauss = nullptr;
  int32_t *status = nullptr;
  int32_t *m = nullptr;
};
std::mutex g_static_mutex;
StaticScratch g_static_ptr[64];
}  // namespace

int trace_heat_static(const double *alpha, const double *beta, const int32_t *m, int nv, int s,
                      int64_t n, const double *t, int nt, double *out, double *se,
                      int32_t *status_out, cudaStream_t st) {
  if (!alpha || !beta || !m || !t || !out) return set_error(SLAQ_EINVAL, "NULL argument");
  if (nv < 1 || nv > kMaxNv || s < 1 || s > kMaxS || (int64_t)nv * s > kStaticMaxNvS)
    return set_error(SLAQ_EINVAL,
                     "nv = %d, s = %d exceed the static scratch of this entry point "
                     "(nv <= %d, s <= %d)",
                     nv, s, kMaxNv, kMaxS);
  if (nt < 1 || n < 1) return set_error(SLAQ_EINVAL, "nt and n must be >= 1");
  int dev = -1;
  SLAQ_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(SLAQ_ENODEVICE, "device index out of range");
  StaticScratch sp;
  {
    std::lock_guard<std::mutex> lk(g_static_mutex);
    StaticScratch &slot = g_static_ptr[dev];
    if (!slot.gauss) {
      void *a = nullptr, *b = nullptr, *c = nullptr;
      cudaError_t e1 = cudaGetSymbolAddress(&a, g_static_gauss);
      if (e1 != cudaSuccess) return cuda_status(e1, "cudaGetSymbolAddress(scratch)");
      cudaError_t e2 = cudaGetSymbolAddress(&b, g_static_status);
      if (e2 != cudaSuccess) return cuda_status(e2, "cudaGetSymbolAddress(status)");
      cudaError_t e3 = cudaGetSymbolAddress(&c, g_static_m);
      if (e3 != cudaSuccess) return cuda_status(e3, "cudaGetSymbolAddress(rule sizes)");
      slot.gauss = static_cast<double *>(a);
      slot.status = static_cast<int32_t *>(b);
      slot.m = static_cast<int32_t *>(c);
    }
    sp = slot;
  }
  ProfScope prof(SLAQ_PROF_TRACE, st);
  double *theta = sp.gauss;
  double *tau2 = sp.gauss + (size_t)nv * s;
  SLAQ_CHECK_CUDA(cudaMemsetAsync(sp.status, 0, sizeof(int32_t), st));  // starts at zero
  ++tl_launches;
  // the caller's m is clamped to [0, s] by k_ritz, and the quadrature reads
  // the clamped copy, so no row is read past s entries whatever m holds
  k_ritz<<<(unsigned)ceil_div(nv, 32), 32, 0, st>>>(alpha, beta, m, nv, s, theta, tau2, sp.status,
                                                    sp.m);
  ++tl_launches;
  k_trace_t<0, false><<<dim3((unsigned)ceil_div(nt, kTT), 1), kTT * kPG, 0, st>>>(
      theta, tau2, sp.m, nv, s, nullptr, (double)n, t, nt, out, se, nullptr);
  if (status_out)
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(status_out, sp.status, sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, st));
  SLAQ_CHECK_LAUNCH("trace_heat_static");
  return SLAQ_OK;
}

}  // namespace slaq
