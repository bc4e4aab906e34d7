// extern "C" entry points of libslaq (declared in include/slaq.h): argument
// checks, device check, error reporting; the work is in build.cu,
// lanczos.cu and quad.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "tridiag.cuh"

namespace slaq {
namespace {
thread_local char g_msg[512] = "no error";
thread_local int g_status = SLAQ_OK;

struct DeviceInfo {
  int checked = 0;  // 0 unknown, 1 ok, 2 wrong device
  int sms = 0;
};
std::mutex g_dev_mutex;
DeviceInfo g_dev[64];
}  // namespace

int set_error(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  g_status = status;
  return status;
}

int cuda_status(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(SLAQ_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  }
  return set_error(SLAQ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_check() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return set_error(SLAQ_ENODEVICE, "no CUDA device available (%s); libslaq has no CPU path",
                     cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  DeviceInfo &d = g_dev[dev];
  if (d.checked == 0) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SLAQ_ENODEVICE, "cannot query CUDA device %d", dev);
    }
    d.checked = (prop.major == 10 && prop.minor == 3) ? 1 : 2;
    d.sms = prop.multiProcessorCount;
    if (d.checked == 1) {
      // keep freed stream-ordered allocations cached in the pool
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      cudaGetLastError();
    }
  }
  if (d.checked != 1)
    return set_error(SLAQ_ENODEVICE,
                     "CUDA device %d is not compute capability 10.3 (GB300); libslaq is built "
                     "for sm_103a only",
                     dev);
  return SLAQ_OK;
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  return std::max(1, g_dev[dev].sms);
}

// ------------------------------------------------------------ allocations
// Every device (and pinned host) allocation of the library goes through
// these functions: they count the allocations the library holds, and a test
// hook (slaq_debug_fail_alloc) can make the n-th one fail as an out-of-memory
// device would, so that every SLAQ_ENOMEM path can be walked.
namespace {
std::atomic<int64_t> g_live_allocs{0};
std::atomic<int64_t> g_fail_at{0};     // 0: off
std::atomic<int64_t> g_alloc_seen{0};  // allocations since the hook was armed
}  // namespace

static int alloc_gate(size_t bytes) {
  const int64_t f = g_fail_at.load();
  if (f > 0 && g_alloc_seen.fetch_add(1) + 1 == f)
    return set_error(SLAQ_ENOMEM, "allocation of %zu bytes failed (injected by slaq_debug_fail_alloc)",
                     bytes);
  return SLAQ_OK;
}

int dalloc(void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  SLAQ_TRY(alloc_gate(bytes));
  cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(SLAQ_ENOMEM, "cudaMallocAsync of %zu bytes failed: %s", bytes,
                     cudaGetErrorString(e));
  }
  ++g_live_allocs;
  return SLAQ_OK;
}

void dfree(void *p, cudaStream_t st) {
  if (!p) return;
  cudaFreeAsync(p, st);
  --g_live_allocs;
}

int dmalloc(void **p, size_t bytes) {
  *p = nullptr;
  SLAQ_TRY(alloc_gate(bytes));
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(SLAQ_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ++g_live_allocs;
  return SLAQ_OK;
}

void dmfree(void *p) {
  if (!p) return;
  cudaFree(p);
  --g_live_allocs;
}

int hmalloc(void **p, size_t bytes) {
  *p = nullptr;
  SLAQ_TRY(alloc_gate(bytes));
  cudaError_t e = cudaMallocHost(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(SLAQ_ENOMEM, "cudaMallocHost of %zu bytes failed: %s", bytes,
                     cudaGetErrorString(e));
  }
  ++g_live_allocs;
  return SLAQ_OK;
}

void hmfree(void *p) {
  if (!p) return;
  cudaFreeHost(p);
  --g_live_allocs;
}

// ---------------------------------------------------------------- profiler
thread_local int64_t tl_launches = 0;
namespace {
thread_local bool tl_prof_paused = false;  // inside a stream capture
struct ProfPair {
  int cat;
  cudaEvent_t a, b;
};
std::mutex g_prof_mutex;
bool g_prof_on = false;
std::vector<ProfPair> g_prof_pairs;
std::vector<cudaEvent_t> g_prof_pool;
std::vector<std::pair<int, cudaEvent_t>> g_prof_open;  // (cat, start) per open scope
double g_prof_ms[SLAQ_PROF_NCAT] = {0};
int64_t g_prof_launch[SLAQ_PROF_NCAT] = {0};

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void prof_collect_locked() {
  for (auto &p : g_prof_pairs) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      g_prof_ms[p.cat] += ms;
    cudaGetLastError();
    g_prof_pool.push_back(p.a);
    g_prof_pool.push_back(p.b);
  }
  g_prof_pairs.clear();
}
}  // namespace

void nvtx_push(int cat) {
  static const char *names[SLAQ_PROF_NCAT] = {"slaq:build",  "slaq:probes", "slaq:spmm",
                                              "slaq:dots",   "slaq:update", "slaq:reduce",
                                              "slaq:ritz",   "slaq:trace",  "slaq:distance"};
  nvtxRangePushA(cat >= 0 && cat < SLAQ_PROF_NCAT ? names[cat] : "slaq");
}
void nvtx_pop() { nvtxRangePop(); }

ProfPause::ProfPause() : saved(tl_prof_paused) { tl_prof_paused = true; }
ProfPause::~ProfPause() { tl_prof_paused = saved; }

void prof_begin(int cat, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  cudaEvent_t e = nullptr;
  if (g_prof_on && !tl_prof_paused) {
    e = prof_event();
    if (e && cudaEventRecord(e, st) != cudaSuccess) {
      cudaGetLastError();
      g_prof_pool.push_back(e);
      e = nullptr;
    }
  }
  g_prof_open.push_back({cat, e});
}

void prof_end(int cat, cudaStream_t st, int64_t launches) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  cudaEvent_t a = nullptr;
  for (size_t i = g_prof_open.size(); i-- > 0;) {
    if (g_prof_open[i].first == cat) {
      a = g_prof_open[i].second;
      g_prof_open.erase(g_prof_open.begin() + i);
      break;
    }
  }
  if (cat >= 0 && cat < SLAQ_PROF_NCAT && !tl_prof_paused) g_prof_launch[cat] += launches;
  if (!a) return;
  cudaEvent_t b = prof_event();
  if (!b || cudaEventRecord(b, st) != cudaSuccess) {
    cudaGetLastError();
    g_prof_pool.push_back(a);
    if (b) g_prof_pool.push_back(b);
    return;
  }
  g_prof_pairs.push_back({cat, a, b});
  if (g_prof_pairs.size() > 4096) prof_collect_locked();
}

}  // namespace slaq

using namespace slaq;

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Device-side outcome of a Lanczos run, read after it completes: word 1
// flags a TMA gather wait that gave up (the run's z vectors are incomplete),
// word 0 a tridiagonal eigensolver that did not converge.
static int run_status(slaq_krylov k, cudaStream_t st) {
  int32_t status[2] = {0, 0};
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(status, k->status, sizeof(status), cudaMemcpyDeviceToHost, st));
  SLAQ_CHECK_CUDA(cudaStreamSynchronize(st));
  if (status[1]) {
    k->ready = false;
    return set_error(SLAQ_ETIMEOUT, "a TMA row-gather wait of the SpMM gave up; rerun the handle");
  }
  if (status[0]) return set_error(SLAQ_ENUMERIC, "tridiagonal eigensolver did not converge");
  return SLAQ_OK;
}

extern "C" {

int slaq_version(void) { return 100; }

int slaq_last_error(char *buf, size_t len) {
  if (buf && len) {
    strncpy(buf, g_msg, len - 1);
    buf[len - 1] = '\0';
  }
  return g_status;
}

int slaq_device_check(void) { return device_check(); }

int slaq_build_laplacian(const int32_t *src, const int32_t *dst, int64_t n_edges, int64_t n_nodes,
                         const double *weights, int kind, int flags, void *stream,
                         slaq_graph *out) {
  SLAQ_TRY(device_check());
  return build_laplacian(src, dst, n_edges, n_nodes, weights, kind, flags, as_stream(stream), out);
}

int slaq_build_laplacian_batch(const int32_t *src, const int32_t *dst,
                               const int64_t *edge_off_host, const int64_t *node_off_host,
                               int n_graphs, const double *weights, int kind, int flags,
                               void *stream, slaq_graph *out) {
  SLAQ_TRY(device_check());
  if (!edge_off_host || !node_off_host || n_graphs < 1)
    return set_error(SLAQ_EINVAL, "a batch needs n_graphs >= 1 and both offset arrays");
  return build_laplacian(src, dst, 0, 0, weights, kind, flags, as_stream(stream), out, n_graphs,
                         edge_off_host, node_off_host);
}

int slaq_graph_batch_info(slaq_graph g, int *n_graphs, int64_t *node_off, double *trace) {
  if (!g) return set_error(SLAQ_EINVAL, "NULL graph");
  if (n_graphs) *n_graphs = g->n_graphs;
  if (node_off) std::memcpy(node_off, g->goff.data(), g->goff.size() * sizeof(int64_t));
  if (trace) std::memcpy(trace, g->gtrace.data(), g->gtrace.size() * sizeof(double));
  return SLAQ_OK;
}

int slaq_krylov_batch_info(slaq_krylov k, int *n_graphs) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  if (n_graphs) *n_graphs = k->n_graphs;
  return SLAQ_OK;
}

int slaq_graph_info(slaq_graph g, int64_t *n, int64_t *nnz, double *trace, int64_t *n_input) {
  if (!g) return set_error(SLAQ_EINVAL, "NULL graph");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (trace) *trace = g->trace;
  if (n_input) *n_input = g->n_input;
  return SLAQ_OK;
}

int slaq_graph_export(slaq_graph g, int64_t *rowptr, int32_t *colidx, double *vals, double *diag,
                      double *scale, int64_t *old_id, void *stream) {
  if (!g) return set_error(SLAQ_EINVAL, "NULL graph");
  SLAQ_TRY(device_check());
  cudaStream_t st = as_stream(stream);
  auto cp = [&](void *dst, const void *src, size_t bytes) -> int {
    if (dst && bytes) SLAQ_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return SLAQ_OK;
  };
  SLAQ_TRY(cp(rowptr, g->rowptr, (g->n + 1) * sizeof(int64_t)));
  SLAQ_TRY(cp(colidx, g->colidx, g->nnz * sizeof(int32_t)));
  SLAQ_TRY(cp(vals, g->vals, g->nnz * sizeof(double)));
  SLAQ_TRY(cp(diag, g->diag, g->n * sizeof(double)));
  SLAQ_TRY(cp(scale, g->scale, g->n * sizeof(double)));
  SLAQ_TRY(cp(old_id, g->old_id, g->n * sizeof(int64_t)));
  return SLAQ_OK;
}

void slaq_graph_destroy(slaq_graph g) {
  if (!g) return;
  cudaDeviceSynchronize();
  graph_free(g, 0);
}

int slaq_lanczos(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision,
                 int reorth_passes, void *stream, slaq_krylov *inout) {
  SLAQ_TRY(device_check());
  cudaStream_t st = as_stream(stream);
  SLAQ_TRY(run_lanczos(g, nv, s, seed, graph_id, precision, reorth_passes, st, inout));
  return run_status((*inout), st);
}

int slaq_lanczos_probes(slaq_graph g, int nv, int probe0, int s, uint64_t seed, int graph_id,
                        int precision, int reorth_passes, void *stream, slaq_krylov *inout) {
  SLAQ_TRY(device_check());
  cudaStream_t st = as_stream(stream);
  SLAQ_TRY(run_lanczos(g, nv, s, seed, graph_id, precision, reorth_passes, st, inout, nullptr,
                       probe0));
  return run_status((*inout), st);
}

int slaq_lanczos_rerun(slaq_krylov k, uint64_t seed, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  cudaStream_t st = as_stream(stream);
  SLAQ_TRY(lanczos_rerun(k, seed, st));
  return run_status(k, st);
}

int slaq_lanczos_batched(const slaq_graph *gs, int count, int nv, int s, uint64_t seed,
                         int graph_id, int precision, int reorth_passes, const char *tune_cache,
                         void *stream, slaq_krylov *inout) {
  SLAQ_TRY(device_check());
  cudaStream_t st = as_stream(stream);
  SLAQ_TRY(lanczos_batched(gs, count, nv, s, seed, graph_id, precision, reorth_passes, tune_cache,
                           st, inout));
  return run_status((*inout), st);
}

int slaq_probes(slaq_graph g, int nv, uint64_t seed, int graph_id, double *out, void *stream) {
  SLAQ_TRY(device_check());
  return probes(g, nv, seed, graph_id, out, as_stream(stream));
}

int slaq_krylov_full_steps(slaq_krylov k, int32_t *full_steps, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  SLAQ_TRY(slaq::full_steps(k, full_steps, as_stream(stream)));
  return SLAQ_OK;
}

int slaq_krylov_export(slaq_krylov k, double *alpha, double *beta, int32_t *m, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  cudaStream_t st = as_stream(stream);
  const size_t ns = (size_t)k->n_graphs * k->nv * k->s;
  if (alpha) SLAQ_CHECK_CUDA(cudaMemcpyAsync(alpha, k->alpha, ns * 8, cudaMemcpyDeviceToDevice, st));
  if (beta) SLAQ_CHECK_CUDA(cudaMemcpyAsync(beta, k->beta, ns * 8, cudaMemcpyDeviceToDevice, st));
  if (m)
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(m, k->m, (size_t)k->n_graphs * k->nv * 4,
                                    cudaMemcpyDeviceToDevice, st));
  return SLAQ_OK;
}

int slaq_ritz_export(slaq_krylov k, double *theta, double *tau2, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  cudaStream_t st = as_stream(stream);
  const size_t ns = (size_t)k->n_graphs * k->nv * k->s;
  if (theta) SLAQ_CHECK_CUDA(cudaMemcpyAsync(theta, k->theta, ns * 8, cudaMemcpyDeviceToDevice, st));
  if (tau2) SLAQ_CHECK_CUDA(cudaMemcpyAsync(tau2, k->tau2, ns * 8, cudaMemcpyDeviceToDevice, st));
  return SLAQ_OK;
}

int slaq_krylov_info(slaq_krylov k, int *nv, int *s, int *precision, int64_t *n) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  if (nv) *nv = k->nv;
  if (s) *s = k->s;
  if (precision) *precision = k->precision;
  if (n) *n = k->n;
  return SLAQ_OK;
}

int slaq_krylov_gathers(slaq_krylov k, int *tma_host) {
  if (!k || !tma_host) return set_error(SLAQ_EINVAL, "NULL Krylov handle or output");
  *tma_host = k->tma ? 1 : 0;
  return SLAQ_OK;
}

int slaq_trace_heat(slaq_krylov k, const double *t, int nt, double *out, double *stderr_,
                    double *per_probe, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return trace_heat(k, t, nt, out, stderr_, per_probe, as_stream(stream));
}

int slaq_trace_heat_cv(slaq_krylov k, const double *t, int nt, int degree, double *out,
                       double *stderr_, double *per_probe, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return trace_heat_cv(k, t, nt, degree, out, stderr_, per_probe, as_stream(stream));
}

int slaq_trace_wave(slaq_krylov k, const double *t, int nt, double *re, double *im,
                    double *stderr_re, double *stderr_im, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return trace_wave(k, t, nt, re, im, stderr_re, stderr_im, as_stream(stream));
}

int slaq_trace_wave_per_probe(slaq_krylov k, const double *t, int nt, double *re_pp,
                              double *im_pp, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  if (!re_pp || !im_pp) return set_error(SLAQ_EINVAL, "per-probe outputs must not be NULL");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return trace_wave(k, t, nt, nullptr, nullptr, nullptr, nullptr, as_stream(stream), re_pp, im_pp);
}

int slaq_trace_vnge(slaq_krylov k, double *out, double *stderr_, double *per_probe, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return trace_vnge(k, out, stderr_, per_probe, as_stream(stream));
}

void slaq_krylov_destroy(slaq_krylov k) {
  if (!k) return;
  cudaDeviceSynchronize();
  krylov_free(k);
}

int slaq_comparators(slaq_krylov k, const double *t, int nt, double *taylor_heat, double *vnge_q,
                     double *finger_bar, double *finger_hat, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return comparators(k, t, nt, taylor_heat, vnge_q, finger_bar, finger_hat, as_stream(stream));
}

int slaq_krylov_monitor(slaq_krylov k, double *ortho_host, double *min_beta_host, void *stream) {
  if (!k) return set_error(SLAQ_EINVAL, "NULL Krylov handle");
  SLAQ_TRY(device_check());
  SLAQ_TRY(krylov_ready(k));
  return krylov_monitor(k, ortho_host, min_beta_host, as_stream(stream));
}

int slaq_distance(const double *a, const double *b, int nt, int kind, double *out, void *stream) {
  SLAQ_TRY(device_check());
  return distance(a, b, nt, kind, out, as_stream(stream));
}

}  // extern "C"

// The Krylov workspace of slaq_descriptors_host's last call on each device,
// kept for the next call (its basis alone is s * n' * nv * 4 bytes: 5 GB at
// R-MAT 2^20 with nv = 100, whose cudaMalloc and cudaFree would otherwise be
// paid on every call).  A call takes the slot's handle (or none), and gives
// it back when it succeeds; a second handle for the same device is freed.
namespace {
constexpr int kCacheDevices = 64;
std::mutex g_host_cache_mu;
slaq_krylov g_host_cache[kCacheDevices] = {};

slaq_krylov host_cache_take(int dev, int nv, int s, int precision) {
  slaq_krylov k = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_host_cache_mu);
    if (dev < 0 || dev >= kCacheDevices) return nullptr;
    k = g_host_cache[dev];
    g_host_cache[dev] = nullptr;
  }
  if (k && (k->nv != nv || k->s != s || k->precision != precision)) {
    krylov_free(k);  // idle: its last call synchronized its stream
    k = nullptr;
  }
  return k;
}

void host_cache_put(int dev, slaq_krylov k) {
  {
    std::lock_guard<std::mutex> lock(g_host_cache_mu);
    if (dev >= 0 && dev < kCacheDevices && !g_host_cache[dev]) {
      g_host_cache[dev] = k;
      return;
    }
  }
  krylov_free(k);
}
}  // namespace

extern "C" {

int slaq_release_cached(void) {
  std::lock_guard<std::mutex> lock(g_host_cache_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < kCacheDevices; ++d) {
    if (!g_host_cache[d]) continue;
    cudaSetDevice(d);
    krylov_free(g_host_cache[d]);
    g_host_cache[d] = nullptr;
  }
  cudaSetDevice(cur);
  return SLAQ_OK;
}

int slaq_descriptors_host(const int32_t *src_host, const int32_t *dst_host, int64_t n_edges,
                          int64_t n_nodes, int kind, int flags, int nv, int s, uint64_t seed,
                          int precision, const double *t_host, int nt, double *heat_host,
                          double *wave_re_host, double *wave_im_host, double *vnge_host,
                          void *stream) {
  SLAQ_TRY(device_check());
  if (n_edges < 0 || (n_edges > 0 && (!src_host || !dst_host)))
    return set_error(SLAQ_EINVAL, "bad edge arrays");
  if ((heat_host || wave_re_host || wave_im_host) && (!t_host || nt < 1))
    return set_error(SLAQ_EINVAL, "traces need t_host and nt >= 1");
  cudaStream_t st = as_stream(stream);
  struct Bufs {
    cudaStream_t st;
    std::vector<void *> p;
    slaq_graph g = nullptr;
    slaq_krylov k = nullptr;
    ~Bufs() {
      cudaStreamSynchronize(st);
      for (void *x : p) dfree(x, st);
      if (k) krylov_free(k);
      if (g) graph_free(g, st);
      cudaStreamSynchronize(st);
    }
  } b{st, {}};
  auto get = [&](void **x, size_t bytes) -> int {
    SLAQ_TRY(dalloc(x, bytes, st));
    b.p.push_back(*x);
    return SLAQ_OK;
  };
  int32_t *src = nullptr, *dst = nullptr;
  double *t = nullptr, *out = nullptr;
  const int ntt = std::max(nt, 1);
  SLAQ_TRY(get((void **)&src, n_edges * sizeof(int32_t)));
  SLAQ_TRY(get((void **)&dst, n_edges * sizeof(int32_t)));
  SLAQ_TRY(get((void **)&t, ntt * sizeof(double)));
  SLAQ_TRY(get((void **)&out, (3 * (size_t)ntt + 1) * sizeof(double)));
  if (n_edges > 0) {
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(src, src_host, n_edges * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(dst, dst_host, n_edges * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  }
  if (t_host && nt > 0)
    SLAQ_CHECK_CUDA(cudaMemcpyAsync(t, t_host, nt * sizeof(double), cudaMemcpyHostToDevice, st));
  SLAQ_TRY(build_laplacian(src, dst, n_edges, n_nodes, nullptr, kind, flags, st, &b.g));
  int dev = 0;
  SLAQ_CHECK_CUDA(cudaGetDevice(&dev));
  b.k = host_cache_take(dev, nv, s, precision);
  SLAQ_TRY(run_lanczos(b.g, nv, s, seed, 0, precision, 1, st, &b.k));
  if (heat_host) SLAQ_TRY(trace_heat(b.k, t, nt, out, nullptr, nullptr, st));
  if (wave_re_host || wave_im_host)
    SLAQ_TRY(trace_wave(b.k, t, nt, out + ntt, out + 2 * ntt, nullptr, nullptr, st));
  if (vnge_host) SLAQ_TRY(trace_vnge(b.k, out + 3 * ntt, nullptr, nullptr, st));
  std::vector<double> h(3 * (size_t)ntt + 1);
  SLAQ_CHECK_CUDA(cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SLAQ_TRY(run_status(b.k, st));
  if (heat_host) std::memcpy(heat_host, h.data(), nt * sizeof(double));
  if (wave_re_host) std::memcpy(wave_re_host, h.data() + ntt, nt * sizeof(double));
  if (wave_im_host) std::memcpy(wave_im_host, h.data() + 2 * ntt, nt * sizeof(double));
  if (vnge_host) *vnge_host = h[3 * ntt];
  host_cache_put(dev, b.k);  // b's destructor synchronizes st before the next call can take it
  b.k = nullptr;
  return SLAQ_OK;
}

int slaq_trace_heat_tridiag_static(const double *alpha, const double *beta, const int32_t *m,
                                   int nv, int s, int64_t n, const double *t, int nt, double *out,
                                   double *stderr_, int32_t *status, void *stream) {
  SLAQ_TRY(device_check());
  return trace_heat_static(alpha, beta, m, nv, s, n, t, nt, out, stderr_, status,
                           as_stream(stream));
}

int slaq_debug_fail_alloc(int64_t nth) {
  g_alloc_seen = 0;
  g_fail_at = nth > 0 ? nth : 0;
  return SLAQ_OK;
}

int64_t slaq_debug_live_allocs(void) { return g_live_allocs.load(); }

int slaq_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  if (on) {
    prof_collect_locked();
    for (int i = 0; i < SLAQ_PROF_NCAT; ++i) {
      g_prof_ms[i] = 0.0;
      g_prof_launch[i] = 0;
    }
  }
  g_prof_on = on != 0;
  return SLAQ_OK;
}

int slaq_profile_gather_peak(int row_bytes, double *tbps_host) {
  SLAQ_TRY(device_check());
  if (!tbps_host) return set_error(SLAQ_EINVAL, "NULL output");
  return profile_gather_peak(row_bytes, tbps_host);
}

int slaq_profile_read(int category, double *ms, int64_t *launches) {
  if (category < 0 || category >= SLAQ_PROF_NCAT)
    return set_error(SLAQ_EINVAL, "unknown profile category %d", category);
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  prof_collect_locked();
  if (ms) *ms = g_prof_ms[category];
  if (launches) *launches = g_prof_launch[category];
  return SLAQ_OK;
}

int slaq_pool_probes_host(const double *values, int nprobe, int len, double *mean,
                          double *stderr_) {
  if (!values || !mean || nprobe < 1 || len < 1)
    return set_error(SLAQ_EINVAL, "pooling needs values, mean, nprobe >= 1 and len >= 1");
  // Welford means and squared deviations over the probe groups p mod 4, then
  // Chan's pairwise combination in group order: the order the device
  // quadrature kernels use, so pooled shards of one run reproduce it.
  constexpr int kGroups = 4;
  for (int j = 0; j < len; ++j) {
    double gm[kGroups] = {0}, g2[kGroups] = {0};
    int gc[kGroups] = {0};
    for (int h = 0; h < kGroups; ++h)
      for (int p = h; p < nprobe; p += kGroups) {
        const double x = values[(size_t)p * len + j];
        ++gc[h];
        const double d = x - gm[h];
        gm[h] += d / gc[h];
        g2[h] += d * (x - gm[h]);
      }
    double M = gm[0], S2 = g2[0];
    int N = gc[0];
    for (int h = 1; h < kGroups; ++h) {
      if (gc[h] == 0) continue;
      const double delta = gm[h] - M;
      const int nn = N + gc[h];
      M += delta * gc[h] / nn;
      S2 += g2[h] + delta * delta * ((double)N * gc[h] / nn);
      N = nn;
    }
    mean[j] = M;
    if (stderr_) stderr_[j] = nprobe > 1 ? std::sqrt(S2 / (nprobe - 1) / nprobe) : NAN;
  }
  return SLAQ_OK;
}

int slaq_set_spmm_gathers(int mode) { return set_spmm_gathers(mode); }

int slaq_debug_tma_giveup(int on) { return debug_tma_giveup(on); }

int slaq_tridiag_gauss_host(const double *alpha, const double *beta, int m, double *theta,
                            double *tau2) {
  if (m < 1 || m > 4096 || !alpha || !theta || !tau2 || (m > 1 && !beta))
    return set_error(SLAQ_EINVAL, "bad arguments to slaq_tridiag_gauss_host");
  std::vector<double> e(std::max(m, 1), 0.0);
  for (int i = 0; i < m; ++i) theta[i] = alpha[i];
  for (int i = 0; i + 1 < m; ++i) e[i] = beta[i];
  if (tridiag_gauss(theta, e.data(), tau2, m) != 0)
    return set_error(SLAQ_ENUMERIC, "tridiagonal eigensolver did not converge");
  return SLAQ_OK;
}

}  // extern "C"
