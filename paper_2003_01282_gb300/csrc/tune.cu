// Batched Lanczos over separately built graphs, and the autotuner that picks
// the kernels' launch shapes for a workload.
//
// A batch is one block-diagonal Laplacian (the graphs' CSRs concatenated on
// the device), so every Lanczos step serves all graphs with the same few
// launches (Sec. 3.1, Algorithm 1, run for many graphs at once).  The launch
// shapes that suit a batch of thousands of small graphs differ from those of
// one large graph: the tuner times a short list of candidates by coordinate
// descent on the real workload and keeps the fastest, and a text cache file
// remembers the choice per workload class.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace slaq {
namespace {

int log2_bucket(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }

// Workload class of a batch: precision, row width, size and degree buckets.
std::string tune_key(slaq_graph g, int nv, int s, int precision, int reorth) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  char buf[160];
  snprintf(buf, sizeof buf, "prec=%d nv=%d s=%d reorth=%d log2n=%d log2deg=%d log2G=%d sms=%d",
           precision, nv, s, reorth, log2_bucket((double)g->n),
           log2_bucket(g->n ? (double)g->nnz / (double)g->n : 0.0), log2_bucket(g->n_graphs), sms);
  return buf;
}

// Cache file: one line per workload class,
// "<key> | spmm upd dots slice align tma" (lines without the last field,
// written before the TMA gathers existed, read as tma = -1).
int read_cache(const char *path, std::map<std::string, slaq_tuning> *out) {
  FILE *f = fopen(path, "r");
  if (!f) {
    if (errno == ENOENT) return SLAQ_OK;  // no cache yet
    return set_error(SLAQ_EINVAL, "cannot read tune cache %s: %s", path, strerror(errno));
  }
  char line[512];
  while (fgets(line, sizeof line, f)) {
    char *bar = strchr(line, '|');
    if (!bar) continue;
    std::string key(line, bar - line);
    while (!key.empty() && key.back() == ' ') key.pop_back();
    slaq_tuning t;
    const int got = sscanf(bar + 1, "%d %d %d %d %d %d", &t.spmm_threads, &t.upd_threads,
                           &t.dots_threads, &t.slice_bytes, &t.spmm_align, &t.spmm_tma);
    if (got == 5) t.spmm_tma = -1;
    if (got == 5 || got == 6) (*out)[key] = t;
  }
  fclose(f);
  return SLAQ_OK;
}

int write_cache(const char *path, const std::map<std::string, slaq_tuning> &all) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return set_error(SLAQ_EINVAL, "cannot write tune cache %s: %s", path, strerror(errno));
  fprintf(f, "# slaq launch-shape cache: <workload class> | spmm_threads upd_threads "
             "dots_threads slice_bytes spmm_align spmm_tma\n");
  for (const auto &kv : all)
    fprintf(f, "%s | %d %d %d %d %d %d\n", kv.first.c_str(), kv.second.spmm_threads,
            kv.second.upd_threads, kv.second.dots_threads, kv.second.slice_bytes,
            kv.second.spmm_align, kv.second.spmm_tma);
  const bool ok = fclose(f) == 0;
  if (!ok || rename(tmp.c_str(), path) != 0)
    return set_error(SLAQ_EINVAL, "cannot write tune cache %s: %s", path, strerror(errno));
  return SLAQ_OK;
}

// Device time of one full Lanczos run with tuning t (the faster of two).
int time_run(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision, int reorth,
             const slaq_tuning &t, cudaStream_t st, slaq_krylov *K, float *ms) {
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
  float best = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {
    SLAQ_CHECK_CUDA(cudaEventRecord(a, st));
    SLAQ_TRY(run_lanczos(g, nv, s, seed, graph_id, precision, reorth, st, K, &t));
    SLAQ_CHECK_CUDA(cudaEventRecord(b, st));
    SLAQ_CHECK_CUDA(cudaEventSynchronize(b));
    float x = 0.0f;
    SLAQ_CHECK_CUDA(cudaEventElapsedTime(&x, a, b));
    best = rep == 0 ? x : std::min(best, x);
  }
  *ms = best;
  return SLAQ_OK;
}

// Coordinate descent over the launch-shape knobs, one pass, starting from
// the defaults; a candidate must win by 2% to replace the incumbent.
int autotune(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision, int reorth,
             cudaStream_t st, slaq_krylov *K, slaq_tuning *out) {
  slaq_tuning best;
  float best_ms = 0.0f;
  SLAQ_TRY(time_run(g, nv, s, seed, graph_id, precision, reorth, best, st, K, &best_ms));
  const int row_bytes = row_ld(nv, precision) * basis_bytes(precision);
  struct Knob {
    int slaq_tuning::*field;
    std::vector<int> values;
  };
  std::vector<Knob> knobs = {
      {&slaq_tuning::spmm_align, {-1, 1, 0}},
      {&slaq_tuning::spmm_threads, {128, 256, 512}},
      {&slaq_tuning::dots_threads, {0, 64, 128, 256}},
      {&slaq_tuning::upd_threads, {128, 256, 512}},
      {&slaq_tuning::slice_bytes, {0}},
  };
  for (int w : {128, 256})
    if (w < row_bytes) knobs.back().values.push_back(w);
  for (const Knob &k : knobs) {
    const int start = best.*(k.field);
    for (int v : k.values) {
      if (v == start) continue;
      slaq_tuning cand = best;
      cand.*(k.field) = v;
      float ms = 0.0f;
      SLAQ_TRY(time_run(g, nv, s, seed, graph_id, precision, reorth, cand, st, K, &ms));
      if (ms < 0.98f * best_ms) {
        best = cand;
        best_ms = ms;
      }
    }
  }
  *out = best;
  return SLAQ_OK;
}

}  // namespace

int lanczos_batched(const slaq_graph *gs, int count, int nv, int s, uint64_t seed, int graph_id,
                    int precision, int reorth, const char *tune_cache, cudaStream_t st,
                    slaq_krylov *inout) {
  if (!inout) return set_error(SLAQ_EINVAL, "NULL output handle");
  // one input handle (a single graph or a batch) runs as it is; a list is
  // concatenated into a union the Krylov handle owns
  slaq_graph u = nullptr;
  slaq_graph input = nullptr;
  if (gs && count == 1) {
    int dev = 0;
    SLAQ_CHECK_CUDA(cudaGetDevice(&dev));
    if (!gs[0]) return set_error(SLAQ_EINVAL, "graph 0 is NULL");
    if (gs[0]->device != dev) return set_error(SLAQ_EINVAL, "graph 0 lives on another device");
    input = gs[0];
  } else {
    SLAQ_TRY(union_graphs(gs, count, st, &u));
  }
  struct Own {
    slaq_graph *u;
    cudaStream_t st;
    ~Own() {
      if (*u) graph_free(*u, st);
    }
  } own{&u, st};
  slaq_graph g = input ? input : u;
  slaq_tuning tune;
  if (tune_cache) {
    std::map<std::string, slaq_tuning> all;
    SLAQ_TRY(read_cache(tune_cache, &all));
    const std::string key = tune_key(g, nv, s, precision, reorth);
    auto it = all.find(key);
    if (it != all.end()) {
      tune = it->second;
    } else {
      SLAQ_TRY(autotune(g, nv, s, seed, graph_id, precision, reorth, st, inout, &tune));
      all[key] = tune;
      SLAQ_TRY(write_cache(tune_cache, all));
    }
  }
  SLAQ_TRY(run_lanczos(g, nv, s, seed, graph_id, precision, reorth, st, inout, &tune));
  // the Krylov handle keeps a union alive until it is destroyed or reused (a
  // single input stays the caller's, as with slaq_lanczos)
  if ((*inout)->owned != u) graph_free((*inout)->owned, st);
  (*inout)->owned = u;
  u = nullptr;
  return SLAQ_OK;
}

}  // namespace slaq
