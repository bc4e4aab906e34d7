// Internal declarations shared by the libslaq translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "slaq.h"

namespace slaq {

// ------------------------------------------------------------------ errors
int set_error(int status, const char *fmt, ...);
int cuda_status(cudaError_t e, const char *what);

#define SLAQ_CHECK_CUDA(call)                                             \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ::slaq::cuda_status(e_, #call);         \
  } while (0)

#define SLAQ_CHECK_LAUNCH(name)                                           \
  do {                                                                    \
    cudaError_t e_ = cudaPeekAtLastError();                               \
    if (e_ != cudaSuccess) return ::slaq::cuda_status(e_, name);          \
  } while (0)

#define SLAQ_TRY(call)                                                    \
  do {                                                                    \
    int st_ = (call);                                                     \
    if (st_ != SLAQ_OK) return st_;                                       \
  } while (0)

int device_check();        // SLAQ_OK on a compute-capability 10.3 device

// Profiler (api.cu): CUDA events around a kernel class on its launch
// stream, and kernel launch counts (every launch site bumps tl_launches).
extern thread_local int64_t tl_launches;
void prof_begin(int cat, cudaStream_t st);
void prof_end(int cat, cudaStream_t st, int64_t launches);
// Suspends the profiler's event records on this thread (inside a capture).
struct ProfPause {
  bool saved;
  ProfPause();
  ~ProfPause();
};
// A kernel class on the host timeline: an NVTX range (visible to Nsight
// tools when one is attached; a no-op otherwise) and, when the profiler is
// on, CUDA events on the launch stream.
void nvtx_push(int cat);
void nvtx_pop();
struct ProfScope {
  int cat;
  cudaStream_t st;
  int64_t start;
  ProfScope(int c, cudaStream_t s) : cat(c), st(s), start(tl_launches) {
    nvtx_push(c);
    prof_begin(c, s);
  }
  ~ProfScope() {
    prof_end(cat, st, tl_launches - start);
    nvtx_pop();
  }
};
int num_sms();             // streaming multiprocessors of the current device

// Allocations (api.cu).  Every allocation of the library goes through these:
// they keep the count slaq_debug_live_allocs reports and honour the test
// hook slaq_debug_fail_alloc.  dalloc/dfree: stream-ordered, from the
// device's default memory pool; dmalloc/dmfree: cudaMalloc/cudaFree;
// hmalloc/hmfree: pinned host memory.  On failure *p is NULL and the status
// is SLAQ_ENOMEM.
int dalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);
int dmalloc(void **p, size_t bytes);
void dmfree(void *p);
int hmalloc(void **p, size_t bytes);
void hmfree(void *p);

template <typename T>
inline int dalloc_t(T **p, size_t count, cudaStream_t st) {
  return dalloc(reinterpret_cast<void **>(p), count * sizeof(T), st);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// --------------------------------------------------------- precision forms
// Basis element type TB and work type TW of each form.
//   FP64: TB = double, TW = double
//   FP32: TB = float,  TW = float
//   BF16: TB = bf16,   TW = float
// Every thread owns one 16-byte vector of a basis row: VE = 16/sizeof(TB)
// probe columns.  The row stride `ld` (elements) makes a basis row a whole
// number of 32-byte sectors.
inline int basis_bytes(int precision) { return precision == SLAQ_FP64 ? 8 : (precision == SLAQ_FP32 ? 4 : 2); }
inline int work_bytes(int precision) { return precision == SLAQ_FP64 ? 8 : 4; }
inline int row_ld(int nv, int precision) {
  int per_sector = 32 / basis_bytes(precision);
  return (int)ceil_div(nv, per_sector) * per_sector;
}
inline int vec_elems(int precision) { return 16 / basis_bytes(precision); }

// ------------------------------------------------------------ graph handle
constexpr int kHeavyChunk = 512;   // nnz per work item of a split (heavy) row

}  // namespace slaq

struct slaq_graph_s {
  uint64_t uid = 0;      // unique over the process (graph_alive)
  int device = -1;
  int64_t n_input = 0;   // n_nodes given at build time (sum over a batch)
  int64_t n = 0;         // kept nodes n' (sum over a batch)
  int64_t nnz = 0;       // stored off-diagonal entries
  int kind = 0;
  int flags = 0;
  bool weighted = false;
  double trace = 0.0;    // tr(L) (of graph 0 for a batch)
  double bound = 0.0;    // Gershgorin bound of the spectrum (largest over a batch)
  // A batch of G graphs is one block-diagonal Laplacian; graph g owns the
  // kept nodes [goff[g], goff[g+1]) in both the canonical and the execution
  // order.  A single graph is the batch G = 1.
  int n_graphs = 1;
  std::vector<int64_t> goff;        // [G+1] host copy
  std::vector<double> gtrace;       // [G] tr(L_g)
  std::vector<double> gtrace2;      // [G] tr(L_g^2) = sum_ij (L_g)_ij^2
  std::vector<double> gbound;       // [G] bound of the spectrum of L_g
  int64_t *goff_dev = nullptr;      // [G+1]
  double *gn_dev = nullptr;         // [G] node counts as double
  double *gtrace_dev = nullptr;     // [G]
  double *gtrace2_dev = nullptr;    // [G]
  double *gbound_dev = nullptr;     // [G]
  int32_t *x_graph = nullptr;       // [n] graph of each execution row
  int64_t *rowptr = nullptr;   // [n+1]
  int32_t *colidx = nullptr;   // [nnz]
  double *vals = nullptr;      // [nnz] off-diagonal values (FP64)
  float *vals32 = nullptr;     // [nnz] FP32 copy (weighted graphs only)
  double *diag = nullptr;      // [n]
  double *scale = nullptr;     // [n]
  float *diag32 = nullptr;     // [n]
  float *scale32 = nullptr;    // [n]
  int64_t *old_id = nullptr;   // [n]
  // Execution copy used by the Lanczos kernels: the same Laplacian with the
  // nodes renumbered by descending entry count (ties by id), so that the
  // most-gathered rows of the basis are contiguous and rows of similar cost
  // run side by side.  The trace functions are permutation invariant; probe
  // signs follow x_old_id, so they are those of the canonical order.
  int64_t *x_rowptr = nullptr;  // [n+1]
  int32_t *x_colidx = nullptr;  // [nnz]
  double *x_vals = nullptr;     // [nnz] (weighted only: unweighted graphs run the pattern form)
  float *x_vals32 = nullptr;    // [nnz] (weighted only)
  double *x_diag = nullptr, *x_scale = nullptr;    // [n]
  float *x_diag32 = nullptr, *x_scale32 = nullptr; // [n]
  int64_t *x_old_id = nullptr;  // [n] original id within its graph
  // SpMM schedule (execution order) for rows with more than heavy_degree
  // entries: each such row is split into chunks of kHeavyChunk entries.
  int64_t heavy_degree = 0;
  int64_t n_heavy = 0;               // heavy rows
  int64_t n_chunks = 0;              // chunks over all heavy rows
  int32_t *heavy_row = nullptr;      // [n_heavy] row id
  int64_t *heavy_first = nullptr;    // [n_heavy+1] first chunk of each heavy row
  int32_t *chunk_slot = nullptr;     // [n_chunks] heavy slot of each chunk
};

// Launch shapes of the Lanczos kernels; slaq_lanczos_batched's autotuner
// picks them per workload, every other call uses these defaults.
struct slaq_tuning {
  int spmm_threads = 256;  // threads of a light-row SpMM block
  int upd_threads = 256;   // threads of an update block
  int dots_threads = 0;    // narrow dots blocks grow row phases up to this many threads
                           // (0: 256 for the BF16 basis, whose threads hold half the rows
                           // in flight, else 128)
  int slice_bytes = 0;     // bytes of a basis row per probe slice (0: whole rows)
  int spmm_align = -1;     // 1: SpMM row teams never straddle two warps, 0: packed
                           // (-1: aligned when a row takes more than 16 threads)
  int spmm_tma = -1;       // light-row gathers: 1 TMA (tile::gather4), else loads
                           // (measured slower on every workload: not a tuner candidate,
                           // set by hand in a cache line)
};

struct slaq_krylov_s {
  int device = -1;
  int nv = 0, s = 0, ld = 0, precision = 0, reorth = 1;  // reorth 0: partial
  int graph_id = 0;
  int probe0 = 0;         // generator index of the first probe (probe ranges)
  bool ready = false;     // the last run completed: its buffers and results are valid
  uint64_t seed = 0;
  int64_t n = 0;          // n' of the last run
  int64_t n_cap = 0;      // rows the workspace holds
  int64_t chunk_cap = 0;  // heavy-row partial rows the workspace holds
  int kind = 0;
  double trace = 0.0, bound = 0.0, tol = 0.0;
  int G = 0;              // row blocks the partials buffer holds
  int dsub = 1;           // pieces per dots chunk in the last dots launch
  int max_chunks_per_graph = 1;
  void *U = nullptr;      // [s][n_cap][ld] basis (TB)
  void *Z = nullptr;      // [n_cap][ld] L u_k (TW)
  float *Y = nullptr;     // [n_cap][ld] s_i u_k[i] (FP32 form, normalized unweighted)
  bool ymode = false;     // the last run gathered Y instead of scale[j] u_k[j]
  const float *yscale = nullptr;  // the run's s_i (execution order), for Y
  void *P = nullptr;      // [chunk_cap][ld] partial sums of split rows (TW)
  double *part = nullptr; // [G][2][s][ld] per-block partial sums (dots, Gram column)
  double *dsum = nullptr; // [s][ld] reduced dot products u_j^T z
  double *coef = nullptr; // [s][ld] projection coefficients
  double *gram = nullptr; // [s][s][ld] Gram matrix u_i^T u_j of the stored basis
  double *proj = nullptr; // [s][s][ld] projected matrix u_i^T L u_j (reduced forms)
  double *rscratch = nullptr;  // Rayleigh-Ritz work space of the reduced forms
  int64_t rscratch_cap = 0;
  double *alpha = nullptr;  // [nv][s]
  double *beta = nullptr;   // [nv][s]
  int32_t *m = nullptr;     // [nv]
  double *theta = nullptr;  // [nv][s]
  double *tau2 = nullptr;   // [nv][s]
  int32_t *status = nullptr;  // [8]: [0] eigensolver flags; [1] SpMM wait timeouts; bytes 8..23: monitor words
  uint32_t *hcount = nullptr; // [n_heavy * slices] arrival counters of split rows (kept zero)
  int64_t hcount_cap = 0;
  // batches: G graphs; per-graph arrays are [G][...] (alpha [G][nv][s], ...)
  int n_graphs = 1;
  double *gn = nullptr;      // [G] node counts
  double *gtrace = nullptr;  // [G] tr(L_g)
  double *gtrace2 = nullptr; // [G] tr(L_g^2)
  double *gbound = nullptr;  // [G] spectral bounds (breakdown tolerance)
  int64_t gcap = 0;          // graphs the per-graph arrays hold
  // row chunks inside one graph: dots (d*) and update (u*) kernels
  std::vector<int64_t> hd_row0, hu_row0;
  std::vector<int32_t> hd_rows, hd_graph, hu_rows, hu_graph;
  std::vector<int32_t> hd_goff;  // [G+1] first dots chunk of each graph
  int64_t *d_row0 = nullptr, *u_row0 = nullptr;
  int32_t *d_rows = nullptr, *u_rows = nullptr, *u_graph = nullptr, *d_goff = nullptr;
  int64_t dcap = 0, ucap = 0;
  int n_dchunks = 0, n_uchunks = 0;
  // partial reorthogonalization (reorth = 0): step k of graph g projects
  // against all previous vectors if pro_full[g][k] (else only u_{k-1}, u_k);
  // pro_any[k] = any graph's flag, read on the host through pro_any_host;
  // omega[g][p][3][s] holds the estimates omega_{i,j} of the last three steps
  int32_t *pro_full = nullptr;      // [G][s+2]
  int32_t *pro_any = nullptr;       // [s+2]
  int32_t *pro_any_host = nullptr;  // [s+2], pinned
  double *omega = nullptr;          // [G][nv][3][s]
  int64_t pro_gcap = 0;             // graphs the partial-reorthogonalization arrays hold
  cudaEvent_t ev_flag = nullptr;    // after the copy of pro_any[k+1]
  // replay of the last run as a CUDA graph (slaq_lanczos_rerun)
  uint64_t *seed_dev = nullptr;     // [1] the probe seed the run reads
  slaq_graph last_g = nullptr;      // graph of the last run (not owned, unless == owned)
  uint64_t last_uid = 0;            // its uid
  cudaGraphExec_t gexec = nullptr;  // captured launches of that run, or null
  int64_t graph_nodes = 0;          // nodes of the captured graph (counted as launches)
  cudaStream_t cap = nullptr;       // private stream the capture runs on
  // light rows through TMA gathers: the tensor map over the gathered vectors
  // and the work items of the last run (tma false: the load path)
  bool tma = false;
  CUtensorMap tma_map;
  int64_t *tma_task = nullptr;  // [tma_ntasks + 1] first row of each work item
  int64_t tma_task_cap = 0;
  int64_t tma_ntasks = 0;
  // side stream on which the split-row SpMM runs beside the light rows
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  slaq_tuning tune;                // launch shapes of the last run
  slaq_graph owned = nullptr;      // union of a slaq_lanczos_batched call
};

namespace slaq {
// internal entry points (definitions in build.cu, lanczos.cu, quad.cu)
int build_laplacian(const int32_t *src, const int32_t *dst, int64_t n_edges, int64_t n_nodes,
                    const double *weights, int kind, int flags, cudaStream_t st,
                    slaq_graph *out, int n_graphs = 1, const int64_t *edge_off_host = nullptr,
                    const int64_t *node_off_host = nullptr);
// frees g's device arrays in stream order on st (every use of g must be
// ordered before that point on st)
void graph_free(slaq_graph g, cudaStream_t st);
void graph_register(slaq_graph g);             // gives g its uid and marks it alive
bool graph_alive(slaq_graph g, uint64_t uid);  // g not freed since it got uid
int run_lanczos(slaq_graph g, int nv, int s, uint64_t seed, int graph_id, int precision,
                int reorth, cudaStream_t st, slaq_krylov *inout,
                const slaq_tuning *tune = nullptr, int probe0 = 0);
int union_graphs(const slaq_graph *gs, int count, cudaStream_t st, slaq_graph *out);
int lanczos_batched(const slaq_graph *gs, int count, int nv, int s, uint64_t seed, int graph_id,
                    int precision, int reorth, const char *tune_cache, cudaStream_t st,
                    slaq_krylov *inout);
void krylov_free(slaq_krylov k);
// SLAQ_OK if k holds a completed run (every buffer a later call reads is in
// place), else SLAQ_EINVAL: a run that failed part-way (for example out of
// memory) leaves the handle destroyable and reusable but not readable
int krylov_ready(slaq_krylov k);
int set_spmm_gathers(int mode);
extern std::atomic<int> g_tma_giveup;  // test hook: TMA waits give up (slaq_debug_tma_giveup)
int debug_tma_giveup(int on);
int probes(slaq_graph g, int nv, uint64_t seed, int graph_id, double *out, cudaStream_t st);
int full_steps(slaq_krylov k, int32_t *out, cudaStream_t st);
int lanczos_rerun(slaq_krylov k, uint64_t seed, cudaStream_t st);
int run_ritz(slaq_krylov k, cudaStream_t st);
int trace_heat(slaq_krylov k, const double *t, int nt, double *out, double *se,
               double *per_probe, cudaStream_t st);
int trace_heat_cv(slaq_krylov k, const double *t, int nt, int degree, double *out, double *se,
                  double *per_probe, cudaStream_t st);
int trace_wave(slaq_krylov k, const double *t, int nt, double *re, double *im, double *se_re,
               double *se_im, cudaStream_t st, double *pp_re = nullptr, double *pp_im = nullptr);
int trace_vnge(slaq_krylov k, double *out, double *se, double *per_probe, cudaStream_t st);
int distance(const double *a, const double *b, int nt, int kind, double *out, cudaStream_t st);
int krylov_monitor(slaq_krylov k, double *ortho, double *min_beta, cudaStream_t st);
int profile_gather_peak(int row_bytes, double *tbps);
int comparators(slaq_krylov k, const double *t, int nt, double *taylor, double *q, double *bar,
                double *hat, cudaStream_t st);
int trace_heat_static(const double *alpha, const double *beta, const int32_t *m, int nv, int s,
                      int64_t n, const double *t, int nt, double *out, double *se,
                      int32_t *status_out, cudaStream_t st);
}  // namespace slaq
