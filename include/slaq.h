/*
 * slaq.h -- C ABI of libslaq: stochastic Lanczos quadrature (SLQ) estimates
 * of spectral trace functions tr f(L) of graph Laplacians on one GPU
 * (NVIDIA GB300, sm_103a).
 *
 * Method: Tsitsulin, Munkhoeva, Perozzi, "Just SLaQ When You Approximate:
 * Accurate Spectral Distances for Web-Scale Graphs", WWW'20 (arXiv
 * 2003.01282), Sec. 3 and Algorithm 1.
 *
 * Conventions (all entry points)
 *   - Every function returns an int status (enum slaq_status); 0 is success.
 *     slaq_last_error() gives a message for the calling thread's last failure.
 *     No C++ exception crosses this boundary.
 *   - Array arguments are DEVICE pointers of the current CUDA device unless
 *     their name ends in _host.  The caller owns every array it passes.
 *   - Handles (slaq_graph, slaq_krylov) own device memory allocated by the
 *     library and are released by their *_destroy function, which waits for
 *     the device to be idle first.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; unless a function says that it
 *     synchronizes, it returns before the GPU work completes.
 *   - There is no CPU fallback: without a compute-capability 10.3 GPU every
 *     compute entry point returns SLAQ_ENODEVICE.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef SLAQ_H
#define SLAQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum slaq_status {
    SLAQ_OK = 0,
    SLAQ_EINVAL = 1,        /* bad argument or malformed input */
    SLAQ_ENOMEM = 2,        /* device allocation failed */
    SLAQ_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SLAQ_ENODEVICE = 4,     /* no sm_103 device current (no CPU fallback) */
    SLAQ_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    SLAQ_EUNSUPPORTED = 6,  /* valid request beyond what this build handles */
    SLAQ_ENUMERIC = 7       /* the tridiagonal eigensolver did not converge */
};

/* Laplacian kinds (Sec. 2): L = D - A, or I - D^{-1/2} A D^{-1/2}. */
enum { SLAQ_NORMALIZED = 0, SLAQ_COMBINATORIAL = 1 };
/* Build flags. */
enum { SLAQ_DROP_ISOLATED = 1 };
/* Arithmetic forms of the Lanczos iteration (the alpha/beta reductions, the
 * tridiagonal eigensolve and the quadrature are FP64 in every form):
 *   SLAQ_FP64           basis, SpMM and reorthogonalization in FP64;
 *   SLAQ_FP32           basis, SpMM and reorthogonalization in FP32;
 *   SLAQ_FP32_BF16BASIS basis stored in BF16, SpMM and updates in FP32.
 * The FP32 and BF16-basis forms run both Laplacian kinds; their heat and
 * wave traces are served for |t| * bound <= 2000 and <= 20 respectively
 * (bound = 2 for the normalized Laplacian, 2 max d for L = D - A), see
 * slaq_trace_heat. */
enum { SLAQ_FP64 = 0, SLAQ_FP32 = 1, SLAQ_FP32_BF16BASIS = 2 };
/* reorth_passes value for partial reorthogonalization (slaq_lanczos). */
enum { SLAQ_REORTH_PARTIAL = 0 };
/* Distance kinds. */
enum { SLAQ_DIST_HEAT = 0, SLAQ_DIST_WAVE = 1, SLAQ_DIST_VNGE = 2 };

typedef struct slaq_graph_s *slaq_graph;    /* CSR Laplacian on the device */
typedef struct slaq_krylov_s *slaq_krylov;  /* Lanczos result + workspace  */

/* Library version as major*10000 + minor*100 + patch. */
int slaq_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to len) into buf_host; returns the status of that error. */
int slaq_last_error(char *buf_host, size_t len);

/* SLAQ_OK if the current CUDA device is compute capability 10.3 (GB300),
 * SLAQ_ENODEVICE otherwise.  Touches no memory. */
int slaq_device_check(void);

/* ---------------------------------------------------------------- graphs */

/* Build the Laplacian of an undirected graph (Sec. 2) as CSR on the device.
 *   src, dst   int32[n_edges] endpoint ids in [0, n_nodes); each pair is an
 *              undirected edge.  Self-loops are dropped; duplicate pairs (in
 *              either orientation) are merged, keeping the largest weight.
 *   weights    float64[n_edges] positive edge weights, or NULL (all 1).
 *   kind       SLAQ_NORMALIZED: diag 1 and off-diagonal -(a_ij s_i) s_j with
 *              s_i = 1/sqrt(d_i); an isolated node gets s_i = 0 and a zero
 *              row.  SLAQ_COMBINATORIAL: diag d_i, off-diagonal -a_ij.
 *   flags      SLAQ_DROP_ISOLATED removes degree-0 nodes and renumbers the
 *              rest in increasing order of their original ids.
 * Degrees of weighted graphs are summed in increasing column order.  The CSR
 * (rows, ascending column ids, values) is canonical, so it is bit-identical
 * to any correct builder's.  Ids outside [0, n_nodes) give SLAQ_EINVAL.
 * Synchronizes `stream` (array sizes are needed on the host).
 * *out receives a new handle. */
int slaq_build_laplacian(const int32_t *src, const int32_t *dst, int64_t n_edges,
                         int64_t n_nodes, const double *weights, int kind, int flags,
                         void *stream, slaq_graph *out);

/* Build the Laplacians of a batch of G graphs as ONE block-diagonal matrix,
 * so that every later call (slaq_lanczos, the traces) serves all graphs
 * with the same launches.  Graph g's edges are src/dst[edge_off_host[g] ..
 * edge_off_host[g+1]) with ids LOCAL to the graph, in [0, n_g), n_g =
 * node_off_host[g+1] - node_off_host[g] >= 1; weights (optional) follow the
 * edges.  kind and flags as for slaq_build_laplacian, applied per graph.
 * 1 <= G <= 65535; offsets are host arrays of G+1 entries starting at 0.
 * Graph g's results match a single-graph run of graph g with graph_id
 * (of slaq_lanczos) increased by g.  A graph that keeps no nodes (all
 * isolated and dropped) stays in the batch with an empty Krylov space:
 * m = 0, zero traces, zero entropy.  Synchronizes `stream`. */
int slaq_build_laplacian_batch(const int32_t *src, const int32_t *dst,
                               const int64_t *edge_off_host, const int64_t *node_off_host,
                               int n_graphs, const double *weights, int kind, int flags,
                               void *stream, slaq_graph *out);

/* Host copies of the batch size G, the kept-node offsets node_off_host[G+1]
 * (graph g owns kept nodes [node_off[g], node_off[g+1]) in exports) and the
 * traces trace_host[G] = tr(L_g).  Any pointer may be NULL. */
int slaq_graph_batch_info(slaq_graph g, int *n_graphs_host, int64_t *node_off_host,
                          double *trace_host);

/* Host copies of: kept node count n', stored off-diagonal count nnz, tr(L),
 * and the n_nodes given at build time (any pointer may be NULL). */
int slaq_graph_info(slaq_graph g, int64_t *n_host, int64_t *nnz_host,
                    double *trace_host, int64_t *n_input_host);

/* Device copies of the CSR: rowptr int64[n'+1], colidx int32[nnz],
 * vals float64[nnz] (off-diagonal values), diag float64[n'], scale float64[n']
 * (s_i; 1 for combinatorial), old_id int64[n'] (original id of each kept
 * node).  Any pointer may be NULL.  For bit-exact checks. */
int slaq_graph_export(slaq_graph g, int64_t *rowptr, int32_t *colidx, double *vals,
                      double *diag, double *scale, int64_t *old_id, void *stream);

void slaq_graph_destroy(slaq_graph g);

/* ---------------------------------------------------------------- Lanczos */

/* Run s-step Lanczos (Sec. 3.1, Algorithm 1 `lanczos`) of the graph's
 * Laplacian from nv Rademacher probes at once, then the Gauss rule of every
 * probe's tridiagonal T (Eq. quadratic: nodes = eigenvalues of T, weights =
 * squared first eigenvector components).  SLAQ_FP64 takes T from the
 * recurrence (alpha, beta below).  The FP32 and BF16-basis forms take the
 * Rayleigh-Ritz matrix of their stored, rounded basis, A = C^-1 M C^-T with
 * M = U^T L U, U^T U = C C^T, reduced to tridiagonal form by Householder
 * reflections that fix the first unit vector: in exact arithmetic A = T,
 * and it removes the first-order effect of the basis rounding on the rule.
 *   Probe p's entry at node i is the sign of SplitMix64 applied to
 *   seed + 0x9E3779B97F4A7C15 * (c + 1), c = graph_id<<48 | p<<32 | orig_id(i)
 *   (-1 where bit 63 is set); the starting vector is that sign vector / sqrt(n').
 *   Every step orthogonalizes the new vector against all previous Lanczos
 *   vectors of its probe by classical Gram-Schmidt (reorth_passes = 1) or
 *   twice (2).  reorth_passes = SLAQ_REORTH_PARTIAL (0) is partial
 *   reorthogonalization (not in the paper; Simon, Math. Comp. 42, 1984):
 *   a step projects the new vector on the previous two only, and every probe
 *   estimates the loss of orthogonality omega_{k,j} ~ q_k^T q_j of its basis
 *   by the recurrence that the symmetry of L imposes on it (measured from
 *   the Gram column on steps that project on all vectors).  When a probe's
 *   max_j |omega_{k,j}| passes sqrt(eps) (eps = 2^-53 FP64, 2^-24 FP32), the
 *   next two steps of its graph project against all previous vectors (their
 *   Gram system with the entries no step measured set to zero; a scaled
 *   pivot below 1/2 there means the basis is too far from orthogonal, as
 *   just after a near-breakdown, and the probe stops as at a breakdown).  The
 *   Gauss rule then comes from the recurrence's T in both forms.  It needs a
 *   host read of one flag per step (the call does not return before the
 *   last step is enqueued); SLAQ_FP32_BF16BASIS with it: SLAQ_EUNSUPPORTED
 *   (BF16 storage rounds at 2^-9, above the FP32 semi-orthogonality level).
 *   A probe whose beta_k falls to tol * bound (tol 1e-10 FP64,
 *   1e-4 FP32 and BF16 basis; bound 2 or 2 max d) stops with m = k+1.
 *   1 <= nv <= 512, 1 <= s <= 64, precision one of SLAQ_FP64/FP32/
 *   FP32_BF16BASIS, graph_id + (graphs in g) - 1 < 65536; the projection
 *   coefficients s * ld * (8 for FP64, else 4) bytes must fit 200 KiB (ld =
 *   nv rounded up to a 32-byte row), else SLAQ_EUNSUPPORTED (FP64 with
 *   nv = 512 allows s <= 50).
 * inout: if *inout is NULL a new handle is created; otherwise *inout must
 * come from an earlier call with the same nv, s and precision, and its
 * device workspace is reused (grown if the graph is larger).
 * The graph handle must stay alive until the work on `stream` completes. */
int slaq_lanczos(slaq_graph g, int nv, int s, uint64_t seed, int graph_id,
                 int precision, int reorth_passes, void *stream, slaq_krylov *inout);

/* slaq_lanczos over a range of the probe generator's probes: column p of the
 * run is generator probe probe0 + p (the probe field of the counter above),
 * so that runs over disjoint ranges of one seed -- one per GPU, or chunks
 * that fit memory -- together hold the probes of one run over their union
 * (Sec. 3.1, Eq. trace: the probes are independent).  Every per-probe output
 * of column p (alpha, beta, m, Gauss rule, per-probe traces) equals that of
 * column probe0 + p of a run from probe 0, up to rounding order (the dot
 * products' summation order depends on the block width nv).
 * 0 <= probe0 and probe0 + nv <= 65536, else SLAQ_EINVAL; everything else as
 * for slaq_lanczos, which is this call with probe0 = 0.  A later
 * slaq_lanczos_rerun keeps the range.  slaq_pool_probes_host combines the
 * ranges' per-probe values into the estimate and standard error over all
 * their probes. */
int slaq_lanczos_probes(slaq_graph g, int nv, int probe0, int s, uint64_t seed, int graph_id,
                        int precision, int reorth_passes, void *stream, slaq_krylov *inout);

/* slaq_lanczos again on the same graph, sizes, form and reorthogonalization
 * as the handle's last slaq_lanczos / slaq_lanczos_batched call, with probes
 * from a new seed: the results equal that call's with `seed` bit for bit.
 * The first rerun captures the run's launches (probe generation, the s
 * Lanczos steps, the Gauss rules) into a CUDA graph; every rerun then copies
 * the seed to the device and launches that graph, so a run costs one launch
 * on the host instead of about 5 s + 10.  The graph handle of the last call
 * must still be alive (a batched call's concatenation of two or more
 * handles is owned by k).  Any slaq_lanczos call on k discards the captured
 * graph.  Not available with
 * partial reorthogonalization (its steps are decided on the host):
 * SLAQ_EUNSUPPORTED.  Synchronizes `stream`; SLAQ_ENUMERIC as for
 * slaq_lanczos. */
int slaq_lanczos_rerun(slaq_krylov k, uint64_t seed, void *stream);

/* slaq_lanczos for a batch of separately built graphs gs[0..count): the
 * graphs (each a single graph or itself a batch) are concatenated on the
 * device into one block-diagonal Laplacian owned by the Krylov handle, and
 * all of them run through the same launches (one handle, count = 1, runs as
 * it is, without a copy).  Graph g of the concatenation
 * (in order, sub-graphs of batch handles expanded) gets probe graph field
 * graph_id + g, so its results equal slaq_lanczos(gs[g], ..., graph_id + g)
 * up to rounding order.  All graphs must share the Laplacian kind and be all
 * weighted or all unweighted; at most 65535 graphs in total.
 * tune_cache: NULL runs the default launch shapes.  Otherwise it names a
 * text file: if it holds a line for this workload class (precision, nv, s,
 * reorth_passes, log2 of n', of nnz/n' and of the graph count, SM count) the
 * launch shapes on it are used (line format "<class> | spmm_threads
 * update_threads dots_threads slice_bytes spmm_align spmm_tma", the last
 * field optional and 1 for the TMA gathers of slaq_set_spmm_gathers); if
 * not, the call first times candidate
 * shapes on this batch (coordinate descent, about a dozen full runs), keeps
 * the fastest and adds its line (the file is rewritten through a temporary
 * beside it).  An unreadable or unwritable file gives SLAQ_EINVAL.
 * The inputs gs may be destroyed once the call returns; only a rerun
 * (slaq_lanczos_rerun) of a call with one input needs that input alive, as
 * after slaq_lanczos.  Synchronizes `stream`; other arguments and errors as
 * for slaq_lanczos. */
int slaq_lanczos_batched(const slaq_graph *gs, int count, int nv, int s, uint64_t seed,
                         int graph_id, int precision, int reorth_passes,
                         const char *tune_cache, void *stream, slaq_krylov *inout);

/* The probe block the Lanczos run starts from, as float64[n'][nv] (+-1),
 * generated on the device exactly as slaq_lanczos does (Eq. trace needs
 * zero-mean, unit-variance probes; the text allows Rademacher signs).
 * For bit-exact checks of the generator. */
int slaq_probes(slaq_graph g, int nv, uint64_t seed, int graph_id, double *out, void *stream);

/* Device copies of alpha float64[nv*s] (row p holds alpha_0..alpha_{m_p-1}),
 * beta float64[nv*s] (beta_0..beta_{m_p-2}) and m int32[nv].  NULL skips.
 * For the FP32 and BF16-basis forms with full reorthogonalization alpha and
 * beta are the diagonal and off-diagonal of the tridiagonal form of the
 * Rayleigh-Ritz matrix (the T whose Gauss rule the traces use); with partial
 * reorthogonalization they are the recurrence's, as in SLAQ_FP64. */
int slaq_krylov_export(slaq_krylov k, double *alpha, double *beta, int32_t *m, void *stream);

/* Which Lanczos steps projected against all previous vectors: full_steps
 * int32[G][s] on the device, 1 where step k of graph g did (every step with
 * reorth_passes 1 or 2, and steps 0 and 1, whose previous vectors are the
 * local pair), else 0 (partial reorthogonalization only).  Steps after a
 * graph's last probe stopped read 0. */
int slaq_krylov_full_steps(slaq_krylov k, int32_t *full_steps, void *stream);

/* Device copies of the Gauss nodes theta float64[nv*s] (ascending within a
 * probe's first m_p entries) and weights tau2 float64[nv*s]. */
int slaq_ritz_export(slaq_krylov k, double *theta, double *tau2, void *stream);

/* Number of graphs G of the run (1 unless the graph was a batch).  For a
 * batch every per-probe output below gains a leading graph axis:
 * alpha, beta, theta, tau2 [G][nv][s], m [G][nv], trace outputs [G][nt],
 * per-probe traces [G][nv][nt], VNGE outputs [G]. */
int slaq_krylov_batch_info(slaq_krylov k, int *n_graphs_host);

/* Host copies of nv, s, precision, n'. */
int slaq_krylov_info(slaq_krylov k, int *nv_host, int *s_host, int *precision_host,
                     int64_t *n_host);

/* Heat trace h_t = tr exp(-t L) (Eq. heat-trace) at nt times t (float64[nt],
 * device) by Eq. slq: out[i] = (n'/nv) sum_p sum_k tau2 exp(-t_i theta);
 * stderr_[i] = sample std over probes / sqrt(nv) (NaN when nv = 1);
 * per_probe float64[nv*nt] (row p = n' sum_k tau2 exp(-t theta)) or NULL.
 * The reduced forms serve |t| * bound <= 20 (BF16 basis) and <= 2000 (FP32)
 * only, with bound 2 for the normalized Laplacian (t <= 10 and t <= 1000)
 * and 2 max d for L = D - A: the basis rounding moves the Ritz values that
 * are not yet converged by about the rounding times bound, which
 * exp(-t theta) turns into errors growing with t * bound (measured within
 * 2.3e-5 (BF16) and 4.4e-7 (FP32, up to t * bound = 1000) of the FP64 form
 * on every graph tried, both Laplacians; the 1e-4 bar first failed at
 * t * bound = 58 (BF16) and 22,000 (FP32)).  A larger t gives
 * SLAQ_EUNSUPPORTED; the reduced forms copy t to the host and synchronize
 * `stream` to check it.  The same holds for slaq_trace_heat_cv,
 * slaq_trace_wave and slaq_trace_wave_per_probe. */
int slaq_trace_heat(slaq_krylov k, const double *t, int nt, double *out, double *stderr_,
                    double *per_probe, void *stream);

/* The heat trace with a polynomial control variate (Sec. 3.1, the "2-term
 * polynomial" variance reduction, whose polynomial the paper does not give).
 * Reading: p_t is the Chebyshev interpolant of degree `degree` (1: c0 + c1 x,
 * 2: + c2 x^2) of exp(-t x) on [0, bound] (bound 2 normalized, 2 max d
 * combinatorial), at the nodes (bound/2)(1 + cos(pi (j + 1/2)/(degree + 1))).
 *   out[i] = (n'/nv) sum_p sum_k tau2 (exp(-t_i theta) - p_t(theta))
 *            + c0 n' + c1 tr L + c2 tr L^2,
 * with tr L^2 = sum_ij L_ij^2 computed by the builder.  Each probe's Gauss
 * rule is exact for p_t, so the estimate stays unbiased; stderr_ is the
 * sample std of the corrected per-probe values / sqrt(nv) (smaller where
 * p_t follows exp(-t x) on the spectrum: small t).  per_probe (or NULL) as
 * for slaq_trace_heat, corrected.  degree other than 1 or 2: SLAQ_EINVAL. */
int slaq_trace_heat_cv(slaq_krylov k, const double *t, int nt, int degree, double *out,
                       double *stderr_, double *per_probe, void *stream);

/* Wave trace tr exp(-i t L): re[i] = sum cos(t lambda), im[i] = -sum sin(t lambda),
 * estimated as above; stderr arrays may be NULL.  The reduced forms'
 * limits on t are those of slaq_trace_heat (measured for the wave with the
 * BF16 basis: below 1e-5 of max |Re| up to its limit, up to 0.28 at t = 100
 * on R-MAT). */
int slaq_trace_wave(slaq_krylov k, const double *t, int nt, double *re, double *im,
                    double *stderr_re, double *stderr_im, void *stream);

/* Per-probe values of the wave trace (as slaq_trace_wave, with its limit on
 * t for the reduced forms, before the mean
 * over probes): re_pp[p][i] = n' sum_k tau2 cos(t_i theta) and im_pp[p][i] =
 * -n' sum_k tau2 sin(t_i theta), float64[nv*nt] each ([G][nv][nt] for a
 * batch).  With the per_probe outputs of the heat trace and the VNGE these
 * are the values slaq_pool_probes_host pools across probe ranges. */
int slaq_trace_wave_per_probe(slaq_krylov k, const double *t, int nt, double *re_pp,
                              double *im_pp, void *stream);

/* Von Neumann graph entropy (Definition 1, Sec. 2.1) of P = L / tr(L) for
 * the Laplacian the graph was built with: -sum mu ln mu over mu = theta/tr(L)
 * > 0 (natural log, 0 ln 0 = 0).  out, stderr_: float64[1]; per_probe
 * float64[nv] or NULL. */
int slaq_trace_vnge(slaq_krylov k, double *out, double *stderr_, double *per_probe,
                    void *stream);

/* Orthogonality monitor of the last run (not in the paper; the quantities
 * that decide whether the Gauss rule of Eq. quadratic can be trusted):
 *   *ortho_host    = max over probes and stored vectors j < k of
 *                    |u_j^T u_k| / (||u_j|| ||u_k||), i.e. max |Q^T Q - I|
 *                    off the diagonal, from the Gram entries the run
 *                    measured (the last vector is left out where the run
 *                    forms only its norm: the FP64 form, and partial
 *                    reorthogonalization, whose unmeasured entries count 0);
 *   *min_beta_host = the smallest beta_k over probes and k < m_p - 1
 *                    (+inf if no probe has two steps).
 * Either pointer may be NULL.  Synchronizes `stream`. */
int slaq_krylov_monitor(slaq_krylov k, double *ortho_host, double *min_beta_host, void *stream);

void slaq_krylov_destroy(slaq_krylov k);

/* The paper's O(m) comparators (Sec. 2.3), for context beside the SLQ
 * estimates, per graph of the run (batches: [G] and [G][nt]); any output
 * may be NULL:
 *   taylor_heat[i] = n' - t_i tr L + (t_i^2 / 2) tr L^2   (Eq. hks-taylor),
 *   vnge_q         = 1 - tr(L^2) / tr(L)^2, the quadratic approximation of
 *                    the VNGE (the two-term expansion x (1 - x) of -x ln x
 *                    over the eigenvalues of P = L / tr L; the printed forms
 *                    of Eq. vnge-taylor and of FINGER's Q are garbled),
 *   finger_bar     = -vnge_q ln(bound / tr L), bound = 2 (normalized) or
 *                    2 max d (combinatorial) (FINGER-Hbar),
 *   finger_hat     = -vnge_q ln(lambda_max / tr L), lambda_max = the largest
 *                    Ritz value of the graph's probes (FINGER-Hhat),
 * with tr L and tr L^2 = sum_ij L_ij^2 as the builder computed them. */
int slaq_comparators(slaq_krylov k, const double *t, int nt, double *taylor_heat, double *vnge_q,
                     double *finger_bar, double *finger_hat, void *stream);

/* --------------------------------------------------------------- distances */

/* Spectral distance between two descriptors (Sec. 4.2):
 *   SLAQ_DIST_HEAT: a, b float64[nt]; out = ||a - b||_2;
 *   SLAQ_DIST_WAVE: a, b float64[2*nt] (re then im); out = ||a - b||_2;
 *   SLAQ_DIST_VNGE: a, b float64[1]; out = |a - b|.
 * out: float64[1] on the device. */
int slaq_distance(const double *a, const double *b, int nt, int kind, double *out,
                  void *stream);

/* ------------------------------------------------------------- host calls */

/* The whole path in one call, from host memory to host memory: copies the
 * edge list and t grid to the device, builds the Laplacian, runs Lanczos and
 * the quadrature, and copies heat[nt], wave_re[nt], wave_im[nt] and vnge[1]
 * back (any output may be NULL).  Synchronizes `stream` before returning.
 * The Krylov workspace of a successful call (s * n' * nv basis values, plus
 * O(n' nv) work vectors) stays allocated for the next call on the same
 * device with the same nv, s and precision, which then skips its allocation;
 * slaq_release_cached frees it. */
/* Frees the workspaces slaq_descriptors_host keeps between calls, on every
 * device.  Must not run concurrently with a slaq_descriptors_host call. */
int slaq_release_cached(void);

int slaq_descriptors_host(const int32_t *src_host, const int32_t *dst_host, int64_t n_edges,
                          int64_t n_nodes, int kind, int flags, int nv, int s, uint64_t seed,
                          int precision, const double *t_host, int nt, double *heat_host,
                          double *wave_re_host, double *wave_im_host, double *vnge_host,
                          void *stream);

/* Hutchinson estimate and standard error over probes (Eq. trace) from
 * per-probe values, on the host (needs no GPU): values_host[nprobe][len],
 * row p holding probe p's values (for example the per-probe heat traces of
 * several slaq_lanczos_probes ranges, concatenated in probe order);
 * mean_host[j] = mean of column j; stderr_host[j] (or NULL) = sample standard
 * deviation / sqrt(nprobe), NaN when nprobe = 1.  The sums run in the fixed
 * order of the device quadrature kernels (Welford over the probe groups
 * p mod 4, combined pairwise in group order), so ranges pooled here reproduce
 * the estimate of one run over all their probes up to the rounding of the
 * per-probe values.  nprobe < 1, len < 1 or NULL values/mean: SLAQ_EINVAL. */
int slaq_pool_probes_host(const double *values_host, int nprobe, int len, double *mean_host,
                          double *stderr_host);

/* ------------------------------------------------ allocation-free variant */

/* Heat trace from Lanczos coefficients without any device allocation.
 * The paper has no counterpart.  Some callers cannot allocate device memory
 * when they call into a library: an application whose own memory manager
 * owns all device memory and hands libraries only buffers it created, or a
 * latency-critical loop where a cudaMalloc (which may synchronize the device
 * or fail once the pool is carved up) is not allowed.  For them this entry
 * point computes what slaq_trace_heat computes after slaq_lanczos, from
 * coefficients the caller holds, and keeps its scratch (the Gauss nodes and
 * weights) in a fixed array inside the library instead of a handle:
 *   out[i] = (n / nv) sum_p sum_k tau2_{p,k} exp(-t_i theta_{p,k}), where
 *   theta_{p,k} and tau2_{p,k} are the eigenvalues and squared first
 *   eigenvector components of probe p's m[p] x m[p] tridiagonal matrix;
 *   stderr_[i] = sample std over the probes / sqrt(nv) (NaN when nv = 1).
 * Arguments (device arrays unless noted):
 *   alpha, beta  float64[nv*s] as written by slaq_krylov_export (row p holds
 *                alpha_0..alpha_{m_p-1} and beta_0..beta_{m_p-2});
 *   m            int32[nv]: each value is clamped to [0, s] before use;
 *   n            the node count n' (host value); t float64[nt];
 *   out, stderr_ float64[nt] (stderr_ may be NULL);
 *   status       int32[1] or NULL: receives 0, or the OR of 1 (an eigensolve
 *                did not converge) and 2 (some m[p] was outside [0, s] and
 *                was clamped).
 * Limits: nv <= 512, s <= 64 (the scratch holds 512 x 64 nodes and
 * weights and 512 rule sizes, about 514 KiB per device, kept until the
 * process exits); larger sizes return SLAQ_EINVAL before any work is
 * enqueued.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.
 * All calls on a device share the one scratch array, which keeps the last
 * call's contents (the call clears its status word itself): calls whose GPU
 * work overlaps (other streams, other threads) race and must be ordered by
 * the caller. */
int slaq_trace_heat_tridiag_static(const double *alpha, const double *beta, const int32_t *m,
                                   int nv, int s, int64_t n, const double *t, int nt, double *out,
                                   double *stderr_, int32_t *status, void *stream);

/* ------------------------------------------------------------ test hooks */

/* Failure injection for the error paths (off by default; for tests): the
 * nth allocation the library makes after this call -- device memory from
 * cudaMalloc or the stream-ordered pool, or pinned host memory -- fails as
 * if the device were out of memory, and the call that makes it returns
 * SLAQ_ENOMEM after releasing what it had allocated.  The hook fires once;
 * nth <= 0 disarms it.  A handle whose run failed this way stays valid to
 * destroy or to run again; reading its results returns SLAQ_EINVAL.
 * Returns SLAQ_OK.  Needs no GPU. */
int slaq_debug_fail_alloc(int64_t nth);

/* Number of allocations the library currently holds (graph and Krylov
 * handles, the temporaries of calls in progress), for leak checks around
 * failing calls.  Needs no GPU. */
int64_t slaq_debug_live_allocs(void);

/* ------------------------------------------------------------- profiling */

/* Kernel classes timed by the profiler. */
enum {
    SLAQ_PROF_BUILD = 0,   /* every kernel of slaq_build_laplacian            */
    SLAQ_PROF_PROBES = 1,  /* probe generation                                */
    SLAQ_PROF_SPMM = 2,    /* L u_k for the probe block (split rows included)  */
    SLAQ_PROF_DOTS = 3,    /* u_j^T z (or u_j^T u_{k+1}) block partial sums    */
    SLAQ_PROF_UPDATE = 4,  /* u_{k+1} = z - sum_j c_j u_j and its norm partials*/
    SLAQ_PROF_REDUCE = 5,  /* partial-sum reductions, alpha, beta, breakdown   */
    SLAQ_PROF_RITZ = 6,    /* tridiagonal Gauss rules                          */
    SLAQ_PROF_TRACE = 7,   /* quadrature: heat, wave, VNGE                     */
    SLAQ_PROF_DIST = 8,    /* distances                                        */
    SLAQ_PROF_NCAT = 9
};

/* on != 0: from now on, bracket every kernel class above with CUDA events
 * recorded on the stream it is launched on; clears all totals (times and
 * launch counts).  on == 0: stop recording (totals are kept). */
int slaq_profile_enable(int on);

/* Host copies of the accumulated device time (ms) and number of kernel
 * launches of one class since the last slaq_profile_enable(1).  Launches
 * are counted whether or not timing is on.  Waits for the recorded events. */
int slaq_profile_read(int category, double *ms_host, int64_t *launches_host);

/* The gather ceiling the SpMM works against (profiling; not part of the
 * method): every stored entry of L gathers one basis row of nv values, far
 * more bytes than reach HBM, and the L2 serves them.  This times random
 * gathers of row_bytes-wide rows (a multiple of 16 in [16, 512], one 16-byte
 * vector per lane, as the SpMM reads them) from an L2-resident 64 MiB table
 * on the current device and writes the rate in TB/s of gathered bytes to
 * *tbps_host.  Allocates and frees its table; synchronizes the device's
 * legacy default stream. */
int slaq_profile_gather_peak(int row_bytes, double *tbps_host);

/* How the SpMM gathers the basis rows of light rows (rows of at most 2048
 * entries), for every later Lanczos run in this process: mode 1 through the
 * tensor memory accelerator (cp.async.bulk.tensor tile::gather4 into a
 * shared-memory ring per warp, Blackwell and later), 0 through 16-byte
 * loads, -1 (the initial state) as the launch-shape tuning of the run says
 * (slaq_lanczos_batched's tune cache; loads otherwise).  A performance
 * choice with the same arithmetic: the two paths differ only in the order
 * the partial sums of a row are added.  Measured on GB300 the TMA path is
 * slower than the loads, from 1.6x (R-MAT 2^24, BF16 basis) to 8x (SBM
 * batches of short rows): its per-row work is serialized per warp.  So the
 * loads are the default and the tuner does not try it.  The TMA path serves the FP32 and
 * BF16-basis forms with rows of at most 256 elements and 32 lanes of 16
 * bytes, unsliced; other runs use loads whatever the mode.  Its waits on
 * the copies are bounded: a wait that gives up fails the run with
 * SLAQ_ETIMEOUT.  A run reads the mode once, when it starts (a replay by
 * slaq_lanczos_rerun keeps its run's path).  SLAQ_EINVAL for a mode outside
 * [-1, 1]. */
int slaq_set_spmm_gathers(int mode);

/* Test hook, off by default: on != 0 makes every warp of the TMA light-row
 * SpMM treat its first wait on a stage as one that ran out of polls (the
 * copies it issued still land: the kernel drains them before it returns), so
 * that a run on the TMA path fails with SLAQ_ETIMEOUT and leaves its handle
 * not ready.  Exercises the bounded-wait error path without faulting the
 * device; on == 0 restores normal waits.  Process-wide. */
int slaq_debug_tma_giveup(int on);

/* *tma_host = 1 if the light rows of k's last run were gathered through
 * TMA (slaq_set_spmm_gathers), 0 if through loads.  Host-side; no GPU work. */
int slaq_krylov_gathers(slaq_krylov k, int *tma_host);

/* Gauss rule of one symmetric tridiagonal matrix on the host, with the same
 * implicit-shift QR code the GPU kernel runs (Golub & Van Loan, Sec. 8.3):
 * alpha_host[m] diagonal, beta_host[m-1] off-diagonal; theta_host[m]
 * ascending eigenvalues, tau2_host[m] squared first eigenvector components.
 * Needs no GPU; for testing the solver on its own.  SLAQ_ENUMERIC if it did
 * not converge. */
int slaq_tridiag_gauss_host(const double *alpha_host, const double *beta_host, int m,
                            double *theta_host, double *tau2_host);

#ifdef __cplusplus
}
#endif

#endif /* SLAQ_H */
