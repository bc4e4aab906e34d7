#!/usr/bin/env python3
"""Benchmark of the SLQ hot path on the R-MAT 2^20 workload.

Workload: R-MAT scale 20 (a, b, c, d = .57, .19, .19, .05), 16 Mi unique
undirected edges, seed 1, isolated nodes dropped, normalized Laplacian;
nv = 100 Rademacher probes, s = 20 Lanczos steps with full reorthogonalization;
heat and wave traces on 256 log-spaced t in [1e-2, 1e2] and the VNGE.

One step = the whole path on device-resident edges: Laplacian build, Lanczos
(SpMM, Gram-Schmidt dots and update, reductions), Gauss rules, quadrature and
the distance of the heat trace to a stored signature.  The metric is
probe-edges per second: nnz * nv * s per step.  The headline form computes
the Lanczos iteration in FP32 (alpha/beta reductions, eigensolve and
quadrature in FP64).  Timed beside it, each with its error against the FP64
form: the FP64 form, the BF16-basis form, and both FP32 and FP64 with
partial reorthogonalization; the heat-trace control variate's standard
errors; the 5000-graph SBM batch (graphs/s); the host-memory entry point.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs the same graph with its own probe
seed (weak scaling over probes); the per-rank estimates are averaged with
one all-reduce of the descriptor vector.  `--impl reference` times the CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

if "--impl" in sys.argv and "reference" in sys.argv or "--cpu-baseline-worker" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "probe-edges/s in Lanczos SpMM (% HBM peak); graphs/s batched; rel err vs FP64"
UNIT = "probe-edges/s"
SCALE, EDGES, GRAPH_SEED = 20, 16 << 20, 1
NV, S, NT, PROBE_SEED = 100, 20, 256, 1
WORKLOAD = ("R-MAT scale 20 (2^20 nodes, 16Mi unique undirected edges, a,b,c,d=.57,.19,.19,.05, "
            "seed 1), isolated nodes dropped, normalized Laplacian; nv=100 Rademacher probes, "
            "s=20 Lanczos steps, full CGS reorthogonalization; heat + wave traces on 256 "
            "log-spaced t in [1e-2,1e2] + VNGE")
CPU_PROBES = 4        # probes of the CPU-oracle sample
REF_PROBES = 1        # probes per step of the reference (oracle) arm
# batched workload: 5000 SBM graphs, nv = 20, s = 15, heat traces at 256 t
SBM_GRAPHS, SBM_NV, SBM_S, SBM_SEED = 5000, 20, 15, 3
SBM_WORKLOAD = ("5000 stochastic-block-model graphs (sizes lognormal, median 300, clipped to "
                "[10, 5000]; 2-6 equal blocks; p_in ~ U[.05,.3], p_out = p_in/U[5,20]; seed 3), "
                "isolated nodes dropped, normalized Laplacians as one block-diagonal batch; "
                "nv=20, s=15; heat traces on 256 log-spaced t")


def make_graph():
    return synth.rmat(SCALE, EDGES, seed=GRAPH_SEED)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------ CPU oracle
def oracle_sample(src, dst, n, probes: int, s: int):
    """Oracle on a bounded sample: CSR build + `probes` probes of Lanczos +
    heat/wave/VNGE quadrature.  Returns (seconds, nnz)."""
    from oracle import descriptors as od
    from oracle.laplacian import build_laplacian
    t = synth.t_grid(NT)
    t0 = time.perf_counter()
    lap = build_laplacian(src, dst, n, drop_isolated=True)
    runs = od.slq_runs(lap, s, probes, PROBE_SEED, probes=range(probes))
    od.heat_trace(runs, lap.n, t)
    od.wave_trace(runs, lap.n, t)
    od.vnge(runs, lap.n, lap.trace)
    return time.perf_counter() - t0, lap.nnz


def cpu_baseline_worker(path: str):
    d = np.load(path)
    sec, nnz = oracle_sample(d["src"], d["dst"], int(d["n"]), CPU_PROBES, S)
    print(json.dumps({"seconds": sec, "nnz": nnz}))


def cpu_baseline(src, dst, n):
    """Run the oracle sample in a child process limited to one thread."""
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "g.npz")
        np.savez(path, src=src, dst=dst, n=n)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", path],
                           capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    pe = out["nnz"] * CPU_PROBES * S
    return {"value": pe / out["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"CSR build of the full graph + {CPU_PROBES} of {NV} probes x {S} Lanczos "
                      f"steps + heat/wave/VNGE quadrature ({out['seconds']:.1f} s, one thread)"}


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample
    (REF_PROBES probes of the workload), timed on one host thread."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import descriptors as od
    from oracle.laplacian import build_laplacian
    src, dst, n = make_graph()
    lap = build_laplacian(src, dst, n, drop_isolated=True)
    t = synth.t_grid(NT)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        runs = od.slq_runs(lap, S, REF_PROBES, PROBE_SEED + i, probes=range(REF_PROBES))
        od.heat_trace(runs, lap.n, t)
        od.wave_trace(runs, lap.n, t)
        od.vnge(runs, lap.n, lap.trace)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = float(np.mean(times))
    value = lap.nnz * REF_PROBES * S / sec
    sample = f"{REF_PROBES} of {NV} probes x {S} Lanczos steps + quadrature per step, one thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nnz": lap.nnz, "n_prime": lap.n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows, self.proc, self.thread = [], None, None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for ts, r in self.rows if t0 <= ts <= t1 and len(r) >= 9] or \
               [r for _, r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ our arm
# DRAM traffic of one SpMM (light-row + split-row kernels, step 16) of the FP32
# R-MAT 2^20 workload, from the ncu capture summarised in
# profiles/kernels_rmat20_fp32_k16.md; it describes the kernels only while
# csrc/lanczos.cu is byte-identical to the source that was captured.
SPMM_TRAFFIC = {
    "bytes_per_spmm": 1955883000 + 350987008 + 561419000 + 8566272,
    "source_sha256": "539318e1736260c06e3e5c38220af5c6f958ea6afc09843f63491855f31327bf",
}


def spmm_traffic(prec):
    import hashlib
    src = os.path.join(ROOT, "paper_2003_01282_gb300", "csrc", "lanczos.cu")
    with open(src, "rb") as f:
        same = hashlib.sha256(f.read()).hexdigest() == SPMM_TRAFFIC["source_sha256"]
    return SPMM_TRAFFIC["bytes_per_spmm"] if (same and prec == "fp32") else None


def algorithmic_bytes(n, nnz, prec, nv=NV, s=S):
    """Algorithmic bytes of one run, per kernel class (useful nv columns)."""
    bq = {"fp64": 8, "fp32": 4, "bf16": 2}[prec]
    bw = 8 if prec == "fp64" else 4
    vec = n * nv
    # the FP32 form gathers y = s * u (written by the update) and reads u_k
    # for the diagonal term: one more vector read per SpMM and one more
    # vector written per update
    yb = bw if prec == "fp32" else 0
    spmm = s * (8 * (n + 1) + 4 * nnz + vec * (bq + bw + yb) + n * 2 * bw)
    # the FP64 form reads only u_{s-1} on the last step; the reduced forms
    # read the whole basis there (the last column of the projected matrix)
    dots = sum(((k + 1 if (k < s - 1 or prec != "fp64") else 1) * bq + bw) * vec for k in range(s))
    update = sum(((k + 1) * bq + bw + bq + yb) * vec for k in range(s - 1))
    return {"spmm": spmm, "dots": dots, "update": update}


def run_batched(args, dev, world=1, rank=0, tdist=None):
    """The SBM batch through one set of launches per step; graphs/s.  Also
    times the same path graph by graph on a subset (per-graph launches).
    Under torchrun every rank runs its own batch (seed + rank): weak scaling
    over graphs, no exchange, the slowest rank's time."""
    import torch
    from paper_2003_01282_gb300 import slaq
    graphs = synth.sbm_batch(SBM_GRAPHS, seed=SBM_SEED + rank)
    srcs = np.concatenate([g[0] for g in graphs])
    dsts = np.concatenate([g[1] for g in graphs])
    edge_off = np.zeros(len(graphs) + 1, np.int64)
    node_off = np.zeros(len(graphs) + 1, np.int64)
    edge_off[1:] = np.cumsum([g[0].size for g in graphs])
    node_off[1:] = np.cumsum([g[2] for g in graphs])
    import ctypes as C
    src = torch.as_tensor(srcs, device=dev)
    dst = torch.as_tensor(dsts, device=dev)
    t = torch.as_tensor(synth.t_grid(NT), device=dev)
    P = slaq.PRECISIONS[args.precision]
    state = {"K": None}

    def step():
        out = C.c_void_p()
        slaq._check(slaq.lib().slaq_build_laplacian_batch(
            C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()), edge_off.ctypes.data_as(C.c_void_p),
            node_off.ctypes.data_as(C.c_void_p), len(graphs), None, slaq.NORMALIZED, slaq.DROP_ISOLATED,
            slaq._stream(None), C.byref(out)))
        g = slaq.Graph(out)
        state["K"] = slaq.lanczos(g, SBM_NV, SBM_S, rank_seed(rank), precision=P,
                                  reuse=state["K"])
        heat, _ = slaq.trace_heat(state["K"], t)
        nnz = g.info["nnz"]
        g.close()
        return heat, nnz

    for _ in range(2):
        _, nnz = step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    slaq.profile_enable(True)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    prof = slaq.profile_read()
    slaq.profile_enable(False)
    ms = e0.elapsed_time(e1) / reps
    if tdist is not None:
        ms = max_over_ranks(ms, dev, tdist)
    # the same path graph by graph on a subset (every 25th graph)
    sub = graphs[::25]
    Ks = None
    e0.record()
    for (sg, dg, ng) in sub:
        g = slaq.build_laplacian(torch.as_tensor(sg, device=dev), torch.as_tensor(dg, device=dev), ng,
                                 flags=slaq.DROP_ISOLATED)
        Ks = slaq.lanczos(g, SBM_NV, SBM_S, PROBE_SEED, precision=P, reuse=Ks)
        slaq.trace_heat(Ks, t)
        g.close()
    e1.record()
    torch.cuda.synchronize(dev)
    ms_sub = e0.elapsed_time(e1)
    return {"workload": SBM_WORKLOAD, "metric": "graphs/s",
            "value": whole_job_value(world, SBM_GRAPHS, ms),
            "ms_per_step": ms, "nnz": int(nnz),
            "probe_edges_per_s": world * nnz * SBM_NV * SBM_S / (ms * 1e-3),
            "kernels_ms_per_step": {k: round(v[0] / reps, 3) for k, v in prof.items()},
            "per_graph_launches": {"graphs": len(sub), "value": len(sub) / (ms_sub * 1e-3),
                                   "unit": "graphs/s"},
            "speedup_over_per_graph": (SBM_GRAPHS / ms) / (len(sub) / ms_sub)}


def small_graph_replay():
    """The small single-graph workload (BA n = 2000, m = 4, seed 0, normalized
    Laplacian, nv = 10, s = 15, full reorthogonalization): wall time of one
    Lanczos run (probes, s steps, Gauss rules; synchronous calls) through
    slaq_lanczos and through slaq_lanczos_rerun, which replays the run's
    captured CUDA graph with a new seed."""
    import torch
    from paper_2003_01282_gb300 import slaq
    s_, d_, n = synth.barabasi_albert(2000, 4, seed=0)
    g = slaq.build_laplacian(torch.as_tensor(s_, device="cuda"), torch.as_tensor(d_, device="cuda"),
                             n, kind=slaq.NORMALIZED)
    out = {"workload": "BA n=2000 m=4 seed 0, normalized; nv=10, s=15, full reorthogonalization"}
    reps = 50
    for name, prec in (("fp64", slaq.FP64), ("fp32", slaq.FP32)):
        K = slaq.lanczos(g, 10, 15, 1, precision=prec)
        for i in range(5):
            slaq.lanczos(g, 10, 15, 2 + i, precision=prec, reuse=K)
            slaq.lanczos_rerun(K, 2 + i)
        t0 = time.perf_counter()
        for i in range(reps):
            slaq.lanczos(g, 10, 15, 100 + i, precision=prec, reuse=K)
        t1 = time.perf_counter()
        slaq.lanczos_rerun(K, 99)                # capture again after the last call
        t2 = time.perf_counter()
        for i in range(reps):
            slaq.lanczos_rerun(K, 100 + i)
        t3 = time.perf_counter()
        a, b_ = (t1 - t0) / reps * 1e3, (t3 - t2) / reps * 1e3
        out[name] = {"ms_per_run_launches": a, "ms_per_run_replay": b_, "speedup": a / b_}
        K.close()
    g.close()
    return out


def rel_errors(a, b, t_np):
    """Error of descriptors a against the FP64 run b (both [heat | wave re |
    wave im | vnge]): heat relative per t, wave relative to its largest
    magnitude (over all t and over t < 10), VNGE relative."""
    lo = t_np < 10.0
    h, h64 = a[:NT], b[:NT]
    wr, wr64 = a[NT:2 * NT], b[NT:2 * NT]
    wi, wi64 = a[2 * NT:3 * NT], b[2 * NT:3 * NT]
    return {
        "heat_max": float(np.max(np.abs(h - h64) / np.abs(h64))),
        "wave_re_max": float(np.max(np.abs(wr - wr64)) / np.max(np.abs(wr64))),
        "wave_im_max": float(np.max(np.abs(wi - wi64)) / np.max(np.abs(wi64))),
        "wave_re_max_t_lt_10": float(np.max(np.abs(wr - wr64)[lo]) / np.max(np.abs(wr64))),
        "vnge": float(abs(a[-1] - b[-1]) / abs(b[-1])),
    }


def kernel_capture(args):
    """Profiling driver: build the workload's graph (R-MAT 2^20, or the SBM
    batch with --capture-batched) and run Lanczos `--kernel-capture` times
    (for ncu captures of single kernels)."""
    import torch
    from paper_2003_01282_gb300 import slaq
    from paper_2003_01282_gb300.build import build
    build()
    if args.capture_batched:
        g = slaq.build_laplacian_batch(synth.sbm_batch(SBM_GRAPHS, seed=SBM_SEED),
                                       flags=slaq.DROP_ISOLATED)
        nv, steps = SBM_NV, SBM_S
    else:
        s_, d_, n = make_graph()
        g = slaq.build_laplacian(torch.as_tensor(s_, device="cuda"), torch.as_tensor(d_, device="cuda"),
                                 n, flags=slaq.DROP_ISOLATED)
        nv, steps = NV, S
    K = None
    for _ in range(args.kernel_capture):
        K = slaq.lanczos(g, nv, steps, PROBE_SEED, precision=slaq.PRECISIONS[args.precision], reuse=K)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_capture": args.kernel_capture, "n_prime": g.info["n"], "nnz": g.info["nnz"]}))


# ---- multi-rank host logic (probe sharding; no data-path collective)
def rank_seed(rank: int) -> int:
    """Probe seed of a rank: every rank draws its own nv probes."""
    return PROBE_SEED + 1000 * rank


def average_over_ranks(desc, world: int, tdist):
    """The per-rank estimates of the same graph are Hutchinson means over
    disjoint probe sets of equal size, so their mean is the estimate over
    all world * nv probes: one all-reduce of the descriptor vector."""
    tdist.all_reduce(desc)
    desc /= world
    return desc


def max_over_ranks(ms: float, device, tdist) -> float:
    """The job's step time: the slowest rank's."""
    import torch
    mt = torch.tensor([ms], device=device, dtype=torch.float64)
    tdist.all_reduce(mt, op=tdist.ReduceOp.MAX)
    return float(mt.item())


def whole_job_value(world: int, units_per_step_per_rank: float, ms: float) -> float:
    """Whole-job throughput: every rank processes its own units each step."""
    return world * units_per_step_per_rank / (ms * 1e-3)


def run_ours(args):
    import torch
    from paper_2003_01282_gb300 import slaq
    from paper_2003_01282_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build()
    slaq.lib()
    if slaq.device_check() != 0:
        raise SystemExit(f"libslaq: {slaq.last_error()[1]}")
    dev = torch.device("cuda", local if dist else torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)

    src_np, dst_np, n_nodes = make_graph()
    src_h = torch.from_numpy(src_np).pin_memory()
    dst_h = torch.from_numpy(dst_np).pin_memory()
    src = src_h.to(dev)
    dst = dst_h.to(dev)
    t_np = synth.t_grid(NT)
    t = torch.as_tensor(t_np, device=dev)
    seed = rank_seed(rank)
    prec = args.precision
    P = slaq.PRECISIONS[prec]

    state = {"K": None, "ref": None}

    def step(precision=P, key="K", reorth=1):
        g = slaq.build_laplacian(src, dst, n_nodes, kind=slaq.NORMALIZED, flags=slaq.DROP_ISOLATED)
        state[key] = slaq.lanczos(g, NV, S, seed, precision=precision, reorth_passes=reorth,
                                  reuse=state.get(key))
        K = state[key]
        heat, _ = slaq.trace_heat(K, t)
        (wr, _), (wi, _) = slaq.trace_wave(K, t)
        vn, _ = slaq.trace_vnge(K)
        desc = torch.cat([heat, wr, wi, vn])
        if dist:
            average_over_ranks(desc, world, tdist)
        if state["ref"] is None:
            state["ref"] = desc[:NT].clone()
        d = slaq.distance(desc[:NT], state["ref"], slaq.DIST_HEAT)
        info = g.info
        g.close()
        return desc, d, info

    for _ in range(args.warmup):
        desc, _, info = step()
    torch.cuda.synchronize(dev)
    n_prime, nnz = info["n"], info["nnz"]

    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(dev.index)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.5)
    slaq.profile_enable(True)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tw0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        desc, dval, _ = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    tw1 = time.perf_counter()
    if dist:
        tdist.barrier()
    prof = slaq.profile_read()
    slaq.profile_enable(False)
    clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        ms = max_over_ranks(ms, dev, tdist)
    pe_step = nnz * NV * S
    value = whole_job_value(world, pe_step, ms)

    # roofline of the dominant Lanczos kernel class
    hbm, peak_src = peaks()
    alg = algorithmic_bytes(n_prime, nnz, prec)
    kernels = {}
    for name in ("spmm", "dots", "update", "reduce", "build", "ritz", "trace", "probes", "dist"):
        kms, kl = prof[name]
        entry = {"ms_per_step": kms / args.steps, "launches_per_step": kl / args.steps}
        if name in alg and kms > 0:
            gbs = alg[name] * args.steps / (kms * 1e-3) / 1e9
            entry.update({"GBps": gbs, "frac": gbs / hbm})
        kernels[name] = entry
    dom = max(("spmm", "dots", "update"), key=lambda k: prof[k][0])
    dom_ms, dom_launch = prof[dom]
    # unit of work: one SpMM (light and split-row kernels, overlapped), one
    # dots pass or one update pass; S, S and S - 1 of them per Lanczos run
    units = {"spmm": S, "dots": S, "update": S - 1}[dom]
    unit_ms = dom_ms / (args.steps * units)
    unit_bytes = alg[dom] / units
    achieved = unit_bytes / (unit_ms * 1e-3) / 1e9
    traffic = spmm_traffic(prec) if dom == "spmm" else None
    launches = sum(v[1] for v in prof.values())

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else ("bf16" if prec == "bf16" else "f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_prime": n_prime, "nnz": nnz, "nv": NV, "s": S, "nt": NT,
                   "precision": prec, "parallelism": f"probes x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (basis %.1f GB, edge list %.0f MB)" % (
                       S * n_prime * NV * {"fp64": 8, "fp32": 4, "bf16": 2}[prec] / 1e9,
                       src.numel() * 8 / 1e6)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic,
                     "unit_of_work": {"spmm": "one SpMM z = L u_k (light-row and split-row kernels)",
                                      "dots": "one dots pass", "update": "one update pass"}[dom],
                     "algorithmic_bytes_per_unit": unit_bytes, "ms_per_unit": unit_ms,
                     "launches_per_unit": dom_launch / (args.steps * units)},
        "kernels": kernels,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(tw0, tw1),
    }

    # the polynomial control variate on the last step's Lanczos run: standard
    # errors against the plain estimate at a few t, and the kernel's time
    if not args.quick:
        K = state["K"]
        tcv = torch.as_tensor([0.01, 0.1, 1.0, 10.0], device=dev, dtype=torch.float64)
        _, se_plain = slaq.trace_heat(K, tcv)
        out = {}
        for degree in (1, 2):
            slaq.trace_heat_cv(K, t, degree)
            torch.cuda.synchronize(dev)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            slaq.trace_heat_cv(K, t, degree)
            c1.record(stream)
            torch.cuda.synchronize(dev)
            _, se_cv = slaq.trace_heat_cv(K, tcv, degree)
            out[f"degree_{degree}"] = {
                "stderr_ratio_plain_over_cv": dict(zip(["t=0.01", "t=0.1", "t=1", "t=10"],
                                                       (se_plain / se_cv).cpu().tolist())),
                "ms_256_t": c0.elapsed_time(c1)}
        result["variance_reduction"] = out

    # FP64 form beside it: time and error of the headline form against it
    if prec != "fp64" and not args.quick:
        for _ in range(1):
            d64, _, _ = step(slaq.FP64, "K64")
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            d64, _, _ = step(slaq.FP64, "K64")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / 2
        b = d64.cpu().numpy()
        result["fp64_form"] = {"ms_per_step": ms64, "value": world * pe_step / (ms64 * 1e-3),
                               "speedup_of_headline": ms64 / ms}
        result["rel_err_vs_fp64"] = rel_errors(desc.double().cpu().numpy(), b, t_np)
        # the BF16-basis form of the same step, against the same FP64 run
        if prec != "bf16":
            step(slaq.FP32_BF16BASIS, "Kbf")
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(2):
                dbf, _, _ = step(slaq.FP32_BF16BASIS, "Kbf")
            e1.record(stream)
            torch.cuda.synchronize(dev)
            msbf = e0.elapsed_time(e1) / 2
            result["bf16_form"] = {"ms_per_step": msbf, "value": world * pe_step / (msbf * 1e-3),
                                   "speedup_over_fp64_form": ms64 / msbf,
                                   "rel_err_vs_fp64": rel_errors(dbf.cpu().numpy(), b, t_np)}
        # partial reorthogonalization (FP32 and FP64 forms): time, the
        # Lanczos kernels' time, how many steps projected against the whole
        # basis, and the error against the FP64 form with full reorthogonalization
        pr = {}
        for name, pp, ms_full in (("fp32", slaq.FP32, ms if prec == "fp32" else None),
                                  ("fp64", slaq.FP64, ms64)):
            key = "Kp" + name
            step(pp, key, slaq.REORTH_PARTIAL)
            torch.cuda.synchronize(dev)
            slaq.profile_enable(True)
            e0.record(stream)
            for _ in range(2):
                dp, _, _ = step(pp, key, slaq.REORTH_PARTIAL)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            kp = slaq.profile_read()
            slaq.profile_enable(False)
            msp = e0.elapsed_time(e1) / 2
            fs = slaq.krylov_full_steps(state[key]).cpu().numpy()
            pr[name] = {"ms_per_step": msp, "value": world * pe_step / (msp * 1e-3),
                        "speedup_over_full_reorth": (ms_full / msp) if ms_full else None,
                        "dots_update_ms_per_step": (kp["dots"][0] + kp["update"][0]) / 2,
                        "full_projection_steps": int(fs.sum()), "of_steps": S - 1,
                        "rel_err_vs_fp64": rel_errors(dp.double().cpu().numpy(), b, t_np)}
        result["partial_reorth"] = pr
        result["graph_replay"] = small_graph_replay()

    # end to end through the host-memory entry point (pinned buffers)
    if not args.quick:
        src_np_p, dst_np_p = src_h.numpy(), dst_h.numpy()
        e2e_times = []
        for i in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            out = slaq.descriptors_host(src_np_p, dst_np_p, n_nodes, t_np, kind=slaq.NORMALIZED,
                                        flags=slaq.DROP_ISOLATED, nv=NV, s=S, seed=seed, precision=P)
            t1 = time.perf_counter()
            if i > 0:
                e2e_times.append(t1 - t0)
        e2e_s = float(np.mean(e2e_times))
        result["e2e"] = {"value": world * pe_step / e2e_s, "unit": UNIT,
                         "h2d_bytes_per_step": int(2 * 4 * src.numel() + 8 * NT),
                         "d2h_bytes_per_step": int(8 * (3 * NT + 1)),
                         "ms_per_step": e2e_s * 1e3}

    if not args.quick and not args.no_batched:
        result["batched_sbm5000"] = run_batched(args, dev, world, rank, tdist if dist else None)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(src_np, dst_np, n_nodes)
    if rank == 0:
        print(json.dumps(result))
    if dist:
        tdist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "bf16"], default="fp32")
    ap.add_argument("--quick", action="store_true", help="skip the FP64-form and end-to-end legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the SBM-batch leg")
    ap.add_argument("--kernel-capture", type=int, default=0,
                    help="profiling driver: run Lanczos this many times on the R-MAT graph and exit")
    ap.add_argument("--capture-batched", action="store_true",
                    help="with --kernel-capture: use the SBM batch instead of the R-MAT graph")
    ap.add_argument("--cpu-baseline-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_worker:
        cpu_baseline_worker(args.cpu_baseline_worker)
        return
    if args.kernel_capture:
        kernel_capture(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
