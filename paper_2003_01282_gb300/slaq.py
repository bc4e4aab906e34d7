"""ctypes binding of libslaq (include/slaq.h): argument marshalling only.

Every function here has the name of the C entry point without the ``slaq_``
prefix and forwards to it; all computation happens in the CUDA library.
Device arrays are torch CUDA tensors (contiguous, of the dtype the header
names); streams default to torch's current stream.  If the library is not
built, importing works but the first call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

NORMALIZED, COMBINATORIAL = 0, 1
DROP_ISOLATED = 1
FP64, FP32, FP32_BF16BASIS = 0, 1, 2
REORTH_PARTIAL = 0  # reorth_passes value: partial reorthogonalization
DIST_HEAT, DIST_WAVE, DIST_VNGE = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": FP32_BF16BASIS}
KINDS = {"normalized": NORMALIZED, "combinatorial": COMBINATORIAL}

STATUS = {0: "SLAQ_OK", 1: "SLAQ_EINVAL", 2: "SLAQ_ENOMEM", 3: "SLAQ_ECUDA",
          4: "SLAQ_ENODEVICE", 5: "SLAQ_ETIMEOUT", 6: "SLAQ_EUNSUPPORTED", 7: "SLAQ_ENUMERIC"}


class SlaqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None
_VP, _I, _I64, _U64, _D, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
_PVP = C.POINTER(C.c_void_p)

_SIGNATURES = {
    "slaq_version": (_I, []),
    "slaq_last_error": (_I, [C.c_char_p, _SZ]),
    "slaq_device_check": (_I, []),
    "slaq_build_laplacian": (_I, [_VP, _VP, _I64, _I64, _VP, _I, _I, _VP, _PVP]),
    "slaq_build_laplacian_batch": (_I, [_VP, _VP, _VP, _VP, _I, _VP, _I, _I, _VP, _PVP]),
    "slaq_graph_batch_info": (_I, [_VP, _VP, _VP, _VP]),
    "slaq_krylov_batch_info": (_I, [_VP, _VP]),
    "slaq_graph_info": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "slaq_graph_export": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "slaq_graph_destroy": (None, [_VP]),
    "slaq_lanczos": (_I, [_VP, _I, _I, _U64, _I, _I, _I, _VP, _PVP]),
    "slaq_lanczos_batched": (_I, [_VP, _I, _I, _I, _U64, _I, _I, _I, C.c_char_p, _VP, _PVP]),
    "slaq_lanczos_probes": (_I, [_VP, _I, _I, _I, _U64, _I, _I, _I, _VP, _PVP]),
    "slaq_trace_wave_per_probe": (_I, [_VP, _VP, _I, _VP, _VP, _VP]),
    "slaq_pool_probes_host": (_I, [_VP, _I, _I, _VP, _VP]),
    "slaq_probes": (_I, [_VP, _I, _U64, _I, _VP, _VP]),
    "slaq_krylov_export": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "slaq_krylov_full_steps": (_I, [_VP, _VP, _VP]),
    "slaq_lanczos_rerun": (_I, [_VP, _U64, _VP]),
    "slaq_ritz_export": (_I, [_VP, _VP, _VP, _VP]),
    "slaq_krylov_info": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "slaq_trace_heat": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP]),
    "slaq_trace_heat_cv": (_I, [_VP, _VP, _I, _I, _VP, _VP, _VP, _VP]),
    "slaq_trace_wave": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "slaq_trace_vnge": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "slaq_krylov_monitor": (_I, [_VP, _VP, _VP, _VP]),
    "slaq_comparators": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "slaq_krylov_destroy": (None, [_VP]),
    "slaq_distance": (_I, [_VP, _VP, _I, _I, _VP, _VP]),
    "slaq_descriptors_host": (_I, [_VP, _VP, _I64, _I64, _I, _I, _I, _I, _U64, _I, _VP, _I,
                                   _VP, _VP, _VP, _VP, _VP]),
    "slaq_tridiag_gauss_host": (_I, [_VP, _VP, _I, _VP, _VP]),
    "slaq_trace_heat_tridiag_static": (_I, [_VP, _VP, _VP, _I, _I, _I64, _VP, _I, _VP, _VP, _VP,
                                            _VP]),
    "slaq_debug_fail_alloc": (_I, [_I64]),
    "slaq_debug_live_allocs": (_I64, []),
    "slaq_profile_enable": (_I, [_I]),
    "slaq_profile_read": (_I, [_I, _VP, _VP]),
    "slaq_profile_gather_peak": (_I, [_I, _VP]),
    "slaq_set_spmm_gathers": (_I, [_I]),
    "slaq_release_cached": (_I, []),
    "slaq_krylov_gathers": (_I, [_VP, _VP]),
    "slaq_debug_tma_giveup": (_I, [_I]),
}

PROF_NAMES = ["build", "probes", "spmm", "dots", "update", "reduce", "ritz", "trace", "dist"]


def lib_path() -> str:
    return LIB


def lib():
    """Load libslaq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with "
                               "paper_2003_01282_gb300.build.build(); there is no CPU fallback")
        h = C.CDLL(LIB)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def last_error() -> tuple[int, str]:
    buf = C.create_string_buffer(512)
    st = lib().slaq_last_error(buf, 512)
    return st, buf.value.decode(errors="replace")


def _check(status: int):
    if status != 0:
        _, msg = last_error()
        raise SlaqError(status, msg)


def _torch():
    import torch
    return torch


def _dev(t, dtype=None, name="array"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return C.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ calls
def version() -> int:
    return lib().slaq_version()


def device_check() -> int:
    return lib().slaq_device_check()


def build_laplacian(src, dst, n_nodes: int, weights=None, kind=NORMALIZED, flags=0, stream=None):
    torch = _torch()
    if isinstance(kind, str):
        kind = KINDS[kind]
    out = C.c_void_p()
    n_edges = int(src.numel())
    if int(dst.numel()) != n_edges:
        raise ValueError("src and dst differ in length")
    _check(lib().slaq_build_laplacian(_dev(src, torch.int32, "src"), _dev(dst, torch.int32, "dst"),
                                      n_edges, int(n_nodes), _dev(weights, torch.float64, "weights"),
                                      int(kind), int(flags), _stream(stream), C.byref(out)))
    return Graph(out)


def build_laplacian_batch(graphs, weights=None, kind=NORMALIZED, flags=0, device="cuda", stream=None):
    """Batch of graphs [(src, dst, n_nodes), ...] (numpy or CPU arrays, local
    ids) as one block-diagonal Laplacian."""
    torch = _torch()
    if isinstance(kind, str):
        kind = KINDS[kind]
    srcs = [np.asarray(g[0], np.int32) for g in graphs]
    dsts = [np.asarray(g[1], np.int32) for g in graphs]
    edge_off = np.zeros(len(graphs) + 1, np.int64)
    node_off = np.zeros(len(graphs) + 1, np.int64)
    edge_off[1:] = np.cumsum([a.size for a in srcs])
    node_off[1:] = np.cumsum([int(g[2]) for g in graphs])
    src = torch.as_tensor(np.concatenate(srcs) if srcs else np.zeros(0, np.int32), device=device)
    dst = torch.as_tensor(np.concatenate(dsts) if dsts else np.zeros(0, np.int32), device=device)
    w = None
    if weights is not None:
        w = torch.as_tensor(np.concatenate([np.asarray(x, np.float64) for x in weights]), device=device)
    out = C.c_void_p()
    _check(lib().slaq_build_laplacian_batch(_dev(src, torch.int32, "src"), _dev(dst, torch.int32, "dst"),
                                            edge_off.ctypes.data_as(C.c_void_p),
                                            node_off.ctypes.data_as(C.c_void_p), len(graphs),
                                            _dev(w, torch.float64, "weights"), int(kind), int(flags),
                                            _stream(stream), C.byref(out)))
    return Graph(out)


def graph_batch_info(g) -> dict:
    G = C.c_int()
    _check(lib().slaq_graph_batch_info(_handle(g), C.byref(G), None, None))
    off = np.zeros(G.value + 1, np.int64)
    tr = np.zeros(G.value)
    _check(lib().slaq_graph_batch_info(_handle(g), C.byref(G), off.ctypes.data_as(C.c_void_p),
                                       tr.ctypes.data_as(C.c_void_p)))
    return {"n_graphs": G.value, "node_off": off, "trace": tr}


def krylov_batch_info(k) -> int:
    G = C.c_int()
    _check(lib().slaq_krylov_batch_info(_handle(k), C.byref(G)))
    return G.value


def graph_info(g) -> dict:
    n, nnz, ni = C.c_int64(), C.c_int64(), C.c_int64()
    tr = C.c_double()
    _check(lib().slaq_graph_info(_handle(g), C.byref(n), C.byref(nnz), C.byref(tr), C.byref(ni)))
    return {"n": n.value, "nnz": nnz.value, "trace": tr.value, "n_input": ni.value}


def graph_export(g, stream=None) -> dict:
    torch = _torch()
    info = graph_info(g)
    n, nnz = info["n"], info["nnz"]
    dev = torch.device("cuda")
    out = {"rowptr": torch.empty(n + 1, dtype=torch.int64, device=dev),
           "colidx": torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
           "vals": torch.empty(max(nnz, 1), dtype=torch.float64, device=dev),
           "diag": torch.empty(max(n, 1), dtype=torch.float64, device=dev),
           "scale": torch.empty(max(n, 1), dtype=torch.float64, device=dev),
           "old_id": torch.empty(max(n, 1), dtype=torch.int64, device=dev)}
    _check(lib().slaq_graph_export(_handle(g), *[_dev(out[k]) for k in
                                                 ("rowptr", "colidx", "vals", "diag", "scale", "old_id")],
                                   _stream(stream)))
    out["colidx"], out["vals"] = out["colidx"][:nnz], out["vals"][:nnz]
    for k in ("diag", "scale", "old_id"):
        out[k] = out[k][:n]
    return out


def graph_destroy(g):
    lib().slaq_graph_destroy(_handle(g))


def lanczos(g, nv: int, s: int, seed: int, graph_id: int = 0, precision=FP64, reorth_passes: int = 1,
            stream=None, reuse=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = C.c_void_p(reuse.ptr.value if reuse is not None else None)
    _check(lib().slaq_lanczos(_handle(g), int(nv), int(s), C.c_uint64(int(seed) & (2**64 - 1)),
                              int(graph_id), int(precision), int(reorth_passes), _stream(stream),
                              C.byref(h)))
    if reuse is not None:
        return reuse
    return Krylov(h)


def lanczos_probes(g, nv: int, probe0: int, s: int, seed: int, graph_id: int = 0, precision=FP64,
                   reorth_passes: int = 1, stream=None, reuse=None):
    """slaq_lanczos_probes: Lanczos over generator probes probe0 .. probe0 + nv - 1."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = C.c_void_p(reuse.ptr.value if reuse is not None else None)
    _check(lib().slaq_lanczos_probes(_handle(g), int(nv), int(probe0), int(s),
                                     C.c_uint64(int(seed) & (2**64 - 1)), int(graph_id),
                                     int(precision), int(reorth_passes), _stream(stream), C.byref(h)))
    if reuse is not None:
        return reuse
    return Krylov(h)


def lanczos_rerun(k, seed: int, stream=None):
    """slaq_lanczos_rerun: the handle's last run again with a new probe seed,
    replayed from a captured CUDA graph."""
    _check(lib().slaq_lanczos_rerun(_handle(k), C.c_uint64(int(seed) & (2**64 - 1)),
                                    _stream(stream)))
    return k


def lanczos_batched(graphs, nv: int, s: int, seed: int, graph_id: int = 0, precision=FP64,
                    reorth_passes: int = 1, tune_cache=None, stream=None, reuse=None):
    """slaq_lanczos_batched: one Lanczos run over the concatenation of the
    graph handles `graphs` (the handle owns the concatenation)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    arr = (C.c_void_p * len(graphs))(*[_handle(g).value for g in graphs])
    h = C.c_void_p(reuse.ptr.value if reuse is not None else None)
    cache = None if tune_cache is None else os.fsencode(tune_cache)
    _check(lib().slaq_lanczos_batched(C.cast(arr, C.c_void_p), len(graphs), int(nv), int(s),
                                      C.c_uint64(int(seed) & (2**64 - 1)), int(graph_id),
                                      int(precision), int(reorth_passes), cache, _stream(stream),
                                      C.byref(h)))
    if reuse is not None:
        return reuse
    return Krylov(h)


def probes(g, nv: int, seed: int, graph_id: int = 0, stream=None):
    torch = _torch()
    n = graph_info(g)["n"]
    out = torch.empty(max(n, 1), nv, dtype=torch.float64, device="cuda")
    _check(lib().slaq_probes(_handle(g), int(nv), C.c_uint64(int(seed) & (2**64 - 1)), int(graph_id),
                             _dev(out), _stream(stream)))
    return out[:n]


def krylov_info(k) -> dict:
    nv, s, pr = C.c_int(), C.c_int(), C.c_int()
    n = C.c_int64()
    _check(lib().slaq_krylov_info(_handle(k), C.byref(nv), C.byref(s), C.byref(pr), C.byref(n)))
    return {"nv": nv.value, "s": s.value, "precision": pr.value, "n": n.value}


def _lead(k):
    """Leading shape of per-graph outputs: () for one graph, (G,) for a batch."""
    G = krylov_batch_info(k)
    return () if G == 1 else (G,)


def krylov_export(k, stream=None):
    torch = _torch()
    info = krylov_info(k)
    nv, s = info["nv"], info["s"]
    lead = _lead(k)
    alpha = torch.empty(*lead, nv, s, dtype=torch.float64, device="cuda")
    beta = torch.empty(*lead, nv, s, dtype=torch.float64, device="cuda")
    m = torch.empty(*lead, nv, dtype=torch.int32, device="cuda")
    _check(lib().slaq_krylov_export(_handle(k), _dev(alpha), _dev(beta), _dev(m), _stream(stream)))
    return alpha, beta, m


def krylov_full_steps(k, stream=None):
    """int32 [(G,) s] on the device: 1 where a Lanczos step projected its new
    vector against all previous ones (slaq_krylov_full_steps)."""
    torch = _torch()
    s = krylov_info(k)["s"]
    out = torch.empty(*_lead(k), s, dtype=torch.int32, device="cuda")
    _check(lib().slaq_krylov_full_steps(_handle(k), _dev(out), _stream(stream)))
    return out


def ritz_export(k, stream=None):
    torch = _torch()
    info = krylov_info(k)
    theta = torch.empty(*_lead(k), info["nv"], info["s"], dtype=torch.float64, device="cuda")
    tau2 = torch.empty_like(theta)
    _check(lib().slaq_ritz_export(_handle(k), _dev(theta), _dev(tau2), _stream(stream)))
    return theta, tau2


def trace_heat(k, t, per_probe: bool = False, stream=None):
    torch = _torch()
    nt = int(t.numel())
    lead = _lead(k)
    out = torch.empty(*lead, nt, dtype=torch.float64, device="cuda")
    se = torch.empty_like(out)
    pp = torch.empty(*lead, krylov_info(k)["nv"], nt, dtype=torch.float64, device="cuda") if per_probe else None
    _check(lib().slaq_trace_heat(_handle(k), _dev(t, torch.float64, "t"), nt, _dev(out), _dev(se),
                                 _dev(pp), _stream(stream)))
    return (out, se, pp) if per_probe else (out, se)


def trace_heat_cv(k, t, degree: int = 2, per_probe: bool = False, stream=None):
    """slaq_trace_heat_cv: the heat trace with the polynomial control variate."""
    torch = _torch()
    nt = int(t.numel())
    lead = _lead(k)
    out = torch.empty(*lead, nt, dtype=torch.float64, device="cuda")
    se = torch.empty_like(out)
    pp = torch.empty(*lead, krylov_info(k)["nv"], nt, dtype=torch.float64, device="cuda") if per_probe else None
    _check(lib().slaq_trace_heat_cv(_handle(k), _dev(t, torch.float64, "t"), nt, int(degree), _dev(out),
                                    _dev(se), _dev(pp) if per_probe else None, _stream(stream)))
    return (out, se, pp) if per_probe else (out, se)


def trace_wave(k, t, stream=None):
    torch = _torch()
    nt = int(t.numel())
    lead = _lead(k)
    re, im = (torch.empty(*lead, nt, dtype=torch.float64, device="cuda") for _ in range(2))
    sre, sim = torch.empty_like(re), torch.empty_like(re)
    _check(lib().slaq_trace_wave(_handle(k), _dev(t, torch.float64, "t"), nt, _dev(re), _dev(im),
                                 _dev(sre), _dev(sim), _stream(stream)))
    return (re, sre), (im, sim)


def trace_wave_per_probe(k, t, stream=None):
    """slaq_trace_wave_per_probe: per-probe Re and Im values, [(G,) nv, nt] each."""
    torch = _torch()
    nt = int(t.numel())
    shape = (*_lead(k), krylov_info(k)["nv"], nt)
    re = torch.empty(*shape, dtype=torch.float64, device="cuda")
    im = torch.empty_like(re)
    _check(lib().slaq_trace_wave_per_probe(_handle(k), _dev(t, torch.float64, "t"), nt, _dev(re),
                                           _dev(im), _stream(stream)))
    return re, im


def trace_vnge(k, per_probe: bool = False, stream=None):
    torch = _torch()
    lead = _lead(k)
    out = torch.empty(*(lead or (1,)), dtype=torch.float64, device="cuda")
    se = torch.empty_like(out)
    pp = torch.empty(*lead, krylov_info(k)["nv"], dtype=torch.float64, device="cuda") if per_probe else None
    _check(lib().slaq_trace_vnge(_handle(k), _dev(out), _dev(se), _dev(pp), _stream(stream)))
    return (out, se, pp) if per_probe else (out, se)


def comparators(k, t, stream=None) -> dict:
    """slaq_comparators: {"taylor_heat": [(G,) nt], "vnge_q", "finger_bar",
    "finger_hat": [(G,)]} (CUDA tensors)."""
    torch = _torch()
    nt = int(t.numel())
    lead = _lead(k)
    out = {"taylor_heat": torch.empty(*lead, nt, dtype=torch.float64, device="cuda")}
    for key in ("vnge_q", "finger_bar", "finger_hat"):
        out[key] = torch.empty(*(lead or (1,)), dtype=torch.float64, device="cuda")
    _check(lib().slaq_comparators(_handle(k), _dev(t, torch.float64, "t"), nt, _dev(out["taylor_heat"]),
                                  _dev(out["vnge_q"]), _dev(out["finger_bar"]), _dev(out["finger_hat"]),
                                  _stream(stream)))
    return out


def krylov_monitor(k, stream=None) -> dict:
    """slaq_krylov_monitor: {"ortho": max |Q^T Q - I| off the diagonal,
    "min_beta": smallest beta} of the last run."""
    o, b = C.c_double(), C.c_double()
    _check(lib().slaq_krylov_monitor(_handle(k), C.byref(o), C.byref(b), _stream(stream)))
    return {"ortho": o.value, "min_beta": b.value}


def krylov_destroy(k):
    lib().slaq_krylov_destroy(_handle(k))


def distance(a, b, kind=DIST_HEAT, stream=None):
    torch = _torch()
    if kind == DIST_WAVE:
        nt = int(a.numel()) // 2
    elif kind == DIST_VNGE:
        nt = 1
    else:
        nt = int(a.numel())
    if int(a.numel()) != int(b.numel()):
        raise ValueError("descriptor lengths differ")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib().slaq_distance(_dev(a, torch.float64, "a"), _dev(b, torch.float64, "b"), nt,
                               int(kind), _dev(out), _stream(stream)))
    return out


def descriptors_host(src, dst, n_nodes: int, t, kind=NORMALIZED, flags=0, nv: int = 10, s: int = 15,
                     seed: int = 0, precision=FP64, stream=None):
    """Host arrays in, host arrays out (numpy); copies happen inside the call."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    if isinstance(kind, str):
        kind = KINDS[kind]
    src, ps = _host(src, np.int32)
    dst, pd = _host(dst, np.int32)
    t, pt = _host(t, np.float64)
    nt = t.size
    heat, wr, wi = (np.empty(nt) for _ in range(3))
    vn = np.empty(1)
    _check(lib().slaq_descriptors_host(ps, pd, src.size, int(n_nodes), int(kind), int(flags), int(nv),
                                       int(s), C.c_uint64(int(seed)), int(precision), pt, nt,
                                       heat.ctypes.data_as(C.c_void_p), wr.ctypes.data_as(C.c_void_p),
                                       wi.ctypes.data_as(C.c_void_p), vn.ctypes.data_as(C.c_void_p),
                                       _stream(stream)))
    return {"heat": heat, "wave_re": wr, "wave_im": wi, "vnge": float(vn[0])}


def pool_probes_host(values):
    """slaq_pool_probes_host: (mean, stderr) over the rows of a [nprobe, len]
    array of per-probe values (numpy, host; no GPU needed)."""
    v, pv = _host(values, np.float64)
    if v.ndim != 2:
        raise ValueError("values must be [nprobe, len]")
    mean, se = np.empty(v.shape[1]), np.empty(v.shape[1])
    _check(lib().slaq_pool_probes_host(pv, v.shape[0], v.shape[1], mean.ctypes.data_as(C.c_void_p),
                                       se.ctypes.data_as(C.c_void_p)))
    return mean, se


def tridiag_gauss_host(alpha, beta):
    """Gauss nodes and weights of one tridiagonal matrix (host, no GPU)."""
    a, pa = _host(alpha, np.float64)
    b, pb = _host(beta if len(beta) else [0.0], np.float64)
    m = a.size
    th, t2 = np.empty(m), np.empty(m)
    _check(lib().slaq_tridiag_gauss_host(pa, pb, m, th.ctypes.data_as(C.c_void_p),
                                         t2.ctypes.data_as(C.c_void_p)))
    return th, t2


def trace_heat_tridiag_static(alpha, beta, m, n: int, t, stream=None):
    """Heat trace from exported Lanczos coefficients; the library allocates
    no device memory for it (see slaq_trace_heat_tridiag_static).
    Returns (out, stderr, status) as CUDA tensors."""
    torch = _torch()
    if alpha.dim() != 2 or tuple(beta.shape) != tuple(alpha.shape):
        raise ValueError("alpha and beta must both be [nv, s]")
    nv, s = int(alpha.shape[0]), int(alpha.shape[1])
    if m.dim() != 1 or int(m.numel()) != nv:
        raise ValueError("m must hold nv entries")
    nt = int(t.numel())
    out = torch.empty(nt, dtype=torch.float64, device=t.device)
    se = torch.empty_like(out)
    status = torch.empty(1, dtype=torch.int32, device=t.device)
    _check(lib().slaq_trace_heat_tridiag_static(_dev(alpha, torch.float64, "alpha"),
                                                _dev(beta, torch.float64, "beta"),
                                                _dev(m, torch.int32, "m"), nv, s, int(n),
                                                _dev(t, torch.float64, "t"), nt, _dev(out), _dev(se),
                                                _dev(status), _stream(stream)))
    return out, se, status


def debug_fail_alloc(nth: int):
    """slaq_debug_fail_alloc: the nth library allocation from now fails (0: off)."""
    _check(lib().slaq_debug_fail_alloc(int(nth)))


def debug_live_allocs() -> int:
    """slaq_debug_live_allocs: allocations the library holds."""
    return int(lib().slaq_debug_live_allocs())


def release_cached():
    """slaq_release_cached: free the workspace descriptors_host keeps between calls."""
    _check(lib().slaq_release_cached())


GATHERS_TUNED, GATHERS_LOADS, GATHERS_TMA = -1, 0, 1


def set_spmm_gathers(mode: int):
    """slaq_set_spmm_gathers: light-row gathers of later runs through TMA
    (GATHERS_TMA), loads (GATHERS_LOADS) or the run's tuning (GATHERS_TUNED)."""
    _check(lib().slaq_set_spmm_gathers(int(mode)))


def debug_tma_giveup(on: bool):
    """slaq_debug_tma_giveup: TMA stage waits give up at once (test hook)."""
    _check(lib().slaq_debug_tma_giveup(1 if on else 0))


def krylov_gathers(k) -> int:
    """slaq_krylov_gathers: 1 if k's last run gathered its light rows through TMA."""
    v = C.c_int()
    _check(lib().slaq_krylov_gathers(_handle(k), C.byref(v)))
    return v.value


def profile_enable(on: bool = True):
    _check(lib().slaq_profile_enable(1 if on else 0))


def profile_gather_peak(row_bytes: int) -> float:
    """slaq_profile_gather_peak: L2 row-gather rate in TB/s for rows of row_bytes."""
    v = C.c_double()
    _check(lib().slaq_profile_gather_peak(int(row_bytes), C.byref(v)))
    return v.value


def profile_read() -> dict:
    """{class name: (device ms, launches)} accumulated since profile_enable(True)."""
    out = {}
    for i, name in enumerate(PROF_NAMES):
        ms, n = C.c_double(), C.c_int64()
        _check(lib().slaq_profile_read(i, C.byref(ms), C.byref(n)))
        out[name] = (ms.value, n.value)
    return out


# --------------------------------------------------------------- handles
def _handle(x):
    return x.ptr if isinstance(x, (Graph, Krylov)) else C.c_void_p(x)


class Graph:
    """Owner of a slaq_graph handle (destroyed with the object)."""

    def __init__(self, ptr: C.c_void_p):
        self.ptr = ptr

    @property
    def info(self):
        return graph_info(self)

    def close(self):
        if self.ptr and self.ptr.value:
            graph_destroy(self)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Krylov:
    """Owner of a slaq_krylov handle (destroyed with the object)."""

    def __init__(self, ptr: C.c_void_p):
        self.ptr = ptr

    @property
    def info(self):
        return krylov_info(self)

    def close(self):
        if self.ptr and self.ptr.value:
            krylov_destroy(self)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
