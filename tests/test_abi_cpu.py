"""CPU checks of the C-ABI library: it builds, loads, exports every symbol the
header declares, reports SLAQ_ENODEVICE without a GPU (no CPU fallback), and
its tridiagonal Gauss-rule solver (the code the GPU kernel runs, compiled for
the host as well) agrees with the oracle's LAPACK-based Gauss rule."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import quadrature
from paper_2003_01282_gb300 import build, slaq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return slaq.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "slaq.h")).read()
    return sorted(set(re.findall(r"\b(slaq_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(slaq.exported_symbols()) == declared


def test_version_and_error_buffer(lib):
    assert slaq.version() == 100
    st, msg = slaq.last_error()
    assert isinstance(msg, str)


def test_no_device_means_enodevice(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert slaq.device_check() == 4
    st, msg = slaq.last_error()
    assert st == 4 and "no CPU path" in msg or "CUDA" in msg
    # a compute call fails loudly instead of falling back to the CPU
    src = (ctypes.c_int32 * 2)(0, 1)
    out = ctypes.c_void_p()
    r = lib.slaq_build_laplacian(src, src, 1, 2, None, 0, 0, None, ctypes.byref(out))
    assert r == 4 and not out.value


@pytest.mark.parametrize("m", [1, 2, 3, 5, 15, 20, 40, 64])
def test_tridiag_gauss_matches_oracle(lib, m):
    rng = np.random.default_rng(m)
    for trial in range(20):
        a = rng.uniform(0, 2, m)
        b = rng.uniform(1e-3, 1, m - 1)
        th, t2 = slaq.tridiag_gauss_host(a, b)
        th_o, t2_o = quadrature.ritz(a, b)
        assert np.all(np.diff(th) >= 0)
        assert np.allclose(th, th_o, atol=1e-13, rtol=0)
        assert np.allclose(t2, t2_o, atol=1e-12, rtol=0)
        assert abs(t2.sum() - 1) < 1e-13


def test_tridiag_gauss_hard_cases(lib):
    # clustered and repeated eigenvalues, tiny couplings, zero diagonal
    cases = [
        (np.zeros(6), np.full(5, 1e-9)),
        (np.ones(8), np.full(7, 1e-14)),
        (np.array([0.0, 0.0]), np.array([1.0])),
        (np.linspace(0, 2, 20), np.full(19, 1e-300)),
        (np.full(20, 1.0), np.full(19, 0.5)),
        (np.array([1e5, 1.0, 1e-5, 3.0]), np.array([1e3, 1e-2, 2.0])),
    ]
    for a, b in cases:
        th, t2 = slaq.tridiag_gauss_host(a, b)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        lam, U = np.linalg.eigh(T)
        scale = max(1.0, np.abs(T).max())
        assert np.allclose(th, lam, atol=1e-13 * scale)
        # weights: compare the Gauss rule's moments, which are unique even
        # when eigenvalues repeat
        for j in range(2 * len(a)):
            x = lam / scale
            y = th / scale
            want = np.sum(U[0] ** 2 * x ** j)
            assert abs(np.sum(t2 * y ** j) - want) < 1e-12 * max(1.0, abs(want))


def test_tridiag_gauss_closed_form_2x2(lib):
    a, b, c = 0.3, 1.1, 0.4
    th, t2 = slaq.tridiag_gauss_host([a, b], [c])
    mid, rad = (a + b) / 2, np.hypot((a - b) / 2, c)
    assert np.allclose(th, [mid - rad, mid + rad], atol=1e-15)
    assert abs(t2[0] - 0.5 * (1 + (b - a) / (2 * rad))) < 1e-14


def test_bad_arguments_rejected(lib):
    with pytest.raises(slaq.SlaqError):
        slaq.tridiag_gauss_host([], [])
