"""Markstein's corrected quotient, as the reduced forms' heat-trace kernel uses
it for its Welford updates, against IEEE division on the host (compiled
with gcc from tests/markstein_check.c; skipped without a C compiler).

The kernel forms q = fl(d r) with r the correctly rounded 1/c, then
fl(q + fl(d - q c) r) through two FMAs, and relies on that being the
correctly rounded d / c (Markstein, IBM J. Res. Dev. 34, 1990), so that host
pooling of per-probe values (plain division) reproduces the device's mean and
standard error bit for bit.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_corrected_quotient_equals_ieee_division(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "markstein_check"
    subprocess.run([cc, "-O2", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(HERE, "markstein_check.c"), "-lm"], check=True)
    # c = 1..512 covers every probe count a trace block divides by (nv <= 512)
    out = subprocess.run([str(exe), "512", "4000"], check=True, capture_output=True, text=True)
    n, bad = (int(x) for x in out.stdout.split())
    assert n == 512 * 4000 and bad == 0
