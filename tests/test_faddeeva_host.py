"""The kernels' FP32 Faddeeva evaluation (the accurate H(a,x) option of
Sect. 3.3.2), compiled as host C++ from the same header the GPU build uses,
against scipy's wofz: H and Im w to 1e-6 relative over a in [1e-6, 1] and x
to 1e5 (nearest-node and residue combination, asymptotic far wing), dH/da and
dH/dx against wofz's derivative identities (central differences of wofz in
the far wing).  CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2001_11252_gb300", "csrc")


def _run(tmp_path, a, x):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "faddeeva_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "faddeeva_check.cpp"),
                           "-o", exe])
    inp = "\n".join("%.17g %.17g" % (ai, xi) for ai, xi in zip(a, x))
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=120).stdout
    return np.array([[float(t) for t in l.split()] for l in out.splitlines() if l.strip()])


def test_faddeeva_fp32_against_wofz(tmp_path):
    from scipy.special import wofz
    rng = np.random.default_rng(8)
    n = 6000
    a = (10 ** rng.uniform(-6, 0, n)).astype(np.float32).astype(np.float64)
    x = np.concatenate([rng.uniform(-9, 9, n // 2), np.sign(rng.uniform(-1, 1, n // 2)) * 10 ** rng.uniform(-1, 5, n // 2)])
    # node midpoints, nodes, the |x| = 8 seam
    x[:10] = [0.0, 0.25, 0.5, -3.25, 7.999, 8.0, 8.001, -8.0, 5.5, 11.0]
    v = _run(tmp_path, a, x)
    assert v.shape == (n, 4)
    xs = x.astype(np.float32).astype(np.float64)
    w = wofz(xs + 1j * a)
    assert np.max(np.abs(v[:, 0] / w.real - 1)) < 1e-6
    assert np.max(np.abs(v[:, 1] - w.imag) / np.abs(w)) < 1e-6
    # references: where |x| <= 8 the derivative identities of w in FP64
    # (dH/da = 2 (x K + a H) - 2/sqrt(pi), dH/dx = 2 (a K - x H)); beyond, where
    # the first cancels even in FP64, central differences of wofz
    H = lambda aa, xx: wofz(xx + 1j * aa).real
    da, dx = 1e-5 * a, 1e-6 * np.maximum(np.abs(xs), 1e-3)
    far = np.abs(xs) > 8
    Ha = np.where(far, (H(a + da, xs) - H(a - da, xs)) / (2 * da), 2 * (xs * w.imag + a * w.real) - 2 / np.sqrt(np.pi))
    Hx = np.where(far, (H(a, xs + dx) - H(a, xs - dx)) / (2 * dx), 2 * (a * w.imag - xs * w.real))
    # the FP32 kernel forms the same identities, which subtract terms of these
    # sizes: the bound scales with them
    sa = np.abs(Ha) + 2 * np.abs(xs * w.imag) + 2 * a * w.real + 2 / np.sqrt(np.pi)
    sx = np.abs(Hx) + 2 * a * np.abs(w.imag) + 2 * np.abs(xs) * w.real + 1e-3 * w.real
    assert np.max(np.abs(v[:, 2] - Ha)[~far] / sa[~far]) < 4e-6
    assert np.max(np.abs(v[:, 3] - Hx)[~far] / sx[~far]) < 4e-6
    # beyond |x| = 8 the series derivative itself is accurate to FP32
    assert np.max(np.abs(v[far, 2] / Ha[far] - 1)) < 1e-5
    assert np.max(np.abs(v[far, 3] / Hx[far] - 1)) < 1e-5


def test_faddeeva_fp32_domain_edge(tmp_path):
    """At a = 2, the edge of the stated domain, H is still within 1e-5."""
    from scipy.special import wofz
    x = np.concatenate([np.linspace(-12, 12, 2001), [20.0, 1e3]])
    a = np.full(x.size, 2.0)
    v = _run(tmp_path, a, x)
    xs = x.astype(np.float32).astype(np.float64)
    assert np.max(np.abs(v[:, 0] / wofz(xs + 2j).real - 1)) < 1e-5
