"""The binary32 erfc of the Ewald real-space kernel (csrc/rbl_erfc_fit.cuh, written by
csrc/erfc_fit.py): erfc(x) = t h(t) exp(-x^2), t = 1 / (1 + P x), h a fitted
polynomial.  Checked on the CPU against scipy's erfc, and against the identities that
fix h at the ends of [0, 1]: h(1) = erfcx(0) = 1 and h(0) = P / sqrt(pi)."""
import math
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2105_04884_gb300", "csrc", "rbl_erfc_fit.cuh")


def _coef():
    txt = open(HDR).read()
    P = float(re.search(r"kErfcP = ([-+0-9.e]+)f", txt).group(1))
    deg = int(re.search(r"kErfcDegree = (\d+)", txt).group(1))
    a = [float(m) for m in re.findall(r"k == \d+ \? ([-+0-9.e]+)f", txt)]
    assert len(a) == deg + 1
    return np.float32(P), np.array(a, dtype=np.float32)


def test_end_values():
    P, a = _coef()
    assert abs(float(np.sum(a.astype(np.float64))) - 1.0) < 1e-6            # h(1) = erfcx(0) = 1
    assert abs(float(a[0]) - float(P) / math.sqrt(math.pi)) < 1e-6          # h(0) = P / sqrt(pi)


def test_relative_error_against_scipy():
    erfc = pytest.importorskip("scipy.special").erfc
    P, a = _coef()
    x = np.linspace(0.0, 6.0, 120001)
    # exact arithmetic with the binary32 coefficients
    t = 1.0 / (1.0 + float(P) * x)
    h = np.polyval(a[::-1].astype(np.float64), t)
    rel = np.abs(t * h * np.exp(-x * x) / erfc(x) - 1.0)
    assert rel.max() < 3e-7
    # the kernel's binary32 sequence (fused multiply-adds rounded once each)
    x32 = x.astype(np.float32)
    t32 = (np.float32(1.0) / (P * x32 + np.float32(1.0))).astype(np.float32)
    hp = np.full_like(t32, a[-1])
    for k in range(len(a) - 2, -1, -1):
        hp = (hp.astype(np.float64) * t32 + float(a[k])).astype(np.float32)
    ex = np.exp(-(x32.astype(np.float64) ** 2)).astype(np.float32)
    approx = (t32 * hp).astype(np.float32) * ex
    rel32 = np.abs(approx.astype(np.float64) / erfc(x32.astype(np.float64)) - 1.0)
    assert rel32[x <= 5.0].max() < 2e-6


def test_header_is_the_generators_output():
    """The committed coefficients are what csrc/erfc_fit.py computes (to binary32
    rounding; the least-squares solve may differ in the last FP64 bits by platform)."""
    pytest.importorskip("scipy.special")
    import importlib.util

    path = os.path.join(os.path.dirname(HDR), "erfc_fit.py")
    spec = importlib.util.spec_from_file_location("erfc_fit", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    P, a = _coef()
    c = mod.fit()
    assert float(P) == pytest.approx(mod.P, rel=1e-7)
    assert len(c) == len(a)
    assert np.allclose(c.astype(np.float32), a, rtol=1e-6, atol=1e-8)
