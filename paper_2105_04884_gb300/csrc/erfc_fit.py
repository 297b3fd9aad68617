"""Writes rbl_erfc_fit.cuh: the binary32 erfc used by the Ewald real-space pair.

erfc(x) = t h(t) exp(-x^2) with t = 1 / (1 + P x) maps x in [0, inf) onto t in
(0, 1]; h(t) = erfcx(x) / t is smooth on [0, 1] (h(1) = 1, h(0) = P / sqrt(pi)), so a
low-degree polynomial fits it to near binary32 precision.  This is the substitution
of Hastings' approximations (Abramowitz & Stegun 7.1.25-7.1.26), with coefficients
of our own: a least-squares fit of the relative error of h at Chebyshev nodes in t
(solved in the Chebyshev basis, then converted to powers of t for Horner's rule),
against scipy.special.erfcx in FP64.  The kernel shares the exp(-x^2) factor with
the force term 2 alpha / sqrt(pi) exp(-alpha^2 r^2), so a pair costs one exponential.

    python erfc_fit.py            # rewrites rbl_erfc_fit.cuh next to this file
"""
from __future__ import annotations

import os

import numpy as np

P = 0.4       # the substitution's scale
DEGREE = 8    # degree of h
NODES = 6000


def fit(p: float = P, degree: int = DEGREE, nodes: int = NODES) -> np.ndarray:
    """Power-series coefficients a_0..a_degree of h(t) ~ sum a_k t^k."""
    from scipy.special import erfcx

    k = np.arange(nodes)
    t = 0.5 * (1.0 - np.cos(np.pi * (k + 0.5) / nodes))  # Chebyshev nodes in (0, 1)
    x = (1.0 / t - 1.0) / p
    h = erfcx(x) / t
    w = 1.0 / h  # relative error
    V = np.polynomial.chebyshev.chebvander(2.0 * t - 1.0, degree)
    c, *_ = np.linalg.lstsq(V * w[:, None], np.ones_like(h), rcond=None)
    poly = np.polynomial.Chebyshev(c, domain=[0.0, 1.0]).convert(kind=np.polynomial.Polynomial)
    return np.asarray(poly.coef, dtype=np.float64)


def header(coef: np.ndarray, p: float = P) -> str:
    lines = [
        "// rbl_erfc_fit.cuh -- generated by erfc_fit.py (do not edit): coefficients of",
        "// erfc(x) = t h(t) exp(-x^2), t = 1 / (1 + P x), h(t) = sum_k A_k t^k, a",
        "// least-squares fit of the relative error of h at Chebyshev nodes (max relative",
        "// error of erfc in exact arithmetic about 1.3e-7 on [0, 10]).",
        "#pragma once",
        "",
        "namespace rbl {",
        "",
        f"constexpr float kErfcP = {float(np.float32(p)):.9e}f;",
        f"constexpr int kErfcDegree = {len(coef) - 1};",
        "",
        "// A_k (a function, so that unrolled device code folds each one to an immediate)",
        "__host__ __device__ constexpr float erfc_fit_coef(int k)",
        "{",
    ]
    for k, a in enumerate(coef):
        lines.append(f"    {'return' if k == 0 else '    '} k == {k} ? {float(np.float32(a)):.9e}f :")
    lines.append("        0.0f;")
    lines += ["}", "", "} // namespace rbl", ""]
    return "\n".join(lines)


def main() -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rbl_erfc_fit.cuh")
    with open(out, "w") as fh:
        fh.write(header(fit()))
    print(out)


if __name__ == "__main__":
    main()
