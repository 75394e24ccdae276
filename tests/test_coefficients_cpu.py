"""The reconstruction coefficients the CUDA kernels are compiled with, checked on the CPU.

The FP32 kernels take their WENO and centered coefficients as compile-time constants
(csrc/weno_coeffs.h, a constexpr derivation in double); the FP64 kernels take the long-double
tables of csrc/coeffs.cpp.  A host-only program built from those two sources dumps both table
sets, and the test checks them against the oracle's exact rational coefficients
(oracle/gen_coeffs.py: finite-volume reconstruction, linear weights, Jiang-Shu indicators;
Appendix B.2, Eq. fifth-order-weno), including the difference form the kernels evaluate
(q_s - t_{r-1} and beta_s as linear and quadratic forms in neighbour differences)."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_14148_gb300", "csrc")
R = 5                                   # highest WENO order 2R-1 = 9

DUMP = r"""
#include <cstdio>
#include "weno_coeffs.h"
int main(int argc, char** argv) {
  ocn::WenoTables<double> t;
  ocn::derive_weno_tables(&t);                      // long double, rounded to double
  FILE* f = std::fopen(argv[1], "wb");
  if (!f) return 1;
  std::fwrite(&ocn::wc::kTables, sizeof(t), 1, f);  // compile-time tables (dbeta packed)
  std::fwrite(&t, sizeof(t), 1, f);
  std::fclose(f);
  return 0;
}
"""

# WenoTables<double> field order and shapes (all doubles, no padding)
FIELDS = [("sub", (R + 1, R, R)), ("d", (R + 1, R)), ("beta", (R + 1, R, R, R)), ("cen", (R + 1, 2 * R)),
          ("gq", (R + 1, R, R - 1)), ("dbeta", (R + 1, R, R - 1, R - 1))]


def _unpack(buf):
    out, o = {}, 0
    for name, shape in FIELDS:
        n = int(np.prod(shape))
        out[name] = buf[o:o + n].reshape(shape)
        o += n
    return out, o


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("coeffs")
    src = d / "dump.cu"
    src.write_text(DUMP)
    exe, out = d / "dump", d / "tables.bin"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(src),
                    os.path.join(CSRC, "coeffs.cpp"), "-o", str(exe)], check=True, capture_output=True)
    subprocess.run([str(exe), str(out)], check=True)
    buf = np.fromfile(out, dtype=np.float64)
    ct, n = _unpack(buf)
    ld, m = _unpack(buf[n:])
    assert n + m == buf.size
    return ct, ld


@pytest.fixture(scope="module")
def exact():
    import sys
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import gen_coeffs as g
    return g


def _packed(dbeta):
    """Upper triangle with off-diagonal terms doubled, as the kernels evaluate the forms."""
    p = np.zeros_like(dbeta)
    for r in range(1, R + 1):
        for s in range(r):
            for a in range(r - 1):
                for b in range(r - 1):
                    p[r, s, a, b] = 2 * dbeta[r, s, a, b] if b > a else (dbeta[r, s, a, b] if a == b else 0.0)
    return p


def test_fp32_kernel_constants_equal_the_long_double_tables(tables):
    ct, ld = tables
    ld = dict(ld, dbeta=_packed(ld["dbeta"]))
    for name in ("gq", "dbeta", "d", "cen", "sub"):
        a, b = ct[name].astype(np.float32), ld[name].astype(np.float32)
        assert np.array_equal(a, b), (name, np.argwhere(a != b)[:5])


def test_tables_against_the_exact_rational_coefficients(tables, exact):
    g = exact
    for side in tables:
        for p in range(1, R + 1):
            ref = np.array([float(x) for x in g.centered(p)])
            assert np.allclose(side["cen"][p, :2 * p], ref, rtol=1e-11, atol=1e-13), ("cen", p)
        for r in range(1, R + 1):
            for s in range(r):
                ref = np.array([float(x) for x in g.reconstruction_coeffs(g.substencil_cells(r, s))])
                assert np.allclose(side["sub"][r, s, :r], ref, rtol=1e-11, atol=1e-12), ("sub", r, s)
            if r > 1:
                ref = np.array([float(x) for x in g.linear_weights(r)])
                assert np.allclose(side["d"][r, :r], ref, rtol=1e-11, atol=1e-13), ("d", r)
                for s in range(r):
                    B = np.array([[float(x) for x in row] for row in g.beta_form(r, s)])
                    scale = np.abs(B).max()
                    assert np.abs(side["beta"][r, s, :r, :r] - B).max() <= 1e-10 * scale, ("beta", r, s)


def test_difference_form_reproduces_the_exact_cell_forms(tables, exact):
    """q_s = t_{r-1} + sum_a gq[s][a] d_{s+a} and beta_s = sum_{a<=b} dbeta[s][a][b] d_{s+a} d_{s+b}
    (packed), d_m = t_{m+1} - t_m, against the exact cell-value forms on random stencils."""
    g = exact
    ct, _ = tables
    rng = np.random.default_rng(7)
    for r in range(2, R + 1):
        subs = [[Fraction(x) for x in g.reconstruction_coeffs(g.substencil_cells(r, s))] for s in range(r)]
        betas = [g.beta_form(r, s) for s in range(r)]
        for _ in range(20):
            t = rng.standard_normal(2 * r - 1) + np.linspace(0.0, rng.standard_normal() * 3.0, 2 * r - 1) ** 2
            tf = [Fraction(float(x)) for x in t]
            dm = np.diff(t)
            for s in range(r):
                q_exact = float(sum(c * tf[s + n] for n, c in enumerate(subs[s])))
                q_diff = t[r - 1] + sum(ct["gq"][r, s, a] * dm[s + a] for a in range(r - 1))
                assert abs(q_diff - q_exact) <= 1e-11 * max(1.0, np.abs(t).max()), ("q", r, s)
                b_exact = float(sum(betas[s][a][b] * tf[s + a] * tf[s + b] for a in range(r) for b in range(r)))
                b_diff = sum(ct["dbeta"][r, s, a, b] * dm[s + a] * dm[s + b]
                             for a in range(r - 1) for b in range(a, r - 1))
                assert abs(b_diff - b_exact) <= 1e-9 * max(1.0, np.abs(t).max() ** 2), ("beta", r, s)
