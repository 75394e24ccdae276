"""Exact-rational generator for the oracle's reconstruction tables.

ORACLE / TEST INFRASTRUCTURE ONLY.  Writes ``oracle/coeffs.h``; nothing in the
CUDA library reads that file or this script.

Everything is derived from definitions, in exact rational arithmetic
(``fractions.Fraction``), in index space (cell width 1, the interface at x=0,
cell n covering [n, n+1]):

* finite-volume reconstruction (paper Appendix B.2, eq. centered-reconstruction
  and eq. upwind-biased): the unique polynomial P of degree s-1 whose averages
  over the s stencil cells equal the cell values, evaluated at the interface.
  With Q(x) = integral of P from the stencil's left edge, Q is the degree-s
  polynomial through the running sums of the cell values at the cell edges, and
  P(0) = Q'(0).
* centered reconstruction of order 2p: cells -p .. p-1 (paper eq.
  centered-reconstruction for p=1).
* upwind-biased substencils for WENO of order 2r-1 with the flow in +x
  (paper eq. fifth-order-weno for r=3): substencil s covers cells -r+s .. s-1,
  s = 0 .. r-1; each contains the upwind cell -1.
* linear ("optimal") weights d_s: the combination of the r substencils that
  equals the upwind-biased stencil of order 2r-1 on cells -r .. r-2.
* Jiang-Shu smoothness indicators: beta_s = sum_{l=1}^{r-1} integral over the
  upwind cell [-1, 0] of (d^l P_s / dx^l)^2 (cell width 1), as a symmetric
  quadratic form in the substencil's r cell values.

Run: ``python oracle/gen_coeffs.py`` (rewrites oracle/coeffs.h).
"""
from fractions import Fraction as F
import os

RMAX = 5   # WENO order up to 9
PMAX = 6   # centered order up to 12


# --- tiny exact polynomial helpers (coefficient lists, lowest power first) ---
def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else F(0)) + (b[i] if i < len(b) else F(0)) for i in range(n)]


def pmul(a, b):
    out = [F(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pscale(a, s):
    return [x * s for x in a]


def pderiv(a):
    return [a[i] * i for i in range(1, len(a))] or [F(0)]


def peval(a, x):
    return sum(c * x ** i for i, c in enumerate(a))


def pint(a, lo, hi):
    """Exact integral of polynomial a over [lo, hi]."""
    return sum(c * (F(hi) ** (i + 1) - F(lo) ** (i + 1)) / (i + 1) for i, c in enumerate(a))


def lagrange_basis(nodes, t):
    """Lagrange basis polynomial L_t for the given nodes."""
    poly = [F(1)]
    for m, xm in enumerate(nodes):
        if m == t:
            continue
        poly = pmul(poly, [F(-xm), F(1)])
        poly = pscale(poly, F(1) / (nodes[t] - xm))
    return poly


def cell_average_basis(cells):
    """phi_l(x) with P(x) = sum_l q_l phi_l(x) for stencil cells n0..n0+s-1.

    Q(x_t) = sum_{l<t} q_l at edges x_t = n0+t, t=0..s; P = Q', so
    phi_l = sum_{t>l} L_t'.
    """
    n0 = cells[0]
    s = len(cells)
    nodes = [F(n0 + t) for t in range(s + 1)]
    dL = [pderiv(lagrange_basis(nodes, t)) for t in range(s + 1)]
    phis = []
    for l in range(s):
        acc = [F(0)]
        for t in range(l + 1, s + 1):
            acc = padd(acc, dL[t])
        phis.append(acc)
    return phis


def reconstruction_coeffs(cells):
    return [peval(phi, F(0)) for phi in cell_average_basis(cells)]


def centered(p):
    return reconstruction_coeffs(list(range(-p, p)))


def substencil_cells(r, s):
    return list(range(-r + s, s))


def linear_weights(r):
    """Solve sum_s d_s c^(s) = c^(full) (exact, by Gaussian elimination)."""
    full = reconstruction_coeffs(list(range(-r, r - 1)))      # 2r-1 cells: -r .. r-2
    # unknowns d_0..d_{r-1}; equations: one per cell -r .. r-2
    rows = []
    for idx, cell in enumerate(range(-r, r - 1)):
        row = []
        for s in range(r):
            cs = substencil_cells(r, s)
            cf = reconstruction_coeffs(cs)
            row.append(cf[cs.index(cell)] if cell in cs else F(0))
        rows.append(row + [full[idx]])
    # least squares is unnecessary: the system is consistent; eliminate.
    m = [r_[:] for r_ in rows]
    nvar = r
    piv_row = 0
    for col in range(nvar):
        sel = next(i for i in range(piv_row, len(m)) if m[i][col] != 0)
        m[piv_row], m[sel] = m[sel], m[piv_row]
        pv = m[piv_row][col]
        m[piv_row] = [x / pv for x in m[piv_row]]
        for i in range(len(m)):
            if i != piv_row and m[i][col] != 0:
                f = m[i][col]
                m[i] = [a - f * b for a, b in zip(m[i], m[piv_row])]
        piv_row += 1
    d = [m[i][nvar] for i in range(nvar)]
    for i in range(nvar, len(m)):          # consistency check
        assert all(x == 0 for x in m[i]), "inconsistent linear-weight system"
    assert sum(d) == 1
    return d


def beta_form(r, s):
    """Symmetric matrix B with beta_s = sum_ab B[a][b] q_a q_b (a,b over the r cells)."""
    phis = cell_average_basis(substencil_cells(r, s))
    B = [[F(0)] * r for _ in range(r)]
    for a in range(r):
        for b in range(r):
            acc = F(0)
            da, db = phis[a], phis[b]
            for _l in range(1, r):
                da, db = pderiv(da), pderiv(db)
                acc += pint(pmul(da, db), -1, 0)
            B[a][b] = acc
    return B


def cfrac(x):
    return f"({x.numerator}.0/{x.denominator}.0)"


def main():
    out = []
    out.append("/* GENERATED by oracle/gen_coeffs.py from exact rational arithmetic. Do not edit.")
    out.append(" * ORACLE / TEST INFRASTRUCTURE ONLY: used by oracle/ocn_oracle.c, never by the CUDA library.")
    out.append(" * Index space: interface at x=0, cell n covers [n, n+1], flow in +x (upwind cell -1).")
    out.append(" */")
    out.append("#ifndef OCN_ORACLE_COEFFS_H")
    out.append("#define OCN_ORACLE_COEFFS_H")
    out.append(f"#define ORC_RMAX {RMAX}")
    out.append(f"#define ORC_PMAX {PMAX}")
    out.append("/* ORC_CENTERED[p][n]: order-2p centered reconstruction, weight of cell n-p (n=0..2p-1). */")
    out.append(f"static const double ORC_CENTERED[{PMAX + 1}][{2 * PMAX}] = {{")
    out.append("  {0},")
    for p in range(1, PMAX + 1):
        c = centered(p)
        assert sum(c) == 1
        out.append("  {" + ", ".join(cfrac(x) for x in c) + "},")
    out.append("};")
    out.append("/* ORC_SUB[r][s][n]: substencil s of WENO(2r-1), weight of cell -r+s+n (n=0..r-1). */")
    out.append(f"static const double ORC_SUB[{RMAX + 1}][{RMAX}][{RMAX}] = {{")
    out.append("  {{0}},")
    for r in range(1, RMAX + 1):
        rows = []
        for s in range(r):
            rows.append("{" + ", ".join(cfrac(x) for x in reconstruction_coeffs(substencil_cells(r, s))) + "}")
        out.append("  {" + ", ".join(rows) + "},")
    out.append("};")
    out.append("/* ORC_D[r][s]: linear weights of WENO(2r-1). */")
    out.append(f"static const double ORC_D[{RMAX + 1}][{RMAX}] = {{")
    out.append("  {0},")
    for r in range(1, RMAX + 1):
        out.append("  {" + ", ".join(cfrac(x) for x in linear_weights(r)) + "},")
    out.append("};")
    out.append("/* ORC_BETA[r][s][a][b]: Jiang-Shu smoothness quadratic form of substencil s (cells -r+s+a, -r+s+b). */")
    out.append(f"static const double ORC_BETA[{RMAX + 1}][{RMAX}][{RMAX}][{RMAX}] = {{")
    out.append("  {{{0}}},")
    for r in range(1, RMAX + 1):
        ss = []
        for s in range(r):
            B = beta_form(r, s)
            ss.append("{" + ", ".join("{" + ", ".join(cfrac(x) for x in row) + "}" for row in B) + "}")
        out.append("  {" + ", ".join(ss) + "},")
    out.append("};")
    out.append("#endif")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "coeffs.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
