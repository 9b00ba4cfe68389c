"""Write se_poly_split.h: the tables that add back the potential of the polynomial
p(r) = sum_n c_n r^(2n), n = 1..3, taken out of the free-space truncated biharmonic
(SE_FLAG_SPLIT_POLY). For a point source at y the stokeslet operator (delta lap - grad grad)
and the stresslet operator ((delta_jl d_m + delta_mj d_l + delta_lm d_j) lap - 2 d_j d_l d_m)
turn r^(2n) (r = x - y) into polynomials in r; expanding (x - y)^gamma in monomials of x and
of y, the summed potential is

    u_j(x) = sum_n c_n sum_a x^a sum_b sum_k T[n][j][a][b][k] M[b][k],
    M[b][k] = sum_sources y^b s_k,

with s = f (stokeslet, k = 0..2) or the 9 products q_l nu_m (stresslet, k = 3 l + m). The
tables list the nonzero coefficients T as (n, j, a, b, k, value); monomials x^a, y^b are
indexed in graded order up to degree 4 (35 of them).

Run from this directory: python gen_poly_split.py  (needs sympy).
"""
import itertools
import os

import sympy as sp

X = sp.symbols("x0:3")
Y = sp.symbols("y0:3")
R = [X[i] - Y[i] for i in range(3)]
R2 = sum(r * r for r in R)


def monomials(deg):
    out = []
    for d in range(deg + 1):
        for e in itertools.product(range(d + 1), repeat=3):
            if sum(e) == d:
                out.append(e)
    # graded, then lexicographically descending in (e0, e1, e2) within a degree
    return sorted(out, key=lambda e: (sum(e), [-v for v in e]))


MONO = monomials(4)
IDX = {e: i for i, e in enumerate(MONO)}


def lap(g, v):
    return sum(sp.diff(g, vi, 2) for vi in v)


def split(expr):
    """expr polynomial in X, Y -> {(a, b): coef}"""
    poly = sp.Poly(sp.expand(expr), *X, *Y)
    out = {}
    for mon, c in poly.terms():
        if c == 0:
            continue
        a, b = tuple(mon[:3]), tuple(mon[3:])
        out[(IDX[a], IDX[b])] = sp.Rational(c)
    return out


def main():
    rows_s, rows_t = [], []
    for n in (1, 2, 3):
        p = R2 ** n
        # derivatives with respect to x (r = x - y)
        for j in range(3):
            for k in range(3):
                g = (sp.KroneckerDelta(j, k) * lap(p, X) - sp.diff(p, X[j], X[k]))
                for (a, b), c in split(g).items():
                    rows_s.append((n, j, a, b, k, c))
            for l in range(3):
                for m in range(3):
                    g = (sp.KroneckerDelta(j, l) * sp.diff(lap(p, X), X[m])
                         + sp.KroneckerDelta(m, j) * sp.diff(lap(p, X), X[l])
                         + sp.KroneckerDelta(l, m) * sp.diff(lap(p, X), X[j])
                         - 2 * sp.diff(p, X[j], X[l], X[m]))
                    for (a, b), c in split(g).items():
                        rows_t.append((n, j, a, b, 3 * l + m, c))
    lines = ["// Generated by gen_poly_split.py: tables of the polynomial split's correction",
             "// (n, j, a, b, k, coefficient): u_j(x) += c_n x^a T M[b][k]; monomials of degree <= 4,",
             "// graded order; k = 0..2 stokeslet strength, k = 3 l + m stresslet product q_l nu_m.",
             "// The includer may set SE_PS_STORAGE (e.g. to place the tables in constant memory).",
             "#pragma once",
             "#ifndef SE_PS_STORAGE",
             "#define SE_PS_STORAGE static",
             "#endif",
             "#define SE_PS_NMONO %d" % len(MONO),
             "#define SE_PS_NMONO3 %d" % sum(1 for e in MONO if sum(e) <= 3),
             "SE_PS_STORAGE const signed char se_ps_mono[%d][3] = {%s};" % (
                 len(MONO), ", ".join("{%d, %d, %d}" % e for e in MONO)),
             "struct SePsTerm { signed char n, j, a, b, k; double c; };",
             "#define SE_PS_NS %d" % len(rows_s),
             "SE_PS_STORAGE const SePsTerm se_ps_stokeslet[%d] = {" % len(rows_s)]
    lines += ["  {%d, %d, %d, %d, %d, %s}," % (n, j, a, b, k, float(c)) for n, j, a, b, k, c in rows_s]
    lines += ["};", "#define SE_PS_NT %d" % len(rows_t),
              "SE_PS_STORAGE const SePsTerm se_ps_stresslet[%d] = {" % len(rows_t)]
    lines += ["  {%d, %d, %d, %d, %d, %s}," % (n, j, a, b, k, float(c)) for n, j, a, b, k, c in rows_t]
    lines += ["};", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "se_poly_split.h")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print(out, len(rows_s), len(rows_t))


if __name__ == "__main__":
    main()
