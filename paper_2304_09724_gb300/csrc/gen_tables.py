"""Writes recon_tables.cuh: exact rational constants of the SHWENO reconstruction used by the
CUDA kernels (Section 2.4 reading: quartic p1 on {I_{j-1}, I_j, I_{j+1}} matching the three
cell averages and the derivative averages of the two outer cells; linear p2, p3; Jiang-Shu
smoothness indicators).  Run:  python gen_tables.py  (needs sympy; output is committed).

In the local coordinate xi in [-1/2, 1/2] the data of cell j are W- = W_{j-1}, W0 = W_j,
W+ = W_{j+1}, v- = h V_{j-1}, v+ = h V_{j+1}.  With the symmetric combinations
  s = W- + W+, dv = v+ - v-   (even part of p1)   and   a = W+ - W-, sv = v- + v+   (odd part)
the monomial coefficients of p1 split into c0, c2, c4 (from W0, s, dv) and c1, c3 (from a, sv).

Both end values of one cell share their arithmetic: the normalised Taylor coefficient m of p1 is
  e_m(+1/2) = U_m + V_m,   e_m(-1/2) = (-1)^m (U_m - V_m),
where U_m (the terms of the even monomials) is a linear form in (W0, s, dv) and V_m (the odd
monomials) one in (a, sv) -- (a, sv, v0) for R1'.  ENDU_/ENDV_ hold those forms.

Reading R1' (option): a quintic p1 that also matches v0 = h V_j.  Its even part is R1's (the
odd monomials do not enter W0, s or dv); its odd part c1, c3, c5 comes from (a, sv, v0).  The
Q-prefixed constants below are that variant.
"""
import os

import sympy as sp

xi = sp.Symbol("xi")
half = sp.Rational(1, 2)


def derive():
    c = sp.symbols("c0:5")
    Wm, W0, Wp, vm, vp = sp.symbols("Wm W0 Wp vm vp")
    P = sum(c[k] * xi ** k for k in range(5))
    eqs = [sp.integrate(P, (xi, l - half, l + half)) - w for l, w in ((-1, Wm), (0, W0), (1, Wp))]
    eqs += [P.subs(xi, l + half) - P.subs(xi, l - half) - w for l, w in ((-1, vm), (1, vp))]
    sol = sp.solve(eqs, c)
    s, dv, a, sv = sp.symbols("s dv a sv")
    # substitute W- = (s - a)/2, W+ = (s + a)/2, v- = (sv - dv)/2, v+ = (sv + dv)/2
    sub = {Wm: (s - a) / 2, Wp: (s + a) / 2, vm: (sv - dv) / 2, vp: (sv + dv) / 2}
    coef = {}
    for k in range(5):
        e = sp.expand(sol[c[k]].subs(sub))
        coef[k] = {v: e.coeff(v) for v in (W0, s, dv, a, sv)}
    # normalised Taylor coefficients of p1 at xi = +1/2 and -1/2 as linear forms in the data
    P1 = P.subs(sol)
    ends = {}
    for tag, x0 in (("P", half), ("M", -half)):
        for m in range(5):
            e = sp.expand(sp.diff(P1, xi, m).subs(xi, x0) / sp.factorial(m))
            ends[(tag, m)] = {v: e.coeff(v) for v in (Wm, W0, Wp, vm, vp)}
    # smoothness indicator of p1 as a quadratic form in c1..c4
    cc = sp.symbols("k0:5")
    Pc = sum(cc[k] * xi ** k for k in range(5))
    beta = sp.expand(sum(sp.integrate(sp.diff(Pc, xi, d) ** 2, (xi, -half, half)) for d in range(1, 5)))
    bq = {}
    for i in range(1, 5):
        for j in range(i, 5):
            bq[(i, j)] = beta.coeff(cc[i], 1).coeff(cc[j], 1) if i != j else beta.coeff(cc[i], 2)
    return coef, bq, (W0, s, dv, a, sv), ends, (Wm, W0, Wp, vm, vp)


def derive_quintic():
    c = sp.symbols("c0:6")
    Wm, W0, Wp, vm, v0, vp = sp.symbols("Wm W0 Wp vm v0 vp")
    P = sum(c[k] * xi ** k for k in range(6))
    eqs = [sp.integrate(P, (xi, l - half, l + half)) - w for l, w in ((-1, Wm), (0, W0), (1, Wp))]
    eqs += [P.subs(xi, l + half) - P.subs(xi, l - half) - w for l, w in ((-1, vm), (0, v0), (1, vp))]
    sol = sp.solve(eqs, c)
    s, dv, a, sv = sp.symbols("s dv a sv")
    sub = {Wm: (s - a) / 2, Wp: (s + a) / 2, vm: (sv - dv) / 2, vp: (sv + dv) / 2}
    coef = {}
    for k in range(6):
        e = sp.expand(sol[c[k]].subs(sub))
        coef[k] = {v: e.coeff(v) for v in (W0, s, dv, a, sv, v0)}
    P1 = P.subs(sol)
    ends = {}
    data = (Wm, W0, Wp, vm, v0, vp)
    for tag, x0 in (("P", half), ("M", -half)):
        for m in range(5):
            e = sp.expand(sp.diff(P1, xi, m).subs(xi, x0) / sp.factorial(m))
            ends[(tag, m)] = {v: e.coeff(v) for v in data}
    cc = sp.symbols("k0:6")
    Pc = sum(cc[k] * xi ** k for k in range(6))
    beta = sp.expand(sum(sp.integrate(sp.diff(Pc, xi, d) ** 2, (xi, -half, half)) for d in range(1, 6)))
    bq = {}
    for i in range(1, 6):
        for j in range(i, 6):
            bq[(i, j)] = beta.coeff(cc[i], 1).coeff(cc[j], 1) if i != j else beta.coeff(cc[i], 2)
    return coef, bq, (W0, s, dv, a, sv, v0), ends, data


def frac(r):
    r = sp.Rational(r)
    if r.q == 1:
        return f"{float(r.p):.1f}"
    return f"({float(r.p):.1f} / {float(r.q):.1f})"


def main():
    coef, bq, names, ends, data = derive()
    g = sp.sqrt(sp.Rational(15)) / 10  # Gauss node offset in [-1/2,1/2]
    lines = [
        "// Generated by gen_tables.py -- exact rational constants of the SHWENO reconstruction.",
        "// Do not edit by hand.",
        "#pragma once",
        "namespace shweno_tables {",
        "// p1 monomial coefficients: c_k = sum of COEF_k_<v> * v over v in {W0, s, dv, a, sv}.",
    ]
    for k in range(5):
        for v in names:
            lines.append(f"constexpr double P1_C{k}_{v} = {frac(coef[k][v])};")
    lines.append("// Taylor coefficient m (d^m p1/dxi^m / m!) at xi = +1/2 (P) and -1/2 (M):")
    lines.append("// END_<P|M>[m][v] over the data v = (W-, W0, W+, v-, v+)")
    for tag in ("P", "M"):
        for m in range(5):
            for iv, v in enumerate(data):
                lines.append(f"constexpr double END_{tag}_{m}_{iv} = {frac(ends[(tag, m)][v])};")
    lines.append("// dot product of row p of END_P (plus) or END_M with the data d[0..4]")
    lines.append("template <bool PLUS>")
    lines.append("__host__ __device__ __forceinline__ double end_dot(int p, const double d[5]) {")
    lines.append("  switch (p) {")
    for m in range(5):
        tp = " + ".join(f"END_P_{m}_{iv} * d[{iv}]" for iv in range(5))
        tm = " + ".join(f"END_M_{m}_{iv} * d[{iv}]" for iv in range(5))
        lines.append(f"    case {m}: return PLUS ? ({tp}) : ({tm});")
    lines.append("  }")
    lines.append("  return 0.0;")
    lines.append("}")
    # even/odd split of the end values: U_m from (W0, s, dv), V_m from (a, sv) (and v0 for R1')
    lines.append("// Even/odd parts of the end values: e_m(+1/2) = U_m + V_m, e_m(-1/2) = (-1)^m (U_m - V_m),")
    lines.append("// U_m = ENDU_m_W0 W0 + ENDU_m_s s + ENDU_m_dv dv, V_m = ENDV_m_a a + ENDV_m_sv sv")
    lines.append("// (R1'; QENDV_m_a a + QENDV_m_sv sv + QENDV_m_v0 v0; U_m is the same).")
    qc, _, qn, _, _ = derive_quintic()
    uv_forms = {}
    for tag, cf, nm, deg in (("", coef, names, 4), ("Q", qc, qn, 5)):
        for m in range(5):
            U, V = {}, {}
            for j in range(m, deg + 1):
                w = sp.binomial(j, m) * half ** (j - m)
                tgt = U if j % 2 == 0 else V
                for v, val in cf[j].items():
                    tgt[v] = tgt.get(v, 0) + w * val
            even_vars, odd_vars = nm[:3], nm[3:]
            assert all(U.get(v, 0) == 0 for v in odd_vars) and all(V.get(v, 0) == 0 for v in even_vars)
            # the split reproduces the end rows
            if tag == "":
                Wm_, W0_, Wp_, vm_, vp_ = data
                back = {nm[0]: W0_, nm[1]: Wm_ + Wp_, nm[2]: vp_ - vm_, nm[3]: Wp_ - Wm_, nm[4]: vm_ + vp_}
                eU = sum(U.get(v, 0) * back[v] for v in nm)
                eV = sum(V.get(v, 0) * back[v] for v in nm)
                for sg, tg in ((1, "P"), (-1, "M")):
                    e = sp.expand(eU + sg * eV) * (1 if sg == 1 else (-1) ** m)
                    assert all(sp.simplify(e.coeff(v) - ends[(tg, m)][v]) == 0 for v in data), (tg, m)
                for v in even_vars:
                    lines.append(f"constexpr double ENDU_{m}_{v} = {frac(U.get(v, 0))};")
            for v in odd_vars:
                lines.append(f"constexpr double {tag}ENDV_{m}_{v} = {frac(V.get(v, 0))};")
            uv_forms[(tag, m)] = (U, V, even_vars, odd_vars)
    # U_m and V_m as functions; a term whose coefficient is zero is left out (x * 0.0 is not
    # folded away by the compiler), a coefficient of +-1 is folded by the compiler itself
    lines.append("// U_m(W0, s, dv) and V_m(a, sv) (R1) or V_m(a, sv, v0) (R1') of the end values")
    lines.append("__host__ __device__ __forceinline__ double end_u(int m, double W0, double s, double dv) {")
    lines.append("  switch (m) {")
    for m in range(5):
        U, _, ev_, _ = uv_forms[("", m)]
        terms = [f"ENDU_{m}_{n} * {n}" for v, n in zip(ev_, ["W0", "s", "dv"]) if U.get(v, 0) != 0]
        lines.append(f"    case {m}: return {' + '.join(terms) if terms else '0.0'};")
    lines.append("  }")
    lines.append("  return 0.0;")
    lines.append("}")
    for tag, nargs in (("", 2), ("Q", 3)):
        fn = "end_v" if tag == "" else "qend_v"
        sig = "double a, double sv" + (", double v0" if tag == "Q" else "")
        lines.append(f"__host__ __device__ __forceinline__ double {fn}(int m, {sig}) {{")
        lines.append("  switch (m) {")
        for m in range(5):
            _, V, _, ov = uv_forms[(tag, m)]
            d = {v: V.get(v, 0) for v in ov}
            names_ = ["a", "sv", "v0"][:nargs]
            terms = [f"{tag}ENDV_{m}_{n} * {n}" for v, n in zip(ov, names_) if d[v] != 0]
            lines.append(f"    case {m}: return {' + '.join(terms) if terms else '0.0'};")
        lines.append("  }")
        lines.append("  return 0.0;")
        lines.append("}")
    lines.append("// smoothness indicator of p1: beta1 = sum_{i<=j} B_ij c_i c_j (i, j >= 1)")
    for (i, j), val in bq.items():
        lines.append(f"constexpr double BETA_{i}{j} = {frac(val)};")
    qcoef, qbq, qnames, qends, qdata = derive_quintic()
    for k in range(6):
        for v in qnames:
            if k % 2 == 0 and k < 5:  # even part: R1's constants
                assert qcoef[k][v] == coef[k].get(v, 0), (k, v)
    lines.append("// Reading R1' (quintic p1, data (W-, W0, W+, v-, v0, v+)): odd monomial coefficients")
    lines.append("// c_k = QP1_C<k>_a a + QP1_C<k>_sv sv + QP1_C<k>_v0 v0 (k = 1, 3, 5); even ones as R1.")
    for k in (1, 3, 5):
        for v in qnames[3:]:
            lines.append(f"constexpr double QP1_C{k}_{v} = {frac(qcoef[k][v])};")
    lines.append("// R1' Taylor coefficients at the ends over (W-, W0, W+, v-, v0, v+)")
    for tag in ("P", "M"):
        for m in range(5):
            for iv, v in enumerate(qdata):
                lines.append(f"constexpr double QEND_{tag}_{m}_{iv} = {frac(qends[(tag, m)][v])};")
    lines.append("template <bool PLUS>")
    lines.append("__host__ __device__ __forceinline__ double qend_dot(int p, const double d[6]) {")
    lines.append("  switch (p) {")
    for m in range(5):
        tp = " + ".join(f"QEND_P_{m}_{iv} * d[{iv}]" for iv in range(6))
        tm = " + ".join(f"QEND_M_{m}_{iv} * d[{iv}]" for iv in range(6))
        lines.append(f"    case {m}: return PLUS ? ({tp}) : ({tm});")
    lines.append("  }")
    lines.append("  return 0.0;")
    lines.append("}")
    lines.append("// R1' smoothness indicator: beta1 = sum_{i<=j} QB_ij c_i c_j (i, j >= 1)")
    for (i, j), val in qbq.items():
        lines.append(f"constexpr double QBETA_{i}{j} = {frac(val)};")
    lines.append("// 3-point Gauss nodes on [-1/2, 1/2] (offset) and weights")
    lines.append("constexpr double GAUSS_G = 0.38729833462074168852;  // sqrt(15)/10")
    lines.append("constexpr double GAUSS_W0 = (5.0 / 18.0), GAUSS_W1 = (8.0 / 18.0);")
    lines.append("// 4-point Gauss-Lobatto nodes and weights on [0, 1]")
    lines.append("constexpr double LOB_L1 = 0.27639320225002103036;  // 1/2 - sqrt(5)/10")
    lines.append("constexpr double LOB_L2 = 0.72360679774997896964;  // 1/2 + sqrt(5)/10")
    lines.append("constexpr double LOB_W0 = (1.0 / 12.0), LOB_W1 = (5.0 / 12.0);")
    lines.append("}  // namespace shweno_tables")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recon_tables.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    # check the printed decimal constants against high-precision values
    assert abs(float(g) - 0.38729833462074168852) < 1e-17
    assert abs(float(half - sp.sqrt(5) / 10) - 0.27639320225002103036) < 1e-17
    print("wrote", out)


if __name__ == "__main__":
    main()
