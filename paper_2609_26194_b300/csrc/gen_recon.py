"""Derive the FAM reconstruction operators and emit them as CUDA device code.

Run:  python paper_2609_26194_b300/csrc/gen_recon.py   (writes fam_recon_gen.cuh)

The operators are derived here from their definitions, not transcribed: for
each order the auxiliary polynomial Q is the unique member of the paper's
ansatz space whose cell averages and scaled first moments match the stencil
data (eq. 5 and eq. 6 in 1D; eq. Qxy_quartic and eq. Qxy_quintic in 2D).  The
FAM-k polynomial is the L2 projection of Q on the central cell onto complete
polynomials of degree k-1 (Sec. 2.4).  Exact rational arithmetic (sympy)
solves each square system once; the generator then writes every coefficient
of the result in the tensor Legendre basis P_a(xi) P_b(eta), with P_a the
monic orthogonal polynomials on [-1/2, 1/2], as common-subexpression-
eliminated C++ code, together with numeric tables (Gauss nodes, weights and
basis values at the points the kernels evaluate).

Local coordinates: xi = (x - x_i)/dx, eta = (y - y_j)/dy.  Stencil arrays in
2D are indexed s = 3*(dj+1) + (di+1) for the neighbour (i+di, j+dj).
"""
from __future__ import annotations

import itertools
import os

import sympy as sp

XI, ETA = sp.symbols("xi eta")
HALF = sp.Rational(1, 2)


def monic_legendre(n):
    """Monic orthogonal polynomials on [-1/2, 1/2] by Gram-Schmidt."""
    P = []
    for d in range(n):
        p = XI ** d
        for q in P:
            p -= sp.integrate(p * q, (XI, -HALF, HALF)) / sp.integrate(q * q, (XI, -HALF, HALF)) * q
        P.append(sp.expand(p))
    return P


LEG = monic_legendre(7)


def _solve_linear(eqs, unknowns, Q):
    """Solve the square moment system M q = rhs exactly (M rational)."""
    M = sp.Matrix([[sp.expand(e.lhs).coeff(u) for u in unknowns] for e in eqs])
    rhs = sp.Matrix([e.rhs for e in eqs])
    assert M.det() != 0, "moment system is singular"
    qv = M.inv() * rhs
    return sp.expand(Q.subs(dict(zip(unknowns, qv))))


def cell_int_1d(expr, s, var=XI):
    """(1/dx) integral over the cell centred at offset s (in cell widths)."""
    return sp.integrate(expr, (var, s - HALF, s + HALF))


# --------------------------------------------------------------------------
# 1D
# --------------------------------------------------------------------------

def derive_1d(k):
    am, a0, ap, mm, m0, mp = sp.symbols("am a0 ap mm m0 mp")
    deg = 3 if k <= 4 else 5
    q = sp.symbols(f"q0:{deg + 1}")
    Q = sum(q[j] * XI ** j for j in range(deg + 1))
    avg = {-1: am, 0: a0, 1: ap}
    mom = {-1: mm, 0: m0, 1: mp}
    eqs = [sp.Eq(cell_int_1d(Q, s), avg[s]) for s in (-1, 0, 1)]
    for s in ((0,) if k <= 4 else (-1, 0, 1)):
        eqs.append(sp.Eq(cell_int_1d(Q * (XI - s), s), mom[s]))
    Qs = _solve_linear(eqs, q, Q)
    # L2 projection onto degree k-1 on the central cell, in the Legendre basis
    coef = []
    for a in range(k):
        coef.append(sp.simplify(cell_int_1d(Qs * LEG[a], 0) / cell_int_1d(LEG[a] ** 2, 0)))
    return (am, a0, ap, mm, m0, mp), coef, Qs


# --------------------------------------------------------------------------
# 2D
# --------------------------------------------------------------------------

def cell_int_2d(expr, si, sj):
    return sp.integrate(sp.integrate(expr, (XI, si - HALF, si + HALF)), (ETA, sj - HALF, sj + HALF))


def derive_2d(k):
    a = sp.symbols("a0:9")
    mx = sp.symbols("mx0:9")
    my = sp.symbols("my0:9")
    if k <= 4:
        monos = [(p, d - p) for d in range(4) for p in range(d + 1)] + [(2, 2)]
        xset = [4]
        yset = [4]
    else:
        monos = [(p, d - p) for d in range(6) for p in range(d + 1)] + [(4, 2), (2, 4)]
        xset = [0, 2, 3, 4, 5, 6, 8]   # I1, I3, I4, I5, I6, I7, I9
        yset = [0, 1, 2, 4, 6, 7, 8]   # I1, I2, I3, I5, I7, I8, I9
    q = sp.symbols(f"q0:{len(monos)}")
    Q = sum(qq * XI ** p * ETA ** r for qq, (p, r) in zip(q, monos))
    eqs = []
    for s in range(9):
        si, sj = s % 3 - 1, s // 3 - 1
        eqs.append(sp.Eq(cell_int_2d(Q, si, sj), a[s]))
        if s in xset:
            eqs.append(sp.Eq(cell_int_2d(Q * (XI - si), si, sj), mx[s]))
        if s in yset:
            eqs.append(sp.Eq(cell_int_2d(Q * (ETA - sj), si, sj), my[s]))
    assert len(eqs) == len(monos)
    Qs = _solve_linear(eqs, q, Q)
    deg = k - 1
    leg_eta = [p.subs(XI, ETA) for p in LEG]

    def coeffs_of(poly, degmax, extra=()):
        out = {}
        pairs = [(p, d - p) for d in range(degmax + 1) for p in range(d + 1)] + list(extra)
        for (p, r) in pairs:
            num = cell_int_2d(poly * LEG[p] * leg_eta[r], 0, 0)
            den = cell_int_2d(LEG[p] ** 2 * leg_eta[r] ** 2, 0, 0)
            out[(p, r)] = sp.expand(num / den)
        return out

    coef = coeffs_of(Qs, deg)
    full = coeffs_of(Qs, 5 if k >= 5 else 3, extra=((4, 2), (2, 4)) if k >= 5 else ((2, 2),))
    return (a, mx, my), coef, full, Qs


# --------------------------------------------------------------------------
# code emission
# --------------------------------------------------------------------------

def cnum(r):
    if isinstance(r, sp.Rational):
        if r.q == 1:
            return f"T({r.p}.0)"
        return f"T({r.p}.0 / {r.q}.0)"
    return f"T({sp.Float(r, 25)})"


def _key(r):
    """Hashable identity of a coefficient ratio (exact if rational)."""
    if isinstance(r, sp.Rational):
        return r
    return sp.Float(r, 18)


def _linear_terms(e):
    e = sp.expand(e)
    d = {}
    for sym_ in e.free_symbols:
        cf = sp.nsimplify(e.diff(sym_))
        if not cf.is_Rational:
            cf = sp.Float(sp.N(cf, 40), 40)
        if cf != 0:
            d[sym_] = cf
    if all(isinstance(c, sp.Rational) for c in d.values()):
        assert sp.expand(e - sum(c * v for v, c in d.items())) == 0
    return d


def emit_linear(name_out, exprs, symbols_map, indent="  ", prefix="t", lead_mul=None):
    """Emit linear forms in the inputs.  A greedy pass extracts shared scaled
    pairs x + r*y (one fused multiply-add each) while any pair occurs in at
    least two forms; each form is then a chain of multiply-adds.  lead_mul
    names a function that computes the product opening a chain (the one
    product that no multiply-add absorbs)."""
    forms = [_linear_terms(e) for e in exprs]
    temps = []
    while True:
        count = {}
        for f in forms:
            keys = sorted(f, key=str)
            for i in range(len(keys)):
                for j in range(i + 1, len(keys)):
                    x, y = keys[i], keys[j]
                    r = _key(f[y] / f[x])
                    count[(x, y, r)] = count.get((x, y, r), 0) + 1
        if not count:
            break
        (x, y, r), n = max(count.items(), key=lambda kv: (kv[1], -len(str(kv[0]))))
        if n < 2:
            break
        t = sp.Symbol(f"{prefix}{len(temps)}")
        temps.append((t, x, y, r))
        for f in forms:
            if x in f and y in f and _key(f[y] / f[x]) == r:
                cx = f.pop(x)
                f.pop(y)
                f[t] = f.get(t, 0) + cx

    def name(v):
        return symbols_map.get(v, str(v))

    def chain(f):
        items = sorted(f.items(), key=lambda kv: str(kv[0]))
        items = [(v, cf) for v, cf in items if cf != 0]
        if not items:
            return "T(0)"
        out = ""
        for v, cf in items:
            if isinstance(cf, sp.Float) and abs(cf - 1) < 1e-30:
                cf = sp.Integer(1)
            if isinstance(cf, sp.Float) and abs(cf + 1) < 1e-30:
                cf = sp.Integer(-1)
            if cf == 1:
                term = f"{name(v)}"
                op = "+"
            elif cf == -1:
                term = f"{name(v)}"
                op = "-"
            else:
                term = f"{cnum(cf)}*{name(v)}"
                if lead_mul and not out:
                    term = f"{lead_mul}({cnum(cf)}, {name(v)})"
                op = "+"
            if not out:
                out = ("-" if op == "-" else "") + term
            else:
                out += f" {op} {term}"
        return out

    lines = []
    for t, x, y, r in temps:
        if r == 1:
            rhs = f"{name(x)} + {name(y)}"
        elif r == -1:
            rhs = f"{name(x)} - {name(y)}"
        else:
            rhs = f"{name(x)} + {cnum(r)}*{name(y)}"
        lines.append(f"{indent}const T {t} = {rhs};")
    for i, f in enumerate(forms):
        lines.append(f"{indent}{name_out}[{i}] = {chain(f)};")
    return lines


def num_literal(x, digits=25):
    v = sp.N(x, digits)
    return f"{sp.Float(v, digits)}"


def gen():
    out = []
    out.append("// GENERATED by gen_recon.py -- do not edit.")
    out.append("// Reconstruction operators of the compact FAM schemes, derived by solving the")
    out.append("// moment-matching systems (eq. 5, 6, Qxy_quartic, Qxy_quintic) in exact")
    out.append("// arithmetic and projecting onto complete polynomials of degree k-1.")
    out.append("#pragma once")
    out.append("")
    # numeric tables
    xg = sorted(sp.Poly(sp.legendre(4, XI)).all_roots())
    nodes = [r / 2 for r in xg]
    wts = [sp.Rational(1, 2) * 2 / ((1 - r ** 2) * sp.diff(sp.legendre(4, XI), XI).subs(XI, r) ** 2) for r in xg]
    out.append("namespace famgen {")
    out.append("// 4-point Gauss-Legendre nodes on [-1/2,1/2] (ascending) and weights (sum 1)")
    out.append("__device__ constexpr double kGaussX[4] = {" + ", ".join(num_literal(sp.nsimplify(x)) for x in nodes) + "};")
    out.append("__device__ constexpr double kGaussW[4] = {" + ", ".join(num_literal(sp.simplify(w)) for w in wts) + "};")
    # basis values P_a at the two positive Gauss nodes and at 1/2
    pos = [nodes[2], nodes[3]]
    out.append("// P_a(x) for the monic orthogonal polynomials on [-1/2,1/2], a = 0..6, at")
    out.append("// x = Gauss node 2 (inner positive), Gauss node 3 (outer positive), 1/2, 0,")
    out.append("// and the positive interior node 1/(2 sqrt 5) of the 4-point Gauss-Lobatto rule.")
    rows = []
    for x in pos + [HALF, sp.Integer(0), 1 / (2 * sp.sqrt(5))]:
        rows.append("{" + ", ".join(num_literal(sp.simplify(LEG[a].subs(XI, x))) for a in range(7)) + "}")
    out.append("__device__ constexpr double kLegAt[5][7] = {" + ", ".join(rows) + "};")
    out.append("}  // namespace famgen")
    out.append("")
    # 1D
    for k in (3, 4, 5, 6):
        syms, coef, _ = derive_1d(k)
        smap = {syms[0]: "am", syms[1]: "a0", syms[2]: "ap", syms[3]: "mm", syms[4]: "m0", syms[5]: "mp"}
        out.append(f"// 1D FAM{k}: Legendre coefficients c[0..{k - 1}] of p_{k - 1}")
        out.append("template <typename T>")
        out.append(f"__device__ __forceinline__ void fam1d_coef_k{k}(T am, T a0, T ap, T mm, T m0, T mp, T* c) {{")
        out += emit_linear("c", coef, smap)
        out.append("}")
        out.append("")
    # 2D
    for k in (3, 4, 5, 6):
        (a, mx, my), coef, full, Qs = derive_2d(k)
        smap = {}
        for s in range(9):
            smap[a[s]] = f"A[{s}]"
            smap[mx[s]] = f"MX[{s}]"
            smap[my[s]] = f"MY[{s}]"
        keys = [(p, d - p) for d in range(k) for p in range(d + 1)]
        out.append(f"// 2D FAM{k}: coefficients of p in the tensor Legendre basis P_a(xi)P_b(eta),")
        out.append(f"// ordered by total degree d, then a = 0..d (b = d - a): " + " ".join(f"({p},{r})" for p, r in keys))
        out.append("template <typename T>")
        out.append(f"__device__ __forceinline__ void fam2d_coef_k{k}(const T* A, const T* MX, const T* MY, T* c) {{")
        # the FP64 kernels evaluate these next to other FP64 work: the opening
        # product of each coefficient runs on the integer pipes (fam::pmul)
        out += emit_linear("c", [coef[key] for key in keys], smap, lead_mul="fam::pmul")
        out.append("}")
        out.append("")
        # traces at the four Gauss points of each face (direct linear forms)
        ppoly = sum(coef[key] * LEG[key[0]] * LEG[key[1]].subs(XI, ETA) for key in keys)
        xg_ = sorted(sp.Poly(sp.legendre(4, XI)).all_roots())
        gn = [r / 2 for r in xg_]
        for face, (fx, fy) in {"xm": (-HALF, None), "xp": (HALF, None), "ym": (None, -HALF), "yp": (None, HALF)}.items():
            tr = []
            for g in gn:
                pt = {XI: fx, ETA: g} if fx is not None else {XI: g, ETA: fy}
                tr.append(sp.expand(ppoly.subs(pt)))
            out.append(f"// 2D FAM{k}: traces of p on face {face} at the 4 Gauss points (ascending)")
            out.append("template <typename T>")
            out.append(f"__device__ __forceinline__ void fam2d_tr_{face}_k{k}(const T* A, const T* MX, const T* MY, T* t) {{")
            out += emit_linear("t", tr, smap)
            out.append("}")
            out.append("")
        # face-centre traces for the OE jumps: xm = u(-1/2,0), xp = u(1/2,0), ym, yp
        variants = [("p", sum(coef[key] * LEG[key[0]] * LEG[key[1]].subs(XI, ETA) for key in keys))]
        if k == 6:
            fullpoly = sum(full[key] * LEG[key[0]] * LEG[key[1]].subs(XI, ETA) for key in full)
            assert sp.expand(fullpoly - Qs) == 0
            variants.append(("q", fullpoly))
        # transpose of the coefficient map: cotangents of the 27 patch inputs
        cb = sp.symbols(f"cb0:{len(keys)}")
        cmap = {c: f"CB[{i}]" for i, c in enumerate(cb)}
        inputs_ = list(a) + list(mx) + list(my)
        forms = [sp.expand(coef[key]) for key in keys]
        tforms = [sum(f.coeff(inp) * cbi for f, cbi in zip(forms, cb)) for inp in inputs_]
        out.append(f"// 2D FAM{k}: transpose of fam2d_coef_k{k}: g[0..8] = avg, g[9..17] = x-moment,")
        out.append("// g[18..26] = y-moment cotangents of the 3x3 patch from the coefficient cotangents CB")
        out.append("template <typename T>")
        out.append(f"__device__ __forceinline__ void fam2d_coefT_k{k}(const T* CB, T* g) {{")
        out += emit_linear("g", tforms, cmap, prefix="s")
        out.append("}")
        out.append("")
        for tag, poly in variants:
            tr = [poly.subs({XI: -HALF, ETA: 0}), poly.subs({XI: HALF, ETA: 0}),
                  poly.subs({XI: 0, ETA: -HALF}), poly.subs({XI: 0, ETA: HALF})]
            tb = sp.symbols("tb0:4")
            tmap = {c: f"TB[{i}]" for i, c in enumerate(tb)}
            trf = [sp.expand(e) for e in tr]
            ttf = [sum(f.coeff(inp) * tbi for f, tbi in zip(trf, tb)) for inp in inputs_]
            out.append(f"// 2D FAM{k}: transpose of fam2d_facec_k{k}{tag} (patch cotangents g[27] from TB[4])")
            out.append("template <typename T>")
            out.append(f"__device__ __forceinline__ void fam2d_facecT_k{k}{tag}(const T* TB, T* g) {{")
            out += emit_linear("g", ttf, tmap, prefix="s")
            out.append("}")
            out.append("")
            out.append(f"// 2D FAM{k}: face-centre traces of {'p_' + str(k) if tag == 'p' else 'the full auxiliary Q6'}")
            out.append("// t[0] = u(-1/2,0), t[1] = u(1/2,0), t[2] = u(0,-1/2), t[3] = u(0,1/2)")
            out.append("template <typename T>")
            out.append(f"__device__ __forceinline__ void fam2d_facec_k{k}{tag}(const T* A, const T* MX, const T* MY, T* t) {{")
            # (the OE kernel's face-centre traces: opening products on the integer pipes)
            out += emit_linear("t", [sp.expand(e) for e in tr], smap, lead_mul="fam::pmul")
            out.append("}")
            out.append("")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    text = gen()
    with open(os.path.join(here, "fam_recon_gen.cuh"), "w") as f:
        f.write(text)
    print("wrote fam_recon_gen.cuh", len(text.splitlines()), "lines")
