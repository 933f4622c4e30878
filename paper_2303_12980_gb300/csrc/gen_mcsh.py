"""Generate mcsh_gen.cuh: straight-line device code for the MCSH angular
probes used by the CUDA kernels.

The MCSH function of order l and component (a, b, c), a+b+c = l, is the
harmonic polynomial S_abc(r) = (-1)^l r^(2l+1) d^a/dx^a d^b/dy^b d^c/dz^c (1/r)
(GMP-Featurizer, Examples: "orders of the MCSH angular probe functions").
This generator works from a closed form of those polynomials and from
recurrences derived by differentiating the identity r^2 d(1/r)/dx = -x/r
(Leibniz rule), NOT from repeated differentiation:

  closed form (traceless Cartesian tensors):
    S_abc = sum_{i,j,k} (-1)^(i+j+k) (2l-2m-1)!! h(a,i) h(b,j) h(c,k)
            x^(a-2i) y^(b-2j) z^(c-2k) r^(2m),   m = i+j+k,
    h(n,i) = n! / (2^i i! (n-2i)!)
  x-raising recurrence (y, z by symmetry):
    S_{a+1,b,c} = (2a+1) x S_abc + 2b y S_{a+1,b-1,c} + 2c z S_{a+1,b,c-1}
                  - r^2 (a^2 S_{a-1,b,c} + b(b-1) S_{a+1,b-2,c} + c(c-1) S_{a+1,b,c-2})

Because every S_abc is traceless (S_{a+2,b,c} + S_{a,b+2,c} + S_{a,b,c+2} = 0),
only the 2l+1 components with a <= 1 are independent; the kernels
accumulate those and rebuild the rest once per center.  The rotation
invariant of one (l, sigma) group is sum over all components of
l!/(a! b! c!) mu_abc^2 (full contraction of the symmetric traceless tensor).

Every emitted recurrence is checked here against the closed form with exact
integer polynomial arithmetic before the header is written.
Run:  python gen_mcsh.py [output_path]
"""
from __future__ import annotations

import math
import os
import sys
from collections import defaultdict

LMAX = 6


# ---------------------------------------------------------------- polynomials
def padd(*ps):
    out = defaultdict(int)
    for coef, p in ps:
        for m, v in p.items():
            out[m] += coef * v
    return {m: v for m, v in out.items() if v}


def pmul_mono(p, m):
    return {(a + m[0], b + m[1], c + m[2]): v for (a, b, c), v in p.items()}


R2 = {(2, 0, 0): 1, (0, 2, 0): 1, (0, 0, 2): 1}


def pmul(p, q):
    out = defaultdict(int)
    for m1, v1 in p.items():
        for m2, v2 in q.items():
            out[(m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2])] += v1 * v2
    return {m: v for m, v in out.items() if v}


def ppow_r2(m):
    p = {(0, 0, 0): 1}
    for _ in range(m):
        p = pmul(p, R2)
    return p


def dfact(n):
    return 1 if n <= 0 else n * dfact(n - 2)


def closed_form(a, b, c):
    l = a + b + c
    out = {}
    h = lambda n, i: math.factorial(n) // (2 ** i * math.factorial(i) * math.factorial(n - 2 * i))
    for i in range(a // 2 + 1):
        for j in range(b // 2 + 1):
            for k in range(c // 2 + 1):
                m = i + j + k
                coef = (-1) ** m * dfact(2 * l - 2 * m - 1) * h(a, i) * h(b, j) * h(c, k)
                term = pmul_mono(ppow_r2(m), (a - 2 * i, b - 2 * j, c - 2 * k))
                out = padd((1, out), (coef, term))
    return out


def all_components(l):
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


def indep_components(l):
    """Independent components of order l: a = 0 first (b descending), then a = 1."""
    comps = [(0, b, l - b) for b in range(l, -1, -1)]
    if l >= 1:
        comps += [(1, b, l - 1 - b) for b in range(l - 1, -1, -1)]
    return comps


def weight(a, b, c):
    return math.factorial(a + b + c) // (math.factorial(a) * math.factorial(b) * math.factorial(c))


# -------------------------------------------------------------- recurrences
def recurrence_terms(t):
    """Terms (coef, kind, src) producing independent component t from
    independent components of lower order.  kind: 'x','y','z' = multiply by
    that coordinate, 'r2' = multiply by r^2, '1' = plain."""
    a, b, c = t
    if (a, b, c) == (0, 0, 0):
        return [(1, "1", None)]
    terms = []
    if a == 1:
        # x-raising from (0, b, c)
        terms.append((1, "x", (0, b, c)))
        if b >= 1:
            terms.append((2 * b, "y", (1, b - 1, c)))
        if c >= 1:
            terms.append((2 * c, "z", (1, b, c - 1)))
        if b >= 2:
            terms.append((-b * (b - 1), "r2", (1, b - 2, c)))
        if c >= 2:
            terms.append((-c * (c - 1), "r2", (1, b, c - 2)))
        return terms
    if b >= 1:
        # y-raising from (0, b-1, c)
        bb = b - 1
        terms.append((2 * bb + 1, "y", (0, bb, c)))
        if c >= 1:
            terms.append((2 * c, "z", (0, bb + 1, c - 1)))
        if bb >= 1:
            terms.append((-bb * bb, "r2", (0, bb - 1, c)))
        if c >= 2:
            terms.append((-c * (c - 1), "r2", (0, bb + 1, c - 2)))
        return terms
    # z-raising from (0, 0, c-1)
    cc = c - 1
    terms.append((2 * cc + 1, "z", (0, 0, cc)))
    if cc >= 1:
        terms.append((-cc * cc, "r2", (0, 0, cc - 1)))
    return terms


MULT = {"x": {(1, 0, 0): 1}, "y": {(0, 1, 0): 1}, "z": {(0, 0, 1): 1}, "r2": R2, "1": {(0, 0, 0): 1}}


def check_recurrences():
    for l in range(LMAX + 2):
        for t in indep_components(l):
            got = {}
            for coef, kind, src in recurrence_terms(t):
                base = {(0, 0, 0): 1} if src is None else closed_form(*src)
                got = padd((1, got), (coef, pmul(base, MULT[kind])))
            want = closed_form(*t)
            assert got == want, (t, got, want)


def reconstruction(l):
    """T[abc] = {k: coef}: each full component as a combination of the
    independent ones, from S_{a,b,c} = -S_{a-2,b+2,c} - S_{a-2,b,c+2}."""
    ind = indep_components(l)
    idx = {t: k for k, t in enumerate(ind)}
    T = {}
    for a in range(0, l + 1):
        for b in range(l - a, -1, -1):
            c = l - a - b
            if a <= 1:
                T[(a, b, c)] = {idx[(a, b, c)]: 1}
            else:
                T[(a, b, c)] = {}
                for src in ((a - 2, b + 2, c), (a - 2, b, c + 2)):
                    for k, v in T[src].items():
                        T[(a, b, c)][k] = T[(a, b, c)].get(k, 0) - v
                T[(a, b, c)] = {k: v for k, v in T[(a, b, c)].items() if v}
    return T


def check_reconstruction():
    for l in range(LMAX + 1):
        ind = indep_components(l)
        T = reconstruction(l)
        for t, combo in T.items():
            got = {}
            for k, v in combo.items():
                got = padd((1, got), (v, closed_form(*ind[k])))
            assert got == closed_form(*t), t


# ------------------------------------------------------------------ emitters
def nind(L):
    return (L + 1) * (L + 1)


def flat(t):
    a, b, c = t
    l = a + b + c
    return l * l + indep_components(l).index(t)


def fnum(v):
    return f"{float(v)!r}f"


def emit_eval_scaled(L):
    """The raising recurrences with the integer coefficient folded into the
    coordinate once per pair (c*x, c*y, c*z, c*r^2 products computed first),
    so that each term of a component costs one FMA: every product and sum
    explicit (the build disables implicit contraction)."""
    lines = [f"__device__ __forceinline__ void gmp_mcsh_indep_{L}(float x, float y, float z, float r2, "
             f"float* __restrict__ S) {{"]
    scaled = {}
    body = []
    for l in range(L + 1):
        for t in indep_components(l):
            k = flat(t)
            rec = recurrence_terms(t)
            if rec[0][1] == "1":
                body.append(f"  S[{k}] = 1.0f;")
                continue
            expr = None
            for coef, kind, src in rec:
                v = "r2" if kind == "r2" else kind
                if coef == 1:
                    m = v
                else:
                    m = f"{v}_{'m' if coef < 0 else ''}{abs(coef)}"
                    scaled[m] = f"__fmul_rn({fnum(coef)}, {v})"
                expr = f"__fmul_rn({m}, S[{flat(src)}])" if expr is None else f"__fmaf_rn({m}, S[{flat(src)}], {expr})"
            body.append(f"  S[{k}] = {expr};")
    for m, e in sorted(scaled.items()):
        lines.append(f"  const float {m} = {e};")
    lines += body
    lines.append("}")
    return "\n".join(lines)


def emit_eval_top(L):
    """Only the components of order L, by the same scaled recurrences, given
    S[0 .. L^2) (orders below L) already evaluated: lets a kernel evaluate
    the orders it contracts first and the next order later."""
    lines = [f"__device__ __forceinline__ void gmp_mcsh_top_{L}(float x, float y, float z, float r2, "
             f"float* __restrict__ S) {{"]
    scaled = {}
    body = []
    for t in indep_components(L):
        k = flat(t)
        expr = None
        for coef, kind, src in recurrence_terms(t):
            v = "r2" if kind == "r2" else kind
            if coef == 1:
                m = v
            else:
                m = f"{v}_{'m' if coef < 0 else ''}{abs(coef)}"
                scaled[m] = f"__fmul_rn({fnum(coef)}, {v})"
            expr = f"__fmul_rn({m}, S[{flat(src)}])" if expr is None else f"__fmaf_rn({m}, S[{flat(src)}], {expr})"
        body.append(f"  S[{k}] = {expr};")
    for m, e in sorted(scaled.items()):
        lines.append(f"  const float {m} = {e};")
    lines += body
    lines.append("}")
    return "\n".join(lines)


def emit_eval_df(L):
    """The same recurrences in double-float arithmetic (gmp_f2, FP32 pairs):
    products of a coordinate and a lower component, integer coefficients
    applied exactly enough by gmp_df_mul_f, sums by gmp_df_add."""
    name = f"gmp_mcsh_indep_df_{L}"
    lines = [f"__device__ __forceinline__ void {name}(gmp_f2 x, gmp_f2 y, gmp_f2 z, gmp_f2 r2, gmp_f2* __restrict__ S) {{"]
    for l in range(L + 1):
        for t in indep_components(l):
            k = flat(t)
            rec = recurrence_terms(t)
            if rec[0][1] == "1":
                lines.append(f"  S[{k}] = gmp_f2{{1.0f, 0.0f}};")
                continue
            expr = None
            for coef, kind, src in rec:
                v = "r2" if kind == "r2" else kind
                prod = f"gmp_df_mul({v}, S[{flat(src)}])"
                term = prod if coef == 1 else f"gmp_df_mul_f({prod}, {fnum(coef)})"
                expr = term if expr is None else f"gmp_df_add({term}, {expr})"
            lines.append(f"  S[{k}] = {expr};")
    lines.append("}")
    return "\n".join(lines)


def emit_feature_df(l):
    """f = sum_all w mu_all^2 from the 2l+1 independent moments, double-float."""
    T_ = reconstruction(l)

    def combo_expr(combo):
        e = None
        for k, v in sorted(combo.items()):
            term = f"mu[{k}]" if v == 1 else f"gmp_df_mul_f(mu[{k}], {fnum(v)})"
            e = term if e is None else f"gmp_df_add({term}, {e})"
        return e

    lines = [f"__device__ __forceinline__ gmp_f2 gmp_mcsh_invariant_df_{l}(const gmp_f2* __restrict__ mu) {{",
             "  gmp_f2 f{0.0f, 0.0f};"]
    for t in all_components(l):
        lines.append(f"  {{ const gmp_f2 m = {combo_expr(T_[t])}; "
                     f"f = gmp_df_add(gmp_df_mul(gmp_df_mul_f(m, {fnum(weight(*t))}), m), f); }}")
    lines += ["  return f;", "}"]
    return "\n".join(lines)


def emit_feature(l, dtype="float"):
    """f = sum_all w mu_all^2 from the 2l+1 independent moments, and the
    adjoint lam_k = g * df/dmu_k (float only)."""
    d = dtype == "double"
    T = "double" if d else "float"
    mul = "__dmul_rn" if d else "__fmul_rn"
    fma = "__fma_rn" if d else "__fmaf_rn"
    lit = (lambda v: f"{float(v)!r}") if d else fnum
    sfx = "_d" if d else ""
    ind = indep_components(l)
    T_ = reconstruction(l)

    def combo_expr(combo):
        e = None
        for k, v in sorted(combo.items()):
            term = f"mu[{k}]" if v == 1 else (f"-mu[{k}]" if v == -1 else f"{mul}({lit(v)}, mu[{k}])")
            if e is None:
                e = term
            else:
                e = f"{fma}({lit(v)}, mu[{k}], {e})"
        return e

    lines = [f"__device__ __forceinline__ {T} gmp_mcsh_invariant{sfx}_{l}(const {T}* __restrict__ mu) {{",
             f"  {T} f = {lit(0)};"]
    for t in all_components(l):
        # (w m) m + f: one rounding where m^2 would be subnormal, instead of
        # w times a rounded subnormal square
        lines.append(f"  {{ const {T} m = {combo_expr(T_[t])}; f = {fma}({mul}({lit(weight(*t))}, m), m, f); }}")
    lines += ["  return f;", "}"]
    if d:
        return "\n".join(lines)
    lines.append(f"__device__ __forceinline__ void gmp_mcsh_invariant_adjoint_{l}("
                 f"const float* __restrict__ mu, float g, float* __restrict__ lam) {{")
    for k in range(len(ind)):
        lines.append(f"  lam[{k}] = 0.0f;")
    for t in all_components(l):
        lines.append(f"  {{ const float m = __fmul_rn({fnum(2 * weight(*t))}, __fmul_rn(g, {combo_expr(T_[t])}));")
        for k, v in sorted(T_[t].items()):
            lines.append(f"    lam[{k}] = __fmaf_rn({fnum(v)}, m, lam[{k}]);")
        lines.append("  }")
    lines.append("}")
    return "\n".join(lines)


def emit_shift_contract_order(l):
    """Same contraction restricted to the components of one order l
    (lam is indexed by the flat independent index)."""
    lines = [f"__device__ __forceinline__ void gmp_mcsh_shift_contract_order_{l}("
             f"const float* __restrict__ lam, const float* __restrict__ S1, float* __restrict__ V) {{",
             "  float vx = 0.0f, vy = 0.0f, vz = 0.0f;"]
    for t in indep_components(l):
        k = flat(t)
        a, b, c = t
        def ref(u):
            if u[0] <= 1:
                return f"S1[{flat(u)}]"
            return f"__fsub_rn(-S1[{flat((0, u[1] + 2, u[2]))}], S1[{flat((0, u[1], u[2] + 2))}])"
        lines.append(f"  vx = __fmaf_rn(lam[{k}], {ref((a + 1, b, c))}, vx);")
        lines.append(f"  vy = __fmaf_rn(lam[{k}], {ref((a, b + 1, c))}, vy);")
        lines.append(f"  vz = __fmaf_rn(lam[{k}], {ref((a, b, c + 1))}, vz);")
    lines += ["  V[0] = vx; V[1] = vy; V[2] = vz;", "}"]
    return "\n".join(lines)


def emit_shift_contract(L):
    """V_v = sum_k lam[k] * S_{k + e_v} for every independent component k of
    orders 0..L, v in (x, y, z), given S1 = independent components of orders
    0..L+1.  Raising a = 1 along x gives the dependent S_{2,b,c}, rebuilt as
    -S_{0,b+2,c} - S_{0,b,c+2}.  Used with r^2 dS_k/dv = (2l+1) v S_k - S_{k+e_v}
    (differentiate (-1)^l r^(2l+1) d^abc(1/r) once more)."""
    lines = [f"__device__ __forceinline__ void gmp_mcsh_shift_contract_{L}("
             f"const float* __restrict__ lam, const float* __restrict__ S1, float* __restrict__ V) {{",
             "  float vx = 0.0f, vy = 0.0f, vz = 0.0f;"]
    for l in range(L + 1):
        for t in indep_components(l):
            k = flat(t)
            a, b, c = t
            def ref(u):
                if u[0] <= 1:
                    return f"S1[{flat(u)}]"
                # a == 2: dependent
                return f"__fsub_rn(-S1[{flat((0, u[1] + 2, u[2]))}], S1[{flat((0, u[1], u[2] + 2))}])"
            lines.append(f"  vx = __fmaf_rn(lam[{k}], {ref((a + 1, b, c))}, vx);")
            lines.append(f"  vy = __fmaf_rn(lam[{k}], {ref((a, b + 1, c))}, vy);")
            lines.append(f"  vz = __fmaf_rn(lam[{k}], {ref((a, b, c + 1))}, vz);")
    lines += ["  V[0] = vx; V[1] = vy; V[2] = vz;", "}"]
    return "\n".join(lines)


def check_shift_identity():
    """r^2 dS/dv == (2l+1) v S - S_{+v} for all components up to LMAX."""
    def deriv(p, ax):
        out = {}
        for m, v in p.items():
            if m[ax]:
                mm = list(m); mm[ax] -= 1
                out[tuple(mm)] = out.get(tuple(mm), 0) + v * m[ax]
        return {m: v for m, v in out.items() if v}
    for l in range(LMAX + 1):
        for t in all_components(l):
            S = closed_form(*t)
            for ax in range(3):
                up = list(t); up[ax] += 1
                lhs = pmul(R2, deriv(S, ax))
                unit = [0, 0, 0]; unit[ax] = 1
                rhs = padd((2 * l + 1, pmul(S, {tuple(unit): 1})), (-1, closed_form(*up)))
                assert lhs == rhs, (t, ax)


def generate() -> str:
    check_shift_identity()
    check_recurrences()
    check_reconstruction()
    out = [
        "// Generated by gen_mcsh.py -- do not edit.  MCSH angular probes (independent",
        "// components a <= 1 of each order), their gradients, and the per-order",
        "// rotation invariant with its adjoint.  See gen_mcsh.py for the derivation.",
        "#pragma once",
        f"#define GMP_MCSH_LMAX {LMAX}",
        "",
    ]
    for L in range(LMAX + 2):
        out.append(emit_eval_scaled(L))
    for L in range(1, LMAX + 2):
        out.append(emit_eval_top(L))
    for L in range(LMAX + 1):
        out.append(emit_eval_df(L))
    for l in range(LMAX + 1):
        out.append(emit_feature(l))
        out.append(emit_feature_df(l))
    for L in range(LMAX + 1):
        out.append(emit_shift_contract(L))
    for l in range(LMAX + 1):
        out.append(emit_shift_contract_order(l))
    out.append("")
    out.append("template <int L> struct GmpMcsh;")
    for L in range(LMAX + 2):
        extra = ""
        if L <= LMAX:
            extra = (f"  static __device__ __forceinline__ void shift_contract(const float* lam, const float* S1,"
                     f" float* V) {{ gmp_mcsh_shift_contract_{L}(lam, S1, V); }}\n")
        out.append(
            f"template <> struct GmpMcsh<{L}> {{\n"
            f"  static constexpr int kInd = {nind(L)};\n"
            f"  static __device__ __forceinline__ void eval(float x, float y, float z, float r2, float* S) "
            f"{{ gmp_mcsh_indep_{L}(x, y, z, r2, S); }}\n"
            + (f"  static __device__ __forceinline__ void eval_top(float x, float y, float z, float r2, float* S) "
               f"{{ gmp_mcsh_top_{L}(x, y, z, r2, S); }}\n" if L >= 1 else "")
            + extra +
            f"}};")
    out.append("")
    out.append("__device__ __forceinline__ float gmp_mcsh_invariant(int l, const float* mu) {")
    out.append("  switch (l) {")
    for l in range(LMAX + 1):
        out.append(f"    case {l}: return gmp_mcsh_invariant_{l}(mu);")
    out.append("    default: return 0.0f;\n  }\n}")
    out.append("__device__ __forceinline__ gmp_f2 gmp_mcsh_invariant_df(int l, const gmp_f2* mu) {")
    out.append("  switch (l) {")
    for l in range(LMAX + 1):
        out.append(f"    case {l}: return gmp_mcsh_invariant_df_{l}(mu);")
    out.append("    default: return gmp_f2{0.0f, 0.0f};\n  }\n}")
    out.append("// independent components of orders 0..l in double-float arithmetic (l <= L of the caller)")
    out.append("__device__ __forceinline__ void gmp_mcsh_indep_df(int l, gmp_f2 x, gmp_f2 y, gmp_f2 z, gmp_f2 r2, gmp_f2* S) {")
    out.append("  switch (l) {")
    for l in range(LMAX + 1):
        out.append(f"    case {l}: gmp_mcsh_indep_df_{l}(x, y, z, r2, S); break;")
    out.append("    default: break;\n  }\n}")
    out.append("__device__ __forceinline__ void gmp_mcsh_shift_contract_order(int l, const float* lam, const float* S1, float* V) {")
    out.append("  switch (l) {")
    for l in range(LMAX + 1):
        out.append(f"    case {l}: gmp_mcsh_shift_contract_order_{l}(lam, S1, V); break;")
    out.append("    default: V[0] = V[1] = V[2] = 0.0f; break;\n  }\n}")
    out.append("__device__ __forceinline__ void gmp_mcsh_invariant_adjoint(int l, const float* mu, float g, float* lam) {")
    out.append("  switch (l) {")
    for l in range(LMAX + 1):
        out.append(f"    case {l}: gmp_mcsh_invariant_adjoint_{l}(mu, g, lam); break;")
    out.append("    default: break;\n  }\n}")
    return "\n".join(out) + "\n"


def main():
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "mcsh_gen.cuh")
    text = generate()
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
