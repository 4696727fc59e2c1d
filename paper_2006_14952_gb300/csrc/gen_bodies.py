"""Write gen_bodies.cuh: straight-line expansion code for orders 1..8.

M2L (M2LBody, M2LLoad, M2LSlices) is described first; P2M, M2M, L2L and L2P
bodies follow at the end of this docstring.

For each order P and output slice g of G, the generated device function takes,
for one (sink, source) pair, the unit separation vector R^ (rx, ry, rz), the
radial prefactors f[0..P] at r^ = 1, the sink factors U[k] = u^(k+1) and the
source multipoles already scaled by v^|m| (Mp), and adds
    acc[n / G] += U[|n|] * sum_m Mp[m] * D^_{n+m}(R^)     (n = g mod G)
with D^_c = sum_{k_d <= c_d/2} prod_d [c_d!/(2^k_d k_d! (c_d-2k_d)!)] R^^(c-2k) f[|c|-|k|]
(the Cartesian derivatives of a radial function, Sec. 2.2 prefactors).  Every
index is a literal, so the arrays live in registers.  Multi-index order: graded,
nx descending, ny descending.

P2MBody<P>:  acc[c] += m u^c for one particle (u = offset / h); finish() applies
             (-1)^|c| / c!  (Eq. p2m, scaled M~ = M / h^|m|).
M2MBody<P>:  out[m] += sum_{n <= m} (x/H)^n / n! 2^-(|m|-|n|) in[m-n] for one
             child, x/H = (sx, sy, sz) / 4, s = +-1 (Eq. m2m, scaled).
L2LBody<P>:  out[n] = 2^-(|n|+1) sum_{|m| <= P-|n|} (x/H)^m / m! Lp[m+n] for one
             child, x/H = (sx, sy, sz) / 4 (Eq. l2l, scaled L~ = L h^(|n|+1)).
L2PBody<P>:  a_d += sum_{|n| <= P-1} Lk[n+e_d] u^n / n! (Eq. l2p gradient).
M2MGenBody<P>: out[m] += sum_{n <= m} d^n / n! rho^(|m|-|n|) in[m-n] for any
             offset d = (z_P - z_C) / H and scale ratio rho = h / H of child
             and parent (the k-d tree's boxes; Eq. m2m, scaled).
L2LGenBody<P>: out[n] += rho^(|n|+1) sum_{|m| <= P-|n|} d^m / m! Lp[m+n],
             d = (z_C - z_P) / H, rho = h / H (Eq. l2l, scaled).
M2LTabBody<P, G, g>: acc[n / G] += sum_m T[n+m] Mp[m] for one pair whose scaled
             operator T_c = D_c h^(|c|+1) comes from the (level, offset) table.
TCStore<P>:  tensor-core M2L operands for one pair: D'_c = u^(|c|+1) D^_c(R^) and
             M'_m = s (v/u)^|m| M~_m, each split x = hi + lo (hi = TF32 rounding),
             stored at row c (or m), column k of K-major 128-byte-swizzled tiles
             (xo[j] = float offset of column k in a row with (row mod 8) = j).
TCStoreBF<P>: the same operands split into BF16 hi = bf16(x), lo = bf16(x - hi),
             64 BF16 columns per 128-byte row.

Run by build.py before nvcc (python3 gen_bodies.py <out>).
"""
from __future__ import annotations

import sys
from math import factorial

SLICES = {1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 2, 8: 8}  # per-pair operator (registers: D and the contraction)
TAB_SLICES = {1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 2, 8: 4}  # table operator (contraction only)
MP_IN_SMEM = {7, 8}  # source multipoles staged per lane in shared memory (register budget)


def ncoef(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def multi(P):
    out = []
    for k in range(P + 1):
        for nx in range(k, -1, -1):
            for ny in range(k - nx, -1, -1):
                out.append((nx, ny, k - nx - ny))
    return out


def idx(n):
    x, y, z = n
    k = x + y + z
    j = y + z
    return (k * (k + 1) * (k + 2)) // 6 + j * (j + 1) // 2 + z


def hco(n, k):
    return factorial(n) // (2 ** k * factorial(k) * factorial(n - 2 * k))


def mono_name(a):
    return "m_%d_%d_%d" % a


def gen_body(P, G, g):
    smem = P in MP_IN_SMEM
    L = []
    mp = (lambda e: f"Mp[{e} * 32]") if smem else (lambda e: f"Mp[{e}]")
    sig_mp = "const float *__restrict__ Mp" if smem else f"const float (&Mp)[{ncoef(P)}]"
    L.append(f"template <> struct M2LBody<{P}, {G}, {g}> {{")
    L.append(f"  static __device__ __forceinline__ void run(float rx, float ry, float rz, const float (&f)[{P + 1}],"
             f" const float (&U)[{P + 1}], {sig_mp}, float (&acc)[{(ncoef(P) + G - 1) // G}]) {{")
    ms = multi(P)
    outs = [n for n in ms if idx(n) % G == g]
    need_c = [c for c in ms if any(all(n[d] <= c[d] for d in range(3)) for n in outs)]
    # monomials R^^a needed by the D terms
    need_m = set()
    for c in need_c:
        for kx in range(c[0] // 2 + 1):
            for ky in range(c[1] // 2 + 1):
                for kz in range(c[2] // 2 + 1):
                    need_m.add((c[0] - 2 * kx, c[1] - 2 * ky, c[2] - 2 * kz))
    # close under the "parent" relation used to build them incrementally
    def parent(a):
        if a[2] > 0:
            return (a[0], a[1], a[2] - 1), "rz"
        if a[1] > 0:
            return (a[0], a[1] - 1, a[2]), "ry"
        return (a[0] - 1, a[1], a[2]), "rx"
    todo = sorted(need_m, key=lambda a: sum(a))
    have = {(0, 0, 0)}
    full = set()
    for a in todo:
        chain = []
        b = a
        while b not in have and b != (0, 0, 0):
            chain.append(b)
            b = parent(b)[0]
        for b in reversed(chain):
            full.add(b)
            have.add(b)
    for a in sorted(full, key=lambda a: (sum(a), -a[0], -a[1])):
        p, v = parent(a)
        src = "1.f" if p == (0, 0, 0) else mono_name(p)
        L.append(f"    const float {mono_name(a)} = {src} * {v};" if p != (0, 0, 0) else
                 f"    const float {mono_name(a)} = {v};")

    def mono(a):
        return "1.f" if a == (0, 0, 0) else mono_name(a)

    for c in need_c:
        ci = idx(c)
        cn = sum(c)
        terms = []
        for kx in range(c[0] // 2 + 1):
            for ky in range(c[1] // 2 + 1):
                for kz in range(c[2] // 2 + 1):
                    co = hco(c[0], kx) * hco(c[1], ky) * hco(c[2], kz)
                    a = (c[0] - 2 * kx, c[1] - 2 * ky, c[2] - 2 * kz)
                    o = cn - kx - ky - kz
                    terms.append((co, a, o))
        parts = []
        for co, a, o in terms:
            t = f"f[{o}]" if a == (0, 0, 0) else f"{mono(a)} * f[{o}]"
            parts.append(t if co == 1 else f"{float(co)}f * {t}")
        expr = " + ".join(parts)
        # D'_c = u^(|c|+1) D^_c; with the sources scaled by (v/u)^|m| every term
        # D'_{n+m} M''_m carries u^(|n|+1) v^|m|: one FMA per term
        L.append(f"    const float D{ci} = U[{cn}] * ({expr});")
        for n in outs:
            if all(n[d] <= c[d] for d in range(3)):
                m = (c[0] - n[0], c[1] - n[1], c[2] - n[2])
                a = idx(n) // G
                L.append(f"    acc[{a}] = fmaf(D{ci}, {mp(idx(m))}, acc[{a}]);")
    L.append("  }")
    L.append("};")
    return "\n".join(L)


def _monomials(P, var, L, prefix="u", include_fact=False):
    """Emit u^a (or u^a / a!) for all |a| <= P as named floats; returns name(a)."""
    names = {}
    for a in multi(P):
        nm = f"{prefix}_{a[0]}_{a[1]}_{a[2]}"
        if a == (0, 0, 0):
            names[a] = "1.f"
            continue
        if a[2] > 0:
            p, v, k = (a[0], a[1], a[2] - 1), var[2], a[2]
        elif a[1] > 0:
            p, v, k = (a[0], a[1] - 1, a[2]), var[1], a[1]
        else:
            p, v, k = (a[0] - 1, a[1], a[2]), var[0], a[0]
        src = names[p]
        if include_fact:
            L.append(f"    const float {nm} = {src} * {v} * {1.0 / k!r}f;")
        else:
            L.append(f"    const float {nm} = {src} * {v};" if src != "1.f" else f"    const float {nm} = {v};")
        names[a] = nm
    return names


def gen_passes(P):
    NC = ncoef(P)
    ms = multi(P)
    out = []
    # ---- P2M
    L = [f"template <> struct P2MBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float ux, float uy, float uz, float m, float (&acc)[{NC}]) {{"]
    nm = _monomials(P, ("ux", "uy", "uz"), L)
    for a in ms:
        c = idx(a)
        L.append(f"    acc[{c}] = fmaf(m, {nm[a]}, acc[{c}]);" if a != (0, 0, 0) else f"    acc[{c}] += m;")
    L.append("  }")
    L.append(f"  static __device__ __forceinline__ void finish(float (&acc)[{NC}]) {{")
    for a in ms:
        co = (-1) ** sum(a) / (factorial(a[0]) * factorial(a[1]) * factorial(a[2]))
        if co != 1.0:
            L.append(f"    acc[{idx(a)}] *= {co!r}f;")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    # ---- M2M
    L = [f"template <> struct M2MBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float sx, float sy, float sz, const float (&in)[{NC}],"
         f" float (&o)[{NC}]) {{"]
    for a in ms:
        k = idx(a)
        L.append(f"    const float i{k} = in[{k}] * {2.0 ** -sum(a)!r}f;")
    for a in ms:
        if a == (0, 0, 0):
            continue
        co = 0.25 ** sum(a) / (factorial(a[0]) * factorial(a[1]) * factorial(a[2]))
        sg = "".join(f" * {v}" for v, e in zip(("sx", "sy", "sz"), a) if e % 2)
        L.append(f"    const float w{idx(a)} = {co!r}f{sg};")
    for m in ms:
        terms = []
        for n in ms:
            if all(n[d] <= m[d] for d in range(3)):
                r = (m[0] - n[0], m[1] - n[1], m[2] - n[2])
                terms.append(f"i{idx(r)}" if n == (0, 0, 0) else f"w{idx(n)} * i{idx(r)}")
        L.append(f"    o[{idx(m)}] += " + " + ".join(terms) + ";")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    # ---- L2L
    L = [f"template <> struct L2LBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float sx, float sy, float sz, const float (&p)[{NC}],"
         f" float (&child)[{NC}]) {{"]
    for a in ms:
        if a == (0, 0, 0):
            continue
        co = 0.25 ** sum(a) / (factorial(a[0]) * factorial(a[1]) * factorial(a[2]))
        sg = "".join(f" * {v}" for v, e in zip(("sx", "sy", "sz"), a) if e % 2)
        L.append(f"    const float w{idx(a)} = {co!r}f{sg};")
    for n in ms:
        terms = []
        for m in ms:
            if sum(m) + sum(n) <= P:
                q = (m[0] + n[0], m[1] + n[1], m[2] + n[2])
                terms.append(f"p[{idx(q)}]" if m == (0, 0, 0) else f"w{idx(m)} * p[{idx(q)}]")
        L.append(f"    child[{idx(n)}] += {2.0 ** -(sum(n) + 1)!r}f * (" + " + ".join(terms) + ");")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    # ---- M2M, any offset and scale ratio
    L = [f"template <> struct M2MGenBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float dx, float dy, float dz, float rho,"
         f" const float (&in)[{NC}], float (&o)[{NC}]) {{",
         "    float rp = 1.f;"]
    for k in range(P + 1):
        for a in ms:
            if sum(a) == k:
                L.append(f"    const float i{idx(a)} = in[{idx(a)}] * rp;" if k else f"    const float i{idx(a)} = in[{idx(a)}];")
        if k < P:
            L.append("    rp *= rho;")
    nm = _monomials(P, ("dx", "dy", "dz"), L, prefix="w", include_fact=True)
    for m in ms:
        terms = []
        for n in ms:
            if all(n[d] <= m[d] for d in range(3)):
                r = (m[0] - n[0], m[1] - n[1], m[2] - n[2])
                terms.append(f"i{idx(r)}" if n == (0, 0, 0) else f"{nm[n]} * i{idx(r)}")
        L.append(f"    o[{idx(m)}] += " + " + ".join(terms) + ";")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    # ---- L2L, any offset and scale ratio
    L = [f"template <> struct L2LGenBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float dx, float dy, float dz, float rho,"
         f" const float (&p)[{NC}], float (&child)[{NC}]) {{"]
    nm = _monomials(P, ("dx", "dy", "dz"), L, prefix="w", include_fact=True)
    L.append("    float rp = rho;")
    for k in range(P + 1):
        for n in ms:
            if sum(n) != k:
                continue
            terms = []
            for m in ms:
                if sum(m) + sum(n) <= P:
                    q = (m[0] + n[0], m[1] + n[1], m[2] + n[2])
                    terms.append(f"p[{idx(q)}]" if m == (0, 0, 0) else f"{nm[m]} * p[{idx(q)}]")
            L.append(f"    child[{idx(n)}] += rp * (" + " + ".join(terms) + ");")
        if k < P:
            L.append("    rp *= rho;")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    # ---- L2P
    L = [f"template <> struct L2PBody<{P}> {{",
         f"  static __device__ __forceinline__ void run(float ux, float uy, float uz, const float (&l)[{NC}],"
         f" float &ax, float &ay, float &az) {{"]
    nm = _monomials(P - 1, ("ux", "uy", "uz"), L, prefix="t", include_fact=True) if P >= 1 else {}
    tx, ty, tz = [], [], []
    for a in multi(P - 1):
        t = nm[a]
        tx.append(f"{t} * l[{idx((a[0] + 1, a[1], a[2]))}]")
        ty.append(f"{t} * l[{idx((a[0], a[1] + 1, a[2]))}]")
        tz.append(f"{t} * l[{idx((a[0], a[1], a[2] + 1))}]")
    L.append("    ax += " + " + ".join(tx) + ";")
    L.append("    ay += " + " + ".join(ty) + ";")
    L.append("    az += " + " + ".join(tz) + ";")
    L.append("  }")
    L.append("};")
    out.append("\n".join(L))
    return "\n\n".join(out)


def gen_tab_body(P, G, g):
    """M2LTabBody<P, G, g>: acc[n / G] += sum_m T[n + m] Mp[m] for the outputs n = g mod G,
    with T one row of the (level, offset) operator table (16-byte aligned, read as float4)."""
    smem = P in MP_IN_SMEM
    mp = (lambda e: f"Mp[{e} * 32]") if smem else (lambda e: f"Mp[{e}]")
    sig_mp = "const float *__restrict__ Mp" if smem else f"const float (&Mp)[{ncoef(P)}]"
    L = [f"template <> struct M2LTabBody<{P}, {G}, {g}> {{",
         f"  static __device__ __forceinline__ void run(const float4 *__restrict__ T4, {sig_mp},"
         f" float (&acc)[{(ncoef(P) + G - 1) // G}]) {{"]
    ms = multi(P)
    outs = [n for n in ms if idx(n) % G == g]
    need_c = [c for c in ms if any(all(n[d] <= c[d] for d in range(3)) for n in outs)]
    loaded = set()
    for c in need_c:
        ci = idx(c)
        q = ci // 4
        if q not in loaded:
            L.append(f"    const float4 q{q} = __ldg(T4 + {q});")
            loaded.add(q)
        comp = "xyzw"[ci % 4]
        for n in outs:
            if all(n[d] <= c[d] for d in range(3)):
                m = (c[0] - n[0], c[1] - n[1], c[2] - n[2])
                a = idx(n) // G
                L.append(f"    acc[{a}] = fmaf(q{q}.{comp}, {mp(idx(m))}, acc[{a}]);")
    L.append("  }")
    L.append("};")
    return "\n".join(L)


def gen_tc(P, bf=False):
    NC = ncoef(P)
    ms = multi(P)
    T = "__nv_bfloat16" if bf else "float"
    row = 64 if bf else 32  # elements per 128-byte row

    def split(v, dst):
        if bf:
            return (f"const __nv_bfloat16 h = __float2bfloat16_rn({v}); hi[{dst}] = h;"
                    f" lo[{dst}] = __float2bfloat16_rn({v} - __bfloat162float(h));")
        return f"const float h = tf32_round({v}); hi[{dst}] = h; lo[{dst}] = {v} - h;"

    L = [f"template <> struct {'TCStoreBF' if bf else 'TCStore'}<{P}> {{",
         f"  static __device__ __forceinline__ void store_d(float rx, float ry, float rz, const float (&f)[{P + 1}],"
         f" const float (&U)[{P + 1}], {T} *__restrict__ hi, {T} *__restrict__ lo, const int (&xo)[8]) {{"]
    nm = {}
    for a in ms:
        if a == (0, 0, 0):
            nm[a] = "1.f"
            continue
        if a[2] > 0:
            p, v = (a[0], a[1], a[2] - 1), "rz"
        elif a[1] > 0:
            p, v = (a[0], a[1] - 1, a[2]), "ry"
        else:
            p, v = (a[0] - 1, a[1], a[2]), "rx"
        name = "m_%d_%d_%d" % a
        L.append(f"    const float {name} = {nm[p]} * {v};" if nm[p] != "1.f" else f"    const float {name} = {v};")
        nm[a] = name
    for c in ms:
        ci = idx(c)
        cn = sum(c)
        parts = []
        for kx in range(c[0] // 2 + 1):
            for ky in range(c[1] // 2 + 1):
                for kz in range(c[2] // 2 + 1):
                    co = hco(c[0], kx) * hco(c[1], ky) * hco(c[2], kz)
                    a = (c[0] - 2 * kx, c[1] - 2 * ky, c[2] - 2 * kz)
                    o = cn - kx - ky - kz
                    t = f"f[{o}]" if a == (0, 0, 0) else f"{nm[a]} * f[{o}]"
                    parts.append(t if co == 1 else f"{float(co)}f * {t}")
        off = (ci >> 3) * 8 * row + (ci & 7) * row
        L.append(f"    {{ const float d = U[{cn}] * ({' + '.join(parts)}); {split('d', f'{off} + xo[{ci & 7}]')} }}")
    L.append("  }")
    L.append(f"  static __device__ __forceinline__ void store_m(const float *__restrict__ Mb, float vr, float s,"
             f" {T} *__restrict__ hi, {T} *__restrict__ lo, const int (&xo)[8]) {{")
    L.append("    float q = s;")
    for k in range(P + 1):
        if k:
            L.append("    q *= vr;")
        for a in ms:
            if sum(a) != k:
                continue
            ci = idx(a)
            off = (ci >> 3) * 8 * row + (ci & 7) * row
            L.append(f"    {{ const float x = __ldg(Mb + {ci}) * q; {split('x', f'{off} + xo[{ci & 7}]')} }}")
    L.append("  }")
    L.append("};")
    return "\n".join(L)


def main(out):
    parts = ["// Generated by gen_bodies.py: do not edit.", "#pragma once", "", "#include <cuda_bf16.h>", "",
             "template <int P, int G, int g> struct M2LBody;", "template <int P> struct M2LLoad;",
             "template <int P, int G, int g> struct M2LTabBody;",
             "template <int P> struct P2MBody;", "template <int P> struct M2MBody;", "template <int P> struct L2LBody;",
             "template <int P> struct L2PBody;", "template <int P> struct M2MGenBody;",
             "template <int P> struct L2LGenBody;", "template <int P> struct TCStore;",
             "template <int P> struct TCStoreBF;", "",
             "__device__ __forceinline__ float tf32_round(float x) {",
             "  uint32_t r;",
             "  asm(\"cvt.rna.tf32.f32 %0, %1;\" : \"=r\"(r) : \"f\"(x));",
             "  return __uint_as_float(r);",
             "}", ""]
    for P in range(1, 9):
        G = SLICES[P]
        for g in range(G):
            parts.append(gen_body(P, G, g))
            parts.append("")
        for g in range(TAB_SLICES[P]):
            parts.append(gen_tab_body(P, TAB_SLICES[P], g))
            parts.append("")
    for P in range(1, 9):
        NC = ncoef(P)
        parts.append(f"template <> struct M2LLoad<{P}> {{")
        parts.append(f"  // dst[c * S] = Mb[c] * v^|c|; Mb is a 16-byte aligned row (float4 loads)")
        parts.append(f"  template <int S, class T> static __device__ __forceinline__ void run(const float *__restrict__ Mb,"
                     f" float v, T &dst) {{")
        parts.append("    const float4 *M4 = reinterpret_cast<const float4 *>(Mb);")
        parts.append("    const float v1 = v;")
        for k in range(2, P + 1):
            parts.append(f"    const float v{k} = v{k - 1} * v;")
        deg = [sum(a) for a in multi(P)]
        for j in range((NC + 3) // 4):
            parts.append(f"    const float4 q{j} = __ldg(M4 + {j});")
        for c in range(NC):
            comp = "q%d.%s" % (c // 4, "xyzw"[c % 4])
            parts.append(f"    dst[{c} * S] = {comp};" if deg[c] == 0 else f"    dst[{c} * S] = {comp} * v{deg[c]};")
        parts.append("  }")
        parts.append("};")
        parts.append("")
    for P in range(1, 9):
        parts.append(gen_passes(P))
        parts.append("")
    for P in range(1, 7):
        parts.append(gen_tc(P))
        parts.append("")
        parts.append(gen_tc(P, bf=True))
        parts.append("")
    g_expr = "1"
    for P in sorted(SLICES, reverse=True):
        if SLICES[P] != 1:
            g_expr = f"(P == {P} ? {SLICES[P]} : {g_expr})"
    s_expr = " || ".join(f"P == {P}" for P in sorted(MP_IN_SMEM)) or "false"
    parts.append("template <int P> struct M2LSlices { static constexpr int G = " + g_expr +
                 "; static constexpr bool kSmem = (" + s_expr + "); };")
    t_expr = "1"
    for P in sorted(TAB_SLICES, reverse=True):
        if TAB_SLICES[P] != 1:
            t_expr = f"(P == {P} ? {TAB_SLICES[P]} : {t_expr})"
    parts.append("template <int P> struct M2LTabSlices { static constexpr int G = " + t_expr + "; };")
    text = "\n".join(parts) + "\n"
    old = None
    try:
        old = open(out).read()
    except OSError:
        pass
    if old != text:
        open(out, "w").write(text)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "gen_bodies.cuh")
