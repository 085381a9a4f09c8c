"""Generate the unrolled moment transforms used by the CUDA kernels.

The non-orthogonal moment set of Eq. e11 is built from raw moments
k_abc = sum_i f_i e_ix^a e_iy^b e_iz^c (Eq. e2) with a, b, c in {0, 1, 2}, plus the
three second-order combinations k200+k020+k002, k200-k020, k200-k002.  Because
every velocity component is -1, 0 or +1, the raw moments factor into three
passes of 1D sums (along z, then y, then x), each turning a triple
(g-, g0, g+) into (g- + g0 + g+, g+ - g-, g+ + g-).  That is 3 adds per triple,
85 adds for the full D3Q27 M instead of the 312 of a row-by-row product with
the 339 non-zeros of Table I.  The inverse runs the three passes backwards
(g+ = (s2 + s1)/2, g- = (s2 - s1)/2, g0 = s0 - s2).  For D3Q19 the missing
corner populations and the eight moments App. C drops are zero; zero terms are
pruned symbolically, and App. C's statement that the D3Q19 M^-1 is the D3Q27
M^-1 restricted makes the pruned inverse exact.

The script checks exactly (rational arithmetic) that the emitted forward code
equals M built from Eq. e11 and that inverse(forward) is the identity, then
writes transform_q19.cuh and transform_q27.cuh next to itself:

    python paper_2306_16274_gb300/csrc/gen_transform.py
"""
import os
from fractions import Fraction

# Eq. e1 ordering (the D3Q19 set is the first 19 entries)
EX = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1)
EY = (0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1)
EZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1)

# Eq. e11 as raw-moment exponents; the three combined second-order moments are marked
MOMENTS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
           "trace", "dxy", "dxz",
           (1, 2, 0), (1, 0, 2), (2, 1, 0), (2, 0, 1), (0, 1, 2), (0, 2, 1), (1, 1, 1),
           (2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1), (1, 1, 2),
           (1, 2, 2), (2, 1, 2), (2, 2, 1), (2, 2, 2)]
KEEP19 = list(range(16)) + [17, 18, 19]


class Emitter:
    """Straight-line code over named values; each value also carries its exact linear form."""

    def __init__(self, prefix):
        self.lines = []
        self.forms = {}      # name -> {basis index: Fraction}
        self.prefix = prefix
        self.n = 0
        self.by_form = {}

    def leaf(self, name, idx):
        self.forms[name] = {idx: Fraction(1)}
        return name

    def _new(self, form, expr):
        key = tuple(sorted(form.items()))
        if not form:
            return None
        if key in self.by_form:
            return self.by_form[key]
        name = f"{self.prefix}{self.n}"
        self.n += 1
        self.lines.append(f"const float {name} = {expr};")
        self.forms[name] = form
        self.by_form[key] = name
        return name

    @staticmethod
    def _comb(*terms):
        out = {}
        for c, f in terms:
            if f is None:
                continue
            for k, v in f.items():
                out[k] = out.get(k, Fraction(0)) + c * v
        return {k: v for k, v in out.items() if v != 0}

    def add(self, a, b):
        if a is None:
            return b
        if b is None:
            return a
        return self._new(self._comb((1, self.forms[a]), (1, self.forms[b])), f"{a} + {b}")

    def sub(self, a, b):
        if b is None:
            return a
        if a is None:
            return self._new(self._comb((-1, self.forms[b])), f"-{b}")
        return self._new(self._comb((1, self.forms[a]), (-1, self.forms[b])), f"{a} - {b}")

    def half_add(self, a, b, sign):
        """0.5 * a + sign * 0.5 * b."""
        fa = self.forms[a] if a is not None else None
        fb = self.forms[b] if b is not None else None
        form = self._comb((Fraction(1, 2), fa), (Fraction(sign, 2), fb))
        if a is None and b is None:
            return None
        if a is None:
            return self._new(form, f"{'' if sign > 0 else '-'}0.5f * {b}")
        if b is None:
            return self._new(form, f"0.5f * {a}")
        return self._new(form, f"0.5f * ({a} {'+' if sign > 0 else '-'} {b})")

    def scale(self, a, num, den, text):
        if a is None:
            return None
        return self._new(self._comb((Fraction(num, den), self.forms[a])), f"{a} * {text}")


def forward(Q):
    em = Emitter("a")
    pops = {}
    for i in range(Q):
        pops[(EX[i], EY[i], EZ[i])] = em.leaf(f"f[{i}]", i)

    def tri(get):
        gm, g0, gp = get(-1), get(0), get(1)
        s = em.add(gp, gm)
        return [em.add(s, g0), em.sub(gp, gm), s]

    tz = {(x, y): tri(lambda z: pops.get((x, y, z))) for x in (-1, 0, 1) for y in (-1, 0, 1)}
    ty = {(x, c): tri(lambda y: tz[(x, y)][c]) for x in (-1, 0, 1) for c in range(3)}
    k = {(a, b, c): tri(lambda x: ty[(x, c)][b])[a] for a in range(3) for b in range(3) for c in range(3)}
    outs = []
    for mk in range(27):
        d = MOMENTS[mk]
        if d == "trace":
            v = em.add(em.add(k[(2, 0, 0)], k[(0, 2, 0)]), k[(0, 0, 2)])
        elif d == "dxy":
            v = em.sub(k[(2, 0, 0)], k[(0, 2, 0)])
        elif d == "dxz":
            v = em.sub(k[(2, 0, 0)], k[(0, 0, 2)])
        else:
            v = k[d]
        outs.append(v)
    keep = list(range(27)) if Q == 27 else KEEP19
    return em, [outs[j] for j in keep]


def inverse(Q):
    em = Emitter("b")
    keep = list(range(27)) if Q == 27 else KEEP19
    m = {mk: None for mk in range(27)}
    for pos, mk in enumerate(keep):
        m[mk] = em.leaf(f"m[{pos}]", pos)
    # second-order raw moments from (trace, dxy, dxz): k200 = (T + Dxy + Dxz)/3
    k200 = em.scale(em.add(em.add(m[7], m[8]), m[9]), 1, 3, "(1.0f / 3.0f)")
    k020 = em.sub(k200, m[8])
    k002 = em.sub(k200, m[9])
    k = {}
    for mk in range(27):
        d = MOMENTS[mk]
        if isinstance(d, tuple):
            k[d] = m[mk]
    k[(2, 0, 0)], k[(0, 2, 0)], k[(0, 0, 2)] = k200, k020, k002

    def itri(s0, s1, s2):
        return {1: em.half_add(s2, s1, +1), -1: em.half_add(s2, s1, -1), 0: em.sub(s0, s2)}

    ty = {}
    for b in range(3):
        for c in range(3):
            r = itri(k[(0, b, c)], k[(1, b, c)], k[(2, b, c)])
            for x in (-1, 0, 1):
                ty[(x, b, c)] = r[x]
    tz = {}
    for x in (-1, 0, 1):
        for c in range(3):
            r = itri(ty[(x, 0, c)], ty[(x, 1, c)], ty[(x, 2, c)])
            for y in (-1, 0, 1):
                tz[(x, y, c)] = r[y]
    f = {}
    for x in (-1, 0, 1):
        for y in (-1, 0, 1):
            r = itri(tz[(x, y, 0)], tz[(x, y, 1)], tz[(x, y, 2)])
            for z in (-1, 0, 1):
                f[(x, y, z)] = r[z]
    return em, [f[(EX[i], EY[i], EZ[i])] for i in range(Q)]


def prune(em, outs):
    """Keep only the lines the outputs depend on."""
    need = set(o for o in outs if o is not None)
    kept = []
    for line in reversed(em.lines):
        name = line.split()[2]
        if name in need:
            kept.append(line)
            rhs = line.split("=", 1)[1]
            for tok in rhs.replace("(", " ").replace(")", " ").replace(";", " ").replace("-", " ").split():
                if tok.startswith(em.prefix):
                    need.add(tok)
    return list(reversed(kept))


def matrix_from_definitions(Q):
    M = []
    for mk in (range(27) if Q == 27 else KEEP19):
        d = MOMENTS[mk]
        row = []
        for i in range(Q):
            ex, ey, ez = EX[i], EY[i], EZ[i]
            if d == "trace":
                v = ex * ex + ey * ey + ez * ez
            elif d == "dxy":
                v = ex * ex - ey * ey
            elif d == "dxz":
                v = ex * ex - ez * ez
            else:
                v = ex ** d[0] * ey ** d[1] * ez ** d[2]
            row.append(Fraction(v))
        M.append(row)
    return M


def check(Q, fem, fouts, iem, iouts):
    M = matrix_from_definitions(Q)
    for r, name in enumerate(fouts):
        form = fem.forms[name] if name is not None else {}
        assert all(form.get(i, 0) == M[r][i] for i in range(Q)), f"forward row {r} wrong"
    # inverse(forward) = identity: compose the linear forms exactly
    Minv = [[iem.forms[name].get(j, Fraction(0)) if name is not None else Fraction(0) for j in range(Q)]
            for name in iouts]
    for a in range(Q):
        for b in range(Q):
            s = sum(M[a][i] * Minv[i][b] for i in range(Q))
            assert s == (1 if a == b else 0), f"M Minv != I at ({a},{b})"
    return M, Minv


def emit(Q):
    fem, fouts = forward(Q)
    iem, iouts = inverse(Q)
    check(Q, fem, fouts, iem, iouts)
    flines = prune(fem, fouts)
    ilines = prune(iem, iouts)
    out = [f"// Unrolled non-orthogonal moment transforms for D3Q{Q}.",
           "// Generated by gen_transform.py (factorised raw-moment sums, exactness checked",
           "// against M built from Eq. e11 in rational arithmetic). Do not edit by hand.",
           "#pragma once", "",
           f"// m = M f   ({len(flines) + sum(1 for o in fouts if o and not o.startswith('a'))} lines)",
           f"__device__ __forceinline__ void moments_from_pops_q{Q}(const float (&f)[{Q}], float (&m)[{Q}]) {{"]
    out += ["    " + ln for ln in flines]
    for r, name in enumerate(fouts):
        out.append(f"    m[{r}] = {name if name is not None else '0.0f'};")
    out += ["}", "",
            f"// f = M^-1 m",
            f"__device__ __forceinline__ void pops_from_moments_q{Q}(const float (&m)[{Q}], float (&f)[{Q}]) {{"]
    out += ["    " + ln for ln in ilines]
    for i, name in enumerate(iouts):
        out.append(f"    f[{i}] = {name if name is not None else '0.0f'};")
    out += ["}", ""]
    return "\n".join(out), len(flines), len(ilines)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for Q in (19, 27):
        text, nf, ni = emit(Q)
        with open(os.path.join(here, f"transform_q{Q}.cuh"), "w") as fh:
            fh.write(text)
        print(f"D3Q{Q}: forward {nf} ops, inverse {ni} ops")


if __name__ == "__main__":
    main()
