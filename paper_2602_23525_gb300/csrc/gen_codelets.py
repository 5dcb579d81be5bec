"""Codelet generator: straight-line radix-R DFT butterflies for the CUDA kernels.

Follows the four phases of the paper's codelet compiler (sec. 5):

* creation  -- the DFT of size R is built symbolically as a linear network
  (a DAG of additions and multiplications by constants), from eq. (2)
  (Cooley-Tukey, recursively, for composite R) or from eq. (1) with the
  conjugate-pair symmetry (for odd prime R);
* simplification -- multiplications by 1, -1, +-i and the 1/sqrt(2) pairs of
  the eighth roots of unity are folded, and every node is hash-consed so equal
  sub-expressions are shared (common-subexpression elimination);
* scheduling -- nodes are emitted in a depth-first topological order from
  the outputs, which keeps live ranges short;
* unparsing -- to CUDA C++ (FP32, ``float2`` registers) and to plain C
  (FP64) for CPU verification of the generator.

Codelets compute the forward transform (w_R = exp(-2 pi i / R)) in place on
an array ``v[0..R-1]``: v_out[k] = sum_r v_in[r] w_R^{r k}.  The backward
transform is obtained by the kernels through conjugation.

Run as a script to (re)write ``codelets.cuh`` next to this file.
"""
from __future__ import annotations

import math
import os
import sys
from fractions import Fraction

RADICES = (2, 3, 4, 5, 7, 8, 9, 11, 13, 16)

# how each composite radix is split by eq. (2): R = n1 * n2
CT_SPLIT = {4: (2, 2), 8: (2, 4), 9: (3, 3), 16: (4, 4)}


class Dag:
    """Hash-consed DAG of real-valued nodes."""

    def __init__(self):
        self.nodes = []      # (op, args...)
        self.index = {}

    def _mk(self, key):
        if key in self.index:
            return self.index[key]
        self.nodes.append(key)
        self.index[key] = len(self.nodes) - 1
        return self.index[key]

    def inp(self, i, part):
        return self._mk(("in", i, part))

    def zero(self):
        return self._mk(("zero",))

    def is_zero(self, a):
        return self.nodes[a][0] == "zero"

    def neg(self, a):
        if self.is_zero(a):
            return a
        if self.nodes[a][0] == "neg":
            return self.nodes[a][1]
        return self._mk(("neg", a))

    def add(self, a, b):
        if self.is_zero(a):
            return b
        if self.is_zero(b):
            return a
        na, nb = self.nodes[a], self.nodes[b]
        if nb[0] == "neg":
            return self.sub(a, nb[1])
        if na[0] == "neg":
            return self.sub(b, na[1])
        if a > b:
            a, b = b, a
        return self._mk(("add", a, b))

    def sub(self, a, b):
        if self.is_zero(b):
            return a
        if self.is_zero(a):
            return self.neg(b)
        nb = self.nodes[b]
        if nb[0] == "neg":
            return self.add(a, nb[1])
        return self._mk(("sub", a, b))

    def mul(self, c, a):
        """c * a for a real constant c (given as an exact key and a float)."""
        if self.is_zero(a):
            return a
        key, val = c
        if val == 1.0:
            return a
        if val == -1.0:
            return self.neg(a)
        if val == 0.0:
            return self.zero()
        if val < 0:
            return self.neg(self._mk(("mul", (key[0], -val), a)))
        return self._mk(("mul", (key[0], val), a))


class Root:
    """w_R^e = exp(-2 pi i e / R) with exact classification of the angle."""

    def __init__(self, e, R):
        self.frac = Fraction(e % R, R)  # turns

    def value(self):
        f = self.frac
        table = {Fraction(0): (1.0, 0.0), Fraction(1, 4): (0.0, -1.0), Fraction(1, 2): (-1.0, 0.0),
                 Fraction(3, 4): (0.0, 1.0)}
        if f in table:
            return table[f]
        a = -2.0 * math.pi * float(f)
        return math.cos(a), math.sin(a)


def const(val):
    return (("c",), float(val))


def cmul_root(dag, root, x):
    """Multiply the complex value x = (re, im) by w = root, folding trivial cases."""
    c, s = root.value()
    xr, xi = x
    if s == 0.0:
        if c == 1.0:
            return x
        return dag.neg(xr), dag.neg(xi)
    if c == 0.0:
        if s == 1.0:   # * i
            return dag.neg(xi), xr
        return xi, dag.neg(xr)  # * (-i)
    if abs(abs(c) - abs(s)) < 1e-15:
        # eighth roots: w = |c| (sc + ss i) with signs sc, ss
        m = abs(c)
        sc = 1.0 if c > 0 else -1.0
        ss = 1.0 if s > 0 else -1.0
        # re = sc*m*xr - ss*m*xi = m*(sc*xr - ss*xi); im = m*(sc*xi + ss*xr)
        re = dag.add(xr if sc > 0 else dag.neg(xr), dag.neg(xi) if ss > 0 else xi)
        im = dag.add(xi if sc > 0 else dag.neg(xi), xr if ss > 0 else dag.neg(xr))
        return dag.mul(const(m), re), dag.mul(const(m), im)
    re = dag.sub(dag.mul(const(c), xr), dag.mul(const(s), xi))
    im = dag.add(dag.mul(const(c), xi), dag.mul(const(s), xr))
    return re, im


def cadd(dag, a, b):
    return dag.add(a[0], b[0]), dag.add(a[1], b[1])


def csub(dag, a, b):
    return dag.sub(a[0], b[0]), dag.sub(a[1], b[1])


def dft_sym(dag, x):
    """Length-R DFT of the list of complex nodes x (forward sign)."""
    R = len(x)
    if R == 1:
        return list(x)
    if R == 2:
        return [cadd(dag, x[0], x[1]), csub(dag, x[0], x[1])]
    if R in CT_SPLIT:
        n1, n2 = CT_SPLIT[R]
        # eq. (2): l = l1 n2 + l2, k = k1 + k2 n1
        inner = []
        for l2 in range(n2):
            sub = dft_sym(dag, [x[l1 * n2 + l2] for l1 in range(n1)])
            inner.append([cmul_root(dag, Root(l2 * k1, R), sub[k1]) for k1 in range(n1)])
        y = [None] * R
        for k1 in range(n1):
            outer = dft_sym(dag, [inner[l2][k1] for l2 in range(n2)])
            for k2 in range(n2):
                y[k1 + k2 * n1] = outer[k2]
        return y
    # odd prime R: conjugate-pair form of eq. (1)
    h = (R - 1) // 2
    t = [cadd(dag, x[j], x[R - j]) for j in range(1, h + 1)]
    u = [csub(dag, x[j], x[R - j]) for j in range(1, h + 1)]
    y = [None] * R
    s0 = x[0]
    for tj in t:
        s0 = cadd(dag, s0, tj)
    y[0] = s0
    for k in range(1, h + 1):
        ar, ai = x[0]
        br, bi = dag.zero(), dag.zero()
        for j in range(1, h + 1):
            ang = 2.0 * math.pi * ((j * k) % R) / R
            cj, sj = math.cos(ang), math.sin(ang)
            ar = dag.add(ar, dag.mul(const(cj), t[j - 1][0]))
            ai = dag.add(ai, dag.mul(const(cj), t[j - 1][1]))
            br = dag.add(br, dag.mul(const(sj), u[j - 1][0]))
            bi = dag.add(bi, dag.mul(const(sj), u[j - 1][1]))
        # y_k = a - i b, y_{R-k} = a + i b ; -i*(br + i bi) = (bi, -br)
        y[k] = (dag.add(ar, bi), dag.sub(ai, br))
        y[R - k] = (dag.sub(ar, bi), dag.add(ai, br))
    return y


def build(R):
    dag = Dag()
    x = [(dag.inp(i, 0), dag.inp(i, 1)) for i in range(R)]
    y = dft_sym(dag, x)
    return dag, y


def schedule(dag, outputs):
    """Depth-first topological order of the nodes reachable from the outputs."""
    order, seen = [], set()

    def visit(a):
        stack = [(a, False)]
        while stack:
            node, done = stack.pop()
            if done:
                order.append(node)
                continue
            if node in seen:
                continue
            seen.add(node)
            stack.append((node, True))
            op = dag.nodes[node]
            kids = []
            if op[0] in ("add", "sub"):
                kids = [op[1], op[2]]
            elif op[0] == "neg":
                kids = [op[1]]
            elif op[0] == "mul":
                kids = [op[2]]
            for k in reversed(kids):
                if k not in seen:
                    stack.append((k, False))

    for re, im in outputs:
        visit(re)
        visit(im)
    return order


def count_ops(dag, outputs):
    adds = muls = 0
    for n in schedule(dag, outputs):
        op = dag.nodes[n][0]
        if op in ("add", "sub"):
            adds += 1
        elif op == "mul":
            muls += 1
    return adds, muls


def _lit(v, target):
    s = repr(float(v))
    if "e" not in s and "." not in s:
        s += ".0"
    return s + ("f" if target == "cuda" else "")


def unparse(R, target):
    """Emit the codelet for radix R as CUDA (float2) or host C (double re/im arrays)."""
    dag, y = build(R)
    order = schedule(dag, y)
    name = {}
    lines = []
    ty = "float" if target == "cuda" else "double"

    def ref(a):
        op = dag.nodes[a]
        if op[0] == "in":
            if target == "cuda":
                return f"v[{op[1]}].{'x' if op[2] == 0 else 'y'}"
            return f"{'re' if op[2] == 0 else 'im'}[{op[1]}]"
        if op[0] == "zero":
            return _lit(0.0, target)
        return name[a]

    for a in order:
        op = dag.nodes[a]
        if op[0] in ("in", "zero"):
            continue
        nm = f"t{len(name)}"
        name[a] = nm
        if op[0] == "add":
            e = f"{ref(op[1])} + {ref(op[2])}"
        elif op[0] == "sub":
            e = f"{ref(op[1])} - {ref(op[2])}"
        elif op[0] == "neg":
            e = f"-{ref(op[1])}"
        else:
            e = f"{_lit(op[1][1], target)} * {ref(op[2])}"
        lines.append(f"    const {ty} {nm} = {e};")
    for k, (re, im) in enumerate(y):
        if target == "cuda":
            lines.append(f"    v[{k}].x = {ref(re)};")
            lines.append(f"    v[{k}].y = {ref(im)};")
        else:
            lines.append(f"    ore[{k}] = {ref(re)};")
            lines.append(f"    oim[{k}] = {ref(im)};")
    adds, muls = count_ops(dag, y)
    head = f"/* radix-{R} forward DFT: {adds} additions, {muls} multiplications */\n"
    if target == "cuda":
        sig = f"__device__ __forceinline__ void gb_dft{R}(float2* v) {{\n"
    else:
        sig = (f"static void host_dft{R}(const double* re, const double* im, double* ore, "
               f"double* oim) {{\n")
    return head + sig + "\n".join(lines) + "\n}\n"


def render_cuda():
    parts = ["/* Generated by gen_codelets.py -- do not edit by hand. */",
             "#pragma once", "#include <cuda_runtime.h>", ""]
    for R in RADICES:
        parts.append(unparse(R, "cuda"))
    return "\n".join(parts)


def render_host_c():
    parts = ["/* Generated by gen_codelets.py for CPU verification. */", ""]
    for R in RADICES:
        parts.append(unparse(R, "c"))
    return "\n".join(parts)


def main(argv):
    here = os.path.dirname(os.path.abspath(__file__))
    out = argv[1] if len(argv) > 1 else os.path.join(here, "codelets.cuh")
    text = render_cuda()
    old = open(out).read() if os.path.exists(out) else None
    if old != text:
        with open(out, "w") as f:
            f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
