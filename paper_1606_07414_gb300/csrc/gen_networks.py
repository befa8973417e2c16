"""Generate tx16_pairnet.cuh: the 44-addition network of the 16-point
approximation (T = P2 M4 M3 M2 P1 M1, Sec. 2.2 of the paper) as straight-line
code on float2 pairs (two blocks at once, Blackwell packed-FP32 builtins).

The generator does symbolically what a compiler cannot do through the packed
builtins:
  * negations (the -I blocks of M3/M4 and the butterflies' minus signs) are
    folded into the adds: every value carries a compile-time sign, a + b is
    emitted as add, sub (an fma by -1, one rounding) or add with the sign
    flipped, so no instruction is spent on a negation;
  * zonal pruning: inputs known to be zero are dropped and only the outputs
    that are used are computed.

Each emitted stage output is one IEEE operation on two stage inputs, exactly as
in the factorisation, so binary32 results are those of the factorisation
evaluated stage by stage.

Run:  python gen_networks.py  (rewrites tx16_pairnet.cuh beside this file)
"""
from __future__ import annotations

import os
import random

# --- the factorisation, 0-indexed (Sec. 2.2) ---------------------------------
G1 = [0, 1, 2, 3, 4, 5, 6, 7, 8, 11, 12, 15, 14, 13, 10, 9]   # P1: b[i] = a[G1[i]]
G2 = [0, 8, 7, 11, 3, 9, 5, 15, 1, 13, 6, 10, 2, 12, 4, 14]   # P2: y[i] = e[G2[i]]
ZERO = None


class Net:
    """Symbolic DAG builder.  A value is ZERO or (node_id, sign)."""

    def __init__(self, cse=False):
        self.nodes = []  # (kind, a_id, b_id) kind in add/sub ; leaves: ("in", name)
        # cse: identical operations share one node; a - b and b - a share one
        # node with opposite signs (binary32 round-to-nearest is symmetric
        # under negation, so this changes no rounded value)
        self.cse = cse
        self.memo = {}

    def leaf(self, name):
        self.nodes.append(("in", name))
        return (len(self.nodes) - 1, 1)

    def _new(self, kind, a, b):
        if self.cse:
            key = (kind, min(a, b), max(a, b)) if kind == "add" else (kind, a, b)
            if key in self.memo:
                return self.memo[key]
        self.nodes.append((kind, a, b))
        if self.cse:
            self.memo[key] = len(self.nodes) - 1
        return len(self.nodes) - 1

    def _sub(self, a, b):
        """Node and sign of a - b."""
        if self.cse and a > b:
            return (self._new("sub", b, a), -1)
        return (self._new("sub", a, b), 1)

    def add(self, x, y):
        if x is ZERO:
            return y
        if y is ZERO:
            return x
        (a, sa), (b, sb) = x, y
        if sa == 1 and sb == 1:
            return (self._new("add", a, b), 1)
        if sa == 1 and sb == -1:
            return self._sub(a, b)
        if sa == -1 and sb == 1:
            return self._sub(b, a)
        return (self._new("add", a, b), -1)

    def neg(self, x):
        return ZERO if x is ZERO else (x[0], -x[1])

    def sub(self, x, y):
        return self.add(x, self.neg(y))

    # -- stages --
    def m1(self, x):
        a = [None] * 16
        for i in range(8):
            a[i] = self.add(x[i], x[15 - i])
            a[8 + i] = self.sub(x[7 - i], x[8 + i])
        return a

    def m2(self, b):
        c = [None] * 16
        for h in (0, 8):
            for i in range(4):
                c[h + i] = self.add(b[h + i], b[h + 7 - i])
                c[h + 4 + i] = self.sub(b[h + 3 - i], b[h + 4 + i])
        return c

    def m3(self, c):
        n = self.neg
        return [self.add(c[0], c[3]), self.add(c[1], c[2]), self.sub(c[1], c[2]), self.sub(c[0], c[3]),
                n(c[4]), n(c[5]), n(c[6]), n(c[7]),
                self.add(c[8], c[11]), self.add(c[9], c[10]), self.sub(c[9], c[10]), self.sub(c[8], c[11]),
                n(c[12]), n(c[13]), n(c[14]), n(c[15])]

    def m4(self, d):
        n = self.neg
        return [self.add(d[0], d[1]), self.sub(d[0], d[1]), n(d[2]), d[3], d[4], d[5], d[6], n(d[7]),
                self.add(d[8], d[9]), self.sub(d[8], d[9]), n(d[10]), n(d[11]), n(d[12]), n(d[13]),
                d[14], n(d[15])]

    def forward(self, x):
        a = self.m1(x)
        b = [a[g] for g in G1]
        e = self.m4(self.m3(self.m2(b)))
        return [e[g] for g in G2]

    def inverse(self, y):
        # T^t = M1 P1^t M2 M3 M4 P2^t (M1..M4 symmetric)
        e = [None] * 16
        for i in range(16):
            e[G2[i]] = y[i]
        c = self.m2(self.m3(self.m4(e)))
        a = [None] * 16
        for i in range(16):
            a[G1[i]] = c[i]
        return self.m1(a)


def emit(net, outputs, in_names, out_name, materialize):
    """C++ statements computing the needed outputs.  Returns (lines, signs)
    where signs[k] is the sign of output k (0: known zero); with
    `materialize`, negative outputs are negated (one fma by -1) so all
    emitted outputs are the true values."""
    live = set()
    stack = [o[0] for o in outputs if o is not ZERO]
    while stack:
        k = stack.pop()
        if k in live:
            continue
        live.add(k)
        if net.nodes[k][0] != "in":
            stack += [net.nodes[k][1], net.nodes[k][2]]
    names = {}
    lines = []
    for k in sorted(live):
        kind = net.nodes[k][0]
        if kind == "in":
            names[k] = in_names[net.nodes[k][1]]
            continue
        a, b = names[net.nodes[k][1]], names[net.nodes[k][2]]
        t = f"t{k}"
        if kind == "add":
            lines.append(f"const float2 {t} = __fadd2_rn({a}, {b});")
        else:  # a - b with one rounding
            lines.append(f"const float2 {t} = sub2({a}, {b});")
        names[k] = t
    signs = []
    for idx, o in enumerate(outputs):
        if o is ZERO:
            lines.append(f"{out_name}[{idx}] = make_float2(0.f, 0.f);")
            signs.append(0)
            continue
        k, s = o
        if materialize and s < 0:
            lines.append(f"{out_name}[{idx}] = __fmul2_rn({names[k]}, pm1());")
            signs.append(1)
        else:
            lines.append(f"{out_name}[{idx}] = {names[k]};")
            signs.append(s)
    adds = sum(1 for k in live if net.nodes[k][0] != "in")
    leaves = {net.nodes[k][1] for k in live if net.nodes[k][0] == "in"}
    return lines, signs, adds, leaves


def check(net, outputs, inputs_value, expect):
    """Evaluate the DAG numerically and compare with the expected outputs."""
    val = {}
    for k, nd in enumerate(net.nodes):
        if nd[0] == "in":
            val[k] = inputs_value[nd[1]]
        elif nd[0] == "add":
            val[k] = val[nd[1]] + val[nd[2]]
        else:
            val[k] = val[nd[1]] - val[nd[2]]
    for o, want in zip(outputs, expect):
        got = 0 if o is ZERO else o[1] * val[o[0]]
        assert got == want, (got, want)


def matrix_from_network(inverse=False):
    """The 16x16 matrix the network realises (column j = image of e_j)."""
    M = [[0] * 16 for _ in range(16)]
    for j in range(16):
        net = Net()
        x = [net.leaf(i) for i in range(16)]
        y = net.inverse(x) if inverse else net.forward(x)
        vals = [1 if i == j else 0 for i in range(16)]
        val = {}
        for k, nd in enumerate(net.nodes):
            val[k] = vals[nd[1]] if nd[0] == "in" else (
                val[nd[1]] + val[nd[2]] if nd[0] == "add" else val[nd[1]] - val[nd[2]])
        for i in range(16):
            M[i][j] = 0 if y[i] is ZERO else y[i][1] * val[y[i][0]]
    return M


def node_values(net, inputs_value):
    """Exact value of every node for the given leaf values."""
    val = {}
    for k, nd in enumerate(net.nodes):
        if nd[0] == "in":
            val[k] = inputs_value[nd[1]]
        elif nd[0] == "add":
            val[k] = val[nd[1]] + val[nd[2]]
        else:
            val[k] = val[nd[1]] - val[nd[2]]
    return val


def emit_nodes(net, outputs, in_names):
    """Packed statements for the nodes the outputs need.  Returns (lines, outs,
    adds) with outs[k] = (variable, sign) of output k, or None if it is zero."""
    live = set()
    stack = [o[0] for o in outputs if o is not ZERO]
    while stack:
        k = stack.pop()
        if k in live:
            continue
        live.add(k)
        if net.nodes[k][0] != "in":
            stack += [net.nodes[k][1], net.nodes[k][2]]
    names = {}
    lines = []
    for k in sorted(live):
        kind = net.nodes[k][0]
        if kind == "in":
            names[k] = in_names[net.nodes[k][1]]
            continue
        a, b = names[net.nodes[k][1]], names[net.nodes[k][2]]
        op = "__fadd2_rn" if kind == "add" else "sub2"
        lines.append(f"const float2 t{k} = {op}({a}, {b});")
        names[k] = f"t{k}"
    outs = [None if o is ZERO else (names[o[0]], o[1]) for o in outputs]
    adds = sum(1 for k in live if net.nodes[k][0] != "in")
    return lines, outs, adds


def _lane(term, h):
    """Scalar lane h of a signed packed value (variable, sign)."""
    name, s = term
    return ("-" if s < 0 else "") + f"{name}.{'xy'[h]}"


class ScalarSums:
    """Scalar additions of lanes, each distinct expression emitted once."""

    def __init__(self, prefix):
        self.prefix = prefix
        self.memo = {}
        self.lines = []

    def add(self, p, q, h):
        # p + q (each a signed term or None) on lane h; returns an expression
        if p is None and q is None:
            return "0.f"
        if p is None or q is None:
            return _lane(p if q is None else q, h)
        a, b = sorted((_lane(p, h), _lane(q, h)))
        key = (a, b)
        if key not in self.memo:
            nm = f"{self.prefix}{len(self.memo)}"
            self.lines.append(f"const float {nm} = __fadd_rn({a}, {b});")
            self.memo[key] = nm
        return self.memo[key]


def emit_transposing(w, T, rnd):
    """Networks of the one-block-per-thread codec, which pairs rows (i, 15 - i)
    in the two lanes of a float2 so that the first butterfly of the column
    pass (rows i and 15 - i) and the last one of the inverse column pass
    become scalar additions across the lanes, writing their results straight
    into the pairing the next pass uses (no register moves).  Samples enter as
    2^23 + 256 x: every node is then a multiple of 256 below 2^32 in
    magnitude, exact in binary32 with no bias correction in M1."""
    # forward row pass on rows (i, 15 - i), then the column M1 across them
    for V in sorted({v for _, v in ZONES}):
        net = Net(cse=True)
        x = [net.leaf(i) for i in range(16)]
        y = net.forward(x)[:V]
        lines, outs, adds = emit_nodes(net, y, [f"X[{i}]" for i in range(16)])
        assert all(o is not None for o in outs)
        for _ in range(20):
            xs = [rnd.randint(0, 255) for _ in range(16)]
            check(net, y, xs, [sum(T[k][m] * xs[m] for m in range(16)) for k in range(V)])
        w(f"// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < {V}, then the")
        w(f"// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with")
        w(f"// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true")
        w(f"// signs); {adds} pair additions and {2 * V} scalar additions")
        w(f"struct FwdRowT{V} {{")
        w(f"  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[{V // 2}], "
          f"float2 (&D)[{V // 2}]) {{")
        for ln in lines:
            w("    " + ln)
        for c in range(V // 2):
            for arr, dsign in (("S", 1), ("D", -1)):
                comps = []
                for h in (0, 1):
                    nm, s = outs[2 * c + h]
                    comps.append(f"__fadd_rn({_lane((nm, s), 0)}, {_lane((nm, s * dsign), 1)})")
                w(f"    {arr}[{c}] = make_float2({comps[0]}, {comps[1]});")
        w("  }")
        w("};")
        w("")
    # forward column pass from the M1 outputs a[0..15]; every output count
    # (a column pair keeps the rows of its taller column's zone)
    for U in range(1, 17):
        net = Net(cse=True)
        a = [net.leaf(i) for i in range(16)]
        b = [a[g] for g in G1]
        e = net.m4(net.m3(net.m2(b)))
        y = [e[g] for g in G2][:U]
        lines, outs, adds = emit_nodes(net, y, [f"a[{i}]" for i in range(16)])
        assert all(o is not None for o in outs)
        for _ in range(20):
            xs = [rnd.randint(-4096, 4096) for _ in range(16)]
            av = [xs[i] + xs[15 - i] for i in range(8)] + [xs[7 - i] - xs[8 + i] for i in range(8)]
            check(net, y, av, [sum(T[k][m] * xs[m] for m in range(16)) for k in range(U)])
        signs = [o[1] for o in outs] + [0] * (16 - U)
        w(f"// forward column pass after M1 (inputs a = M1 x), outputs u < {U}:")
        w(f"// n[u] = sign[u] * (T x)[u]; {adds} pair additions")
        w(f"struct FwdColM{U} {{")
        w(sign_fn(signs))
        w(f"  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[{U}]) {{")
        for ln in lines:
            w("    " + ln)
        for u in range(U):
            w(f"    n[{u}] = {outs[u][0]};")
        w("  }")
        w("};")
        w("")
    # inverse column pass with its last butterfly (M1) scalar, into row pairs
    for U in range(1, 17):
        net = Net(cse=True)
        ins = [net.leaf(i) if i < U else ZERO for i in range(16)]
        e = [None] * 16
        for i in range(16):
            e[G2[i]] = ins[i]
        c = net.m2(net.m3(net.m4(e)))
        pre = [None] * 16
        for i in range(16):
            pre[G1[i]] = c[i]
        lines, outs, adds = emit_nodes(net, pre, [f"w[{i}]" for i in range(16)])
        ss = ScalarSums("s")
        body = []
        for i in range(8):
            p, q = outs[i], outs[15 - i]
            qn = None if q is None else (q[0], -q[1])
            for h in (0, 1):
                zi = ss.add(p, q, h)
                zj = ss.add(p, qn, h)
                body.append(f"Z[{i}][{h}] = make_float2({zi}, {zj});")
        for _ in range(20):
            ws = [rnd.randint(-5000, 5000) if i < U else 0 for i in range(16)]
            val = node_values(net, ws)
            pv = [0 if o is ZERO else o[1] * val[o[0]] for o in pre]
            z = [pv[i] + pv[15 - i] for i in range(8)] + [pv[7 - i] - pv[8 + i] for i in range(8)]
            assert z == [sum(T[m][k] * ws[m] for m in range(16)) for k in range(16)]
        w(f"// inverse column pass, inputs u < {U} (true values; lanes: columns 2c, 2c+1), with its")
        w(f"// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;")
        w(f"// {adds} pair additions and {len(ss.memo)} scalar additions")
        w(f"struct InvColT{U} {{")
        w(f"  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {{")
        for ln in lines + ss.lines + body:
            w("    " + ln)
        w("  }")
        w("};")
        w("")
    w("// the column-pass networks of a column pair keeping rows u < H")
    w("template <int H>")
    w("struct ColNets;")
    for U in range(1, 17):
        w(f"template <>")
        w(f"struct ColNets<{U}> {{")
        w(f"  using FC = FwdColM{U};")
        w(f"  using IC = InvColT{U};")
        w("};")
    w("")


# --- the 8-point approximation T8 (Sec. 2.1): the first halves of M2, M3, M4 --
# (those stages are block diagonal across the split of their 16 inputs into
# 0..7 and 8..15), with output k of T8 the first-half output that P2 sends to
# row 2k of T
G8 = [G2[2 * k] for k in range(8)]


def t8_forward(net, x):
    e = net.m4(net.m3(net.m2(list(x) + [ZERO] * 8)))
    return [e[g] for g in G8]


def t8_inverse(net, y):
    e = [ZERO] * 16
    for k in range(8):
        e[G8[k]] = y[k]
    return net.m2(net.m3(net.m4(e)))[:8]


def emit_t8(w, T, rnd):
    """Networks of T8 on float2 pairs for the mixed 8/16 tiling codec, which
    holds a 16x16 region per thread with rows (i, 15 - i) in the lanes: lane x
    walks the upper 8x8 blocks top-down, lane y the lower ones bottom-up.  The
    column networks take the eight row pairs in order; the first stage of T8
    (M2) pairs rows k and 7 - k of a block, which both lanes see, and lane y
    then carries the odd-frequency half negated (rows 3 - k and 4 + k come in
    swapped order).  The quantiser is odd-symmetric and the inverse column
    network undoes the same swap in its last stage, so lane y's output pair m
    is row 7 - m of the lower block with its true value: outputs come back in
    the (i, 15 - i) pairing."""
    T8 = [[T[2 * k][j] for j in range(8)] for k in range(8)]
    # T8 is the even rows of T on the sums x_j + x_(15-j)
    for k in range(8):
        assert all(T[2 * k][j] == T[2 * k][15 - j] for j in range(8))
    G = [[sum(T8[a][j] * T8[b][j] for j in range(8)) for b in range(8)] for a in range(8)]
    assert all(G[a][b] == 0 for a in range(8) for b in range(8) if a != b), "T8 T8^t is not diagonal"
    fsign = None
    for V in range(1, 9):  # forward row pass, outputs v < V (signed)
        net = Net(cse=True)
        x = [net.leaf(i) for i in range(8)]
        y = t8_forward(net, x)[:V]
        lines, outs, adds = emit_nodes(net, y, [f"X[{i}]" for i in range(8)])
        for _ in range(20):
            xs = [rnd.randint(0, 255) for _ in range(8)]
            check(net, y, xs, [sum(T8[k][m] * xs[m] for m in range(8)) for k in range(V)])
        signs = [o[1] for o in outs] + [0] * (16 - V)
        if V == 8:
            fsign = signs[:8]
        w(f"// T8 on one half row of both lanes, outputs v < {V}: R[v] = sign[v] * (T8 x)[v];")
        w(f"// {adds} pair additions")
        w(f"struct FwdRow8T{V} {{")
        w(sign_fn(signs))
        w(f"  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[{V}]) {{")
        for ln in lines:
            w("    " + ln)
        for v in range(V):
            w(f"    R[{v}] = {outs[v][0]};")
        w("  }")
        w("};")
        w("")
    for H in range(1, 9):  # forward column pass over the 8 row pairs, outputs u < H (signed)
        net = Net(cse=True)
        a = [net.leaf(i) for i in range(8)]
        y = t8_forward(net, a)[:H]
        lines, outs, adds = emit_nodes(net, y, [f"a[{i}]" for i in range(8)])
        for _ in range(20):
            xs = [rnd.randint(-4096, 4096) for _ in range(8)]
            check(net, y, xs, [sum(T8[k][m] * xs[m] for m in range(8)) for k in range(H)])
        signs = [o[1] for o in outs] + [0] * (16 - H)
        assert signs[:H] == fsign[:H]  # the same network: the same output signs
        w(f"// T8 down a column of the eight row pairs, outputs u < {H}: n[u] = sign[u] * (T8 a)[u]")
        w(f"// per lane (lane y: odd u negated, see the row-pair note); {adds} pair additions")
        w(f"struct FwdCol8M{H} {{")
        w(sign_fn(signs))
        w(f"  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[{H}]) {{")
        for ln in lines:
            w("    " + ln)
        for u in range(H):
            w(f"    n[{u}] = {outs[u][0]};")
        w("  }")
        w("};")
        w("")
    for H in range(1, 9):  # inverse column pass, inputs u < H (true values), outputs true
        net = Net()
        ins = [net.leaf(i) if i < H else ZERO for i in range(8)]
        z = t8_inverse(net, ins)
        lines, outs, adds = emit_nodes(net, z, [f"w[{i}]" for i in range(8)])
        assert all(o is not None and o[1] == 1 for o in outs), "inverse column outputs must be true values"
        for _ in range(20):
            ws = [rnd.randint(-5000, 5000) if i < H else 0 for i in range(8)]
            check(net, z, ws, [sum(T8[m][k] * ws[m] for m in range(8)) for k in range(8)])
        w(f"// T8^t down a column, inputs u < {H}: z[m] = (T8^t w)[m] per lane, true values; "
          f"{adds} pair additions")
        w(f"struct InvCol8T{H} {{")
        w(f"  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {{")
        for ln in lines:
            w("    " + ln)
        for m in range(8):
            w(f"    z[{m}] = {outs[m][0]};")
        w("  }")
        w("};")
        w("")
    for V in range(1, 9):  # inverse row pass, inputs v < V (true values), outputs signed
        net = Net()
        ins = [net.leaf(i) if i < V else ZERO for i in range(8)]
        z = t8_inverse(net, ins)
        lines, outs, adds = emit_nodes(net, z, [f"w[{i}]" for i in range(8)])
        assert all(o is not None for o in outs)
        for _ in range(20):
            ws = [rnd.randint(-5000, 5000) if i < V else 0 for i in range(8)]
            check(net, z, ws, [sum(T8[m][k] * ws[m] for m in range(8)) for k in range(8)])
        signs = [o[1] for o in outs] + [0] * 8
        w(f"// T8^t on a half row, inputs v < {V}: z[j] = sign[j] * (T8^t w)[j]; {adds} pair additions")
        w(f"struct InvRow8T{V} {{")
        w(sign_fn(signs))
        w(f"  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {{")
        for ln in lines:
            w("    " + ln)
        for j in range(8):
            w(f"    z[{j}] = {outs[j][0]};")
        w("  }")
        w("};")
        w("")
    for u in range(8):  # row u of T8 is symmetric for even u, antisymmetric for odd u
        assert all(T8[u][7 - j] == (-1) ** u * T8[u][j] for j in range(8)), "T8 row parity"
    w("// T8 itself (rows: frequencies u; columns: samples j), for column passes that")
    w("// accumulate T8 x term by term; row u is symmetric for even u, antisymmetric")
    w("// for odd u")
    w("constexpr int kT8[8][8] = {")
    for u in range(8):
        w("    {" + ", ".join(str(x) for x in T8[u]) + "},")
    w("};")
    w("// the T8 networks of the mixed tiling codec: a column keeping rows u < H,")
    w("// a half row keeping columns v < V")
    w("template <int H>")
    w("struct Col8Nets;")
    for H in range(1, 9):
        w("template <>")
        w(f"struct Col8Nets<{H}> {{")
        w(f"  using FC = FwdCol8M{H};")
        w(f"  using IC = InvCol8T{H};")
        w("};")
    w("template <int V>")
    w("struct Row8Nets;")
    for V in range(1, 9):
        w("template <>")
        w(f"struct Row8Nets<{V}> {{")
        w(f"  using FR = FwdRow8T{V};")
        w(f"  using IR = InvRow8T{V};")
        w("};")
    w("")


ZONES = [(3, 4), (5, 6), (7, 8), (11, 10), (16, 16)]  # (rows U, columns V) kept


def sign_fn(signs):
    neg = sum(1 << i for i, x in enumerate(signs) if x < 0)
    zero = sum(1 << i for i, x in enumerate(signs) if x == 0)
    return (f"  __host__ __device__ static constexpr int sign(int i) {{ return sign_of(0x{neg:04x}u, "
            f"0x{zero:04x}u, i); }}")


def main(path=None):
    """Write the header (to `path`, default tx16_pairnet.cuh beside this file),
    checking every emitted network against the matrix it realises."""
    T = matrix_from_network(False)
    Tt = matrix_from_network(True)
    assert all(Tt[i][j] == T[j][i] for i in range(16) for j in range(16)), "inverse is not T^t"
    rnd = random.Random(1606)
    out = []
    w = out.append
    w("// GENERATED by gen_networks.py -- do not edit.  The 44-addition network of")
    w("// T = P2 M4 M3 M2 P1 M1 (Sec. 2.2) on float2 pairs, negations folded into the")
    w("// additions and pruned to the zonal extents used by the fused codec.")
    w("#pragma once")
    w("#include <cuda_runtime.h>")
    w("namespace tx16 {")
    w("namespace pairnet {")
    w("__device__ __forceinline__ float2 pm1() { return make_float2(-1.f, -1.f); }")
    w("__device__ __forceinline__ float2 pbias() { return make_float2(-16777216.f, -16777216.f); }  // -2^24")
    w("// a - b and RD(a - b) per lane: a packed addition of the negated operand")
    w("// (one rounding; the negation folds into the instruction)")
    w("__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }")
    w("__device__ __forceinline__ float2 sub2_rd(float2 a, float2 b) { return __fadd2_rd(a, make_float2(-b.x, -b.y)); }")
    w("// sign of output i encoded as bit masks (negative / known zero)")
    w("__host__ __device__ constexpr int sign_of(unsigned neg, unsigned zero, int i) {")
    w("  return ((zero >> i) & 1u) ? 0 : (((neg >> i) & 1u) ? -1 : 1);")
    w("}")
    w("")
    # forward row pass: inputs are biased samples X = 2^23 + x.  M1 is special:
    #   x_i + x_j = (X_i - 2^24) + X_j  (both steps exact), x_i - x_j = X_i - X_j.
    fwd_sign = None
    for V in sorted({v for _, v in ZONES}):
        # M1 on biased inputs is emitted by hand below; the rest symbolically
        net2 = Net()
        aa = [net2.leaf(i) for i in range(16)]  # a[0..15] as leaves
        b = [aa[g] for g in G1]
        e = net2.m4(net2.m3(net2.m2(b)))
        y = [e[g] for g in G2]
        outs = y[:V] + [ZERO] * (16 - V)
        lines, signs, adds, live_a = emit(net2, outs, [f"a{i}" for i in range(16)], "y", materialize=False)
        # numeric self-check of the composite (M1 by hand + the rest)
        for _ in range(20):
            xs = [rnd.randint(0, 255) for _ in range(16)]
            av = [xs[i] + xs[15 - i] for i in range(8)] + [xs[7 - i] - xs[8 + i] for i in range(8)]
            expect = [sum(T[k][m] * xs[m] for m in range(16)) if k < V else 0 for k in range(16)]
            check(net2, outs, av, expect)
        w(f"// forward row pass, outputs v < {V}: y[v] = sign[v] * (T x)[v]; {adds} pair additions after M1")
        w(f"struct FwdRow{V} {{")
        w(sign_fn(signs))
        w("  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {")
        for i in range(8):
            j = 15 - i
            if i in live_a:
                w(f"    const float2 a{i} = __fadd2_rn(__fadd2_rn(X[{i}], pbias()), X[{j}]);")
            if (8 + (7 - i)) in live_a:
                # a[8 + k] = x[7 - k] - x[8 + k] with k = 7 - i  ->  x[i] - x[15 - i]
                w(f"    const float2 a{8 + (7 - i)} = sub2(X[{i}], X[{j}]);")
        for ln in lines:
            w("    " + ln)
        w("  }")
        w("};")
        w("")
        if V == 16:
            fwd_sign = signs
    # forward column pass: 16 plain inputs, outputs u < U
    col_sign = None
    for U in sorted({u for u, _ in ZONES}):
        net = Net()
        x = [net.leaf(i) for i in range(16)]
        y = net.forward(x)
        outs = y[:U] + [ZERO] * (16 - U)
        lines, signs, adds, _ = emit(net, outs, [f"x[{i}]" for i in range(16)], "y", materialize=False)
        for _ in range(20):
            xs = [rnd.randint(-4096, 4096) for _ in range(16)]
            check(net, outs, xs, [sum(T[k][m] * xs[m] for m in range(16)) if k < U else 0 for k in range(16)])
        w(f"// forward column pass, outputs u < {U}: y[u] = sign[u] * (T x)[u]; {adds} pair additions")
        w(f"struct FwdCol{U} {{")
        w(sign_fn(signs))
        w("  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {")
        for ln in lines:
            w("    " + ln)
        w("  }")
        w("};")
        w("")
        if U == 16:
            col_sign = signs
    # inverse column pass: inputs u < U carry the forward column signs
    for U in sorted({u for u, _ in ZONES}):
        net = Net()
        ins = [(net.leaf(i)[0], col_sign[i]) if i < U else ZERO for i in range(16)]
        y = net.inverse(ins)
        lines, signs, adds, _ = emit(net, y, [f"w[{i}]" for i in range(16)], "z", materialize=True)
        for _ in range(20):
            # true coefficient W_u = col_sign[u] * (stored node value)
            ws = [rnd.randint(-5000, 5000) if i < U else 0 for i in range(16)]
            node_vals = [col_sign[i] * ws[i] for i in range(16)]
            check(net, y, node_vals, [sum(T[m][k] * ws[m] for m in range(16)) for k in range(16)])
        w(f"// inverse column pass, inputs u < {U} (node values, signs of the forward column")
        w(f"// pass), outputs z[i] = (T^t w)[i] materialised; {adds} pair additions")
        w(f"struct InvCol{U} {{")
        w("  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {")
        for ln in lines:
            w("    " + ln)
        w("  }")
        w("};")
        w("")
    # inverse row pass: inputs v < V positive, outputs with signs
    for V in sorted({v for _, v in ZONES}):
        net = Net()
        ins = [net.leaf(i) if i < V else ZERO for i in range(16)]
        y = net.inverse(ins)
        lines, signs, adds, _ = emit(net, y, [f"w[{i}]" for i in range(16)], "z", materialize=False)
        for _ in range(20):
            ws = [rnd.randint(-5000, 5000) if i < V else 0 for i in range(16)]
            check(net, y, ws, [sum(T[m][k] * ws[m] for m in range(16)) for k in range(16)])
        w(f"// inverse row pass, inputs v < {V}: z[j] = sign[j] * (T^t w)[j]; {adds} pair additions")
        w(f"struct InvRow{V} {{")
        w(sign_fn(signs))
        w("  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {")
        for ln in lines:
            w("    " + ln)
        w("  }")
        w("};")
        w("")
    emit_transposing(w, T, rnd)
    emit_t8(w, T, rnd)
    w(f"// sign of each output of the (unpruned) forward network: row-pass outputs")
    w(f"// are stored unsigned; the column thread folds this sign into its scale.")
    w(f"constexpr unsigned kFwdNegMask = 0x{sum(1 << i for i, x in enumerate(fwd_sign) if x < 0):04x}u;")
    w("}  // namespace pairnet")
    w("}  // namespace tx16")
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tx16_pairnet.cuh")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
