"""Writes sbox_lut3.h: the bitsliced S-box circuit mapped onto three-input lookup tables,
and the linear maps the rounds need as programs of two- and three-input XORs.

The bitsliced kernel spends most of its integer-ALU instructions in the S-box
circuit (bitsliced.h, `sbox_circuit`: Boyar and Peralta's depth-16 circuit, 34
ANDs and 94 XORs).  A GPU evaluates any Boolean function of three 32-bit
operands in one LOP3 instruction, so the cheapest program for the circuit is a
cover of its gates by three-input cones.  This script

  1. reads the gate list of `sbox_circuit` from bitsliced.h (one source for the
     circuit; its exhaustive compile-time check stays where it is),
  2. builds the network the kernel evaluates per state byte: the S-box without
     its affine constant, F, with a round-key plane XORed onto each output bit.
     Decryption runs the same network: it works on A^-1 of the state (A the
     S-box's affine matrix), where the inverse S-box A^-1 F(A^-1 x) leaves F
     alone and the two A^-1 move into the linear map around it (bitsliced.h,
     decrypt_half),
  3. re-brackets the XOR sums the circuit computes once (maximal trees of XOR
     gates whose inner results feed nothing else: any bracketing of the same
     terms gives the same sum), each tree as recorded in SHAPES below,
  4. maps the network onto three-input lookup tables: every 3-feasible cut of
     every gate is enumerated, each gate takes the cut of least area flow, and
     passes of exact-area recovery then re-choose cuts where that frees the most
     tables (the standard cut-based technology-mapping method of FPGA tools),
  5. emits each table as one `lop(a, b, c, truth_table)` call, the truth table in
     PTX's lop3 encoding (bit i = F(i >> 2 & 1, i >> 1 & 1, i & 1) for operands
     a, b, c), in the order the network computes them.

The linear maps -- MixColumns on a column's 32 bit planes, the decryption's
column map A^-1 InvMixColumns A^-1 (A^-1 on each byte), and A^-1 on one byte --
are written as straight-line programs by a greedy method in the manner of
Paar's (1997) common-subexpression algorithm, adapted to three-input gates:
while some output still needs more than one gate, create the XOR of the pair or
triple of available signals whose creation lowers the remaining three-input-gate
count most, ties broken by a seeded jitter; each output then sums its remaining
signals three at a time.  MIX_SEEDS records the jitter seed with the fewest
gates among those tried (`--search-mix`, 64 seeds per run).  MixColumns takes
55 tables per column where its xtime form took 76; the decryption's column map
117, and with it each inverse S-box is the 81-table forward network instead of
a 102-table one.

The bracketings in SHAPES come from `--search`: a hill climb that re-draws one
tree's bracketing at a time and keeps the draw when the mapped table count does
not grow (91 -> 81 tables from the circuit's own bracketing).  A tree's entry
seeds the splitmix64 generator that picks which two of its remaining terms to
XOR next; trees without an entry keep the circuit's bracketing.

Run from anywhere: python gen_sbox_lut3.py [--out PATH]  (default: rewrites sbox_lut3.h next to it);
python gen_sbox_lut3.py --search [--iters N] [--seed S] prints a new SHAPES entry;
python gen_sbox_lut3.py --search-mix mix|dec_mix|affine_inv [--seed S] prints the best of 64 seeds from S.
"""
import argparse
import itertools
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))


def circuit_gates():
    """(out, op, a, b) for each gate of sbox_circuit, inputs u0..u7, outputs s0..s7."""
    src = open(os.path.join(HERE, "bitsliced.h")).read()
    body = src[src.index("GBAES_HD constexpr void sbox_circuit"):]
    body = body[:body.index("\n}\n")]
    gates, seen = [], set()
    for m in re.finditer(r"(\w+(?:\[\d\])?)\s*=\s*(\w+(?:\[\d\])?)\s*([\^&])\s*(\w+(?:\[\d\])?)", body):
        out, a, op, b = (re.sub(r"\[(\d)\]", r"\1", g) for g in m.groups())
        if out not in seen:
            seen.add(out)
            gates.append((out, op, a, b))
    assert len(gates) == 128 and sum(g[1] == "&" for g in gates) == 34
    return gates


def affine_inverse_rows():
    """Rows of A^-1 over GF(2): bit j of row i = coefficient of x_j in y_i."""
    a = [(1 << i) | (1 << ((i + 4) & 7)) | (1 << ((i + 5) & 7)) | (1 << ((i + 6) & 7)) | (1 << ((i + 7) & 7))
         for i in range(8)]
    m, inv = a[:], [1 << i for i in range(8)]
    for col in range(8):
        piv = next(r for r in range(col, 8) if (m[r] >> col) & 1)
        m[col], m[piv] = m[piv], m[col]
        inv[col], inv[piv] = inv[piv], inv[col]
        for r in range(8):
            if r != col and (m[r] >> col) & 1:
                m[r] ^= m[col]
                inv[r] ^= inv[col]
    return inv


class Net:
    """A network of two-input gates over named primary inputs."""

    def __init__(self, pis):
        self.pis = list(pis)
        self.gates = {}  # name -> (op, a, b)
        self.order = []
        self.outs = []

    def gate(self, name, op, a, b):
        assert name not in self.gates and name not in self.pis
        self.gates[name] = (op, a, b)
        self.order.append(name)
        return name

    def xor_chain(self, prefix, terms):
        acc = terms[0]
        for i, t in enumerate(terms[1:]):
            acc = self.gate(f"{prefix}_{i}", "^", acc, t)
        return acc

    def add_circuit(self, tag, u):
        """The S-box circuit on planes u[0..7] (u[0] = most significant bit); returns its 8 outputs."""
        ren = {f"u{i}": u[i] for i in range(8)}
        for out, op, a, b in circuit_gates():
            ren[out] = self.gate(f"{tag}{out}", op, ren.get(a, a), ren.get(b, b))
        return [ren[f"s{i}"] for i in range(8)]


def encrypt_net():
    """x[t] (bit t) -> S(x)[t] ^ k[t], the affine constant left to the round keys."""
    net = Net([f"x{t}" for t in range(8)] + [f"k{t}" for t in range(8)])
    o = net.add_circuit("c_", [f"x{7 - i}" for i in range(8)])
    for t in range(8):
        net.outs.append(net.gate(f"y{t}", "^", o[7 - t], f"k{t}"))
    return net


class SplitMix64:
    """The splitmix64 generator (Steele, Lea, Flood 2014): a 64-bit state stepped by a constant, mixed."""

    def __init__(self, seed):
        self.state = seed & (2 ** 64 - 1)

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & (2 ** 64 - 1)
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2 ** 64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2 ** 64 - 1)
        return z ^ (z >> 31)

    def below(self, n):
        return self.next() % n


def xor_trees(net):
    """{root: terms} for each maximal tree of XOR gates whose inner nodes feed only the tree (> 2 terms)."""
    fanout = {}
    for n in net.order:
        for x in net.gates[n][1:]:
            fanout[x] = fanout.get(x, 0) + 1
    for o in net.outs:
        fanout[o] = fanout.get(o, 0) + 1
    inner = {x for n in net.order if net.gates[n][0] == "^" for x in net.gates[n][1:]
             if x in net.gates and net.gates[x][0] == "^" and fanout[x] == 1}

    def terms(n):
        out = []
        for x in net.gates[n][1:]:
            out += terms(x) if x in inner else [x]
        return out

    trees = {n: terms(n) for n in net.order if net.gates[n][0] == "^" and n not in inner}
    return {r: t for r, t in trees.items() if len(t) > 2}


def reshape(net, shapes):
    """A copy of net with the XOR trees named in shapes re-bracketed by their seeds."""
    trees = xor_trees(net)
    new = Net(net.pis)
    done, count = {}, [0]

    def build(n):
        if n in net.pis:
            return n
        if n not in done:
            op, a, b = net.gates[n]
            if n in trees and shapes.get(n):
                terms = [build(x) for x in trees[n]]
                rng = SplitMix64(shapes[n])
                while len(terms) > 2:
                    i = rng.below(len(terms))
                    j = rng.below(len(terms) - 1)
                    j += j >= i
                    count[0] += 1
                    g = new.gate(f"{n}__{count[0]}", "^", terms[i], terms[j])
                    terms = [x for m, x in enumerate(terms) if m not in (i, j)] + [g]
                done[n] = new.gate(n, "^", terms[0], terms[1])
            else:
                done[n] = new.gate(n, op, build(a), build(b))
        return done[n]

    for o in net.outs:
        build(o)
    new.outs = [done[o] for o in net.outs]
    return new


def search(net, iters, seed):
    """Hill climb over the trees' bracketings; returns the shapes of the best network found."""
    roots = sorted(xor_trees(net))
    rng, shapes = SplitMix64(seed), {}
    cur = len(map_lut3(reshape(net, shapes), passes=3))
    for _ in range(iters):
        r = roots[rng.below(len(roots))]
        old = shapes.get(r)
        shapes[r] = rng.next() | 1
        c = len(map_lut3(reshape(net, shapes), passes=3))
        if c <= cur:
            cur = c
        elif old is None:
            del shapes[r]
        else:
            shapes[r] = old
    return shapes


def map_lut3(net, passes=8):
    """Cut-based mapping onto 3-input tables; returns {node: leaves} for the chosen cover."""
    fanout = {}
    for n in net.order:
        for x in net.gates[n][1:]:
            fanout[x] = fanout.get(x, 0) + 1
    for o in net.outs:
        fanout[o] = fanout.get(o, 0) + 1
    cuts = {p: [frozenset([p])] for p in net.pis}
    for n in net.order:
        _, a, b = net.gates[n]
        cs = sorted({c1 | c2 for c1 in cuts[a] for c2 in cuts[b] if len(c1 | c2) <= 3}, key=len)
        keep = []
        for c in cs:
            if not any(k <= c for k in keep):
                keep.append(c)
        cuts[n] = keep + [frozenset([n])]

    def choices(n):
        return [c for c in cuts[n] if c != frozenset([n])]

    flow = {p: 0.0 for p in net.pis}
    best = {}
    for n in net.order:
        v, c = min(((1 + sum(flow[x] / max(1, fanout.get(x, 1)) for x in c), sorted(c)) for c in choices(n)))
        flow[n], best[n] = v, frozenset(c)

    def cover():
        req, stack = set(), list(net.outs)
        while stack:
            n = stack.pop()
            if n in net.pis or n in req:
                continue
            req.add(n)
            stack.extend(best[n])
        return req

    def refs():
        r = {}
        for n in cover():
            for x in best[n]:
                r[x] = r.get(x, 0) + 1
        for o in net.outs:
            r[o] = r.get(o, 0) + 1
        return r

    def deref(n, r):
        area = 1
        for x in best[n]:
            if x not in net.pis:
                r[x] -= 1
                if r[x] == 0:
                    area += deref(x, r)
        return area

    def ref(n, r):
        area = 1
        for x in best[n]:
            if x not in net.pis:
                r[x] = r.get(x, 0) + 1
                if r[x] == 1:
                    area += ref(x, r)
        return area

    for _ in range(passes):
        r = refs()
        for n in net.order:
            if r.get(n, 0) == 0:
                continue
            deref(n, r)
            scored = []
            for c in choices(n):
                old, best[n] = best[n], c
                scored.append((ref(n, r), sorted(c), c))
                deref(n, r)
                best[n] = old
            best[n] = min(scored)[2]
            ref(n, r)
    return {n: sorted(best[n]) for n in cover()}


def truth_table(net, node, leaves):
    """lop3 immediate of node as a function of its cut's leaves, padded to three operands with the first."""
    ops = (leaves + [leaves[0]] * 3)[:3]
    imm = 0
    for i in range(8):
        assign = {}
        for j, leaf in enumerate(ops):
            bit = (i >> (2 - j)) & 1
            if assign.setdefault(leaf, bit) != bit:
                assign = None  # a combination the padding rules out: leave its bit 0
                break
        if assign is None:
            continue
        memo = dict(assign)

        def ev(n):
            if n not in memo:
                op, a, b = net.gates[n]
                memo[n] = (ev(a) & ev(b)) if op == "&" else (ev(a) ^ ev(b))
            return memo[n]

        imm |= ev(node) << i
    return ops, imm


def emit(net, cover, fname):
    topo = [n for n in net.order if n in cover]
    names = {f"x{t}": f"x[{t}]" for t in range(8)}
    names.update({f"k{t}": f"k[{t}]" for t in range(8)})
    lines = []
    for i, n in enumerate(topo):
        ops, imm = truth_table(net, n, cover[n])
        names[n] = f"v{i}"
        lines.append(f"    const uint32_t v{i} = lop({names[ops[0]]}, {names[ops[1]]}, {names[ops[2]]}, Tt<0x{imm:02x}>{{}});")
    for t, o in enumerate(net.outs):
        lines.append(f"    x[{t}] = {names[o]};")
    head = (f"template <class Lop>\nGBAES_HD constexpr void {fname}(uint32_t* x, const uint32_t (&k)[8], "
            f"const Lop& lop) {{  // {len(topo)} tables")
    return head + "\n" + "\n".join(lines) + "\n}\n"


# ------------------------------------------------------- MixColumns as XOR programs


def gf_mul(a, b):
    """Product in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1."""
    r = 0
    for i in range(8):
        if (b >> i) & 1:
            r ^= a << i
    for i in range(15, 7, -1):
        if (r >> i) & 1:
            r ^= 0x11B << (i - 8)
    return r


def column_rows(coef):
    """The 32x32 GF(2) matrix of a column map out_q = sum_j coef[j] a_{q+j}: row 8q+t (output byte q,
    bit t) as a bit mask over input bit 8q'+t' (byte q', bit t')."""
    rows = []
    for q in range(4):
        for t in range(8):
            m = 0
            for j, c in enumerate(coef):
                for tp in range(8):
                    if (gf_mul(c, 1 << tp) >> t) & 1:
                        m |= 1 << (8 * ((q + j) % 4) + tp)
            rows.append(m)
    return rows


def xor_program(rows, seed, n_in=32):
    """A straight-line program of XORs of two or three signals computing every row (greedy: repeatedly
    create the sum of the pair or triple of signals that lowers the three-input-gate cost of the
    remaining rows most, a seeded jitter breaking ties).  Returns (steps, rows as signal sets); step k
    creates signal n_in + k as the XOR of its operands."""
    rng = SplitMix64(seed)
    rows_s = [set(i for i in range(n_in) if (r >> i) & 1) for r in rows]

    def cost(k):
        return k // 2 if k > 1 else 0  # three-input gates to sum k signals: ceil((k - 1) / 2)

    steps = []
    while True:
        cands = set()
        for rs in rows_s:
            if len(rs) > 1:
                srt = sorted(rs)
                cands.update(itertools.combinations(srt, 2))
                cands.update(itertools.combinations(srt, 3))
        best, best_v = None, 0.0
        for c in sorted(cands):
            gain = sum(cost(len(rs)) - cost(len(rs) - len(c) + 1) for rs in rows_s
                       if len(rs) > 1 and all(x in rs for x in c))
            v = gain - 1 + (rng.next() >> 11) / float(1 << 53) * 0.5
            if v > best_v:
                best, best_v = c, v
        if best is None:
            break
        new = n_in + len(steps)
        steps.append(best)
        for rs in rows_s:
            if len(rs) > 1 and all(x in rs for x in best):
                rs.difference_update(best)
                rs.add(new)
    return steps, rows_s


def emit_linear(fname, what, steps, rows_s, n_in=32):
    """The program as lop calls on n_in planes in place."""
    lines = [f"    const uint32_t i{i} = x[{i}];" for i in range(n_in)]
    names = {i: f"i{i}" for i in range(n_in)}
    xor2, xor3 = 0x3C, 0x96  # a ^ b (third operand repeats a), a ^ b ^ c
    n = 0

    def lop(ops):
        nonlocal n
        v = f"w{n}"
        n += 1
        if len(ops) == 2:
            lines.append(f"    const uint32_t {v} = lop({ops[0]}, {ops[1]}, {ops[0]}, Tt<0x{xor2:02x}>{{}});")
        else:
            lines.append(f"    const uint32_t {v} = lop({ops[0]}, {ops[1]}, {ops[2]}, Tt<0x{xor3:02x}>{{}});")
        return v

    for k, ops in enumerate(steps):
        names[n_in + k] = lop([names[o] for o in ops])
    outs = []
    for rs in rows_s:
        terms = [names[o] for o in sorted(rs)]
        while len(terms) > 1:
            take = terms[:3]
            terms = [lop(take)] + terms[3:]
        outs.append(terms[0])
    lines += [f"    x[{i}] = {o};" for i, o in enumerate(outs)]
    head = (f"// {what}\ntemplate <class Lop>\nGBAES_HD constexpr void {fname}(uint32_t* x, const Lop& lop) {{  "
            f"// {n} tables")
    return head + "\n" + "\n".join(lines) + "\n}\n", n


def affine_inverse_byte(v):
    """A^-1 applied to one byte (bit i of the result = parity of row i of A^-1 and v)."""
    rows = affine_inverse_rows()
    return sum((bin(rows[i] & v).count("1") & 1) << i for i in range(8))


def matrix_rows(f, n):
    """Rows (bit masks over the n input bits) of the GF(2)-linear map f on n-bit vectors."""
    cols = [f(1 << j) for j in range(n)]
    return [sum(((cols[j] >> r) & 1) << j for j in range(n)) for r in range(n)]


def bytewise(f):
    return lambda v: sum(f((v >> (8 * q)) & 0xFF) << (8 * q) for q in range(4))


def linear_maps():
    """name -> (rows, inputs): MixColumns of a column; the decryption column map A^-1 InvMixColumns A^-1
    (bytewise A^-1 on both sides, see bitsliced.h); A^-1 on one byte."""
    inv_rows = column_rows((14, 11, 13, 9))

    def apply(rows, v):
        return sum((bin(row & v).count("1") & 1) << r for r, row in enumerate(rows))

    ainv = bytewise(affine_inverse_byte)
    return {
        "mix": (column_rows((2, 3, 1, 1)), 32),
        "dec_mix": (matrix_rows(lambda v: ainv(apply(inv_rows, ainv(v))), 32), 32),
        "affine_inv": (matrix_rows(affine_inverse_byte, 8), 8),
    }


# Seeds of the greedy XOR programs, chosen by --search-mix runs (the program with the fewest gates among
# the seeds tried: 0-575 for MixColumns, 0-1087 for the decryption column map).
MIX_SEEDS = {"mix": 117, "dec_mix": 236, "affine_inv": 0}


# Bracketings found by --search (seed 1, 1,500 steps): tree root -> splitmix64 seed.
SHAPES = {
    "enc": {
        "c_l6": 8411996437093593279,
        "c_m20": 6036339614689729693,
        "c_m21": 2927808880244328445,
        "c_m22": 12944380480760822807,
        "c_m23": 14618154987885078747,
        "c_m38": 2243067523905852675,
        "c_m40": 961137476199508239,
        "c_t19": 5039539338173171385,
        "c_t22": 1163728296864529161,
        "y0": 13290268570847108467,
        "y1": 15053352997926904907,
        "y2": 17407377188203331605,
        "y3": 11924832088314853027,
        "y4": 4621030392246333243,
        "y5": 15563214200757333989,
        "y6": 65468312225334051,
        "y7": 5208041666417506291,
    },
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "sbox_lut3.h"))
    ap.add_argument("--search", action="store_true", help="hill-climb the S-box network's bracketings")
    ap.add_argument("--search-mix", choices=tuple(MIX_SEEDS))
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()
    maps = linear_maps()
    if args.search_mix:
        rows, n_in = maps[args.search_mix]
        counts = []
        for sd in range(args.seed, args.seed + 64):
            steps, rows_s = xor_program(rows, sd, n_in)
            counts.append((len(steps) + sum(len(r) // 2 for r in rows_s if len(r) > 1), sd))
        print("fewest gates, seed:", min(counts))
        return
    if args.search:
        net = encrypt_net()
        shapes = search(net, args.iters, args.seed)
        print(len(map_lut3(reshape(net, shapes))), "tables;", dict(sorted(shapes.items())))
        return
    out = args.out
    enc = reshape(encrypt_net(), SHAPES["enc"])
    enc_cover = map_lut3(enc)
    code, count = {}, {}
    what = {
        "mix": ("mix_column_lut3", "MixColumns of one column in place: out_q = 02 a_q + 03 a_q+1 + a_q+2 + a_q+3."),
        "dec_mix": ("dec_mix_column_lut3", "Decryption's column map in place: A^-1 InvMixColumns A^-1 (A^-1 bytewise)."),
        "affine_inv": ("affine_inv_byte_lut3", "A^-1 (the inverse of the S-box's affine matrix) on one byte in place."),
    }
    for name, (rows, n_in) in maps.items():
        code[name], count[name] = emit_linear(what[name][0], what[name][1],
                                              *xor_program(rows, MIX_SEEDS[name], n_in), n_in=n_in)
    text = f"""// Generated by gen_sbox_lut3.py from sbox_circuit in bitsliced.h -- do not edit.
//
// The bitsliced S-box network as three-input lookup tables (one LOP3 each on
// the GPU): sbox_key_lut3 computes x[t] = F(x)[t] ^ k[t], F the S-box without its
// affine constant ({len(enc_cover)} tables for the {len(enc.gates)} two-input gates of the circuit plus
// the key XORs).  Planes are indexed by bit (x[0] = least significant).  The
// linear maps as greedy programs of two- and three-input XORs: mix_column_lut3
// is MixColumns ({count["mix"]} tables) and dec_mix_column_lut3 the decryption's
// A^-1 InvMixColumns A^-1 ({count["dec_mix"]}), on the 32 planes of one state column
// (x[8q + t] = bit t of row q); affine_inv_byte_lut3 is A^-1 on one byte's 8
// planes ({count["affine_inv"]}).  lop(a, b, c, Tt<imm>) returns the function whose truth
// table imm lists F(a, b, c) at bit 4a + 2b + c (the table travels as a type, so
// that it stays a compile-time constant).
#pragma once

#include <cstdint>
#include <type_traits>

#ifndef GBAES_HD
#ifdef __CUDACC__
#define GBAES_HD __host__ __device__
#else
#define GBAES_HD
#endif
#endif

namespace gbaes {{
namespace bs {{

template <uint32_t V>
using Tt = std::integral_constant<uint32_t, V>;

{emit(enc, enc_cover, "sbox_key_lut3")}
{code["mix"]}
{code["dec_mix"]}
{code["affine_inv"]}
}}  // namespace bs
}}  // namespace gbaes
"""
    with open(out, "w") as f:
        f.write(text)
    print(f"{os.path.basename(out)}: S-box {len(enc_cover)} tables; "
          + ", ".join(f"{k} {v}" for k, v in count.items()))


if __name__ == "__main__":
    main()
