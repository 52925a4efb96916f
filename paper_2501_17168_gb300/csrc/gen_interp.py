"""Generates the forward register-machine interpreter (interp_fwd.cuh) and
its instruction-set header (isa_fwd.cuh).

The forward instruction set.  A compiled tree is a sequence of 64-bit words
run by one warp over 32*K data points (K per lane).  The value of a subtree
evaluated at nesting level d lives in register group G[d] (K floats per lane);
level d is chosen by the stage compiler so that a binary node whose children
are both subtrees evaluates the child that needs more levels first into G[d]
and the other into G[d+1] (Sethi-Ullman order), then combines them into
G[d].  Nothing is ever copied between groups, so evaluation order costs no
moves.  Levels 0..NREG-1 are registers; deeper nesting (trees whose
Sethi-Ullman number exceeds NREG) saves G[NREG-1] on a memory stack and
combines with it later (the first NSM entries in per-warp shared-memory
rows, deeper ones in local memory).
Leaves never get an instruction of their own: a leaf operand rides in its
parent's word (feature index or constant bits), and a binary node with two
leaf children is one instruction (two words when the operands need more than
32 bits).  A Modi node (Sec. IV-C) adds its function value into its output
accumulator and leaves its rightmost child's value in the group.

Word layout: .x = opcode | out_index << 16 (Modi forms only), .y = operand.
Opcodes are form_base + sub * NREG + d for the level forms (sub = function
index) and form_base + sub for the memory-stack forms (push and pop through
a stack-pointer register).

Why PTX: the instruction stream is warp-uniform, so the ideal dispatch is
one indirect branch per instruction; a C++ switch is lowered to a compare
tree and shuffles the register groups at every case.  A hand-written loop
keeps every group in fixed registers and dispatches with one brx.idx over a
.branchtargets table.

The FP32 function bodies:
  add/sub/mul   add.rn / sub.rn / mul.rn (never contracted)
  pdiv(a,b)     |b| > 1e-6f ? a * rcp.approx(b) : 1  (flush to zero)
  max           max.f32 (a NaN operand yields the other one)
  sin/cos(a)    Cody-Waite reduction r = a - k*C1 - k*C2, k = rint(a/(2pi))
                (rint by the 1.5*2^23 addition trick, so it stays on the FMA
                pipe), then sin.approx / cos.approx of r
  plog(a)       |a| > 1e-6f ? lg2.approx(|a|) * ln2 : 0
  cexp(a)       ex2.approx.ftz(min(a, 80) * log2 e)
  tan(a)        sin.approx(r) * rcp.approx(cos.approx(r))
Every add, sub, mul and fma of these bodies (and of the Modi accumulation)
runs on two points at once as the packed f32x2 form, each half rounded like
the scalar instruction; the issue slots it saves are what bounds this
interpreter.  max, the guards and the approximations stay scalar (PTX has no
packed form of them).

The OP_* constants below are the accumulator-and-slots instruction set that
the adjoint kernel runs (tgp_internal.cuh, enum Op); gen_interp_bwd.py
imports them together with the function constants.

Run `python gen_interp.py` to regenerate (the build does it when stale).
"""
from __future__ import annotations

import os
import struct

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "interp_fwd.cuh")
OUT_ISA = os.path.join(HERE, "isa_fwd.cuh")

R = 8
F_ADD, F_SUB, F_MUL, F_PDIV, F_MAX, F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN, F_ITE = range(11)
BIN = [F_ADD, F_SUB, F_MUL, F_PDIV, F_MAX]   # binary functions of the adjoint set
UNA = [F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN]
# binary forms of the forward set: the binary functions, then ite's branch
# selection (its condition is pushed by a CD form before the branches)
FBIN = BIN + [F_ITE]

# opcode layout (must match enum Op in tgp_internal.cuh)
OP_END_ROOT, OP_END_MODI, OP_LDV, OP_LDC = 0, 1, 2, 3
OP_UN, OP_UNV, OP_BV, OP_BC, OP_RV, OP_RC = 4, 9, 14, 19, 24, 29
OP_UN_M, OP_BV_M, OP_BC_M, OP_RV_M, OP_RC_M = 34, 39, 44, 49, 54
OP_SPV, OP_SPC, OP_BS, OP_RS, OP_BS_M, OP_RS_M = 59, 67, 75, 115, 155, 195
OP_COUNT = 235


def fhex(x: float) -> str:
    return "0f%08X" % struct.unpack(">I", struct.pack(">f", x))[0]


GUARD = fhex(1e-6)
ONE = fhex(1.0)
ZERO = fhex(0.0)
CLAMP = fhex(80.0)
LOG2E = fhex(1.442695)        # log2(e) rounded to float
LN2 = fhex(0.6931472)         # ln(2) rounded to float
INV2PI = fhex(0.15915494)     # 1/(2pi) rounded to float
C1 = fhex(6.28125)            # 2pi split: 8 significant bits ...
C2 = fhex(1.9353072e-3)       # ... and the rest, rounded to float
MAGIC = fhex(12582912.0)      # 1.5 * 2^23: x + MAGIC - MAGIC = rint(x) for |x| < 2^22


# ------------------------------------------------------------------ forward ISA
NREG = 3          # nesting levels held in registers
MAXS = 6          # local-memory stack entries: trees of <= 1024 nodes need <= 9 levels
NC = [F_SUB, F_PDIV, F_ITE]   # non-commutative binary forms (max is symmetric in PTX)
NB = len(FBIN)


def bi(f):
    """Sub-index of a binary form's function."""
    return FBIN.index(f)

# (name, number of sub-forms); level forms come first, then memory forms
LEVEL_FORMS = [
    ("LDV", 1), ("LDC", 1),                       # G[d] = x[v] / c (only a lone leaf)
    ("UN", 5), ("UNV", 5), ("UNC", 5),            # G[d] = f(G[d]) / f(x[v]) / f(c)
    ("BV", NB), ("BC", NB),                       # G[d] = f(G[d], x[v]) / f(G[d], c)
    ("RV", 3), ("RC", 3),                         # G[d] = f(x[v], G[d]) / f(c, G[d])
    ("VV", NB),                                   # G[d] = f(x[v1], x[v2]), y = v1 | v2 << 16
    ("VC", NB), ("CV", 3),                        # f(x[v], c) / f(c, x[v]); second word .x = v
    ("CC", NB),                                   # f(c1, c2); second word .x = bits of c2
    ("BS", NB), ("RS", 3),                        # G[d] = f(G[d], G[d+1]) / f(G[d+1], G[d])
    ("UN_M", 5), ("UNV_M", 5), ("UNC_M", 5),      # Modi: out += f(.), G[d] = the operand
    ("BV_M", NB), ("BC_M", NB), ("RV_M", NB), ("RC_M", NB),
    ("BS_M", NB), ("RS_M", NB),
    ("CD", 1), ("CDV", 1), ("CDC", 1),            # push the sign bits of G[d] / x[v] / c > 0
]
NSM = 1           # memory-stack entries held in shared memory (the deeper ones in local memory)
MEM_FORMS = [
    ("SAVE", 1),                                  # push G[NREG-1] (local memory)
    ("MS", NB), ("SM", 3),                        # pop m: G = f(m, G) / f(G, m)  (G = G[NREG-1])
    ("MS_M", NB), ("SM_M", NB),
    ("SAVES", NSM),                               # the same for entry s < NSM in shared memory
    ("MSS", NB * NSM), ("SMS", 3 * NSM),          #   (sub = f * NSM + s)
    ("MSS_M", NB * NSM), ("SMS_M", NB * NSM),
    ("PUSHS", None), ("PUSHL", None),             # push G[NREG-1] (shared-memory entry 0 / local
                                                  # memory), then run a subtree's first instruction
]
# The forms that can start a subtree (its first instruction loads a leaf), in
# the order of the PUSHS/PUSHL sub-forms: the instruction after a push is
# always one of these at level NREG-1, so the push rides in its word
START_FORMS = [("LDV", 1), ("LDC", 1), ("CDV", 1), ("CDC", 1), ("UNV", 5), ("UNC", 5),
               ("UNV_M", 5), ("UNC_M", 5), ("VV", NB), ("VC", NB), ("CV", 3), ("CC", NB)]
NSTART = sum(n for _, n in START_FORMS)
assert NSM == 1  # the fused pushes address shared-memory entry 0 only
MEM_FORMS = [(name, NSTART if n is None else n) for name, n in MEM_FORMS]
MAXC = 8          # pending ite conditions: 64 condition bits, 8 points per lane


def isa_layout():
    base, op = {}, 2
    for name, n in LEVEL_FORMS:
        base[name] = op
        op += n * NREG
    for name, n in MEM_FORMS:
        base[name] = op
        op += n
    return base, op


FX_BASE, FX_COUNT = isa_layout()


def fx(name, sub, lvl):
    n = dict(LEVEL_FORMS + MEM_FORMS)[name]
    assert 0 <= sub < n
    if name in dict(MEM_FORMS):
        assert lvl == 0
        return FX_BASE[name] + sub
    assert 0 <= lvl < NREG
    return FX_BASE[name] + sub * NREG + lvl


def layout_key(op):
    """Position of a case in the generated code.  The interpreter is bound
    by instruction fetch, and the order of the cases in the code matters:
    level-major order (all forms of level 0, then level 1, ...; within a
    level the forms in LEVEL_FORMS order, then the function) with the
    rarely used tan forms moved to the end measured fastest among the
    orders tried (generation order, form-major, hot-forms-first,
    function-major within a level, frequency order within a level)."""
    names = sorted(FX_BASE.items(), key=lambda kv: kv[1])
    name, base = max(((n, b) for n, b in names if b <= op), key=lambda nb: nb[1])
    order = [n for n, _ in LEVEL_FORMS + MEM_FORMS].index(name)
    if name in dict(MEM_FORMS):
        sub, lvl = op - base, NREG
    else:
        sub, lvl = divmod(op - base, NREG)
    cold = name in ("UN", "UNV", "UNC", "UN_M", "UNV_M", "UNC_M") and UNA[sub] == F_TAN
    # ite's forms are rare (and absent from most function sets): kept cold
    cold |= name in ("CD", "CDV", "CDC")
    binf = {"BV", "BC", "VV", "VC", "CC", "BS", "BV_M", "BC_M", "RV_M", "RC_M", "BS_M", "RS_M",
            "MS", "MS_M", "SM_M"}
    if name in binf:
        cold |= sub == bi(F_ITE)
    if name in ("MSS", "MSS_M", "SMS_M"):
        cold |= sub // NSM == bi(F_ITE)
    if name in ("RV", "RC", "CV", "RS", "SM"):
        cold |= sub == NC.index(F_ITE)
    if name == "SMS":
        cold |= sub // NSM == NC.index(F_ITE)
    return (1 if cold else 0, lvl, order, sub)


class Gen:
    def __init__(self, K: int, modi: bool):
        self.K = K
        self.modi = modi
        self.lines: list[str] = []
        self.defined: set[int] = set()
        self.chunks: list = []

    def e(self, s: str):
        self.lines.append(s)

    # ---- register names
    @staticmethod
    def G(d):
        return lambda j: f"G{d}_{j}"

    @staticmethod
    def named(p):
        return lambda j: f"{p}{j}"

    # ---- operand loads
    def load_x(self, dst, idx):
        """dst[j] = X tile value of the lane's point j, feature = register idx."""
        self.e(f"mad.lo.u32 r_ad, {idx}, r_xstr, r_xc;")
        for h in range(self.K // 4):
            off = f"+{512 * h}" if h else ""
            self.e(f"ld.shared.v4.f32 {{{dst(4*h)}, {dst(4*h+1)}, {dst(4*h+2)}, {dst(4*h+3)}}}, [r_ad{off}];")

    def refetch(self):
        """Skips the second word of a two-word instruction (already in r_nx)."""
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr+8];")
        self.e("add.u32 r_ptr, r_ptr, 8;")

    def movs(self, dst, src):
        for j in range(self.K):
            self.e(f"mov.f32 {dst(j)}, {src(j)};")

    def mem_pop(self, dst):
        """dst = top of the memory stack (r_sp = local address one past it)."""
        K = self.K
        self.e(f"sub.u32 r_sp, r_sp, {K * 4};")
        for h in range(K // 4):
            self.e(f"ld.local.v4.f32 {{{dst(4*h)}, {dst(4*h+1)}, {dst(4*h+2)}, {dst(4*h+3)}}}, "
                   f"[r_sp+{16 * h}];")

    def mem_push(self, src):
        K = self.K
        for h in range(K // 4):
            self.e(f"st.local.v4.f32 [r_sp+{16 * h}], "
                   f"{{{src(4*h)}, {src(4*h+1)}, {src(4*h+2)}, {src(4*h+3)}}};")
        self.e(f"add.u32 r_sp, r_sp, {K * 4};")

    # ---- function bodies: out[j] = f(a[j], b[j]); a, b, out are name functions
    def fn2(self, f, out, a, b):
        if f == F_ITE:
            # pop the condition bits of the K points: out = cond ? a : b
            self.e("cvt.u32.u64 r_c, r_cs;")
            for j in range(self.K):
                self.e(f"and.b32 r_ct, r_c, {1 << j};")
                self.e(f"setp.ne.u32 P{j}, r_ct, 0;")
                self.e(f"selp.f32 {out(j)}, {a(j)}, {b(j)}, P{j};")
            self.e(f"shr.b64 r_cs, r_cs, {self.K};")
            return
        if f in (F_ADD, F_SUB, F_MUL):
            name = {F_ADD: "add", F_SUB: "sub", F_MUL: "mul"}[f]
            for h in range(self.K // 2):
                self.p2(f"{name}.rn.f32x2", out, h, a, b)
            return
        for j in range(self.K):
            o, x, y = out(j), a(j), b(j)
            if f == F_MAX:
                self.e(f"max.f32 {o}, {x}, {y};")
            elif f == F_PDIV:
                # a * rcp(b) in flush-to-zero arithmetic: for |b| > 2^126
                # the reciprocal is subnormal and flushes to 0, a deviation
                # of at most |a| 2^-126 (the oracle's pdiv allowance)
                self.e(f"abs.f32 V{j}, {y};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"rcp.approx.ftz.f32 V{j}, {y};")
        if f == F_PDIV:
            V = self.named("V")
            for h in range(self.K // 2):
                self.p2("mul.rn.f32x2", V, h, a, V)
            for j in range(self.K):
                self.e(f"selp.f32 {out(j)}, V{j}, {ONE}, P{j};")

    # ---- packed FP32 (f32x2: two points per instruction, each rounded as
    # the scalar operation would be)
    def pair(self, src, h):
        """A .b64 operand holding src's points 2h and 2h+1: a packed register
        pair, or a constant (hex float literal) in both halves."""
        if isinstance(src, str):
            return "0x" + src[2:] * 2
        return "{" + f"{src(2 * h)}, {src(2 * h + 1)}" + "}"

    def p2(self, op, out, h, *srcs):
        """out[2h, 2h+1] = op(srcs...) on the pair of points 2h, 2h+1."""
        names = []
        for i, s_ in enumerate(srcs):
            self.e(f"mov.b64 QP{i}, {self.pair(s_, h)};")
            names.append(f"QP{i}")
        self.e(f"{op} QP3, {', '.join(names)};")
        self.e(f"mov.b64 {{{out(2 * h)}, {out(2 * h + 1)}}}, QP3;")

    def reduce(self, a):
        """V[j] = a[j] reduced by 2pi (Cody-Waite), W[j] scratch, two points
        per instruction."""
        V, W = self.named("V"), self.named("W")
        for h in range(self.K // 2):
            self.p2("mul.rn.f32x2", W, h, a, INV2PI)
            self.p2("add.rn.f32x2", W, h, W, MAGIC)
            self.p2("sub.rn.f32x2", W, h, MAGIC, W)      # -rint(x / 2pi)
            self.p2("fma.rn.f32x2", V, h, W, C1, a)
            self.p2("fma.rn.f32x2", V, h, W, C2, V)

    def fn1(self, f, out, a):
        K = self.K
        V, W = self.named("V"), self.named("W")
        if f in (F_SIN, F_COS, F_TAN):
            self.reduce(a)
            for j in range(K):
                if f == F_SIN:
                    self.e(f"sin.approx.ftz.f32 {out(j)}, V{j};")
                elif f == F_COS:
                    self.e(f"cos.approx.ftz.f32 {out(j)}, V{j};")
                else:
                    self.e(f"cos.approx.ftz.f32 W{j}, V{j};")
                    self.e(f"sin.approx.ftz.f32 V{j}, V{j};")
                    self.e(f"rcp.approx.ftz.f32 W{j}, W{j};")
            if f == F_TAN:
                for h in range(K // 2):
                    self.p2("mul.rn.f32x2", out, h, V, W)
        elif f == F_PLOG:
            for j in range(K):
                self.e(f"abs.f32 V{j}, {a(j)};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"lg2.approx.ftz.f32 V{j}, V{j};")
            for h in range(K // 2):
                self.p2("mul.rn.f32x2", V, h, V, LN2)
            for j in range(K):
                self.e(f"selp.f32 {out(j)}, V{j}, {ZERO}, P{j};")
        elif f == F_CEXP:
            for j in range(K):
                self.e(f"min.f32 V{j}, {a(j)}, {CLAMP};")
            for h in range(K // 2):
                self.p2("mul.rn.f32x2", V, h, V, LOG2E)
            for j in range(K):
                self.e(f"ex2.approx.ftz.f32 {out(j)}, V{j};")

    def modi_add(self, src):
        """out[o][lane points] += src[j] (o from bits 16..23 of the word)."""
        K = self.K
        self.e("bfe.u32 r_moo, r_ix, 16, 8;")
        self.e(f"mad.lo.u32 r_ma, r_moo, {128 * K}, r_mo;")
        for h in range(K // 4):
            regs = [f"M{4 * h + q}" for q in range(4)]
            off = f"+{512 * h}" if h else ""
            self.e(f"ld.shared.v4.f32 {{{', '.join(regs)}}}, [r_ma{off}];")
        M = self.named("M")
        for h in range(K // 2):
            self.p2("add.rn.f32x2", M, h, M, src)
        for h in range(K // 4):
            regs = [f"M{4 * h + q}" for q in range(4)]
            off = f"+{512 * h}" if h else ""
            self.e(f"st.shared.v4.f32 [r_ma{off}], {{{', '.join(regs)}}};")

    def cond(self, src, scalar=False):
        """Pushes the K sign bits (value > 0; NaN is not) of src onto the
        condition stack r_cs (K bits per entry, the newest in the low bits)."""
        K = self.K
        if scalar:
            self.e(f"setp.gt.f32 P0, {src(0)}, 0f00000000;")
            self.e(f"selp.u32 r_cb, {(1 << K) - 1}, 0, P0;")
        else:
            self.e("mov.u32 r_cb, 0;")
            for j in range(K):
                self.e(f"setp.gt.f32 P{j}, {src(j)}, 0f00000000;")
                self.e(f"selp.u32 r_ct, {1 << j}, 0, P{j};")
                self.e("or.b32 r_cb, r_cb, r_ct;")
        self.e("cvt.u64.u32 r_cb64, r_cb;")
        self.e(f"shl.b64 r_cs, r_cs, {K};")
        self.e("or.b64 r_cs, r_cs, r_cb64;")

    def case(self, op, body, then=None):
        """Label C<op>, its body, then back to the dispatch (or on to `then`:
        another case's opcode or a body label)."""
        assert op not in self.defined
        self.defined.add(op)
        start = len(self.lines)
        self.e(f"C{op}:")
        body()
        if then is None:
            self.e("bra.uni LOOP;")
        else:
            self.e(f"bra.uni {then};" if isinstance(then, str) else f"bra.uni C{then};")
        self.chunks.append((layout_key(op), self.lines[start:]))
        del self.lines[start:]

    def body(self, label, body):
        """A combining body reached only by bra from cases; placed with the
        memory-stack cases."""
        start = len(self.lines)
        self.e(f"{label}:")
        body()
        self.e("bra.uni LOOP;")
        self.chunks.append(((0, NREG, -1, len(self.chunks)), self.lines[start:]))
        del self.lines[start:]

    def build(self) -> str:
        K = self.K
        G = self.G
        L, T = self.named("L"), self.named("T")
        cv = lambda j: "cv"
        c2 = lambda j: "c2v"
        top = NREG - 1
        self.e("{")
        temps = [f"{p}{j}" for p in "LTVWM" for j in range(K)]
        self.e(".reg .f32 " + ", ".join(temps) + ", cv, c2v;")
        self.e(".reg .f32 " + ", ".join(G(d)(j) for d in range(NREG) for j in range(K)) + ";")
        self.e(".reg .pred " + ", ".join(f"P{j}" for j in range(K)) + ";")
        self.e(".reg .b64 QP0, QP1, QP2, QP3;")
        self.e(".reg .u32 r_ptr, r_ix, r_iy, r_nx, r_ny, r_op, r_ad, r_xc, r_xstr, r_mo, r_moo, "
               "r_ma, r_flag, r_t, r_sp, r_sb, r_c, r_cb, r_ct;")
        self.e(".reg .b64 r_cs, r_cb64;")
        self.e("mov.b64 r_cs, 0;")
        # the Modi kernel keeps the NSM shared-memory entries in local memory too
        n_local = MAXS + (NSM if self.modi else 0)
        self.e(f".local .align 16 .b8 gm[{n_local * K * 4}];")
        self.e("mov.u32 r_sp, gm;")
        self.e("mov.u32 r_sb, %{sb};")
        self.e("mov.u32 r_ptr, %{pg};")
        self.e("mov.u32 r_xc, %{xc};")
        self.e("mov.u32 r_xstr, %{xstr};")
        self.e("mov.u32 r_mo, %{mo};")
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr];")
        self.e("LOOP:")
        self.e("mov.b32 r_ix, r_nx;")
        self.e("mov.b32 r_iy, r_ny;")
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr+8];")
        self.e("add.u32 r_ptr, r_ptr, 8;")
        self.e("mov.b32 cv, r_iy;")
        if self.modi:
            self.e("and.b32 r_op, r_ix, 65535;")
            self.e("brx.idx.uni r_op, TS;")
        else:
            # plain programs carry nothing above the opcode
            self.e("brx.idx.uni r_ix, TS;")

        self.e("C0:")
        self.e("mov.u32 r_flag, 0;")
        self.e("bra.uni DONE;")
        self.e("C1:")
        self.e("mov.u32 r_flag, 1;")
        self.e("bra.uni DONE;")
        self.defined.update((0, 1))

        for d in range(NREG):
            Gd = G(d)
            self.case(fx("LDV", 0, d), lambda: self.load_x(Gd, "r_iy"))
            self.case(fx("LDC", 0, d), lambda: self.movs(Gd, cv))
            # ite's condition: G[d] holds nothing live until the branches, so
            # a leaf condition is loaded there
            self.case(fx("CD", 0, d), lambda: self.cond(Gd))
            self.case(fx("CDV", 0, d), lambda: (self.load_x(Gd, "r_iy"), self.cond(Gd)))
            self.case(fx("CDC", 0, d), lambda: self.cond(cv, scalar=True))
            for u, f in enumerate(UNA):
                un = fx("UN", u, d)
                self.case(un, lambda f=f: self.fn1(f, Gd, Gd))
                self.case(fx("UNV", u, d), lambda: self.load_x(Gd, "r_iy"), then=un)
                self.case(fx("UNC", u, d), lambda: self.movs(Gd, cv), then=un)
            # levels above d hold no live value while an instruction of level d
            # runs, so below the top level a leaf operand is loaded into
            # G[d+1] and the slot-combining body of BS/RS is reused
            Gn = G(d + 1) if d < top else L
            for f in FBIN:
                bv, bc = fx("BV", bi(f), d), fx("BC", bi(f), d)
                if d < top:
                    self.case(bv, lambda: self.load_x(Gn, "r_iy"), then=fx("BS", bi(f), d))
                else:
                    self.case(bv, lambda f=f: (self.load_x(L, "r_iy"), self.fn2(f, Gd, Gd, L)))
                self.case(bc, lambda f=f: self.fn2(f, Gd, Gd, cv))

                def vv():
                    self.e("and.b32 r_t, r_iy, 65535;")
                    self.load_x(Gd, "r_t")
                    self.e("shr.u32 r_iy, r_iy, 16;")
                    if d < top:
                        self.load_x(Gn, "r_iy")

                self.case(fx("VV", bi(f), d), vv, then=fx("BS", bi(f), d) if d < top else bv)

                def vc():
                    self.load_x(Gd, "r_nx")
                    self.refetch()

                self.case(fx("VC", bi(f), d), vc, then=bc)

                def cc(f=f):
                    self.e("mov.b32 c2v, r_nx;")
                    self.refetch()
                    self.fn2(f, Gd, cv, c2)

                self.case(fx("CC", bi(f), d), cc)
                if d < top:
                    self.case(fx("BS", bi(f), d), lambda f=f: self.fn2(f, Gd, Gd, G(d + 1)))
            for i, f in enumerate(NC):
                rc = fx("RC", i, d)
                if d < top:
                    self.case(fx("RV", i, d), lambda: self.load_x(Gn, "r_iy"), then=fx("RS", i, d))
                else:
                    self.case(fx("RV", i, d), lambda f=f: (self.load_x(L, "r_iy"), self.fn2(f, Gd, L, Gd)))
                self.case(rc, lambda f=f: self.fn2(f, Gd, cv, Gd))

                def cvx():
                    self.load_x(Gd, "r_nx")
                    self.refetch()

                self.case(fx("CV", i, d), cvx, then=rc)
                if d < top:
                    self.case(fx("RS", i, d), lambda f=f: self.fn2(f, Gd, G(d + 1), Gd))
            if not self.modi:
                continue
            for u, f in enumerate(UNA):
                unm = fx("UN_M", u, d)
                self.case(unm, lambda f=f: (self.fn1(f, T, Gd), self.modi_add(T)))
                self.case(fx("UNV_M", u, d), lambda: self.load_x(Gd, "r_iy"), then=unm)
                self.case(fx("UNC_M", u, d), lambda: self.movs(Gd, cv), then=unm)
            for f in FBIN:
                def bvm(f=f):
                    self.load_x(L, "r_iy")
                    self.fn2(f, T, Gd, L)
                    self.modi_add(T)
                    self.movs(Gd, L)

                def bcm(f=f):
                    self.fn2(f, T, Gd, cv)
                    self.modi_add(T)
                    self.movs(Gd, cv)

                def rvm(f=f):
                    self.load_x(L, "r_iy")
                    self.fn2(f, T, L, Gd)
                    self.modi_add(T)

                def rcm(f=f):
                    self.fn2(f, T, cv, Gd)
                    self.modi_add(T)

                if d < top:
                    # the leaf operand goes to G[d+1]; BS_M/RS_M do the rest
                    self.case(fx("BV_M", bi(f), d), lambda: self.load_x(Gn, "r_iy"), then=fx("BS_M", bi(f), d))
                    self.case(fx("BC_M", bi(f), d), lambda: self.movs(Gn, cv), then=fx("BS_M", bi(f), d))
                    self.case(fx("RV_M", bi(f), d), lambda: self.load_x(Gn, "r_iy"), then=fx("RS_M", bi(f), d))
                    self.case(fx("RC_M", bi(f), d), lambda: self.movs(Gn, cv), then=fx("RS_M", bi(f), d))
                else:
                    self.case(fx("BV_M", bi(f), d), bvm)
                    self.case(fx("BC_M", bi(f), d), bcm)
                    self.case(fx("RV_M", bi(f), d), rvm)
                    self.case(fx("RC_M", bi(f), d), rcm)
                if d < top:
                    def bsm(f=f):
                        self.fn2(f, T, Gd, G(d + 1))
                        self.modi_add(T)
                        self.movs(Gd, G(d + 1))

                    def rsm(f=f):
                        self.fn2(f, T, G(d + 1), Gd)
                        self.modi_add(T)

                    self.case(fx("BS_M", bi(f), d), bsm)
                    self.case(fx("RS_M", bi(f), d), rsm)

        # memory stack: entry s < NSM in the warp's shared-memory rows, deeper
        # entries in local memory; a pop loads the entry into L and goes on
        # in a combining body shared by both kinds of entry
        Gt = G(top)
        sm_off = lambda q, h: f"[r_sb+{q * 128 * K + 512 * h}]"

        # (the Modi kernel keeps the whole stack in local memory: its shared
        # memory holds the Modi accumulators; the order of pushes and pops is
        # the same, so the shared-memory forms become local pushes and pops)
        def sm_push(q):
            if self.modi:
                return self.mem_push(Gt)
            for h in range(K // 4):
                regs = ", ".join(Gt(4 * h + i) for i in range(4))
                self.e(f"st.shared.v4.f32 {sm_off(q, h)}, {{{regs}}};")

        def sm_pop(q):
            if self.modi:
                return self.mem_pop(L)
            for h in range(K // 4):
                regs = ", ".join(L(4 * h + i) for i in range(4))
                self.e(f"ld.shared.v4.f32 {{{regs}}}, {sm_off(q, h)};")

        self.case(fx("SAVE", 0, 0), lambda: self.mem_push(Gt))
        for q in range(NSM):
            self.case(fx("SAVES", q, 0), lambda q=q: sm_push(q))
        for f in FBIN:
            self.body(f"MSB{f}", lambda f=f: self.fn2(f, Gt, L, Gt))
            self.case(fx("MS", bi(f), 0), lambda: self.mem_pop(L), then=f"MSB{f}")
            for q in range(NSM):
                self.case(fx("MSS", bi(f) * NSM + q, 0), lambda q=q: sm_pop(q), then=f"MSB{f}")
        for i, f in enumerate(NC):
            self.body(f"SMB{i}", lambda f=f: self.fn2(f, Gt, Gt, L))
            self.case(fx("SM", i, 0), lambda: self.mem_pop(L), then=f"SMB{i}")
            for q in range(NSM):
                self.case(fx("SMS", i * NSM + q, 0), lambda q=q: sm_pop(q), then=f"SMB{i}")
        if self.modi:
            for f in FBIN:
                def msm(f=f):
                    self.fn2(f, T, L, Gt)
                    self.modi_add(T)

                def smm(f=f):
                    self.fn2(f, T, Gt, L)
                    self.modi_add(T)
                    self.movs(Gt, L)

                self.body(f"MSMB{f}", msm)
                self.body(f"SMMB{f}", smm)
                self.case(fx("MS_M", bi(f), 0), lambda: self.mem_pop(L), then=f"MSMB{f}")
                self.case(fx("SM_M", bi(f), 0), lambda: self.mem_pop(L), then=f"SMMB{f}")
                for q in range(NSM):
                    self.case(fx("MSS_M", bi(f) * NSM + q, 0), lambda q=q: sm_pop(q), then=f"MSMB{f}")
                    self.case(fx("SMS_M", bi(f) * NSM + q, 0), lambda q=q: sm_pop(q), then=f"SMMB{f}")

        # a push fused into the first instruction of the subtree that follows
        # it: store G[NREG-1], then go on in that instruction's own case
        i = 0
        for name, n in START_FORMS:
            for sub in range(n):
                target = fx(name, sub, top)
                if target in self.defined:
                    self.case(fx("PUSHS", i, 0), lambda: sm_push(0), then=target)
                    self.case(fx("PUSHL", i, 0), lambda: self.mem_push(Gt), then=target)
                i += 1

        # the cases in code order (see layout_key)
        for _, chunk in sorted(self.chunks, key=lambda c: c[0]):
            self.lines.extend(chunk)
        # opcodes the stage compiler never emits for this kernel: end with NaN
        self.e("CBAD:")
        for j in range(K):
            self.e(f"mov.f32 G0_{j}, 0f7FC00000;")
        self.e("mov.u32 r_flag, 0;")
        self.e("bra.uni DONE;")
        self.e("DONE:")
        for j in range(K):
            self.e(f"mov.f32 %{{a{j}}}, G0_{j};")
        self.e("mov.u32 %{flag}, r_flag;")
        self.e("}")
        # the jump table goes right after the dispatch
        table = "TS: .branchtargets " + ", ".join(
            (f"C{k}" if k in self.defined else "CBAD") for k in range(FX_COUNT)) + ";"
        i = self.lines.index("C0:")
        self.lines.insert(i - 3 if self.modi else i - 2, table)
        return "\n".join(self.lines)


def operand_map(K):
    names = [f"a{j}" for j in range(K)] + ["flag", "pg", "xc", "xstr", "mo", "sb"]
    return {n: i for i, n in enumerate(names)}


def render(K: int, modi: bool) -> str:
    body = Gen(K, modi).build()
    m = operand_map(K)
    for n, i in m.items():
        body = body.replace("%{" + n + "}", f"%{i}")
    # C string literal, one PTX line per source line
    lit = "\n".join('      "' + l.replace("\\", "\\\\").replace('"', '\\"') + '\\n"' for l in body.split("\n"))
    outs = ", ".join([f'"=f"(acc[{j}])' for j in range(K)] + ['"=r"(flag)'])
    ins = '"r"(pg), "r"(xc), "r"(xstr), "r"(mo), "r"(sb)'
    return f"""template <>
__device__ __forceinline__ unsigned interp_fwd<{K}, {'true' if modi else 'false'}>(
    unsigned pg, unsigned xc, unsigned xstr, unsigned mo, unsigned sb, float (&acc)[{K}]) {{
  unsigned flag;
  asm volatile(
{lit}
      : {outs}
      : {ins}
      : "memory");
  return flag;
}}
"""


def render_isa() -> str:
    out = [
        "// isa_fwd.cuh -- GENERATED by gen_interp.py; do not edit by hand.",
        "// Opcodes of the forward instruction set run by interp_fwd (level registers",
        "// G[0..NREG-1], a memory stack of NSM shared-memory entries per warp and",
        "// MAXS local-memory entries per thread).  A level form's",
        "// opcode is base + sub * NREG + d, a memory form's base + sub; sub is the",
        "// unary index f - F_SIN, the binary function f, or for the forms that exist",
        "// only for non-commutative functions nc_index(f), bin_index(f) for the",
        "// others.  Word: .x = opcode |",
        "// out_index << 16 (Modi forms), .y = operand; VC/CV/CC take a second word",
        "// whose .x is the feature index (VC, CV) or the bits of the second constant",
        "// (CC).",
        "#pragma once",
        "#include <cstdint>",
        "namespace tgp {",
        "namespace fx {",
        f"constexpr int NREG = {NREG};",
        f"constexpr int MAXS = {MAXS};",
        f"constexpr int NSM = {NSM};   // stack entries in shared memory (SAVES/MSS/SMS forms; the",
        "                           // Modi kernel keeps them in local memory)",
        "enum : uint32_t {",
        "  END_ROOT = 0,  // output := G[0] (one output, no Modi node)",
        "  END_MODI = 1,  // outputs are the Modi accumulators",
    ]
    for name, _ in LEVEL_FORMS + MEM_FORMS:
        out.append(f"  {name} = {FX_BASE[name]},")
    out.append(f"  COUNT = {FX_COUNT}")
    out.append("};")
    out.append("// index of a non-commutative binary form's function among the RV/RC/CV/RS/SM forms")
    out.append("__host__ __device__ constexpr int nc_index(int f) { return f == 1 ? 0 : f == 3 ? 1 : f == 10 ? 2 : -1; }")
    out.append("// index of a binary form's function (ite's branch selection after the binary functions)")
    out.append("__host__ __device__ constexpr int bin_index(int f) { return f <= 4 ? f : f == 10 ? 5 : -1; }")
    out.append(f"constexpr int MAXC = {MAXC};   // pending ite conditions the 64-bit condition stack holds")
    out.append(f"constexpr int NSTART = {NSTART};  // forms that can start a subtree (PUSHS/PUSHL sub-forms)")
    out.append("// The fused form \"push G[NREG-1] (to shared-memory entry 0, or to local")
    out.append("// memory when `local`), then run op\" for a subtree's first instruction op at")
    out.append("// level NREG-1; 0 when op has none (the push is then a word of its own).")
    out.append("__host__ __device__ constexpr uint32_t push_form(uint32_t op, bool local) {")
    out.append("  const uint32_t pb = local ? PUSHL : PUSHS;")
    i = 0
    for name, n in START_FORMS:
        out.append(f"  if (op >= {name} && op < {name} + {n} * NREG && (op - {name}) % NREG == NREG - 1)")
        out.append(f"    return pb + {i} + (op - {name}) / NREG;")
        i += n
    out.append("  return 0;")
    out.append("}")
    # the same map as a table for the stage compiler's serial emission loop
    # (one constant-memory load instead of the range checks)
    vals = []
    for op in range(FX_COUNT):
        v = 0
        i = 0
        for name, n in START_FORMS:
            for sub in range(n):
                if fx(name, sub, NREG - 1) == op:
                    v = FX_BASE["PUSHS"] + i
                i += 1
        vals.append(v)
    out.append("#ifdef __CUDACC__")
    out.append("// push_form(op, false) for every opcode; push_form(op, true) is that + NSTART")
    out.append("// where it is not 0")
    out.append("static __constant__ uint16_t PUSH_FORM_TABLE[COUNT] = {")
    for k in range(0, FX_COUNT, 16):
        out.append("    " + ", ".join(str(v) for v in vals[k:k + 16]) + ",")
    out.append("};")
    out.append("#endif")
    out.append("}  // namespace fx")
    out.append("}  // namespace tgp")
    return "\n".join(out) + "\n"


def main():
    parts = [
        "// interp_fwd.cuh -- GENERATED by gen_interp.py; do not edit by hand.",
        "// Forward interpreter loop of the level-register machine (isa_fwd.cuh).",
        "// interp_fwd<K, MODI>(pg, xc, xstr, mo, sb, acc): pg = shared address of",
        "// the program, xc = shared address of the lane's first point of feature 0,",
        "// xstr = bytes between feature rows, mo = shared address of the lane's Modi",
        "// accumulators, sb = shared address of the lane's 16 bytes in the warp's",
        "// memory-stack rows (NSM entries of K*128 bytes); returns 1 when the",
        "// outputs are the Modi sums, else 0 with the single output in acc.",
        "#pragma once",
        "namespace tgp {",
        "template <int K, bool MODI>",
        "__device__ __forceinline__ unsigned interp_fwd(unsigned pg, unsigned xc, unsigned xstr,",
        "                                               unsigned mo, unsigned sb, float (&acc)[K]);",
    ]
    for K, modi in ((8, False), (4, False), (4, True)):  # the kernels instantiated in eval.cu
        parts.append(render(K, modi))
    parts.append("}  // namespace tgp")
    open(OUT, "w").write("\n".join(parts) + "\n")
    open(OUT_ISA, "w").write(render_isa())
    return OUT


if __name__ == "__main__":
    print(main())
