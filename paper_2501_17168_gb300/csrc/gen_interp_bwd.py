"""Generates interp_bwd.cuh: the two inline-PTX loops of the adjoint kernel.

Both keep the eight slots in the warp's shared-memory slot area (one case
per instruction family, the slot number taken from the opcode), which keeps
the two loops small enough for the instruction cache.
bwd_forward<K, MODI>  runs a compiled program like the forward interpreter
                      and, per instruction, appends the local partials the
                      reverse sweep will need to a per-thread tape in local
                      memory (at most one entry per tree node):
                        unary f          f'(a)            (1 entry)
                        leaf-binary      mul/pdiv/max: the accumulator operand (1)
                        slot-binary      mul/pdiv/max: both operands (2)
                        add/sub, leaves  nothing
bwd_reverse<K, MODI>  walks the program from its last instruction to its
                      first with the adjoint of the accumulator in registers
                      (G, K points per lane) and of the eight slots, the
                      mirror image of the forward register machine: a slot
                      written by a spill in the forward is read back by that
                      spill's reverse, after the reverse of its consumer has
                      stored the slot's adjoint there.  Variable leaves add
                      their adjoint into the CTA's shared-memory gradient tile
                      of X (red.shared.add); constant leaves add the
                      warp-summed adjoint into a per-warp shared array
                      indexed by the leaf's node position.
Local derivatives (ties of max go to the operand fmax returned, left on a
tie; the guards of pdiv and plog and the clamp of cexp give zero
derivatives on their constant branches):
  add (1, 1)   sub (1, -1)   mul (b, a)   pdiv (1/b, -a/b^2)
  sin cos(a)   cos -sin(a)   plog 1/a   cexp exp(a) (a <= 80)   tan 1 + tan^2
Modi nodes (Sec. IV-C): the function value's adjoint is the seed of its
output; the value handed to the parent (the rightmost child) keeps the
parent's adjoint.
As in the forward interpreter, the adds, subtractions, multiplies and fmas
run as packed f32x2 pairs of points; the per-warp sums of constant
gradients keep their scalar order.
"""
from __future__ import annotations

import os

from gen_interp import (BIN, C1, C2, CLAMP, F_ADD, F_CEXP, F_COS, F_MAX, F_MUL, F_PDIV, F_PLOG,
                        F_SIN, F_SUB, F_TAN, GUARD, INV2PI, LN2, LOG2E, MAGIC, ONE, OP_BC, OP_BC_M,
                        OP_BS, OP_BS_M, OP_BV, OP_BV_M, OP_COUNT, OP_END_MODI, OP_END_ROOT, OP_LDC,
                        OP_LDV, OP_RC, OP_RC_M, OP_RS, OP_RS_M, OP_RV, OP_RV_M, OP_SPC, OP_SPV, OP_UN,
                        OP_UN_M, OP_UNV, R, UNA, ZERO, fhex)

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "interp_bwd.cuh")

NEEDS_OPERAND = (F_MUL, F_PDIV, F_MAX)


class Base:
    def __init__(self, K: int, modi: bool):
        assert K in (4, 8)
        self.K = K
        self.modi = modi
        self.lines: list[str] = []

    def e(self, s):
        self.lines.append(s)

    def vec(self, p, n=None):
        return lambda j: f"{p}{j}"

    def load_x(self, dst):
        self.e("mad.lo.u32 r_ad, r_iy, r_xstr, r_xc;")
        self.e(f"ld.shared.v4.f32 {{{dst(0)}, {dst(1)}, {dst(2)}, {dst(3)}}}, [r_ad];")
        if self.K == 8:
            self.e(f"ld.shared.v4.f32 {{{dst(4)}, {dst(5)}, {dst(6)}, {dst(7)}}}, [r_ad+512];")

    def tape_put(self, src):
        for h in range(self.K // 4):
            regs = ", ".join(src(4 * h + q) for q in range(4))
            self.e(f"st.local.v4.f32 [r_tape+{16 * h}], {{{regs}}};")
        self.e(f"add.u32 r_tape, r_tape, {4 * self.K};")

    def tape_get(self, dst):
        self.e(f"sub.u32 r_tape, r_tape, {4 * self.K};")
        for h in range(self.K // 4):
            regs = ", ".join(dst(4 * h + q) for q in range(4))
            self.e(f"ld.local.v4.f32 {{{regs}}}, [r_tape+{16 * h}];")

    # ---- packed FP32 (f32x2: two points per instruction, each rounded as
    # the scalar operation would be)
    @staticmethod
    def pair(src, h):
        if isinstance(src, str):          # a constant (hex float literal) in both halves
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

    def pk(self, op, out, *srcs):
        for h in range(self.K // 2):
            self.p2(op, out, h, *srcs)

    def reduce(self, a):
        """V[j] = a[j] reduced by 2pi (Cody-Waite), W[j] scratch."""
        V, W = self.vec("V"), self.vec("W")
        for h in range(self.K // 2):
            self.p2("mul.rn.f32x2", W, h, a, INV2PI)
            self.p2("add.rn.f32x2", W, h, W, MAGIC)
            self.p2("sub.rn.f32x2", W, h, MAGIC, W)
            self.p2("fma.rn.f32x2", V, h, W, C1, a)
            self.p2("fma.rn.f32x2", V, h, W, C2, V)

    def fn2(self, f, out, a, b):
        if f in (F_ADD, F_SUB, F_MUL):
            self.pk({F_ADD: "add", F_SUB: "sub", F_MUL: "mul"}[f] + ".rn.f32x2", out, a, b)
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
            V = self.vec("V")
            self.pk("mul.rn.f32x2", V, a, V)
            for j in range(self.K):
                self.e(f"selp.f32 {out(j)}, V{j}, {ONE}, P{j};")

    def fn1d(self, f, out, a, d):
        """out[j] = f(a[j]) and d[j] = f'(a[j]) (a is read before out is written)."""
        K = self.K
        V, W = self.vec("V"), self.vec("W")
        if f in (F_SIN, F_COS, F_TAN):
            self.reduce(a)
            for j in range(K):
                o, dd = out(j), d(j)
                if f == F_SIN:
                    self.e(f"cos.approx.ftz.f32 {dd}, V{j};")
                    self.e(f"sin.approx.ftz.f32 {o}, V{j};")
                elif f == F_COS:
                    self.e(f"sin.approx.ftz.f32 {dd}, V{j};")
                    self.e(f"neg.f32 {dd}, {dd};")
                    self.e(f"cos.approx.ftz.f32 {o}, V{j};")
                else:
                    self.e(f"cos.approx.ftz.f32 W{j}, V{j};")
                    self.e(f"sin.approx.ftz.f32 V{j}, V{j};")
                    self.e(f"rcp.approx.ftz.f32 W{j}, W{j};")
            if f == F_TAN:
                self.pk("mul.rn.f32x2", out, V, W)
                self.pk("fma.rn.f32x2", d, out, out, ONE)
        elif f == F_PLOG:
            for j in range(K):
                x = a(j)
                self.e(f"abs.f32 V{j}, {x};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"rcp.approx.ftz.f32 W{j}, {x};")
                self.e(f"selp.f32 {d(j)}, W{j}, {ZERO}, P{j};")
                self.e(f"lg2.approx.ftz.f32 V{j}, V{j};")
            self.pk("mul.rn.f32x2", V, V, LN2)
            for j in range(K):
                self.e(f"selp.f32 {out(j)}, V{j}, {ZERO}, P{j};")
        elif f == F_CEXP:
            for j in range(K):
                x = a(j)
                self.e(f"setp.le.f32 P{j}, {x}, {CLAMP};")
                self.e(f"min.f32 V{j}, {x}, {CLAMP};")
            self.pk("mul.rn.f32x2", V, V, LOG2E)
            for j in range(K):
                self.e(f"ex2.approx.ftz.f32 {out(j)}, V{j};")
                self.e(f"selp.f32 {d(j)}, {out(j)}, {ZERO}, P{j};")

    def modi_add(self, src):
        self.e("bfe.u32 r_moo, r_ix, 8, 8;")
        self.e(f"mad.lo.u32 r_ma, r_moo, {128 * self.K}, r_mo;")
        M = self.vec("M")
        for h in range(self.K // 4):
            regs = [f"M{4 * h + q}" for q in range(4)]
            off = f"+{512 * h}" if h else ""
            self.e(f"ld.shared.v4.f32 {{{', '.join(regs)}}}, [r_ma{off}];")
        self.pk("add.rn.f32x2", M, M, src)
        for h in range(self.K // 4):
            regs = [f"M{4 * h + q}" for q in range(4)]
            off = f"+{512 * h}" if h else ""
            self.e(f"st.shared.v4.f32 [r_ma{off}], {{{', '.join(regs)}}};")


class Fwd(Base):
    """forward interpreter that also records the tape"""

    def case(self, op, body):
        self.e(f"FC{op}:")
        body()
        self.e("bra.uni FLOOP;")

    def build(self):
        K = self.K
        A, L, T, c = self.vec("A"), self.vec("L"), self.vec("T"), (lambda j: "cv")
        S = lambda d: (lambda j: f"S{d}_{j}")
        regs = [f"{p}{j}" for p in ("A", "L", "T", "V", "W", "M", "SV") for j in range(K)]
        self.e("{")
        self.e(".reg .f32 " + ", ".join(regs) + ", cv;")
        self.e(".reg .pred " + ", ".join(f"P{j}" for j in range(K)) + ";")
        self.e(".reg .b64 QP0, QP1, QP2, QP3;")
        self.e(".reg .u32 r_ptr, r_ix, r_iy, r_nx, r_ny, r_op, r_ad, r_xc, r_xstr, r_mo, r_moo, r_ma, r_flag, r_tape, r_slot, r_d, r_sl;")
        self.e("mov.u32 r_slot, %{slot};")
        self.e("mov.u32 r_ptr, %{pg};")
        self.e("mov.u32 r_xc, %{xc};")
        self.e("mov.u32 r_xstr, %{xstr};")
        self.e("mov.u32 r_mo, %{mo};")
        self.e("mov.u32 r_tape, %{tape};")
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr];")
        self.e("FLOOP:")
        self.e("mov.b32 r_ix, r_nx;")
        self.e("mov.b32 r_iy, r_ny;")
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr+8];")
        self.e("add.u32 r_ptr, r_ptr, 8;")
        self.e("mov.b32 cv, r_iy;")
        self.e("and.b32 r_op, r_ix, 255;")
        self.e("FTS: .branchtargets " + ", ".join(fwd_label(k) for k in range(OP_COUNT)) + ";")
        self.e("brx.idx.uni r_op, FTS;")
        self.e(f"FC{OP_END_ROOT}:")
        self.e("mov.u32 r_flag, 0;")
        self.e("bra.uni FDONE;")
        self.e(f"FC{OP_END_MODI}:")
        self.e("mov.u32 r_flag, 1;")
        self.e("bra.uni FDONE;")
        self.case(OP_LDV, lambda: self.load_x(A))
        self.case(OP_LDC, lambda: [self.e(f"mov.f32 A{j}, cv;") for j in range(K)])
        for f in UNA:
            def un(f=f):
                self.fn1d(f, A, A, T)
                self.tape_put(T)

            def unv(f=f):
                self.load_x(L)
                self.fn1d(f, A, L, T)
                self.tape_put(T)

            def unm(f=f):
                if not self.modi:
                    return
                self.fn1d(f, L, A, T)        # value into L (scratch), derivative into T
                self.tape_put(T)
                self.modi_add(L)

            self.case(OP_UN + f - F_SIN, un)
            self.case(OP_UNV + f - F_SIN, unv)
            self.case(OP_UN_M + f - F_SIN, unm)
        for f in BIN:
            need = f in NEEDS_OPERAND

            def bv(f=f, need=need, modi=False):
                self.load_x(L)
                if need:
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, A, L)
                    self.modi_add(T)
                    for j in range(K):
                        self.e(f"mov.f32 A{j}, L{j};")
                else:
                    self.fn2(f, A, A, L)

            def bc(f=f, need=need, modi=False):
                if need:
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, A, c)
                    self.modi_add(T)
                    for j in range(K):
                        self.e(f"mov.f32 A{j}, cv;")
                else:
                    self.fn2(f, A, A, c)

            def rv(f=f, need=need, modi=False):
                self.load_x(L)
                if need:
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, L, A)
                    self.modi_add(T)
                else:
                    self.fn2(f, A, L, A)

            def rc(f=f, need=need, modi=False):
                if need:
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, c, A)
                    self.modi_add(T)
                else:
                    self.fn2(f, A, c, A)

            self.case(OP_BV + f, bv)
            self.case(OP_BC + f, bc)
            self.case(OP_RV + f, rv)
            self.case(OP_RC + f, rc)
            for op, fn in ((OP_BV_M, bv), (OP_BC_M, bc), (OP_RV_M, rv), (OP_RC_M, rc)):
                self.case(op + f, (lambda fn=fn: fn(modi=True)) if self.modi else (lambda: None))
        # slots live in the warp's shared-memory slot area ([R][32 lanes][K]);
        # one case per family, the slot index comes from the opcode
        def slot_addr(base):
            self.e(f"sub.u32 r_d, r_op, {base};")
            self.e(f"mad.lo.u32 r_sl, r_d, {128 * K}, r_slot;")

        def st_slot(src):
            for h in range(K // 4):
                regs = ", ".join(src(4 * h + q) for q in range(4))
                self.e(f"st.shared.v4.f32 [r_sl+{512 * h}], {{{regs}}};")

        def ld_slot(dst):
            for h in range(K // 4):
                regs = ", ".join(dst(4 * h + q) for q in range(4))
                self.e(f"ld.shared.v4.f32 {{{regs}}}, [r_sl+{512 * h}];")

        SV = self.vec("SV")
        self.e("FSPV:")
        slot_addr(OP_SPV)
        st_slot(A)
        self.load_x(A)
        self.e("bra.uni FLOOP;")
        self.e("FSPC:")
        slot_addr(OP_SPC)
        st_slot(A)
        for j in range(K):
            self.e(f"mov.f32 A{j}, cv;")
        self.e("bra.uni FLOOP;")
        for f in BIN:
            need = f in NEEDS_OPERAND

            def bs(f=f, need=need, modi=False, base=None):
                slot_addr(base)
                ld_slot(SV)
                if need:
                    self.tape_put(SV)
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, SV, A)
                    self.modi_add(T)
                else:
                    self.fn2(f, A, SV, A)

            def rs(f=f, need=need, modi=False, base=None):
                slot_addr(base)
                ld_slot(SV)
                if need:
                    self.tape_put(SV)
                    self.tape_put(A)
                if modi:
                    self.fn2(f, T, A, SV)
                    self.modi_add(T)
                    for j in range(K):
                        self.e(f"mov.f32 A{j}, SV{j};")
                else:
                    self.fn2(f, A, A, SV)

            for lab, fn, base, modi in ((f"FBS{f}", bs, OP_BS + f * R, False), (f"FRS{f}", rs, OP_RS + f * R, False),
                                        (f"FBSM{f}", bs, OP_BS_M + f * R, True), (f"FRSM{f}", rs, OP_RS_M + f * R, True)):
                self.e(f"{lab}:")
                if not modi or self.modi:
                    fn(modi=modi, base=base)
                self.e("bra.uni FLOOP;")
        self.e("FDONE:")
        for j in range(K):
            self.e(f"mov.f32 %{{a{j}}}, A{j};")
        self.e("mov.u32 %{flag}, r_flag;")
        self.e("mov.u32 %{tend}, r_tape;")
        self.e("}")
        return "\n".join(self.lines)


class Rev(Base):
    """reverse sweep"""

    def case(self, op, body):
        self.e(f"RC{op}:")
        body()
        self.e("bra.uni RLOOP;")

    # ---- accumulation targets
    def gx_add(self, vals):
        """gradient tile of X at the lane's points of feature r_iy += vals.
        The tile is laid out [feature][chunk][j][lane] (r_gx already points
        at the lane's word of the chunk), so the 32 lanes of one reduction
        hit 32 different banks."""
        self.e("mad.lo.u32 r_ad, r_iy, r_xstr, r_gx;")
        for j in range(self.K):
            self.e(f"red.shared.add.f32 [r_ad+{128 * j}], {vals(j)};")

    def gc_add(self, vals):
        """per-warp constant gradient [node] += sum over the warp's points"""
        K = self.K
        self.e(f"add.f32 q_s, {vals(0)}, {vals(1)};")
        for j in range(2, K):
            self.e(f"add.f32 q_s, q_s, {vals(j)};")
        for m in (16, 8, 4, 2, 1):
            self.e(f"shfl.sync.bfly.b32 q_t, q_s, {m}, 31, -1;")
            self.e("add.f32 q_s, q_s, q_t;")
        self.e("shr.u32 r_nd, r_ix, 16;")
        self.e("mad.lo.u32 r_ca, r_nd, 4, r_cg;")
        self.e("@PL ld.shared.f32 q_t, [r_ca];")
        self.e("@PL add.f32 q_t, q_t, q_s;")
        self.e("@PL st.shared.f32 [r_ca], q_t;")

    def seed(self, dst):
        """dst = seed of the output of this Modi instruction at the lane's points"""
        self.e("bfe.u32 r_moo, r_ix, 8, 8;")
        self.e(f"mad.lo.u32 r_ma, r_moo, {128 * self.K}, r_sd;")
        for h in range(self.K // 4):
            regs = ", ".join(dst(4 * h + q) for q in range(4))
            off = f"+{512 * h}" if h else ""
            self.e(f"ld.shared.v4.f32 {{{regs}}}, [r_ma{off}];")

    def dfn2(self, f, a, b, g, da, db):
        """da[j] = g*df/da, db[j] = g*df/db at (a[j], b[j]); None skips one"""
        K = self.K
        if f == F_MUL:
            if da: self.pk("mul.rn.f32x2", da, g, b)
            if db: self.pk("mul.rn.f32x2", db, g, a)
            return
        if f == F_PDIV:
            V, W = self.vec("V"), self.vec("W")
            for j in range(K):
                y = b(j)
                self.e(f"abs.f32 V{j}, {y};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"rcp.approx.ftz.f32 V{j}, {y};")
            self.pk("mul.rn.f32x2", W, g, V)                  # g / b
            if db:
                self.pk("mul.rn.f32x2", V, a, V)              # a / b
                self.pk("mul.rn.f32x2", V, W, V)
                for j in range(K):
                    self.e(f"neg.f32 V{j}, V{j};")
                    self.e(f"selp.f32 {db(j)}, V{j}, {ZERO}, P{j};")
            if da:
                for j in range(K):
                    self.e(f"selp.f32 {da(j)}, W{j}, {ZERO}, P{j};")
            return
        for j in range(K):
            x, y, gg = a(j), b(j), g(j)
            if f == F_ADD:
                if da: self.e(f"mov.f32 {da(j)}, {gg};")
                if db: self.e(f"mov.f32 {db(j)}, {gg};")
            elif f == F_SUB:
                if da: self.e(f"mov.f32 {da(j)}, {gg};")
                if db: self.e(f"neg.f32 {db(j)}, {gg};")
            elif f == F_MAX:
                self.e(f"setp.ge.f32 P{j}, {x}, {y};")
                self.e(f"setp.nan.f32 Q{j}, {y}, {y};")
                self.e(f"or.pred P{j}, P{j}, Q{j};")
                if da: self.e(f"selp.f32 {da(j)}, {gg}, {ZERO}, P{j};")
                if db: self.e(f"selp.f32 {db(j)}, {ZERO}, {gg}, P{j};")

    def addv(self, out, x, y):
        self.pk("add.rn.f32x2", out, x, y)

    def build(self):
        K = self.K
        G, L, T1, T2 = self.vec("G"), self.vec("L"), self.vec("T"), self.vec("U")
        DA, DB, SD = self.vec("DA"), self.vec("DB"), self.vec("SD")
        GS = lambda d: (lambda j: f"GS{d}_{j}")
        c = lambda j: "cv"
        regs = [f"{p}{j}" for p in ("G", "L", "T", "U", "V", "W", "DA", "DB", "SD", "GSV") for j in range(K)]
        self.e("{")
        self.e(".reg .f32 " + ", ".join(regs) + ", cv, q_s, q_t;")
        self.e(".reg .pred " + ", ".join([f"P{j}" for j in range(K)] + [f"Q{j}" for j in range(K)]) + ", PL;")
        self.e(".reg .b64 QP0, QP1, QP2, QP3;")
        self.e(".reg .u32 r_ptr, r_ix, r_iy, r_nx, r_ny, r_op, r_ad, r_xc, r_xstr, r_gx, r_cg, r_sd, r_moo, r_ma, r_tape, r_nd, r_ca, r_lane, r_beg, r_slot, r_d, r_sl;")
        self.e("mov.u32 r_slot, %{slot};")
        self.e("mov.u32 r_ptr, %{plast};")
        self.e("mov.u32 r_beg, %{pg};")
        self.e("mov.u32 r_xc, %{xc};")
        self.e("mov.u32 r_xstr, %{xstr};")
        self.e("mov.u32 r_gx, %{gx};")
        self.e("mov.u32 r_cg, %{cg};")
        self.e("mov.u32 r_sd, %{sd};")
        self.e("mov.u32 r_tape, %{tend};")
        self.e("mov.u32 r_lane, %{lane};")
        self.e("setp.eq.u32 PL, r_lane, 0;")
        for j in range(K):
            self.e(f"mov.f32 G{j}, %{{s{j}}};")
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr];")
        self.e("RLOOP:")
        self.e("mov.b32 r_ix, r_nx;")
        self.e("mov.b32 r_iy, r_ny;")
        # prefetch the previous instruction (below the program start this
        # reads the pad word in front of it, which is never executed)
        self.e("ld.shared.v2.u32 {r_nx, r_ny}, [r_ptr+-8];")
        self.e("sub.u32 r_ptr, r_ptr, 8;")
        self.e("mov.b32 cv, r_iy;")
        self.e("and.b32 r_op, r_ix, 255;")
        self.e("RTR: .branchtargets " + ", ".join(rev_label(k) for k in range(OP_COUNT)) + ";")
        self.e("brx.idx.uni r_op, RTR;")

        # the program's terminator starts the sweep: the root's adjoint (END_ROOT)
        # is the seed already in G; Modi trees start from zero
        self.case(OP_END_ROOT, lambda: None)
        self.case(OP_END_MODI, lambda: [self.e(f"mov.f32 G{j}, {ZERO};") for j in range(K)])

        def done_if_first():
            # the first instruction of a program loads a leaf into acc; its
            # reverse ends the sweep
            self.e("bra.uni RDONE;")

        def ldv():
            self.gx_add(G)

        def ldc():
            self.gc_add(G)

        self.e(f"RC{OP_LDV}:")
        ldv()
        done_if_first()
        self.e(f"RC{OP_LDC}:")
        ldc()
        done_if_first()
        for f in UNA:
            def un(f=f):
                self.tape_get(T1)
                self.pk("mul.rn.f32x2", G, G, T1)

            def unv(f=f):
                self.tape_get(T1)
                self.pk("mul.rn.f32x2", DA, G, T1)
                self.gx_add(DA)

            def unm(f=f):
                if not self.modi:
                    return
                self.tape_get(T1)
                self.seed(SD)
                self.pk("fma.rn.f32x2", G, SD, T1, G)

            self.case(OP_UN + f - F_SIN, un)
            self.e(f"RC{OP_UNV + f - F_SIN}:")
            unv()
            done_if_first()
            self.case(OP_UN_M + f - F_SIN, unm)

        for f in BIN:
            need = f in NEEDS_OPERAND

            # BV: acc = f(a = acc_before, b = x)
            def bv(f=f, need=need):
                self.load_x(L)
                if need:
                    self.tape_get(T1)
                self.dfn2(f, T1, L, G, DA, DB)
                self.gx_add(DB)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            def bc(f=f, need=need):
                if need:
                    self.tape_get(T1)
                self.dfn2(f, T1, c, G, DA, DB)
                self.gc_add(DB)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            # RV: acc = f(a = x, b = acc_before)
            def rv(f=f, need=need):
                self.load_x(L)
                if need:
                    self.tape_get(T1)
                self.dfn2(f, L, T1, G, DA, DB)
                self.gx_add(DA)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DB{j};")

            def rc(f=f, need=need):
                if need:
                    self.tape_get(T1)
                self.dfn2(f, c, T1, G, DA, DB)
                self.gc_add(DA)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DB{j};")

            # Modi forms: the function value's adjoint is the output's seed
            def bvm(f=f, need=need):      # out += f(acc, x); acc = x
                self.load_x(L)
                if need:
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, T1, L, SD, DA, DB)
                self.addv(DB, DB, G)
                self.gx_add(DB)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            def bcm(f=f, need=need):      # out += f(acc, c); acc = c
                if need:
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, T1, c, SD, DA, DB)
                self.addv(DB, DB, G)
                self.gc_add(DB)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            def rvm(f=f, need=need):      # out += f(x, acc); acc unchanged
                self.load_x(L)
                if need:
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, L, T1, SD, DA, DB)
                self.gx_add(DA)
                self.addv(G, G, DB)

            def rcm(f=f, need=need):      # out += f(c, acc); acc unchanged
                if need:
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, c, T1, SD, DA, DB)
                self.gc_add(DA)
                self.addv(G, G, DB)

            self.case(OP_BV + f, bv)
            self.case(OP_BC + f, bc)
            self.case(OP_RV + f, rv)
            self.case(OP_RC + f, rc)
            for op, fn in ((OP_BV_M, bvm), (OP_BC_M, bcm), (OP_RV_M, rvm), (OP_RC_M, rcm)):
                self.case(op + f, fn if self.modi else (lambda: None))

        def slot_addr(base):
            self.e(f"sub.u32 r_d, r_op, {base};")
            self.e(f"mad.lo.u32 r_sl, r_d, {128 * K}, r_slot;")

        def st_slot(src):
            for h in range(K // 4):
                regs = ", ".join(src(4 * h + q) for q in range(4))
                self.e(f"st.shared.v4.f32 [r_sl+{512 * h}], {{{regs}}};")

        def ld_slot(dst):
            for h in range(K // 4):
                regs = ", ".join(dst(4 * h + q) for q in range(4))
                self.e(f"ld.shared.v4.f32 {{{regs}}}, [r_sl+{512 * h}];")

        GSV = self.vec("GSV")
        self.e("RSPV:")
        slot_addr(OP_SPV)
        self.gx_add(G)
        ld_slot(G)
        self.e("bra.uni RLOOP;")
        self.e("RSPC:")
        slot_addr(OP_SPC)
        self.gc_add(G)
        ld_slot(G)
        self.e("bra.uni RLOOP;")
        for f in BIN:
            need = f in NEEDS_OPERAND

            def bs(f=f, need=need):
                if need:
                    self.tape_get(T2)        # acc_before (b)
                    self.tape_get(T1)        # s[d] (a)
                self.dfn2(f, T1, T2, G, GSV, DB)
                st_slot(GSV)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DB{j};")

            def rs(f=f, need=need):
                if need:
                    self.tape_get(T2)        # acc_before (a)
                    self.tape_get(T1)        # s[d] (b)
                self.dfn2(f, T2, T1, G, DA, GSV)
                st_slot(GSV)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            def bsm(f=f, need=need):         # out += f(s[d], acc); acc unchanged
                if need:
                    self.tape_get(T2)
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, T1, T2, SD, GSV, DB)
                st_slot(GSV)
                self.addv(G, G, DB)

            def rsm(f=f, need=need):         # out += f(acc, s[d]); acc = s[d]
                if need:
                    self.tape_get(T2)
                    self.tape_get(T1)
                self.seed(SD)
                self.dfn2(f, T2, T1, SD, DA, DB)
                self.addv(GSV, DB, G)
                st_slot(GSV)
                for j in range(K):
                    self.e(f"mov.f32 G{j}, DA{j};")

            for lab, fn, base, modi in ((f"RBS{f}", bs, OP_BS + f * R, False), (f"RRS{f}", rs, OP_RS + f * R, False),
                                        (f"RBSM{f}", bsm, OP_BS_M + f * R, True), (f"RRSM{f}", rsm, OP_RS_M + f * R, True)):
                self.e(f"{lab}:")
                if not modi or self.modi:
                    slot_addr(base)
                    fn()
                self.e("bra.uni RLOOP;")
        self.e("RDONE:")
        self.e("}")
        return "\n".join(self.lines)


def _family(k):
    """(family, f) of a slot-indexed opcode, or None"""
    if OP_SPV <= k < OP_SPV + R:
        return ("SPV", None)
    if OP_SPC <= k < OP_SPC + R:
        return ("SPC", None)
    for base, name in ((OP_BS, "BS"), (OP_RS, "RS"), (OP_BS_M, "BSM"), (OP_RS_M, "RSM")):
        if base <= k < base + 5 * R:
            return (name, (k - base) // R)
    return None


def fwd_label(k):
    fam = _family(k)
    if fam is None:
        return f"FC{k}"
    return f"F{fam[0]}" + ("" if fam[1] is None else str(fam[1]))


def rev_label(k):
    fam = _family(k)
    if fam is None:
        return f"RC{k}"
    return f"R{fam[0]}" + ("" if fam[1] is None else str(fam[1]))


def _literal(body: str) -> str:
    return "\n".join('      "' + l.replace("\\", "\\\\").replace('"', '\\"') + '\\n"'
                     for l in body.split("\n"))


def render_fwd(K, modi):
    body = Fwd(K, modi).build()
    names = [f"a{j}" for j in range(K)] + ["flag", "tend", "pg", "xc", "xstr", "mo", "tape", "slot"]
    for i, n in enumerate(names):
        body = body.replace("%{" + n + "}", f"%{i}")
    outs = ", ".join([f'"=f"(acc[{j}])' for j in range(K)] + ['"=r"(flag)', '"=r"(tend)'])
    return f"""template <>
__device__ __forceinline__ unsigned bwd_forward<{K}, {'true' if modi else 'false'}>(
    unsigned pg, unsigned xc, unsigned xstr, unsigned mo, unsigned tape, unsigned slot,
    float (&acc)[{K}], unsigned& tend) {{
  unsigned flag;
  asm volatile(
{_literal(body)}
      : {outs}
      : "r"(pg), "r"(xc), "r"(xstr), "r"(mo), "r"(tape), "r"(slot)
      : "memory");
  return flag;
}}
"""


def render_rev(K, modi):
    body = Rev(K, modi).build()
    names = ["plast", "pg", "xc", "xstr", "gx", "cg", "sd", "tend", "lane", "slot"] + [f"s{j}" for j in range(K)]
    for i, n in enumerate(names):
        body = body.replace("%{" + n + "}", f"%{i}")
    ins = ", ".join(['"r"(plast)', '"r"(pg)', '"r"(xc)', '"r"(xstr)', '"r"(gx)', '"r"(cg)', '"r"(sd)',
                     '"r"(tend)', '"r"(lane)', '"r"(slot)'] + [f'"f"(seed[{j}])' for j in range(K)])
    return f"""template <>
__device__ __forceinline__ void bwd_reverse<{K}, {'true' if modi else 'false'}>(
    unsigned plast, unsigned pg, unsigned xc, unsigned xstr, unsigned gx, unsigned cg, unsigned sd,
    unsigned tend, unsigned lane, unsigned slot, const float (&seed)[{K}]) {{
  asm volatile(
{_literal(body)}
      :
      : {ins}
      : "memory");
}}
"""


def main():
    parts = [
        "// interp_bwd.cuh -- GENERATED by gen_interp_bwd.py; do not edit by hand.",
        "// Forward-with-tape and reverse sweeps of the adjoint kernel (adjoint.cu).",
        "#pragma once",
        "namespace tgp {",
        "template <int K, bool MODI>",
        "__device__ __forceinline__ unsigned bwd_forward(unsigned pg, unsigned xc, unsigned xstr,",
        "                                                unsigned mo, unsigned tape, unsigned slot,",
        "                                                float (&acc)[K], unsigned& tend);",
        "template <int K, bool MODI>",
        "__device__ __forceinline__ void bwd_reverse(unsigned plast, unsigned pg, unsigned xc,",
        "                                            unsigned xstr, unsigned gx, unsigned cg,",
        "                                            unsigned sd, unsigned tend, unsigned lane,",
        "                                            unsigned slot, const float (&seed)[K]);",
    ]
    for K, modi in ((4, False), (4, True)):
        parts.append(render_fwd(K, modi))
        parts.append(render_rev(K, modi))
    parts.append("}  // namespace tgp")
    open(OUT, "w").write("\n".join(parts) + "\n")
    return OUT


if __name__ == "__main__":
    import sys
    sys.path.insert(0, HERE)
    print(main())
