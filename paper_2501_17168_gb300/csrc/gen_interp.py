"""Generates interp_fwd.cuh: the forward register-machine interpreter as one
inline-PTX loop with a jump-table dispatch (brx.idx over .branchtargets).

Why PTX: the instruction stream of a compiled tree is warp-uniform, so the
ideal dispatch is one indirect branch per instruction.  A C++ `switch` over
the 235 opcodes is lowered to a compare-and-branch tree and, with 72+
loop-carried floats (the accumulator and eight slots of K points), to
register shuffling at every case; a hand-written loop keeps every slot in a
fixed register and dispatches with one brx.idx.

Semantics per opcode are the ones listed in tgp_internal.cuh (enum Op).  The
FP32 function bodies:
  add/sub/mul   add.rn / sub.rn / mul.rn (never contracted)
  pdiv(a,b)     |b| > 1e-6f ? a * rcp.approx(b) : 1
  max           max.f32 (a NaN operand yields the other one)
  sin/cos(a)    Cody-Waite reduction r = a - k*C1 - k*C2, k = rint(a/(2pi))
                (rint by the 1.5*2^23 addition trick, so it stays on the FMA
                pipe), then sin.approx / cos.approx of r
  plog(a)       |a| > 1e-6f ? lg2.approx(|a|) * ln2 : 0
  cexp(a)       ex2.approx.ftz(min(a, 80) * log2 e)
  tan(a)        sin.approx(r) * rcp.approx(cos.approx(r))

Run `python gen_interp.py` to regenerate (the build does it when stale).
"""
from __future__ import annotations

import os
import struct

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "interp_fwd.cuh")

R = 8
F_ADD, F_SUB, F_MUL, F_PDIV, F_MAX, F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN = range(10)
BIN = [F_ADD, F_SUB, F_MUL, F_PDIV, F_MAX]
UNA = [F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN]

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


class Gen:
    def __init__(self, K: int, modi: bool):
        self.K = K
        self.modi = modi
        self.lines: list[str] = []

    def e(self, s: str):
        self.lines.append(s)

    # register names
    def A(self, j):
        return f"A{j}"

    def S(self, d, j):
        return f"S{d}_{j}"

    def Lr(self, j):
        return f"L{j}"

    def T(self, j):
        return f"T{j}"

    def U(self, j):
        return f"U{j}"

    # ---- operand loads
    def load_x(self, dst):
        """dst[j] = X tile value of the lane's point j, feature = iy."""
        K = self.K
        self.e("mad.lo.u32 r_ad, r_iy, r_xstr, r_xc;")
        self.e(f"ld.shared.v4.f32 {{{dst(0)}, {dst(1)}, {dst(2)}, {dst(3)}}}, [r_ad];")
        if K == 8:
            self.e(f"ld.shared.v4.f32 {{{dst(4)}, {dst(5)}, {dst(6)}, {dst(7)}}}, [r_ad+512];")

    # ---- function bodies: out[j] = f(a[j], b[j]); a, b, out are name functions
    def fn2(self, f, out, a, b):
        K = self.K
        for j in range(K):
            o, x, y = out(j), a(j), b(j)
            if f == F_ADD:
                self.e(f"add.rn.f32 {o}, {x}, {y};")
            elif f == F_SUB:
                self.e(f"sub.rn.f32 {o}, {x}, {y};")
            elif f == F_MUL:
                self.e(f"mul.rn.f32 {o}, {x}, {y};")
            elif f == F_MAX:
                self.e(f"max.f32 {o}, {x}, {y};")
            elif f == F_PDIV:
                self.e(f"abs.f32 V{j}, {y};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"rcp.approx.ftz.f32 V{j}, {y};")
                self.e(f"mul.rn.f32 V{j}, {x}, V{j};")
                self.e(f"selp.f32 {o}, V{j}, {ONE}, P{j};")

    def reduce(self, j, x):
        """V{j} = x reduced by 2pi (Cody-Waite), using W{j} as scratch."""
        self.e(f"mul.rn.f32 W{j}, {x}, {INV2PI};")
        self.e(f"add.rn.f32 W{j}, W{j}, {MAGIC};")
        self.e(f"sub.rn.f32 W{j}, {MAGIC}, W{j};")       # -rint(x / 2pi)
        self.e(f"fma.rn.f32 V{j}, W{j}, {C1}, {x};")
        self.e(f"fma.rn.f32 V{j}, W{j}, {C2}, V{j};")

    def fn1(self, f, out, a):
        K = self.K
        for j in range(K):
            o, x = out(j), a(j)
            if f == F_SIN:
                self.reduce(j, x)
                self.e(f"sin.approx.ftz.f32 {o}, V{j};")
            elif f == F_COS:
                self.reduce(j, x)
                self.e(f"cos.approx.ftz.f32 {o}, V{j};")
            elif f == F_PLOG:
                self.e(f"abs.f32 V{j}, {x};")
                self.e(f"setp.gt.f32 P{j}, V{j}, {GUARD};")
                self.e(f"lg2.approx.ftz.f32 V{j}, V{j};")
                self.e(f"mul.rn.f32 V{j}, V{j}, {LN2};")
                self.e(f"selp.f32 {o}, V{j}, {ZERO}, P{j};")
            elif f == F_CEXP:
                self.e(f"min.f32 V{j}, {x}, {CLAMP};")
                self.e(f"mul.rn.f32 V{j}, V{j}, {LOG2E};")
                self.e(f"ex2.approx.ftz.f32 {o}, V{j};")
            elif f == F_TAN:
                self.reduce(j, x)
                self.e(f"cos.approx.ftz.f32 W{j}, V{j};")
                self.e(f"sin.approx.ftz.f32 V{j}, V{j};")
                self.e(f"rcp.approx.ftz.f32 W{j}, W{j};")
                self.e(f"mul.rn.f32 {o}, V{j}, W{j};")

    def modi_add(self, src):
        """out[o][lane points] += src[j] (o from bits 8..15 of ix)."""
        K = self.K
        self.e("bfe.u32 r_moo, r_ix, 8, 8;")
        self.e(f"mad.lo.u32 r_ma, r_moo, {128 * K}, r_mo;")
        for h in range(K // 4):
            regs = [f"M{4 * h + q}" for q in range(4)]
            off = f"+{512 * h}" if h else ""
            self.e(f"ld.shared.v4.f32 {{{', '.join(regs)}}}, [r_ma{off}];")
            for q in range(4):
                self.e(f"add.rn.f32 {regs[q]}, {regs[q]}, {src(4 * h + q)};")
            self.e(f"st.shared.v4.f32 [r_ma{off}], {{{', '.join(regs)}}};")

    def case(self, op, body):
        self.e(f"C{op}:")
        body()
        self.e("bra.uni LOOP;")

    def build(self) -> str:
        K = self.K
        A, Lr, T = self.A, self.Lr, self.T
        c = lambda j: "cv"
        self.e("{")
        self.e(".reg .f32 " + ", ".join([f"A{j}" for j in range(K)] + [f"L{j}" for j in range(K)] +
                                      [f"T{j}" for j in range(K)] + [f"V{j}" for j in range(K)] +
                                      [f"W{j}" for j in range(K)] + [f"M{j}" for j in range(K)]) + ", cv;")
        self.e(".reg .f32 " + ", ".join(self.S(d, j) for d in range(R) for j in range(K)) + ";")
        self.e(".reg .pred " + ", ".join(f"P{j}" for j in range(K)) + ";")
        self.e(".reg .u32 r_ptr, r_ix, r_iy, r_nx, r_ny, r_op, r_ad, r_xc, r_xstr, r_mo, r_moo, r_ma, r_flag;")
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
        self.e("TS: .branchtargets " + ", ".join(f"C{k}" for k in range(OP_COUNT)) + ";")
        if self.modi:
            self.e("and.b32 r_op, r_ix, 255;")
            self.e("brx.idx.uni r_op, TS;")
        else:
            # programs for the plain kernel carry nothing above the opcode
            self.e("brx.idx.uni r_ix, TS;")

        # ---- terminators and leaf loads
        self.e(f"C{OP_END_ROOT}:")
        self.e("mov.u32 r_flag, 0;")
        self.e("bra.uni DONE;")
        self.e(f"C{OP_END_MODI}:")
        self.e("mov.u32 r_flag, 1;")
        self.e("bra.uni DONE;")
        self.case(OP_LDV, lambda: self.load_x(A))
        self.case(OP_LDC, lambda: [self.e(f"mov.f32 A{j}, cv;") for j in range(K)])
        # ---- unary / fused unary-of-variable
        for f in UNA:
            self.case(OP_UN + f - F_SIN, lambda f=f: self.fn1(f, A, A))
            self.case(OP_UNV + f - F_SIN, lambda f=f: (self.load_x(Lr), self.fn1(f, A, Lr)))
        # ---- binary with a leaf operand
        for f in BIN:
            self.case(OP_BV + f, lambda f=f: (self.load_x(Lr), self.fn2(f, A, A, Lr)))
            self.case(OP_BC + f, lambda f=f: self.fn2(f, A, A, c))
            self.case(OP_RV + f, lambda f=f: (self.load_x(Lr), self.fn2(f, A, Lr, A)))
            self.case(OP_RC + f, lambda f=f: self.fn2(f, A, c, A))
        # ---- Modi forms (only reachable in the Modi kernel)
        for f in UNA:
            self.case(OP_UN_M + f - F_SIN,
                      lambda f=f: (self.fn1(f, T, A), self.modi_add(T)) if self.modi else None)
        for f in BIN:
            def bvm(f=f):
                if not self.modi:
                    return
                self.load_x(Lr)
                self.fn2(f, T, A, Lr)
                self.modi_add(T)
                for j in range(K):
                    self.e(f"mov.f32 A{j}, L{j};")

            def bcm(f=f):
                if not self.modi:
                    return
                self.fn2(f, T, A, c)
                self.modi_add(T)
                for j in range(K):
                    self.e(f"mov.f32 A{j}, cv;")

            def rvm(f=f):
                if not self.modi:
                    return
                self.load_x(Lr)
                self.fn2(f, T, Lr, A)
                self.modi_add(T)

            def rcm(f=f):
                if not self.modi:
                    return
                self.fn2(f, T, c, A)
                self.modi_add(T)

            self.case(OP_BV_M + f, bvm)
            self.case(OP_BC_M + f, bcm)
            self.case(OP_RV_M + f, rvm)
            self.case(OP_RC_M + f, rcm)
        # ---- spill + leaf load
        for d in range(R):
            def spv(d=d):
                for j in range(K):
                    self.e(f"mov.f32 {self.S(d, j)}, A{j};")
                self.load_x(A)

            def spc(d=d):
                for j in range(K):
                    self.e(f"mov.f32 {self.S(d, j)}, A{j};")
                    self.e(f"mov.f32 A{j}, cv;")

            self.case(OP_SPV + d, spv)
            self.case(OP_SPC + d, spc)
        # ---- binary on a slot
        for f in BIN:
            for d in range(R):
                Sd = lambda j, d=d: self.S(d, j)
                self.case(OP_BS + f * R + d, lambda f=f, Sd=Sd: self.fn2(f, A, Sd, A))
        for f in BIN:
            for d in range(R):
                Sd = lambda j, d=d: self.S(d, j)
                self.case(OP_RS + f * R + d, lambda f=f, Sd=Sd: self.fn2(f, A, A, Sd))
        for f in BIN:
            for d in range(R):
                Sd = lambda j, d=d: self.S(d, j)

                def bsm(f=f, Sd=Sd):
                    if not self.modi:
                        return
                    self.fn2(f, T, Sd, A)
                    self.modi_add(T)

                self.case(OP_BS_M + f * R + d, bsm)
        for f in BIN:
            for d in range(R):
                Sd = lambda j, d=d: self.S(d, j)

                def rsm(f=f, Sd=Sd, d=d):
                    if not self.modi:
                        return
                    self.fn2(f, T, A, Sd)
                    self.modi_add(T)
                    for j in range(K):
                        self.e(f"mov.f32 A{j}, {self.S(d, j)};")

                self.case(OP_RS_M + f * R + d, rsm)
        self.e("DONE:")
        for j in range(K):
            self.e(f"mov.f32 %{{a{j}}}, A{j};")
        self.e("mov.u32 %{flag}, r_flag;")
        self.e("}")
        return "\n".join(self.lines)


def operand_map(K):
    names = [f"a{j}" for j in range(K)] + ["flag", "pg", "xc", "xstr", "mo"]
    return {n: i for i, n in enumerate(names)}


def render(K: int, modi: bool) -> str:
    body = Gen(K, modi).build()
    m = operand_map(K)
    for n, i in m.items():
        body = body.replace("%{" + n + "}", f"%{i}")
    # C string literal, one PTX line per source line
    lit = "\n".join('      "' + l.replace("\\", "\\\\").replace('"', '\\"') + '\\n"' for l in body.split("\n"))
    outs = ", ".join([f'"=f"(acc[{j}])' for j in range(K)] + ['"=r"(flag)'])
    ins = '"r"(pg), "r"(xc), "r"(xstr), "r"(mo)'
    return f"""template <>
__device__ __forceinline__ unsigned interp_fwd<{K}, {'true' if modi else 'false'}>(
    unsigned pg, unsigned xc, unsigned xstr, unsigned mo, float (&acc)[{K}]) {{
  unsigned flag;
  asm volatile(
{lit}
      : {outs}
      : {ins}
      : "memory");
  return flag;
}}
"""


def main():
    parts = [
        "// interp_fwd.cuh -- GENERATED by gen_interp.py; do not edit by hand.",
        "// Forward interpreter loop of the register machine (see tgp_internal.cuh).",
        "// interp_fwd<K, MODI>(pg, xc, xstr, mo, acc): pg = shared address of the",
        "// program, xc = shared address of the lane's first point of feature 0,",
        "// xstr = bytes between feature rows, mo = shared address of the lane's Modi",
        "// accumulators; returns 1 when the outputs are the Modi sums, else 0 with",
        "// the single output in acc.",
        "#pragma once",
        "namespace tgp {",
        "template <int K, bool MODI>",
        "__device__ __forceinline__ unsigned interp_fwd(unsigned pg, unsigned xc, unsigned xstr,",
        "                                               unsigned mo, float (&acc)[K]);",
    ]
    for K, modi in ((8, False), (4, False), (4, True), (8, True)):
        parts.append(render(K, modi))
    parts.append("}  // namespace tgp")
    open(OUT, "w").write("\n".join(parts) + "\n")
    return OUT


if __name__ == "__main__":
    print(main())
