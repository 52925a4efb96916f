"""The forward instruction set's fused pushes, checked on the host (no GPU).

The stage compiler never emits a push of G[NREG-1] as a word of its own
when the instruction after it (the first instruction of the next subtree,
which loads a leaf at level NREG-1) has a fused form: it emits that form's
PUSHS/PUSHL opcode instead, as given by push_form() in the generated
isa_fwd.cuh.  These tests tie the three places that must agree:
  * push_form() in the header, compiled here with the host compiler;
  * the generator's table of subtree-starting forms;
  * the generated interpreters, where each fused case must store G[NREG-1]
    to the right place and then jump into exactly the case it stands for.
"""
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_17168_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_interp as gi  # noqa: E402


def _expected_push_form(op, local):
    """The fused opcode for op, from the generator's tables, or 0."""
    top = gi.NREG - 1
    i = 0
    for name, n in gi.START_FORMS:
        for sub in range(n):
            if gi.fx(name, sub, top) == op:
                return gi.FX_BASE["PUSHL" if local else "PUSHS"] + i
            i += 1
    return 0


@pytest.fixture(scope="module")
def header_push_form(tmp_path_factory):
    """push_form(op, local) for every opcode, from the header compiled by g++."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("isa")
    hdr = d / "isa_fwd.cuh"
    hdr.write_text(gi.render_isa())
    src = d / "t.cpp"
    src.write_text(
        "#define __host__\n#define __device__\n#include <cstdio>\n#include \"isa_fwd.cuh\"\n"
        "int main() { for (unsigned op = 0; op < tgp::fx::COUNT; ++op)\n"
        "  std::printf(\"%u %u %u\\n\", op, tgp::fx::push_form(op, false), tgp::fx::push_form(op, true));\n"
        "  return 0; }\n")
    exe = d / "t"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-o", str(exe), str(src)], cwd=str(d))
    out = subprocess.check_output([str(exe)], text=True)
    table = {}
    for line in out.split("\n"):
        if line.strip():
            op, s, l = map(int, line.split())
            table[op] = (s, l)
    return table


def test_header_push_form_matches_the_generator(header_push_form):
    assert len(header_push_form) == gi.FX_COUNT
    n_fused = 0
    for op, (s, l) in header_push_form.items():
        assert s == _expected_push_form(op, False), op
        assert l == _expected_push_form(op, True), op
        n_fused += s != 0
    # every subtree-starting form at the top level has exactly one fused form
    assert n_fused == gi.NSTART


def test_device_table_matches_push_form(header_push_form):
    """The stage compiler reads the fused opcodes from a constant-memory
    table; it must hold push_form(op, false) for every opcode."""
    text = gi.render_isa()
    body = text[text.index("PUSH_FORM_TABLE[COUNT] = {"):]
    body = body[body.index("{") + 1:body.index("};")]
    table = [int(t) for t in body.replace("\n", " ").split(",") if t.strip()]
    assert len(table) == gi.FX_COUNT
    for op, v in enumerate(table):
        assert v == header_push_form[op][0], op
        if v:
            assert header_push_form[op][1] == v + gi.NSTART


def test_fused_opcodes_are_distinct_and_in_range(header_push_form):
    seen = set()
    for s, l in header_push_form.values():
        for f in (s, l):
            if f:
                assert gi.FX_BASE["PUSHS"] <= f < gi.FX_COUNT
                assert f not in seen
                seen.add(f)
    assert len(seen) == 2 * gi.NSTART


def _cases(text):
    """{label: [lines]} of the generated interpreter's cases."""
    out, cur = {}, None
    for line in text.split("\n"):
        m = re.fullmatch(r"(C\d+):", line)
        if m:
            cur = m.group(1)
            out[cur] = []
        elif cur is not None:
            out[cur].append(line)
            if line.startswith("bra.uni") or line.startswith("brx"):
                cur = None
    return out


@pytest.mark.parametrize("K,modi", [(8, False), (4, False), (4, True)])
def test_fused_cases_store_then_enter_their_instruction(K, modi):
    gen = gi.Gen(K, modi)
    cases = _cases(gen.build())
    top = gi.NREG - 1
    i = 0
    n_checked = 0
    for name, n in gi.START_FORMS:
        for sub in range(n):
            target = gi.fx(name, sub, top)
            for kind in ("PUSHS", "PUSHL"):
                op = gi.FX_BASE[kind] + i
                if target not in gen.defined:
                    # a form this kernel never runs (Modi forms in the plain
                    # kernels): its fused form must not exist either
                    assert f"C{op}" not in cases
                    continue
                body = cases[f"C{op}"]
                assert body[-1] == f"bra.uni C{target};", (kind, name, sub)
                stores = [l for l in body if l.startswith("st.")]
                # G[top] goes out whole: K/4 16-byte stores of its K floats
                assert len(stores) == K // 4
                regs = sorted(re.findall(rf"G{top}_(\d+)", " ".join(stores)), key=int)
                assert regs == [str(j) for j in range(K)]
                # the plain kernels keep entry 0 in shared memory; the Modi
                # kernel keeps its whole stack in local memory
                shared = kind == "PUSHS" and not modi
                assert all(l.startswith("st.shared" if shared else "st.local") for l in stores)
                if not shared:
                    assert f"add.u32 r_sp, r_sp, {4 * K};" in body
                n_checked += 1
            i += 1
    assert n_checked >= 2 * (gi.NSTART - (0 if modi else 10))
