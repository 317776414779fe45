"""CPU model of the evaluator's group interpreters, for testing without a
GPU.

`group_asm(path, fn)` expands the hand-written inline-PTX string of
`groups_u8` (the byte-code group loop) or `group_u32` (upper trees) in
gp_eval.cu, its macros included, into plain text by compiling a small C
program that prints the same string literal.  `run` interprets that text
for one lane (each 64-bit stack entry is a pair of float32) over the dozen
PTX forms the interpreter uses.  `push_pop` is the interpreter's intended
meaning written plainly: codes read right to left (Sec. 2.2's single-pass
EVAL in postfix order), a leaf pushes the top of stack and loads its
table row, an operator pops its second argument and combines it with the
top of stack (its first); protected division gives the problem's value for
a zero divisor (Table gp.details)."""
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np

F = np.float32
M32 = 0xFFFFFFFF


def group_asm(src_path, fn="groups_u8"):
    """The inline-PTX text of `fn` (groups_u8: the byte-code group loop;
    group_u32: upper trees, whose value-buffer leaves read staged entries)."""
    s = open(src_path).read()
    g = s.index(f"__device__ __forceinline__ int {fn}(")
    tmpl = s.rindex("template <uint32_t S>", 0, g)
    marks = ("#define GP_UNODE",) if fn == "group_u32" else ("#define GP_BN(",)
    first = min(i for i in (s.find(m) for m in marks) if 0 <= i < tmpl)
    a = s.index("asm volatile(", g) + len("asm volatile(")
    b = s.index(': "+l"(tos)', a)
    c_src = ("#include <stdio.h>\n" + s[first:tmpl] + "\nint main(void) { fputs(\n" + s[a:b]
             + ", stdout); return 0; }\n")
    cc = shutil.which("gcc") or shutil.which("cc")
    with tempfile.TemporaryDirectory() as d:
        cpath, exe = os.path.join(d, "emit.c"), os.path.join(d, "emit")
        open(cpath, "w").write(c_src)
        subprocess.run([cc, "-O0", "-o", exe, cpath], check=True, capture_output=True)
        return subprocess.run([exe], check=True, capture_output=True, text=True).stdout


def parse(text):
    prog, labels, tables = [], {}, {}
    for raw in text.splitlines():
        ln = raw.strip()
        if not ln or ln in ("{", "}") or ln.startswith(".reg"):
            continue
        m = re.match(r"^(\w+):\s*\.branchtargets\s+(.*);$", ln)
        if m:
            tables[m.group(1)] = [x.strip() for x in m.group(2).split(",")]
            continue
        m = re.match(r"^(\w+):$", ln)
        if m:
            labels[m.group(1)] = len(prog)
            continue
        prog.append(ln.rstrip(";"))
    return prog, labels, tables


def _addr(r, expr):
    """A shared address [a+b*c+...] of registers and immediates."""
    total = 0
    for term in expr.strip("[]").split("+"):
        prod = 1
        for f in term.split("*"):
            prod *= _val(r, f)
        total += prod
    return total & M32


def _val(r, tok):
    tok = tok.strip()
    if tok in r:
        return r[tok]
    if tok.startswith("0f"):
        return np.frombuffer(int(tok[2:], 16).to_bytes(4, "little"), dtype=F)[0]
    if "+" in tok:                                  # constant expression, e.g. 16+3
        return sum(int(x, 0) for x in tok.split("+"))
    return int(tok, 0)


M64 = (1 << 64) - 1


def run(parsed, regs, shared, gmem=None, max_steps=100000):
    """Interpret parsed PTX; regs maps the operands %0.. (and gets the named
    registers), shared maps byte address -> (float32, float32), gmem maps a
    16-byte aligned global address -> its 16 bytes."""
    prog, labels, tables = parsed
    r, pc = dict(regs), 0
    for _ in range(max_steps):
        if pc >= len(prog):
            return r
        ins = prog[pc]
        pc += 1
        if ins.startswith("@"):
            pred, ins = ins.split(None, 1)
            if not r[pred[1:]]:
                continue
        op, _, rest = ins.partition(" ")
        args = [x.strip() for x in re.split(r",(?![^{]*})", rest)] if rest else []
        v = lambda k: _val(r, args[k])          # noqa: E731
        if op == "bra.uni":
            pc = labels[args[0]]
        elif op == "brx.idx.uni":
            pc = labels[tables[args[1]][v(0) & M32]]
        elif op == "bfe.u32":
            r[args[0]] = (v(1) >> v(2)) & ((1 << v(3)) - 1)
        elif op == "prmt.b32":
            src = (v(1) & M32) | ((v(2) & M32) << 32)
            sel = v(3)
            out = 0
            for i in range(4):
                k = (sel >> (4 * i)) & 7
                out |= ((src >> (8 * k)) & 0xFF) << (8 * i)
            r[args[0]] = out
        elif op == "ld.global.nc.v4.u32":
            dst = [x.strip() for x in args[0].strip("{}").split(",")]
            blk = gmem[_val(r, args[1].strip("[]"))]
            for i, d in enumerate(dst):
                r[d] = int.from_bytes(bytes(blk[4 * i:4 * i + 4]), "little")
        elif op == "sub.u64":
            r[args[0]] = (v(1) - v(2)) & M64
        elif op.startswith("setp.") and op.endswith(".u64"):
            _, cmp, _ = op.split(".")
            a, b = v(1) & M64, v(2) & M64
            r[args[0]] = {"gt": a > b, "le": a <= b, "lt": a < b, "eq": a == b}[cmp]
        elif op.startswith("setp."):
            _, cmp, ty = op.split(".")
            a, b = v(1), v(2)
            if ty == "u32":
                r[args[0]] = {"gt": (a & M32) > (b & M32), "lt": (a & M32) < (b & M32),
                              "eq": (a & M32) == (b & M32)}[cmp]
            elif cmp == "neu":
                r[args[0]] = bool(np.isnan(a) or np.isnan(b) or a != b)
            else:
                raise ValueError(ins)
        elif op in ("sub.u32", "add.u32"):
            r[args[0]] = (v(1) - v(2) if op == "sub.u32" else v(1) + v(2)) & M32
        elif op == "mad.lo.u32":
            r[args[0]] = (v(1) * v(2) + v(3)) & M32
        elif op == "ld.shared.b64":
            r[args[0]] = shared[_addr(r, args[1])]
        elif op == "st.shared.b64":
            shared[_addr(r, args[0])] = v(1)
        elif op in ("mov.b32", "mov.u32", "mov.s32", "mov.b64"):
            d, s = args
            if d.startswith("{"):
                lo, hi = [x.strip() for x in d.strip("{}").split(",")]
                r[lo], r[hi] = _val(r, s)
            elif s.startswith("{"):
                lo, hi = [x.strip() for x in s.strip("{}").split(",")]
                r[d] = (r[lo], r[hi])
            else:
                r[d] = _val(r, s)
        elif op in ("add.rn.f32x2", "sub.rn.f32x2", "mul.rn.f32x2"):
            a, b = v(1), v(2)
            f = {"add": np.add, "sub": np.subtract, "mul": np.multiply}[op.split(".")[0]]
            with np.errstate(all="ignore"):
                r[args[0]] = (F(f(a[0], b[0])), F(f(a[1], b[1])))
        elif op == "div.rn.f32":
            with np.errstate(all="ignore"):
                r[args[0]] = F(np.divide(v(1), v(2)))
        elif op == "selp.f32":
            r[args[0]] = v(1) if v(3) else v(2)
        else:
            raise ValueError(f"instruction outside the model: {ins}")
    raise RuntimeError("step limit")
