"""Generate tmem_gen.cuh: TMEM row load/store helpers of W consecutive 32-bit columns.

Each helper is one inline-PTX block that issues every tcgen05.ld (or .st) chunk of the row
(32x32b shapes .x32/.x16/.x8/.x4) and then a single tcgen05.wait, so a whole pencil's
accumulator moves between TMEM and registers with one wait and the destination registers
cannot be used before the wait.  Run: python gen_tmem.py > tmem_gen.cuh
"""
import sys

WIDTHS = (4, 6, 8, 10, 12, 16, 18, 20, 24, 32, 36, 40, 48)  # n or 2n floats of one pencil, n in {4..24} even


def chunks(w):
    out, col = [], 0
    for c in (32, 16, 8, 4, 2, 1):
        while w - col >= c:
            out.append((col, c))
            col += c
    assert col == w, w
    return out


def gen_load(w):
    lines = [f"__device__ __forceinline__ void tmem_load_row{w}(uint32_t taddr, float* v) {{",
             f"  uint32_t r[{w}];"]
    body, reg = [], 0
    cs = chunks(w)
    for ci, (col, c) in enumerate(cs):
        regs = ", ".join(f"%{reg + i}" for i in range(c))
        body.append(f'"tcgen05.ld.sync.aligned.32x32b.x{c}.b32 {{{regs}}}, [%{w + ci}];\\n\\t"')
        reg += c
    body.append('"tcgen05.wait::ld.sync.aligned;"')
    outs = ", ".join(f'"=r"(r[{i}])' for i in range(w))
    addrs = ", ".join(f'"r"(taddr + {col}u)' for col, _ in cs)
    lines.append("  asm volatile(" + "\n               ".join(body))
    lines.append(f"               : {outs}")
    lines.append(f"               : {addrs}")
    lines.append('               : "memory");')
    lines.append(f"#pragma unroll\n  for (int i = 0; i < {w}; ++i) v[i] = __uint_as_float(r[i]);")
    lines.append("}")
    return "\n".join(lines)


def gen_store(w):
    lines = [f"__device__ __forceinline__ void tmem_store_row{w}(uint32_t taddr, const float* v) {{"]
    cs = chunks(w)
    body, reg = [], len(cs)
    for ci, (col, c) in enumerate(cs):
        regs = ", ".join(f"%{reg + i}" for i in range(c))
        body.append(f'"tcgen05.st.sync.aligned.32x32b.x{c}.b32 [%{ci}], {{{regs}}};\\n\\t"')
        reg += c
    body.append('"tcgen05.wait::st.sync.aligned;"')
    ins = ", ".join(f'"r"(__float_as_uint(v[{i}]))' for i in range(w))
    addrs = ", ".join(f'"r"(taddr + {col}u)' for col, _ in cs)
    lines.append("  asm volatile(" + "\n               ".join(body))
    lines.append(f'               :: {addrs}, {ins}')
    lines.append('               : "memory");')
    lines.append("}")
    return "\n".join(lines)


def main():
    out = ["// tmem_gen.cuh - generated by gen_tmem.py; do not edit.",
           "// Row helpers: W consecutive 32-bit TMEM columns of this thread's lane, one wait each.",
           "#pragma once", "#include <stdint.h>", "", "namespace hse {", ""]
    for w in WIDTHS:
        out.append(gen_load(w))
        out.append("")
        out.append(gen_store(w))
        out.append("")
    out.append("template <int W> struct TmemRow;")
    for w in WIDTHS:
        out.append(f"template <> struct TmemRow<{w}> {{")
        out.append(f"  static __device__ __forceinline__ void load(uint32_t a, float* v) {{ tmem_load_row{w}(a, v); }}")
        out.append(f"  static __device__ __forceinline__ void store(uint32_t a, const float* v) {{ tmem_store_row{w}(a, v); }}")
        out.append("};")
    out.append("")
    out.append("}  // namespace hse")
    sys.stdout.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
