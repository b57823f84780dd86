"""Writes chains.cuh: the carry-flag chains of the p-bit arithmetic, each one
inline-PTX statement per word count W in {4, 8, 16, 32} (p = 32 W bits).

A chain of add.cc / addc.cc / mad*.cc instructions passes its carry in the
condition-code flag, which nothing outside the chain may write; emitting the
whole chain as one asm statement makes that hold by construction instead of
depending on the compiler placing nothing between separate statements.  PTX
operands are positional, so one string per W serves every call site.

Run:  python gen_chains.py   (rewrites chains.cuh beside this file)
"""
import os

WS = (4, 8, 16, 32)
HERE = os.path.dirname(os.path.abspath(__file__))


def asm(lines):
    return "\n".join(f'      "{ln}\\n\\t"' for ln in lines)


def inc_chain(W):
    # m[0..W) += inc; c = carry out.  Operands: %0..%W-1 m (in/out), %W c, %W+1 inc
    lines = [f"add.cc.u32 %0, %0, %{W + 1};"]
    lines += [f"addc.cc.u32 %{k}, %{k}, 0;" for k in range(1, W)]
    lines += [f"addc.u32 %{W}, 0, 0;"]
    outs = ", ".join(f'"+r"(m[{k}])' for k in range(W)) + ', "=r"(c)'
    return f"""template <>
__device__ __forceinline__ uint32_t chain_inc<{W}>(uint32_t (&m)[{W}], uint32_t inc) {{
  uint32_t c;
  asm volatile(
{asm(lines)}
      : {outs}
      : "r"(inc));
  return c;
}}
"""


def borrow_chain(W):
    # 1 when a < b (the borrow out of a - b).  %0 t (scratch), %1 borrow, a %2.., b %W+2..
    a0, b0 = 2, 2 + W
    lines = [f"sub.cc.u32 %0, %{a0}, %{b0};"]
    lines += [f"subc.cc.u32 %0, %{a0 + k}, %{b0 + k};" for k in range(1, W)]
    lines += ["subc.u32 %1, 0, 0;"]
    ins = ", ".join(f'"r"(a[{k}])' for k in range(W)) + ", " + ", ".join(
        f'"r"(b[{k}])' for k in range(W))
    return f"""template <>
__device__ __forceinline__ uint32_t chain_borrow<{W}>(const uint32_t (&a)[{W}],
                                                      const uint32_t (&b)[{W}]) {{
  uint32_t t, bw;
  asm volatile(
{asm(lines)}
      : "=r"(t), "=r"(bw)
      : {ins});
  return bw & 1u;
}}
"""


def add_frame_chain(W):
    # T[0] = y[0] + c0; T[k] = x[k] + y[k] (k = 1..W); T[W+1] = carry out.
    # Operands: %0..%W+1 T, y %W+2..%2W+2, x[1..W] %2W+3..%3W+2, c0 %3W+3
    t0, y0, x1, c0 = 0, W + 2, 2 * W + 3, 3 * W + 3
    lines = [f"add.cc.u32 %{t0}, %{y0}, %{c0};"]
    lines += [f"addc.cc.u32 %{t0 + k}, %{x1 + k - 1}, %{y0 + k};" for k in range(1, W + 1)]
    lines += [f"addc.u32 %{t0 + W + 1}, 0, 0;"]
    outs = ", ".join(f'"=r"(T[{k}])' for k in range(W + 2))
    ins = ", ".join(f'"r"(y[{k}])' for k in range(W + 1)) + ", " + ", ".join(
        f'"r"(x[{k}])' for k in range(1, W + 1)) + ', "r"(c0)'
    return f"""template <>
__device__ __forceinline__ void chain_add_frame<{W}>(uint32_t (&T)[{W + 2}],
                                                     const uint32_t (&x)[{W + 1}],
                                                     const uint32_t (&y)[{W + 1}], uint32_t c0) {{
  asm volatile(
{asm(lines)}
      : {outs}
      : {ins});
}}
"""


def mul_row_chain(W):
    # Row of the schoolbook product: r[0..W] += lo(a b[j]) at r[j] (carry into
    # r[W]), then r[1..W] += hi(a b[j]) at r[j+1], carry out into r[W+1].
    # Operands: %0..%W+1 r (in/out; r[W+1] out only as the carry, written
    # even for the top row where it is discarded), a %W+2, b %W+3..%2W+2
    a, b0 = W + 2, W + 3
    lines = [f"mad.lo.cc.u32 %0, %{a}, %{b0}, %0;"]
    lines += [f"madc.lo.cc.u32 %{j}, %{a}, %{b0 + j}, %{j};" for j in range(1, W)]
    lines += [f"addc.u32 %{W}, %{W}, 0;"]
    lines += [f"mad.hi.cc.u32 %1, %{a}, %{b0}, %1;"]
    lines += [f"madc.hi.cc.u32 %{j + 1}, %{a}, %{b0 + j}, %{j + 1};" for j in range(1, W)]
    lines += [f"addc.u32 %{W + 1}, 0, 0;"]
    outs = ", ".join(f'"+r"(r[{k}])' for k in range(W + 1)) + f', "=r"(r[{W + 1}])'
    ins = '"r"(a), ' + ", ".join(f'"r"(b[{j}])' for j in range(W))
    return f"""template <>
__device__ __forceinline__ void chain_mul_row<{W}>(uint32_t (&r)[{W + 2}], uint32_t a,
                                                   const uint32_t (&b)[{W}]) {{
  asm volatile(
{asm(lines)}
      : {outs}
      : {ins});
}}
"""


def main():
    parts = ["""// chains.cuh -- written by gen_chains.py; do not edit by hand.
//
// Carry-flag chains of the p-bit arithmetic (mpdev.cuh), one inline-PTX
// statement per chain so that no instruction outside the chain can come
// between its add.cc / addc.cc / mad*.cc steps and the carry flag they pass.
//   chain_inc<W>(m, inc):      m += inc over W words, returns the carry out
//   chain_borrow<W>(a, b):     1 when a < b (W-word naturals)
//   chain_add_frame<W>(T,x,y,c0): T[0] = y[0] + c0, T[k] = x[k] + y[k] with
//                              carries (k = 1..W), T[W+1] = the carry out
//   chain_mul_row<W>(r, a, b): one schoolbook row on a window r[0..W+1]:
//                              r[0..W] += a * b (W words of b) with the low
//                              halves at r[j] and the high halves at r[j+1];
//                              r[W+1] receives the row's final carry (its
//                              value on entry is ignored)
#pragma once
#include <cstdint>

namespace mpk {

template <int W>
__device__ __forceinline__ uint32_t chain_inc(uint32_t (&m)[W], uint32_t inc);
template <int W>
__device__ __forceinline__ uint32_t chain_borrow(const uint32_t (&a)[W], const uint32_t (&b)[W]);
template <int W>
__device__ __forceinline__ void chain_add_frame(uint32_t (&T)[W + 2], const uint32_t (&x)[W + 1],
                                                const uint32_t (&y)[W + 1], uint32_t c0);
template <int W>
__device__ __forceinline__ void chain_mul_row(uint32_t (&r)[W + 2], uint32_t a,
                                              const uint32_t (&b)[W]);
"""]
    for W in WS:
        parts += [inc_chain(W), borrow_chain(W), add_frame_chain(W), mul_row_chain(W)]
    parts.append("}  // namespace mpk\n")
    with open(os.path.join(HERE, "chains.cuh"), "w") as f:
        f.write("\n".join(parts))


if __name__ == "__main__":
    main()
