// chains.cuh -- written by gen_chains.py; do not edit by hand.
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

template <>
__device__ __forceinline__ uint32_t chain_inc<4>(uint32_t (&m)[4], uint32_t inc) {
  uint32_t c;
  asm volatile(
      "add.cc.u32 %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.u32 %4, 0, 0;\n\t"
      : "+r"(m[0]), "+r"(m[1]), "+r"(m[2]), "+r"(m[3]), "=r"(c)
      : "r"(inc));
  return c;
}

template <>
__device__ __forceinline__ uint32_t chain_borrow<4>(const uint32_t (&a)[4],
                                                      const uint32_t (&b)[4]) {
  uint32_t t, bw;
  asm volatile(
      "sub.cc.u32 %0, %2, %6;\n\t"
      "subc.cc.u32 %0, %3, %7;\n\t"
      "subc.cc.u32 %0, %4, %8;\n\t"
      "subc.cc.u32 %0, %5, %9;\n\t"
      "subc.u32 %1, 0, 0;\n\t"
      : "=r"(t), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
  return bw & 1u;
}

template <>
__device__ __forceinline__ void chain_add_frame<4>(uint32_t (&T)[6],
                                                     const uint32_t (&x)[5],
                                                     const uint32_t (&y)[5], uint32_t c0) {
  asm volatile(
      "add.cc.u32 %0, %6, %15;\n\t"
      "addc.cc.u32 %1, %11, %7;\n\t"
      "addc.cc.u32 %2, %12, %8;\n\t"
      "addc.cc.u32 %3, %13, %9;\n\t"
      "addc.cc.u32 %4, %14, %10;\n\t"
      "addc.u32 %5, 0, 0;\n\t"
      : "=r"(T[0]), "=r"(T[1]), "=r"(T[2]), "=r"(T[3]), "=r"(T[4]), "=r"(T[5])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(c0));
}

template <>
__device__ __forceinline__ void chain_mul_row<4>(uint32_t (&r)[6], uint32_t a,
                                                   const uint32_t (&b)[4]) {
  asm volatile(
      "mad.lo.cc.u32 %0, %6, %7, %0;\n\t"
      "madc.lo.cc.u32 %1, %6, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %9, %2;\n\t"
      "madc.lo.cc.u32 %3, %6, %10, %3;\n\t"
      "addc.u32 %4, %4, 0;\n\t"
      "mad.hi.cc.u32 %1, %6, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %6, %8, %2;\n\t"
      "madc.hi.cc.u32 %3, %6, %9, %3;\n\t"
      "madc.hi.cc.u32 %4, %6, %10, %4;\n\t"
      "addc.u32 %5, 0, 0;\n\t"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "=r"(r[5])
      : "r"(a), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
}

template <>
__device__ __forceinline__ uint32_t chain_inc<8>(uint32_t (&m)[8], uint32_t inc) {
  uint32_t c;
  asm volatile(
      "add.cc.u32 %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.cc.u32 %4, %4, 0;\n\t"
      "addc.cc.u32 %5, %5, 0;\n\t"
      "addc.cc.u32 %6, %6, 0;\n\t"
      "addc.cc.u32 %7, %7, 0;\n\t"
      "addc.u32 %8, 0, 0;\n\t"
      : "+r"(m[0]), "+r"(m[1]), "+r"(m[2]), "+r"(m[3]), "+r"(m[4]), "+r"(m[5]), "+r"(m[6]), "+r"(m[7]), "=r"(c)
      : "r"(inc));
  return c;
}

template <>
__device__ __forceinline__ uint32_t chain_borrow<8>(const uint32_t (&a)[8],
                                                      const uint32_t (&b)[8]) {
  uint32_t t, bw;
  asm volatile(
      "sub.cc.u32 %0, %2, %10;\n\t"
      "subc.cc.u32 %0, %3, %11;\n\t"
      "subc.cc.u32 %0, %4, %12;\n\t"
      "subc.cc.u32 %0, %5, %13;\n\t"
      "subc.cc.u32 %0, %6, %14;\n\t"
      "subc.cc.u32 %0, %7, %15;\n\t"
      "subc.cc.u32 %0, %8, %16;\n\t"
      "subc.cc.u32 %0, %9, %17;\n\t"
      "subc.u32 %1, 0, 0;\n\t"
      : "=r"(t), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  return bw & 1u;
}

template <>
__device__ __forceinline__ void chain_add_frame<8>(uint32_t (&T)[10],
                                                     const uint32_t (&x)[9],
                                                     const uint32_t (&y)[9], uint32_t c0) {
  asm volatile(
      "add.cc.u32 %0, %10, %27;\n\t"
      "addc.cc.u32 %1, %19, %11;\n\t"
      "addc.cc.u32 %2, %20, %12;\n\t"
      "addc.cc.u32 %3, %21, %13;\n\t"
      "addc.cc.u32 %4, %22, %14;\n\t"
      "addc.cc.u32 %5, %23, %15;\n\t"
      "addc.cc.u32 %6, %24, %16;\n\t"
      "addc.cc.u32 %7, %25, %17;\n\t"
      "addc.cc.u32 %8, %26, %18;\n\t"
      "addc.u32 %9, 0, 0;\n\t"
      : "=r"(T[0]), "=r"(T[1]), "=r"(T[2]), "=r"(T[3]), "=r"(T[4]), "=r"(T[5]), "=r"(T[6]), "=r"(T[7]), "=r"(T[8]), "=r"(T[9])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]), "r"(y[8]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(c0));
}

template <>
__device__ __forceinline__ void chain_mul_row<8>(uint32_t (&r)[10], uint32_t a,
                                                   const uint32_t (&b)[8]) {
  asm volatile(
      "mad.lo.cc.u32 %0, %10, %11, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %12, %1;\n\t"
      "madc.lo.cc.u32 %2, %10, %13, %2;\n\t"
      "madc.lo.cc.u32 %3, %10, %14, %3;\n\t"
      "madc.lo.cc.u32 %4, %10, %15, %4;\n\t"
      "madc.lo.cc.u32 %5, %10, %16, %5;\n\t"
      "madc.lo.cc.u32 %6, %10, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %10, %18, %7;\n\t"
      "addc.u32 %8, %8, 0;\n\t"
      "mad.hi.cc.u32 %1, %10, %11, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %12, %2;\n\t"
      "madc.hi.cc.u32 %3, %10, %13, %3;\n\t"
      "madc.hi.cc.u32 %4, %10, %14, %4;\n\t"
      "madc.hi.cc.u32 %5, %10, %15, %5;\n\t"
      "madc.hi.cc.u32 %6, %10, %16, %6;\n\t"
      "madc.hi.cc.u32 %7, %10, %17, %7;\n\t"
      "madc.hi.cc.u32 %8, %10, %18, %8;\n\t"
      "addc.u32 %9, 0, 0;\n\t"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "=r"(r[9])
      : "r"(a), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
}

template <>
__device__ __forceinline__ uint32_t chain_inc<16>(uint32_t (&m)[16], uint32_t inc) {
  uint32_t c;
  asm volatile(
      "add.cc.u32 %0, %0, %17;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.cc.u32 %4, %4, 0;\n\t"
      "addc.cc.u32 %5, %5, 0;\n\t"
      "addc.cc.u32 %6, %6, 0;\n\t"
      "addc.cc.u32 %7, %7, 0;\n\t"
      "addc.cc.u32 %8, %8, 0;\n\t"
      "addc.cc.u32 %9, %9, 0;\n\t"
      "addc.cc.u32 %10, %10, 0;\n\t"
      "addc.cc.u32 %11, %11, 0;\n\t"
      "addc.cc.u32 %12, %12, 0;\n\t"
      "addc.cc.u32 %13, %13, 0;\n\t"
      "addc.cc.u32 %14, %14, 0;\n\t"
      "addc.cc.u32 %15, %15, 0;\n\t"
      "addc.u32 %16, 0, 0;\n\t"
      : "+r"(m[0]), "+r"(m[1]), "+r"(m[2]), "+r"(m[3]), "+r"(m[4]), "+r"(m[5]), "+r"(m[6]), "+r"(m[7]), "+r"(m[8]), "+r"(m[9]), "+r"(m[10]), "+r"(m[11]), "+r"(m[12]), "+r"(m[13]), "+r"(m[14]), "+r"(m[15]), "=r"(c)
      : "r"(inc));
  return c;
}

template <>
__device__ __forceinline__ uint32_t chain_borrow<16>(const uint32_t (&a)[16],
                                                      const uint32_t (&b)[16]) {
  uint32_t t, bw;
  asm volatile(
      "sub.cc.u32 %0, %2, %18;\n\t"
      "subc.cc.u32 %0, %3, %19;\n\t"
      "subc.cc.u32 %0, %4, %20;\n\t"
      "subc.cc.u32 %0, %5, %21;\n\t"
      "subc.cc.u32 %0, %6, %22;\n\t"
      "subc.cc.u32 %0, %7, %23;\n\t"
      "subc.cc.u32 %0, %8, %24;\n\t"
      "subc.cc.u32 %0, %9, %25;\n\t"
      "subc.cc.u32 %0, %10, %26;\n\t"
      "subc.cc.u32 %0, %11, %27;\n\t"
      "subc.cc.u32 %0, %12, %28;\n\t"
      "subc.cc.u32 %0, %13, %29;\n\t"
      "subc.cc.u32 %0, %14, %30;\n\t"
      "subc.cc.u32 %0, %15, %31;\n\t"
      "subc.cc.u32 %0, %16, %32;\n\t"
      "subc.cc.u32 %0, %17, %33;\n\t"
      "subc.u32 %1, 0, 0;\n\t"
      : "=r"(t), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]));
  return bw & 1u;
}

template <>
__device__ __forceinline__ void chain_add_frame<16>(uint32_t (&T)[18],
                                                     const uint32_t (&x)[17],
                                                     const uint32_t (&y)[17], uint32_t c0) {
  asm volatile(
      "add.cc.u32 %0, %18, %51;\n\t"
      "addc.cc.u32 %1, %35, %19;\n\t"
      "addc.cc.u32 %2, %36, %20;\n\t"
      "addc.cc.u32 %3, %37, %21;\n\t"
      "addc.cc.u32 %4, %38, %22;\n\t"
      "addc.cc.u32 %5, %39, %23;\n\t"
      "addc.cc.u32 %6, %40, %24;\n\t"
      "addc.cc.u32 %7, %41, %25;\n\t"
      "addc.cc.u32 %8, %42, %26;\n\t"
      "addc.cc.u32 %9, %43, %27;\n\t"
      "addc.cc.u32 %10, %44, %28;\n\t"
      "addc.cc.u32 %11, %45, %29;\n\t"
      "addc.cc.u32 %12, %46, %30;\n\t"
      "addc.cc.u32 %13, %47, %31;\n\t"
      "addc.cc.u32 %14, %48, %32;\n\t"
      "addc.cc.u32 %15, %49, %33;\n\t"
      "addc.cc.u32 %16, %50, %34;\n\t"
      "addc.u32 %17, 0, 0;\n\t"
      : "=r"(T[0]), "=r"(T[1]), "=r"(T[2]), "=r"(T[3]), "=r"(T[4]), "=r"(T[5]), "=r"(T[6]), "=r"(T[7]), "=r"(T[8]), "=r"(T[9]), "=r"(T[10]), "=r"(T[11]), "=r"(T[12]), "=r"(T[13]), "=r"(T[14]), "=r"(T[15]), "=r"(T[16]), "=r"(T[17])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]), "r"(y[8]), "r"(y[9]), "r"(y[10]), "r"(y[11]), "r"(y[12]), "r"(y[13]), "r"(y[14]), "r"(y[15]), "r"(y[16]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]), "r"(x[16]), "r"(c0));
}

template <>
__device__ __forceinline__ void chain_mul_row<16>(uint32_t (&r)[18], uint32_t a,
                                                   const uint32_t (&b)[16]) {
  asm volatile(
      "mad.lo.cc.u32 %0, %18, %19, %0;\n\t"
      "madc.lo.cc.u32 %1, %18, %20, %1;\n\t"
      "madc.lo.cc.u32 %2, %18, %21, %2;\n\t"
      "madc.lo.cc.u32 %3, %18, %22, %3;\n\t"
      "madc.lo.cc.u32 %4, %18, %23, %4;\n\t"
      "madc.lo.cc.u32 %5, %18, %24, %5;\n\t"
      "madc.lo.cc.u32 %6, %18, %25, %6;\n\t"
      "madc.lo.cc.u32 %7, %18, %26, %7;\n\t"
      "madc.lo.cc.u32 %8, %18, %27, %8;\n\t"
      "madc.lo.cc.u32 %9, %18, %28, %9;\n\t"
      "madc.lo.cc.u32 %10, %18, %29, %10;\n\t"
      "madc.lo.cc.u32 %11, %18, %30, %11;\n\t"
      "madc.lo.cc.u32 %12, %18, %31, %12;\n\t"
      "madc.lo.cc.u32 %13, %18, %32, %13;\n\t"
      "madc.lo.cc.u32 %14, %18, %33, %14;\n\t"
      "madc.lo.cc.u32 %15, %18, %34, %15;\n\t"
      "addc.u32 %16, %16, 0;\n\t"
      "mad.hi.cc.u32 %1, %18, %19, %1;\n\t"
      "madc.hi.cc.u32 %2, %18, %20, %2;\n\t"
      "madc.hi.cc.u32 %3, %18, %21, %3;\n\t"
      "madc.hi.cc.u32 %4, %18, %22, %4;\n\t"
      "madc.hi.cc.u32 %5, %18, %23, %5;\n\t"
      "madc.hi.cc.u32 %6, %18, %24, %6;\n\t"
      "madc.hi.cc.u32 %7, %18, %25, %7;\n\t"
      "madc.hi.cc.u32 %8, %18, %26, %8;\n\t"
      "madc.hi.cc.u32 %9, %18, %27, %9;\n\t"
      "madc.hi.cc.u32 %10, %18, %28, %10;\n\t"
      "madc.hi.cc.u32 %11, %18, %29, %11;\n\t"
      "madc.hi.cc.u32 %12, %18, %30, %12;\n\t"
      "madc.hi.cc.u32 %13, %18, %31, %13;\n\t"
      "madc.hi.cc.u32 %14, %18, %32, %14;\n\t"
      "madc.hi.cc.u32 %15, %18, %33, %15;\n\t"
      "madc.hi.cc.u32 %16, %18, %34, %16;\n\t"
      "addc.u32 %17, 0, 0;\n\t"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "=r"(r[17])
      : "r"(a), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]));
}

template <>
__device__ __forceinline__ uint32_t chain_inc<32>(uint32_t (&m)[32], uint32_t inc) {
  uint32_t c;
  asm volatile(
      "add.cc.u32 %0, %0, %33;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.cc.u32 %4, %4, 0;\n\t"
      "addc.cc.u32 %5, %5, 0;\n\t"
      "addc.cc.u32 %6, %6, 0;\n\t"
      "addc.cc.u32 %7, %7, 0;\n\t"
      "addc.cc.u32 %8, %8, 0;\n\t"
      "addc.cc.u32 %9, %9, 0;\n\t"
      "addc.cc.u32 %10, %10, 0;\n\t"
      "addc.cc.u32 %11, %11, 0;\n\t"
      "addc.cc.u32 %12, %12, 0;\n\t"
      "addc.cc.u32 %13, %13, 0;\n\t"
      "addc.cc.u32 %14, %14, 0;\n\t"
      "addc.cc.u32 %15, %15, 0;\n\t"
      "addc.cc.u32 %16, %16, 0;\n\t"
      "addc.cc.u32 %17, %17, 0;\n\t"
      "addc.cc.u32 %18, %18, 0;\n\t"
      "addc.cc.u32 %19, %19, 0;\n\t"
      "addc.cc.u32 %20, %20, 0;\n\t"
      "addc.cc.u32 %21, %21, 0;\n\t"
      "addc.cc.u32 %22, %22, 0;\n\t"
      "addc.cc.u32 %23, %23, 0;\n\t"
      "addc.cc.u32 %24, %24, 0;\n\t"
      "addc.cc.u32 %25, %25, 0;\n\t"
      "addc.cc.u32 %26, %26, 0;\n\t"
      "addc.cc.u32 %27, %27, 0;\n\t"
      "addc.cc.u32 %28, %28, 0;\n\t"
      "addc.cc.u32 %29, %29, 0;\n\t"
      "addc.cc.u32 %30, %30, 0;\n\t"
      "addc.cc.u32 %31, %31, 0;\n\t"
      "addc.u32 %32, 0, 0;\n\t"
      : "+r"(m[0]), "+r"(m[1]), "+r"(m[2]), "+r"(m[3]), "+r"(m[4]), "+r"(m[5]), "+r"(m[6]), "+r"(m[7]), "+r"(m[8]), "+r"(m[9]), "+r"(m[10]), "+r"(m[11]), "+r"(m[12]), "+r"(m[13]), "+r"(m[14]), "+r"(m[15]), "+r"(m[16]), "+r"(m[17]), "+r"(m[18]), "+r"(m[19]), "+r"(m[20]), "+r"(m[21]), "+r"(m[22]), "+r"(m[23]), "+r"(m[24]), "+r"(m[25]), "+r"(m[26]), "+r"(m[27]), "+r"(m[28]), "+r"(m[29]), "+r"(m[30]), "+r"(m[31]), "=r"(c)
      : "r"(inc));
  return c;
}

template <>
__device__ __forceinline__ uint32_t chain_borrow<32>(const uint32_t (&a)[32],
                                                      const uint32_t (&b)[32]) {
  uint32_t t, bw;
  asm volatile(
      "sub.cc.u32 %0, %2, %34;\n\t"
      "subc.cc.u32 %0, %3, %35;\n\t"
      "subc.cc.u32 %0, %4, %36;\n\t"
      "subc.cc.u32 %0, %5, %37;\n\t"
      "subc.cc.u32 %0, %6, %38;\n\t"
      "subc.cc.u32 %0, %7, %39;\n\t"
      "subc.cc.u32 %0, %8, %40;\n\t"
      "subc.cc.u32 %0, %9, %41;\n\t"
      "subc.cc.u32 %0, %10, %42;\n\t"
      "subc.cc.u32 %0, %11, %43;\n\t"
      "subc.cc.u32 %0, %12, %44;\n\t"
      "subc.cc.u32 %0, %13, %45;\n\t"
      "subc.cc.u32 %0, %14, %46;\n\t"
      "subc.cc.u32 %0, %15, %47;\n\t"
      "subc.cc.u32 %0, %16, %48;\n\t"
      "subc.cc.u32 %0, %17, %49;\n\t"
      "subc.cc.u32 %0, %18, %50;\n\t"
      "subc.cc.u32 %0, %19, %51;\n\t"
      "subc.cc.u32 %0, %20, %52;\n\t"
      "subc.cc.u32 %0, %21, %53;\n\t"
      "subc.cc.u32 %0, %22, %54;\n\t"
      "subc.cc.u32 %0, %23, %55;\n\t"
      "subc.cc.u32 %0, %24, %56;\n\t"
      "subc.cc.u32 %0, %25, %57;\n\t"
      "subc.cc.u32 %0, %26, %58;\n\t"
      "subc.cc.u32 %0, %27, %59;\n\t"
      "subc.cc.u32 %0, %28, %60;\n\t"
      "subc.cc.u32 %0, %29, %61;\n\t"
      "subc.cc.u32 %0, %30, %62;\n\t"
      "subc.cc.u32 %0, %31, %63;\n\t"
      "subc.cc.u32 %0, %32, %64;\n\t"
      "subc.cc.u32 %0, %33, %65;\n\t"
      "subc.u32 %1, 0, 0;\n\t"
      : "=r"(t), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(a[16]), "r"(a[17]), "r"(a[18]), "r"(a[19]), "r"(a[20]), "r"(a[21]), "r"(a[22]), "r"(a[23]), "r"(a[24]), "r"(a[25]), "r"(a[26]), "r"(a[27]), "r"(a[28]), "r"(a[29]), "r"(a[30]), "r"(a[31]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]), "r"(b[16]), "r"(b[17]), "r"(b[18]), "r"(b[19]), "r"(b[20]), "r"(b[21]), "r"(b[22]), "r"(b[23]), "r"(b[24]), "r"(b[25]), "r"(b[26]), "r"(b[27]), "r"(b[28]), "r"(b[29]), "r"(b[30]), "r"(b[31]));
  return bw & 1u;
}

template <>
__device__ __forceinline__ void chain_add_frame<32>(uint32_t (&T)[34],
                                                     const uint32_t (&x)[33],
                                                     const uint32_t (&y)[33], uint32_t c0) {
  asm volatile(
      "add.cc.u32 %0, %34, %99;\n\t"
      "addc.cc.u32 %1, %67, %35;\n\t"
      "addc.cc.u32 %2, %68, %36;\n\t"
      "addc.cc.u32 %3, %69, %37;\n\t"
      "addc.cc.u32 %4, %70, %38;\n\t"
      "addc.cc.u32 %5, %71, %39;\n\t"
      "addc.cc.u32 %6, %72, %40;\n\t"
      "addc.cc.u32 %7, %73, %41;\n\t"
      "addc.cc.u32 %8, %74, %42;\n\t"
      "addc.cc.u32 %9, %75, %43;\n\t"
      "addc.cc.u32 %10, %76, %44;\n\t"
      "addc.cc.u32 %11, %77, %45;\n\t"
      "addc.cc.u32 %12, %78, %46;\n\t"
      "addc.cc.u32 %13, %79, %47;\n\t"
      "addc.cc.u32 %14, %80, %48;\n\t"
      "addc.cc.u32 %15, %81, %49;\n\t"
      "addc.cc.u32 %16, %82, %50;\n\t"
      "addc.cc.u32 %17, %83, %51;\n\t"
      "addc.cc.u32 %18, %84, %52;\n\t"
      "addc.cc.u32 %19, %85, %53;\n\t"
      "addc.cc.u32 %20, %86, %54;\n\t"
      "addc.cc.u32 %21, %87, %55;\n\t"
      "addc.cc.u32 %22, %88, %56;\n\t"
      "addc.cc.u32 %23, %89, %57;\n\t"
      "addc.cc.u32 %24, %90, %58;\n\t"
      "addc.cc.u32 %25, %91, %59;\n\t"
      "addc.cc.u32 %26, %92, %60;\n\t"
      "addc.cc.u32 %27, %93, %61;\n\t"
      "addc.cc.u32 %28, %94, %62;\n\t"
      "addc.cc.u32 %29, %95, %63;\n\t"
      "addc.cc.u32 %30, %96, %64;\n\t"
      "addc.cc.u32 %31, %97, %65;\n\t"
      "addc.cc.u32 %32, %98, %66;\n\t"
      "addc.u32 %33, 0, 0;\n\t"
      : "=r"(T[0]), "=r"(T[1]), "=r"(T[2]), "=r"(T[3]), "=r"(T[4]), "=r"(T[5]), "=r"(T[6]), "=r"(T[7]), "=r"(T[8]), "=r"(T[9]), "=r"(T[10]), "=r"(T[11]), "=r"(T[12]), "=r"(T[13]), "=r"(T[14]), "=r"(T[15]), "=r"(T[16]), "=r"(T[17]), "=r"(T[18]), "=r"(T[19]), "=r"(T[20]), "=r"(T[21]), "=r"(T[22]), "=r"(T[23]), "=r"(T[24]), "=r"(T[25]), "=r"(T[26]), "=r"(T[27]), "=r"(T[28]), "=r"(T[29]), "=r"(T[30]), "=r"(T[31]), "=r"(T[32]), "=r"(T[33])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]), "r"(y[8]), "r"(y[9]), "r"(y[10]), "r"(y[11]), "r"(y[12]), "r"(y[13]), "r"(y[14]), "r"(y[15]), "r"(y[16]), "r"(y[17]), "r"(y[18]), "r"(y[19]), "r"(y[20]), "r"(y[21]), "r"(y[22]), "r"(y[23]), "r"(y[24]), "r"(y[25]), "r"(y[26]), "r"(y[27]), "r"(y[28]), "r"(y[29]), "r"(y[30]), "r"(y[31]), "r"(y[32]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]), "r"(x[16]), "r"(x[17]), "r"(x[18]), "r"(x[19]), "r"(x[20]), "r"(x[21]), "r"(x[22]), "r"(x[23]), "r"(x[24]), "r"(x[25]), "r"(x[26]), "r"(x[27]), "r"(x[28]), "r"(x[29]), "r"(x[30]), "r"(x[31]), "r"(x[32]), "r"(c0));
}

template <>
__device__ __forceinline__ void chain_mul_row<32>(uint32_t (&r)[34], uint32_t a,
                                                   const uint32_t (&b)[32]) {
  asm volatile(
      "mad.lo.cc.u32 %0, %34, %35, %0;\n\t"
      "madc.lo.cc.u32 %1, %34, %36, %1;\n\t"
      "madc.lo.cc.u32 %2, %34, %37, %2;\n\t"
      "madc.lo.cc.u32 %3, %34, %38, %3;\n\t"
      "madc.lo.cc.u32 %4, %34, %39, %4;\n\t"
      "madc.lo.cc.u32 %5, %34, %40, %5;\n\t"
      "madc.lo.cc.u32 %6, %34, %41, %6;\n\t"
      "madc.lo.cc.u32 %7, %34, %42, %7;\n\t"
      "madc.lo.cc.u32 %8, %34, %43, %8;\n\t"
      "madc.lo.cc.u32 %9, %34, %44, %9;\n\t"
      "madc.lo.cc.u32 %10, %34, %45, %10;\n\t"
      "madc.lo.cc.u32 %11, %34, %46, %11;\n\t"
      "madc.lo.cc.u32 %12, %34, %47, %12;\n\t"
      "madc.lo.cc.u32 %13, %34, %48, %13;\n\t"
      "madc.lo.cc.u32 %14, %34, %49, %14;\n\t"
      "madc.lo.cc.u32 %15, %34, %50, %15;\n\t"
      "madc.lo.cc.u32 %16, %34, %51, %16;\n\t"
      "madc.lo.cc.u32 %17, %34, %52, %17;\n\t"
      "madc.lo.cc.u32 %18, %34, %53, %18;\n\t"
      "madc.lo.cc.u32 %19, %34, %54, %19;\n\t"
      "madc.lo.cc.u32 %20, %34, %55, %20;\n\t"
      "madc.lo.cc.u32 %21, %34, %56, %21;\n\t"
      "madc.lo.cc.u32 %22, %34, %57, %22;\n\t"
      "madc.lo.cc.u32 %23, %34, %58, %23;\n\t"
      "madc.lo.cc.u32 %24, %34, %59, %24;\n\t"
      "madc.lo.cc.u32 %25, %34, %60, %25;\n\t"
      "madc.lo.cc.u32 %26, %34, %61, %26;\n\t"
      "madc.lo.cc.u32 %27, %34, %62, %27;\n\t"
      "madc.lo.cc.u32 %28, %34, %63, %28;\n\t"
      "madc.lo.cc.u32 %29, %34, %64, %29;\n\t"
      "madc.lo.cc.u32 %30, %34, %65, %30;\n\t"
      "madc.lo.cc.u32 %31, %34, %66, %31;\n\t"
      "addc.u32 %32, %32, 0;\n\t"
      "mad.hi.cc.u32 %1, %34, %35, %1;\n\t"
      "madc.hi.cc.u32 %2, %34, %36, %2;\n\t"
      "madc.hi.cc.u32 %3, %34, %37, %3;\n\t"
      "madc.hi.cc.u32 %4, %34, %38, %4;\n\t"
      "madc.hi.cc.u32 %5, %34, %39, %5;\n\t"
      "madc.hi.cc.u32 %6, %34, %40, %6;\n\t"
      "madc.hi.cc.u32 %7, %34, %41, %7;\n\t"
      "madc.hi.cc.u32 %8, %34, %42, %8;\n\t"
      "madc.hi.cc.u32 %9, %34, %43, %9;\n\t"
      "madc.hi.cc.u32 %10, %34, %44, %10;\n\t"
      "madc.hi.cc.u32 %11, %34, %45, %11;\n\t"
      "madc.hi.cc.u32 %12, %34, %46, %12;\n\t"
      "madc.hi.cc.u32 %13, %34, %47, %13;\n\t"
      "madc.hi.cc.u32 %14, %34, %48, %14;\n\t"
      "madc.hi.cc.u32 %15, %34, %49, %15;\n\t"
      "madc.hi.cc.u32 %16, %34, %50, %16;\n\t"
      "madc.hi.cc.u32 %17, %34, %51, %17;\n\t"
      "madc.hi.cc.u32 %18, %34, %52, %18;\n\t"
      "madc.hi.cc.u32 %19, %34, %53, %19;\n\t"
      "madc.hi.cc.u32 %20, %34, %54, %20;\n\t"
      "madc.hi.cc.u32 %21, %34, %55, %21;\n\t"
      "madc.hi.cc.u32 %22, %34, %56, %22;\n\t"
      "madc.hi.cc.u32 %23, %34, %57, %23;\n\t"
      "madc.hi.cc.u32 %24, %34, %58, %24;\n\t"
      "madc.hi.cc.u32 %25, %34, %59, %25;\n\t"
      "madc.hi.cc.u32 %26, %34, %60, %26;\n\t"
      "madc.hi.cc.u32 %27, %34, %61, %27;\n\t"
      "madc.hi.cc.u32 %28, %34, %62, %28;\n\t"
      "madc.hi.cc.u32 %29, %34, %63, %29;\n\t"
      "madc.hi.cc.u32 %30, %34, %64, %30;\n\t"
      "madc.hi.cc.u32 %31, %34, %65, %31;\n\t"
      "madc.hi.cc.u32 %32, %34, %66, %32;\n\t"
      "addc.u32 %33, 0, 0;\n\t"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "=r"(r[33])
      : "r"(a), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]), "r"(b[16]), "r"(b[17]), "r"(b[18]), "r"(b[19]), "r"(b[20]), "r"(b[21]), "r"(b[22]), "r"(b[23]), "r"(b[24]), "r"(b[25]), "r"(b[26]), "r"(b[27]), "r"(b[28]), "r"(b[29]), "r"(b[30]), "r"(b[31]));
}

}  // namespace mpk
