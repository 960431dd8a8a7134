// Warp-level tensor-core helpers for FP32 stage products: mma.sync m16n8k8
// with TF32 operands and FP32 accumulation, each FP32 operand split into a
// TF32 high part and a TF32 remainder ("3xTF32": hi*hi + hi*lo + lo*hi),
// which keeps the products at FP32 accuracy.
// Fragment layout (PTX ISA, mma.m16n8k8, .tf32): with g = lane / 4 and
// q = lane % 4, A holds (g, q), (g + 8, q), (g, q + 4), (g + 8, q + 4); B holds
// (k = q, n = g), (k = q + 4, n = g); C holds (g, 2q), (g, 2q + 1), (g + 8, 2q),
// (g + 8, 2q + 1).
#pragma once

#include <cstdint>

namespace gq {
namespace dev {

__device__ __forceinline__ uint32_t tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

struct Tf32Pair {
  uint32_t hi, lo;
};

__device__ __forceinline__ Tf32Pair tf32_split(float x) {
  Tf32Pair p;
  p.hi = tf32_hi(x);
  p.lo = tf32_hi(x - __uint_as_float(p.hi));
  return p;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// c += A(16 x 8 tile) * B(8 x 8 tile) in 3xTF32; fa(r, k) and fb(k, n) give
// the tile elements (zero outside the matrices)
template <class FA, class FB>
__device__ __forceinline__ void mma3_tile(float (&c)[4], int lane, FA fa, FB fb) {
  const int g = lane >> 2, q = lane & 3;
  const Tf32Pair a0 = tf32_split(fa(g, q)), a1 = tf32_split(fa(g + 8, q));
  const Tf32Pair a2 = tf32_split(fa(g, q + 4)), a3 = tf32_split(fa(g + 8, q + 4));
  const Tf32Pair b0 = tf32_split(fb(q, g)), b1 = tf32_split(fb(q + 4, g));
  const uint32_t ahi[4] = {a0.hi, a1.hi, a2.hi, a3.hi}, alo[4] = {a0.lo, a1.lo, a2.lo, a3.lo};
  const uint32_t bhi[2] = {b0.hi, b1.hi}, blo[2] = {b0.lo, b1.lo};
  mma_tf32(c, alo, bhi);
  mma_tf32(c, ahi, blo);
  mma_tf32(c, ahi, bhi);
}

}  // namespace dev
}  // namespace gq
