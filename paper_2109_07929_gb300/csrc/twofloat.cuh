// Error-free transformations in FP32, for arithmetic on unevaluated pairs of floats.
//
// two_sum is Knuth's branch-free sum (The Art of Computer Programming, vol. 2, Sec. 4.2.2):
// s = fl(a + b) and e with s + e = a + b exactly.  two_prod uses the fused multiply-add:
// p = fl(a b) and e = fma(a, b, -p) = a b - p exactly (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005), as long as a b does not underflow.
// The _rn intrinsics keep the compiler from contracting or reordering these sequences.
#pragma once

namespace mca {

__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return s;
}

__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

}  // namespace mca
