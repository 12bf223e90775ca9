// Error-free binary32 transformations and the triple-binary32 accumulator
// used by the FP64-accurate residuals (no FP64 instruction in their loops).
#pragma once

namespace ebv {
namespace {

// Knuth's TwoSum, s + e == a + b exactly.  The _rn intrinsics are never
// contracted into fused multiply-adds, which would break the identity.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// p + e == a * b exactly (TwoProduct through the fused multiply-add).
__device__ __forceinline__ void two_prod_f(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}

// Accumulation of long dot products whose partial sums are O(1) while the
// result is tiny (a residual b - Ax near convergence), in binary32 only.
//
// A double-float (h, l) pair is not enough: once a large term (the diagonal
// of a dominant row) has entered, each TwoSum error of h is ~2^-25 |h|, the
// low word grows to ~sqrt(k) 2^-25 |h| after k terms and its own binary32
// rounding random-walks to ~1e-13 |h| and beyond.  (Restarting the pair every
// 16 terms and merging it into a triple still leaves ~2^-43 |h| in the block
// that holds the large term.)  TripleF gives every first-order quantity an
// error-free level: the products go into h by TwoSum, the TwoSum errors of h
// and the product errors / cross terms (both ~2^-24 |a x|) go into m by
// TwoSum, and only second-order errors (~2^-48 |partial sums|) reach the
// plain word l.  About 25 binary32 operations per multiply-add, with no FP64
// instruction in the loop.
struct TripleF {
  float h, m, l;
  __device__ __forceinline__ void zero() { h = m = l = 0.f; }
  // += (a_h + a_l) * (x_h + x_l), dropping a_l * x_l (relative 2^-47 or less).
  __device__ __forceinline__ void fma_split(float a_h, float a_l, float x_h, float x_l) {
    float p, pe, s, e1, t, e2, u, e3;
    two_prod_f(a_h, x_h, p, pe);
    const float c = pe + fmaf(a_h, x_l, a_l * x_h);  // rounding ~2^-48 |a x|
    two_sum_f(h, p, s, e1);
    two_sum_f(m, e1, t, e2);
    two_sum_f(t, c, u, e3);
    h = s;
    m = u;
    l += e2 + e3;
  }
  // += v (a single binary32 value), exact up to the rounding of l.
  __device__ __forceinline__ void add1(float v) {
    float s, e1, t, e2;
    two_sum_f(h, v, s, e1);
    two_sum_f(m, e1, t, e2);
    h = s;
    m = t;
    l += e2;
  }
  __device__ __forceinline__ void add(const TripleF &o) {
    float s, e1, t, e2, u, e3;
    two_sum_f(h, o.h, s, e1);
    two_sum_f(m, o.m, t, e2);
    two_sum_f(t, e1, u, e3);
    h = s;
    m = u;
    l += o.l + e2 + e3;
  }
  __device__ __forceinline__ double value() const { return (double)h + ((double)m + (double)l); }
};

}  // namespace
}  // namespace ebv
