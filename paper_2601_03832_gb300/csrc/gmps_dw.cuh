// Double-word ("float-float") arithmetic on the FP32 pipes.
//
// GB300's FP64 pipe issues one warp instruction per ~64 cycles and a
// dependent DFMA takes ~64 cycles; FP64 divide/sqrt take 440-690 cycles
// (measured on this part).  A value x = h + l held as two floats with
// |l| <= ulp(h)/2 carries a ~48-bit significand and runs on the FP32 pipes
// (1 warp instruction per cycle, 4-cycle latency).
//
// The algorithms are the double-word building blocks of M. Joldes,
// J.-M. Muller and V. Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
// 2Sum (Knuth), Fast2Sum (Dekker), 2Prod via FMA, DWPlusDW (accurate
// version), DWTimesDW with FMA and DWDivDW; sqrt uses one Newton correction
// of the correctly rounded FP32 square root (Karp & Markstein, "High
// precision division and square root", TOMS 1997).  Every float operation
// uses the _rn intrinsics so that no contraction or reassociation can break
// the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace gmps {

using ::fma;
using ::sqrt;
using ::rsqrt;
using ::fmax;

struct dw {
  float h, l;
  __device__ __forceinline__ dw() {}
  __device__ __forceinline__ dw(float hh, float ll) : h(hh), l(ll) {}
  __device__ __forceinline__ dw(float f) : h(f), l(0.f) {}
  __device__ __forceinline__ dw(int i) : h((float)i), l(0.f) {}
  // from FP64 (used only off the hot path: loads of FP64 parameters)
  __device__ __forceinline__ explicit dw(double d) {
    h = __double2float_rn(d);
    l = __double2float_rn(d - (double)h);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
  __device__ __forceinline__ explicit operator float() const { return h; }
};

// complex element stored as two double-words (16 bytes)
struct __align__(16) dw2 {
  float rh, rl, ih, il;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
  float sh, sl, th, tl, vh, vl;
  two_sum(x.h, y.h, sh, sl);
  two_sum(x.l, y.l, th, tl);
  const float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = __fadd_rn(tl, vl);
  dw z;
  fast_two_sum(vh, w, z.h, z.l);
  return z;
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.h, -x.l); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl0 = __fmul_rn(x.l, y.l);
  const float tl1 = __fmaf_rn(x.h, y.l, tl0);
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  const float cl3 = __fadd_rn(cl1, cl2);
  dw z;
  fast_two_sum(ch, cl3, z.h, z.l);
  return z;
}
// DW times a float
__device__ __forceinline__ dw mul_f(dw x, float y) {
  const float ch = __fmul_rn(x.h, y);
  const float cl1 = __fmaf_rn(x.h, y, -ch);
  const float cl3 = __fmaf_rn(x.l, y, cl1);
  dw z;
  fast_two_sum(ch, cl3, z.h, z.l);
  return z;
}
__device__ __forceinline__ dw operator/(dw x, dw y) {
  const float th = __fdiv_rn(x.h, y.h);
  const dw r = mul_f(y, th);
  const float ph = __fsub_rn(x.h, r.h);
  const float dl = __fsub_rn(x.l, r.l);
  const float d = __fadd_rn(ph, dl);
  const float tl = __fdiv_rn(d, y.h);
  dw z;
  fast_two_sum(th, tl, z.h, z.l);
  return z;
}
__device__ __forceinline__ dw& operator+=(dw& a, dw b) { return a = a + b; }
__device__ __forceinline__ dw& operator-=(dw& a, dw b) { return a = a - b; }
__device__ __forceinline__ dw& operator*=(dw& a, dw b) { return a = a * b; }
__device__ __forceinline__ dw fma(dw a, dw b, dw c) { return a * b + c; }
__device__ __forceinline__ bool operator>(dw a, dw b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
__device__ __forceinline__ bool operator<(dw a, dw b) { return b > a; }
__device__ __forceinline__ bool operator==(dw a, dw b) { return a.h == b.h && a.l == b.l; }
__device__ __forceinline__ bool operator!=(dw a, dw b) { return !(a == b); }
__device__ __forceinline__ dw fmax(dw a, dw b) { return a > b ? a : b; }

// sqrt: s = RN(sqrt(h)); one Newton correction (x - s^2) / (2 s) in FP32.
__device__ __forceinline__ dw sqrt(dw x) {
  if (!(x.h > 0.f)) return dw(0.f, 0.f);
  const float s = __fsqrt_rn(x.h);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p), pe), x.l);
  const float c = __fdiv_rn(r, __fmul_rn(2.f, s));
  dw z;
  fast_two_sum(s, c, z.h, z.l);
  return z;
}
__device__ __forceinline__ dw rsqrt(dw x) { return dw(1.f) / sqrt(x); }

__device__ __forceinline__ dw shx(dw v, int o) {
  return dw(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

}  // namespace gmps
