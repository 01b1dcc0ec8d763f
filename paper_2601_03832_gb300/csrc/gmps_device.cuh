#pragma once
// Device code of the iterative-Grover MPS engine for sm_103a (included by
// one gmps_form_*.cu per arithmetic form, which instantiates it).
//
// One thread block owns one instance for a whole launch and applies all of
// its Grover iterations without returning to the host (Sec. III-A: the
// state is replaced by G|state> once per iteration, G = D O of Sec. II,
// Eq. 3).  Each operator is contracted into the site tensors, then the chain
// is recompressed by a canonicalising Householder-QR sweep (left to right)
// and a truncated one-sided-Jacobi SVD sweep (right to left), as the MPS
// backend of Sec. III-B-2 describes ("tensors are locally updated, and
// truncation is applied ...").  The chain is sequential along the sites, so
// the block's threads parallelise inside each small factorisation: lane
// groups own matrix columns (QR) or row pairs (Jacobi) and reduce with warp
// shuffles; all working matrices live in shared memory and, for small
// instances, the whole chain does too.  Steps small enough for one warp run
// in registers instead (gmps_tiny.cuh), and a second warp then takes the
// work off the sweep's critical path (Q formation, target environments).
//
// Arithmetic forms (template parameters): T = real type of the QR/SVD and
// scalar bookkeeping (double, or the double-word dw), S = storage type of a
// complex site element (double2, float2 or dw2), CR = real type of the
// contractions (double, float or dw).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include <type_traits>

#include "gmps_forms.h"

namespace cg = cooperative_groups;

namespace gmps {

// ------------------------------------------------------------------ complex
template <class T>
struct cx {
  T re, im;
};
template <class T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.re = a;
  r.im = b;
  return r;
}
template <class T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <class T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <class T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
template <class T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk<T>(a.re * s, a.im * s); }
// acc + a*b
template <class T>
__device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <class T>
__device__ __forceinline__ cx<T> cmacc(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <class T>
__device__ __forceinline__ T abs2(cx<T> a) { return fma(a.re, a.re, a.im * a.im); }

// storage <-> compute conversion
template <class T>
__device__ __forceinline__ cx<T> ld(const double2* p) {
  double2 v = *p;
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ __forceinline__ cx<T> ld(const float2* p) {
  float2 v = *p;
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ __forceinline__ void st(double2* p, cx<T> v) { *p = make_double2((double)v.re, (double)v.im); }
template <class T>
__device__ __forceinline__ void st(float2* p, cx<T> v) { *p = make_float2((float)v.re, (float)v.im); }
// double-word storage: exact for DW values, FP64 values are split on store
template <class T>
__device__ __forceinline__ cx<T> ld(const dw2* p) {
  const dw2 v = *p;
  return mk<T>((T)((double)v.rh + (double)v.rl), (T)((double)v.ih + (double)v.il));
}
template <>
__device__ __forceinline__ cx<dw> ld<dw>(const dw2* p) {
  const dw2 v = *p;
  return mk<dw>(dw(v.rh, v.rl), dw(v.ih, v.il));
}
__device__ __forceinline__ void st(dw2* p, cx<dw> v) {
  dw2 o;
  o.rh = v.re.h;
  o.rl = v.re.l;
  o.ih = v.im.h;
  o.il = v.im.l;
  *p = o;
}
__device__ __forceinline__ void st(dw2* p, cx<double> v) { st(p, mk<dw>(dw(v.re), dw(v.im))); }

// Murmur3's 64-bit finaliser (Appleby): a counter-based hash for the
// stochastic rounding of complex64 stores.
__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}
// x rounded to FP32 stochastically: up (away from zero) with probability
// equal to the dropped fraction of an FP32 unit, using 29 random bits r.
// Integer operations only (FP64 conversions would occupy the FP64 pipe).
// Outside FP32's normal range: round to nearest.
__device__ __forceinline__ float sr_f32(double x, unsigned r) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  if (mag < 0x3810000000000000ull || mag >= 0x47e0000000000000ull) return (float)x;  // |x| < 2^-126 or >= 2^127
  b += (unsigned long long)(r >> 3);      // 29 random bits below the FP32 significand
  b &= ~((1ull << 29) - 1ull);            // truncate: now exactly an FP32 value
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float((hi & 0x80000000u) | ((e - 1023u + 127u) << 23) | m);
}
// Store of a site-tensor element: round to nearest, except complex64 storage,
// which rounds stochastically.  The rounding of FP32 storage repeats nearly
// the same error every iteration on a slowly changing state, so with round to
// nearest it adds up linearly over k; stochastic rounding (random bits from
// the per-store key and the element's index) makes it a random walk.
template <class V>
__device__ __forceinline__ void st_site(double2* p, V v, unsigned long long, unsigned) { st(p, v); }
template <class V>
__device__ __forceinline__ void st_site(dw2* p, V v, unsigned long long, unsigned) { st(p, v); }
template <class T>
__device__ __forceinline__ void st_site(float2* p, cx<T> v, unsigned long long key, unsigned e) {
  const unsigned long long h = fmix64(key ^ ((unsigned long long)e * 0x9e3779b97f4a7c15ull));
  *p = make_float2(sr_f32((double)v.re, (unsigned)h), sr_f32((double)v.im, (unsigned)(h >> 32)));
}
template <class A, class B>
__device__ __forceinline__ cx<A> cvt(cx<B> v) { return mk<A>((A)v.re, (A)v.im); }
template <>
__device__ __forceinline__ cx<dw> cvt<dw, dw>(cx<dw> v) { return v; }

// per-type constants
template <class T>
struct K;
template <>
struct K<double> {
  static __device__ __forceinline__ double isq2() { return 0.70710678118654752440; }
  // Jacobi convergence: |<x_p,x_q>| <= tol sqrt(|x_p|^2 |x_q|^2)
  static __device__ __forceinline__ double jtol() { return 8.0 * 2.220446049250313e-16; }
  static __device__ __forceinline__ float jtolf() { return 1.7763568e-15f; }
  // squared column norm below which a Householder column counts as zero
  static __device__ __forceinline__ double tiny2() { return 0.0; }
  // |x0|^2 <= phase_floor |x|^2: the pivot is negligible, its phase is taken as 1
  // (keeps |x0|^2 out of the denormal range, where rsqrt is inaccurate)
  static __device__ __forceinline__ double phase_floor() { return 7.52316384526264e-37; }  // 2^-120
  // Householder columns are scaled by a power of two first (needed only when
  // the exponent range is FP32's)
  static constexpr bool kScaleColumns = false;
};
template <>
struct K<float> {
  static __device__ __forceinline__ float isq2() { return 0.70710677f; }
  static __device__ __forceinline__ float jtol() { return 8.f * 1.1920929e-07f; }
  static __device__ __forceinline__ float jtolf() { return 9.536743e-07f; }
  static __device__ __forceinline__ float tiny2() { return 0.f; }
  static __device__ __forceinline__ float phase_floor() { return 8.6736174e-19f; }  // 2^-60
  static constexpr bool kScaleColumns = true;
};
template <>
struct K<dw> {
  static __device__ __forceinline__ dw isq2() { return dw(0.70710677f, 1.2101617e-08f); }
  static __device__ __forceinline__ dw jtol() { return dw(5.6843419e-14f); }  // 2^-44
  static __device__ __forceinline__ float jtolf() { return 5.6843419e-14f; }
  static __device__ __forceinline__ dw tiny2() { return dw(0.f); }
  static __device__ __forceinline__ dw phase_floor() { return dw(7.8886091e-31f); }  // 2^-100
  // squares of entries below ~1e-16 are FP32 denormals: the reflector is built
  // from the column scaled to O(1) by an exact power of two
  static constexpr bool kScaleColumns = true;
};

// -------------------------------------------------------------- reductions
__device__ __forceinline__ double shx(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shx(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shx_m(double v, int o, unsigned m) { return __shfl_xor_sync(m, v, o); }
__device__ __forceinline__ float shx_m(float v, int o, unsigned m) { return __shfl_xor_sync(m, v, o); }
__device__ __forceinline__ dw shx_m(dw v, int o, unsigned m) {
  return dw(__shfl_xor_sync(m, v.h, o), __shfl_xor_sync(m, v.l, o));
}
__device__ __forceinline__ double shidx(double v, int i) { return __shfl_sync(0xffffffffu, v, i); }
__device__ __forceinline__ float shidx(float v, int i) { return __shfl_sync(0xffffffffu, v, i); }
__device__ __forceinline__ dw shidx(dw v, int i) {
  return dw(__shfl_sync(0xffffffffu, v.h, i), __shfl_sync(0xffffffffu, v.l, i));
}
template <class T>
__device__ __forceinline__ T gsum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += shx(v, o);
  return v;
}
__device__ __forceinline__ int pow2_cap32(int x) {
  int g = 1;
  while (g < x && g < 32) g <<= 1;
  return g;
}

// Lane groups: G consecutive lanes (G a power of two <= 32) work on one task.
struct Grp {
  int G, gid, lg, ng;
};
__device__ __forceinline__ Grp make_grp(int G) {
  Grp g;
  g.G = G;
  g.lg = threadIdx.x & (G - 1);
  g.gid = threadIdx.x / G;
  g.ng = blockDim.x / G;
  return g;
}
// Lanes per task for a block-wide sweep of `ntask` column tasks over `rows`
// rows (Householder updates, norms, Q formation): the power of two G <= 32
// minimising passes x (rows per lane x 10 + 3 log2 G), the FP64 instructions
// a warp issues per pass (dot, update and norm per element; three shuffle
// reductions per task).  Wide groups leave lanes idle on short columns and
// serialise few tasks; narrow ones take every task in one pass.
__device__ __forceinline__ int pick_g(int rows, int ntask) {
  int best = 32, bestc = 0x7fffffff;
#pragma unroll
  for (int lg = 0; lg <= 5; ++lg) {
    const int G = 1 << lg, ng = blockDim.x >> lg;
    const int cost = ((ntask + ng - 1) / ng) * (((rows + G - 1) >> lg) * 10 + 3 * lg);
    if (cost < bestc) {
      bestc = cost;
      best = G;
    }
  }
  return best;
}

// Device clock in ns and the SM id, for the per-instance busy-time record.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return (int)r;
}

// ----------------------------------------------------------- device state
template <class T, class S>
struct Blk {
  const InstDesc* d;
  int n;
  S* sites;                // slab base (shared or global)
  const int* off;          // slot offsets (shared copy)
  int* chi;                // [n+1] bond after the last SVD sweep (shared)
  int* qb;                 // [n+1] bonds after the QR sweep (shared)
  unsigned long long* tbits;  // direct-sum product terms
  int* tplus;
  cx<T>* tcoef;
  cx<T>* amps;
  cx<T>* Rp;               // R carried by the QR sweep
  cx<T>* W;                // QR work matrix
  T* tau;
  cx<T>* beta;
  cx<T>* Mat;              // SVD work matrix
  cx<T>* U;                // accumulated Jacobi rotations
  cx<T>* US;               // U*S carried by the SVD sweep
  T* sig;
  int* perm;
  int* qperm;              // QR column pivots
  T* qcn;                  // QR trailing column norms
  unsigned char* tbuf;     // two buffers: 32 lanes' reflector registers + (p, m) of a small QR step
  int* misc;               // [0] status, [1] max sweeps, [2] sweeps sum, [3] svd count, [4] k kept
  double* dmisc;           // [0] log_norm, [1] discarded, [2..5] phase coefficients
  unsigned long long rng;  // key of this sweep pair's stochastic rounding (complex64 storage)
  int csize;               // CTAs of the cluster sharing the large QR steps (1: this block alone)
  T* tmisc;                // [0] rank-rule eps, [1] tol, [2] discarded weight, [3..6] e^{i phi}-1 and 1-e^{i psi},
                           // [7] 2^{-n/2}, [8] Jacobi skip floor, [9] squared norm of the swept matrices
  __device__ S* slot(int l) const { return sites + off[l]; }
  // key of the stores into site l in one pass (0: QR sweep, 1: SVD sweep)
  __device__ unsigned long long key(int l, int pass) const {
    return fmix64(rng + (((unsigned long long)l << 2) | (unsigned long long)pass));
  }
};

// ------------------------------------------------- exponent / scaling helpers
// Exponent of a positive value and its scaled FP32 image, by integer bit
// manipulation (no FP64 conversion instructions: on this part those run on
// the FP64 pipe).  Scaled images truncate toward zero; underflow gives 0.
__device__ __forceinline__ int expo_of(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }
__device__ __forceinline__ int expo_of(dw x) { return ((__float_as_int(x.h) >> 23) & 0xff) - 127; }
__device__ __forceinline__ float f32_scaled(double x, int sh) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = (hi >> 20) & 0x7ff;
  if (e == 0) return 0.f;
  const int fe = e - 1023 - sh + 127;
  if (fe <= 0) return 0.f;
  if (fe >= 255) return __int_as_float((hi & 0x80000000) | 0x7f800000);
  const unsigned m = ((unsigned)(hi & 0xfffff) << 3) | ((unsigned)lo >> 29);
  return __uint_as_float(((unsigned)hi & 0x80000000u) | ((unsigned)fe << 23) | m);
}
__device__ __forceinline__ float f32_scaled(dw x, int sh) {
  const int u = __float_as_int(x.h);
  const int e = (u >> 23) & 0xff;
  if (e == 0) return 0.f;
  const int fe = e - sh;
  if (fe <= 0) return 0.f;
  if (fe >= 255) return __int_as_float((u & 0x80000000) | 0x7f800000);
  return __int_as_float((u & 0x807fffff) | (fe << 23));
}
// exact widening of a normal float (denormals -> 0)
template <class T>
__device__ __forceinline__ T widen(float f);
template <>
__device__ __forceinline__ double widen<double>(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xff;
  if (e == 0) return 0.0;
  const unsigned m = u & 0x7fffffu;
  return __hiloint2double((int)((u & 0x80000000u) | ((e - 127 + 1023) << 20) | (m >> 3)), (int)(m << 29));
}
template <>
__device__ __forceinline__ dw widen<dw>(float f) { return dw(f); }
// exact 2^e
template <class T>
__device__ __forceinline__ T pow2(int e);
template <>
__device__ __forceinline__ double pow2<double>(int e) { return __hiloint2double((e + 1023) << 20, 0); }
template <>
__device__ __forceinline__ float pow2<float>(int e) { return __int_as_float((e + 127) << 23); }
template <>
__device__ __forceinline__ dw pow2<dw>(int e) { return dw(__int_as_float((e + 127) << 23)); }
__device__ __forceinline__ int expo_abs(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }
__device__ __forceinline__ int expo_abs(float x) { return ((__float_as_int(x) >> 23) & 0xff) - 127; }
__device__ __forceinline__ int expo_abs(dw x) { return ((__float_as_int(x.h) >> 23) & 0xff) - 127; }

// ----------------------------------------------------------- Householder QR
// Householder reflectors H_j = I - tau_j v_j v_j^dag with v_j = x - beta_j e_j,
// beta_j = -e^{i arg x_j}|x|, tau_j = 1/(|x| (|x| + |x_j|)), so that H_j x =
// beta_j e_j.  The QR is rank-revealing: column pivoting (largest remaining
// column first), stopped once the largest remaining column norm is at or
// below the rank rule's noise floor, max(m, n) eps times the largest input
// column norm -- the directions left carry zero weight up to rounding (for
// the Grover iterate they are the rounding of its two-dimensional span).
// Column norms of the trailing block are recomputed by the lane group that
// updates each column.  In place on A (m x ncol, leading dim lda): on return
// perm[c] is the original index of the column now at position c; the first
// `rank` columns hold v_j from row j down, the leading `rank` rows the
// upper-trapezoidal R of the permuted matrix (diagonal in beta).  cn is
// scratch for ncol norms; ctl for 4 ints.  pref (npref entries, or null): the
// pivot sequence this step took in the previous iteration; step j takes
// column pref[j] again while its norm is at least half the largest remaining
// one, so that the sequence -- and the row basis it gives the next site --
// stays put between iterations (the stop test still uses the largest norm).
template <class T>
__device__ int qr_rank_revealing(cx<T>* A, int m, int ncol, int lda, T* tau, cx<T>* beta, int* perm, T* cn,
                                 int* ctl, T floor_rel2, const int* pref = nullptr, int npref = 0) {
  const int pmax = min(m, ncol);
  const int G = pow2_cap32(m);  // lanes on the pivot column
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  // initial column norms
  {
    const Grp g = make_grp(pick_g(m, ncol));
    for (int t0 = 0; t0 < ncol; t0 += g.ng) {
      const int c = t0 + g.gid;
      T s2 = 0;
      if (c < ncol)
        for (int i = g.lg; i < m; i += g.G) s2 += abs2(A[i * lda + c]);
      s2 = gsum(s2, g.G);
      if (c < ncol && g.lg == 0) {
        cn[c] = s2;
        perm[c] = c;
      }
    }
  }
  __syncthreads();
  T floor2 = 0;
  int rank = pmax;
  for (int j = 0; j < pmax; ++j) {
    if (threadIdx.x == 0) {
      // pivot: largest remaining norm (compared through exact FP32 images)
      const int want = j < npref ? pref[j] : -1;
      int best = j, keep = perm[j] == want ? j : -1;
      float bv = f32_scaled(cn[j], 0);
      for (int c = j + 1; c < ncol; ++c) {
        const float v = f32_scaled(cn[c], 0);
        if (v > bv) {
          bv = v;
          best = c;
        }
        if (perm[c] == want) keep = c;
      }
      if (j == 0) {
        ctl[1] = 0;
        // floor relative to the largest column norm of the input
        *(T*)(ctl + 2) = cn[best] * floor_rel2;
      }
      ctl[1] = (j > 0 && !(cn[best] > *(T*)(ctl + 2))) ? 1 : 0;
      if (keep >= 0 && f32_scaled(cn[keep], 0) >= 0.5f * bv) best = keep;
      ctl[0] = best;
      if (ctl[1] == 0 && best != j) {
        const T tc = cn[j];
        cn[j] = cn[best];
        cn[best] = tc;
        const int tp = perm[j];
        perm[j] = perm[best];
        perm[best] = tp;
      }
    }
    __syncthreads();
    if (ctl[1]) {
      rank = j;
      break;
    }
    const int best = ctl[0];
    if (best != j)
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const cx<T> t = A[i * lda + j];
        A[i * lda + j] = A[i * lda + best];
        A[i * lda + best] = t;
      }
    __syncthreads();
    if (threadIdx.x < G) {
      int em = -2000;
      if (K<T>::kScaleColumns) {
        for (int i = j + threadIdx.x; i < m; i += G) {
          const cx<T> x = A[i * lda + j];
          if (x.re != (T)0) em = max(em, expo_abs(x.re));
          if (x.im != (T)0) em = max(em, expo_abs(x.im));
        }
        for (int o = G >> 1; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(gmask, em, o));
      }
      const bool scl = K<T>::kScaleColumns && em > -2000;
      const T sc = scl ? pow2<T>(-em) : (T)1;
      // the pivot column's norm (rows >= j) is cn[j] unless the column was rescaled
      T s = 0;
      if (scl) {
        for (int i = j + threadIdx.x; i < m; i += G) {
          cx<T> x = cscale(A[i * lda + j], sc);
          A[i * lda + j] = x;
          s += abs2(x);
        }
        for (int o = G >> 1; o > 0; o >>= 1) s += shx_m(s, o, gmask);
      } else {
        s = cn[j];
      }
      if (threadIdx.x == 0) {
        cx<T> x0 = A[j * lda + j];
        T a2 = abs2(x0);
        cx<T> b = mk<T>(0, 0);
        T t = 0;
        if (s > K<T>::tiny2()) {
          T inv = rsqrt(s);
          T nrm = s * inv;
          cx<T> ph = mk<T>(1, 0);
          T ax0 = 0;
          if (a2 > K<T>::phase_floor() * s) {
            T ia = rsqrt(a2);
            ax0 = a2 * ia;
            ph = cscale(x0, ia);
          }
          b = cscale(ph, -nrm);
          t = (T)1 / (nrm * (nrm + ax0));
          A[j * lda + j] = csub(x0, b);
        }
        beta[j] = scl ? cscale(b, pow2<T>(em)) : b;
        tau[j] = t;
      }
    }
    __syncthreads();
    const T tj = tau[j];
    const int ntask = ncol - j - 1;
    const Grp g = make_grp(pick_g(m - j, ntask));
    for (int t0 = 0; t0 < ntask; t0 += g.ng) {
      const int c = j + 1 + t0 + g.gid;
      const bool act = (t0 + g.gid) < ntask;
      cx<T> w = mk<T>(0, 0);
      if (act)
        for (int i = j + g.lg; i < m; i += g.G) w = cmacc(w, A[i * lda + j], A[i * lda + c]);
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      T s2 = 0;
      if (act) {
        const cx<T> tw = cscale(w, -tj);
        for (int i = j + g.lg; i < m; i += g.G) {
          cx<T> x = A[i * lda + c];
          if (tj != (T)0) x = cmac(x, A[i * lda + j], tw);
          A[i * lda + c] = x;
          if (i > j) s2 += abs2(x);
        }
      }
      s2 = gsum(s2, g.G);
      if (act && g.lg == 0) cn[c] = s2;
    }
    __syncthreads();
  }
  return rank;
}

// ------------------------------------------------------ QR over a cluster
// A large rank-revealing QR (a generic MPO's expanded bond in the hundreds or
// thousands of columns) split over the CTAs of a thread-block cluster: CTA r
// owns a contiguous slice of the columns of the work matrix W (global memory,
// m x ncol), keeps their norms in its shared memory and updates them; the
// pivot choice and the pivot's Householder reflector are exchanged through the
// instance's work area.  Per reflector step: every CTA posts its best column,
// a cluster barrier, every CTA picks the same global best (largest norm,
// lowest column on ties) and the same stop decision; the owner builds the
// reflector into refl[:, j]; a cluster barrier; every CTA applies it to its
// remaining columns.  Columns are not swapped: R comes out in the original
// column order (R P^T), as the single-CTA routine leaves it in Rp.  All loop
// counts are decided from data every CTA reads after the same barrier, so the
// CTAs always meet the same barriers.  Returns the rank, or maxrank + 1 when
// the columns left after maxrank reflectors are still above the floor.
struct ClusterCand {
  float key;   // FP32 image of the squared column norm (-1: no column left)
  int col;
  double val;  // the squared norm
};
struct ClusterCtl {
  int op;      // 0: exit, 1: QR of the work matrix
  int m, ncol;
  int pad;
  double floor_rel2;
  double pad2[3];
  ClusterCand cand[kMaxCluster];
};
static_assert(sizeof(ClusterCtl) <= kClusterCtlBytes, "cluster control block");

template <class T>
struct ClusterView {
  ClusterCtl* c;
  int* piv;       // column pivoted at step j
  T* tau;
  cx<T>* beta;
};
template <class T>
__device__ __forceinline__ ClusterView<T> cluster_view(unsigned char* work, const SmemPlan& P, int rcap) {
  unsigned char* b = work + P.off_ctl;
  ClusterView<T> v;
  v.c = (ClusterCtl*)b;
  b += kClusterCtlBytes;
  v.piv = (int*)b;
  b += align_up(sizeof(int) * (size_t)rcap, 16);
  v.tau = (T*)b;
  b += align_up(sizeof(T) * (size_t)rcap, 16);
  v.beta = (cx<T>*)b;
  return v;
}

// complex load that bypasses L1 (written by another CTA of the cluster)
__device__ __forceinline__ cx<double> ldcg_cx(const cx<double>* p) {
  const double2 v = __ldcg((const double2*)p);
  return mk<double>(v.x, v.y);
}

template <class T>
__device__ __noinline__ int cluster_qr(cx<T>* W, int m, int ncol, cx<T>* Rp, cx<T>* refl, int ldr, const ClusterView<T>& cv,
                          T floor_rel2, int maxrank, T* cn, int* pstep) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
  const int per = (ncol + csize - 1) / csize;
  const int c0 = min(ncol, crank * per), c1 = min(ncol, c0 + per);
  const int nloc = c1 - c0;
  const int pmax = min(m, ncol);
  {
    const Grp g = make_grp(pick_g(m, nloc));
    for (int t0 = 0; t0 < nloc; t0 += g.ng) {
      const int lc = t0 + g.gid;
      T s2 = 0;
      if (lc < nloc)
        for (int i = g.lg; i < m; i += g.G) s2 += abs2(W[i * ncol + c0 + lc]);
      s2 = gsum(s2, g.G);
      if (lc < nloc && g.lg == 0) {
        cn[lc] = s2;
        pstep[lc] = -1;
      }
    }
  }
  __syncthreads();
  T floor2 = 0;
  int rank = pmax;
  for (int j = 0; j < pmax; ++j) {
    if (threadIdx.x == 0) {
      int best = -1;
      float bv = -1.f;
      for (int lc = 0; lc < nloc; ++lc) {
        if (pstep[lc] >= 0) continue;
        const float v = f32_scaled(cn[lc], 0);
        if (v > bv) {
          bv = v;
          best = lc;
        }
      }
      cv.c->cand[crank].key = bv;
      cv.c->cand[crank].col = best < 0 ? -1 : c0 + best;
      cv.c->cand[crank].val = best < 0 ? 0.0 : (double)cn[best];
      __threadfence();
    }
    cl.sync();  // candidates posted
    float bk = -1.f;
    int bc = -1;
    double bval = 0.0;
    for (int r = 0; r < csize; ++r) {
      const float k = __ldcg(&cv.c->cand[r].key);
      const int col = __ldcg(&cv.c->cand[r].col);
      if (col >= 0 && (k > bk || (k == bk && col < bc))) {
        bk = k;
        bc = col;
        bval = __ldcg(&cv.c->cand[r].val);
      }
    }
    if (j == 0) floor2 = (T)bval * floor_rel2;
    if (bc < 0 || (j > 0 && !((T)bval > floor2))) {
      rank = j;
      break;
    }
    if (j == maxrank) {  // a further direction above the floor: capacity exceeded
      rank = maxrank + 1;
      break;
    }
    const bool mine = bc >= c0 && bc < c1;
    if (mine) {
      if (threadIdx.x == 0) {
        // H = I - tau v v^dag with v = x - beta e_j, beta = -e^{i arg x_j} |x|
        const T s = cn[bc - c0];
        const cx<T> x0 = W[j * ncol + bc];
        const T a2 = abs2(x0);
        cx<T> b = mk<T>(0, 0);
        T t = 0;
        if (s > K<T>::tiny2()) {
          const T inv = rsqrt(s);
          const T nrm = s * inv;
          cx<T> ph = mk<T>(1, 0);
          T ax0 = 0;
          if (a2 > K<T>::phase_floor() * s) {
            const T ia = rsqrt(a2);
            ax0 = a2 * ia;
            ph = cscale(x0, ia);
          }
          b = cscale(ph, -nrm);
          t = (T)1 / (nrm * (nrm + ax0));
          W[j * ncol + bc] = csub(x0, b);
        }
        cv.tau[j] = t;
        cv.beta[j] = b;
        cv.piv[j] = bc;
        pstep[bc - c0] = j;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) refl[i * ldr + j] = i < j ? mk<T>(0, 0) : W[i * ncol + bc];
      __threadfence();
    }
    cl.sync();  // reflector j posted
    const T tj = __ldcg(&cv.tau[j]);
    const Grp g = make_grp(pick_g(m - j, nloc));
    for (int t0 = 0; t0 < nloc; t0 += g.ng) {
      const int lc = t0 + g.gid;
      const bool act = lc < nloc && pstep[lc] < 0;
      const int c = c0 + lc;
      cx<T> w = mk<T>(0, 0);
      if (act)
        for (int i = j + g.lg; i < m; i += g.G) w = cmacc(w, ldcg_cx(refl + i * ldr + j), W[i * ncol + c]);
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      T s2 = 0;
      if (act) {
        const cx<T> tw = cscale(w, -tj);
        for (int i = j + g.lg; i < m; i += g.G) {
          cx<T> x = W[i * ncol + c];
          if (tj != (T)0) x = cmac(x, ldcg_cx(refl + i * ldr + j), tw);
          W[i * ncol + c] = x;
          if (i > j) s2 += abs2(x);
        }
      }
      s2 = gsum(s2, g.G);
      if (act && g.lg == 0) cn[lc] = s2;
    }
    __syncthreads();
  }
  // R P^T into Rp (rows < rank, this CTA's columns): a column pivoted at step
  // i' holds R above row i', beta at row i' and its reflector below
  const int rows = min(rank, maxrank);
  for (int e = threadIdx.x; e < rows * nloc; e += blockDim.x) {
    const int i = e / nloc, lc = e % nloc, c = c0 + lc;
    const int ps = pstep[lc];
    cx<T> v;
    if (ps < 0 || i < ps)
      v = W[i * ncol + c];
    else if (i == ps)
      v = ldcg_cx(&cv.beta[i]);
    else
      v = mk<T>(0, 0);
    Rp[i * ncol + c] = v;
  }
  __threadfence();
  cl.sync();  // R and the reflectors complete
  return rank;
}

// A cluster CTA other than the first: waits for the first CTA's commands and
// takes its share of each large QR until told to stop.
template <class T>
__device__ __noinline__ void cluster_worker(const InstDesc& d, unsigned char* smem) {
  cg::cluster_group cl = cg::this_cluster();
  const SmemPlan P = make_plan(d.n, d.M, d.xcap, d.chicap, d.rcap, sizeof(T), 0, true);
  unsigned char* work = (unsigned char*)d.work;
  const ClusterView<T> cv = cluster_view<T>(work, P, d.rcap);
  T* cn = (T*)smem;
  int* pstep = (int*)(smem + align_up(sizeof(T) * (size_t)d.xcap, 16));
  for (;;) {
    cl.sync();  // a command is posted
    if (__ldcg(&cv.c->op) == 0) break;
    const int m = __ldcg(&cv.c->m), ncol = __ldcg(&cv.c->ncol);
    const T fl2 = (T)__ldcg(&cv.c->floor_rel2);
    cluster_qr<T>((cx<T>*)(work + P.off_w), m, ncol, (cx<T>*)(work + P.off_rprev), (cx<T>*)(work + P.off_refl),
                  d.rcap, cv, fl2, d.rcap, cn, pstep);
  }
}

// qr_form_q for reflectors that other CTAs of the cluster wrote (A in global
// memory): every read of A bypasses L1.
__device__ inline void qr_form_q_cluster(cx<double>* A, int m, int p, int lda, const double* tau) {
  for (int j = p - 1; j >= 0; --j) {
    const double tj = tau[j];
    const int ntask = p - j - 1;
    const Grp g = make_grp(pick_g(m - j, ntask));
    for (int t0 = 0; t0 < ntask; t0 += g.ng) {
      const int c = j + 1 + t0 + g.gid;
      const bool act = (t0 + g.gid) < ntask;
      cx<double> w = mk<double>(0, 0);
      if (act)
        for (int i = j + g.lg; i < m; i += g.G) w = cmacc(w, ldcg_cx(A + i * lda + j), ldcg_cx(A + i * lda + c));
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      if (act && tj != 0.0) {
        const cx<double> tw = cscale(w, -tj);
        for (int i = j + g.lg; i < m; i += g.G)
          A[i * lda + c] = cmac(ldcg_cx(A + i * lda + c), ldcg_cx(A + i * lda + j), tw);
      }
    }
    __syncthreads();
    const cx<double> vj = ldcg_cx(A + j * lda + j);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      cx<double> q;
      if (i < j) {
        q = mk<double>(0, 0);
      } else if (i == j) {
        q = mk<double>(1.0 - tj * abs2(vj), 0);
      } else {
        const cx<double> vi = ldcg_cx(A + i * lda + j);
        q = mk<double>(-tj * fma(vi.re, vj.re, vi.im * vj.im), -tj * fma(vi.im, vj.re, -vi.re * vj.im));
      }
      A[i * lda + j] = q;
    }
    __threadfence_block();
    __syncthreads();
  }
}

// Overwrite the reflectors in A (m x p block, leading dim lda) with the thin
// Q = H_0 H_1 ... H_{p-1} [I_p; 0], right to left (reflector storage reused).
template <class T>
__device__ void qr_form_q(cx<T>* A, int m, int p, int lda, const T* tau) {
  for (int j = p - 1; j >= 0; --j) {
    const T tj = tau[j];
    const int ntask = p - j - 1;
    const Grp g = make_grp(pick_g(m - j, ntask));
    for (int t0 = 0; t0 < ntask; t0 += g.ng) {
      const int c = j + 1 + t0 + g.gid;
      const bool act = (t0 + g.gid) < ntask;
      cx<T> w = mk<T>(0, 0);
      if (act)
        for (int i = j + g.lg; i < m; i += g.G) w = cmacc(w, A[i * lda + j], A[i * lda + c]);
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      if (act && tj != (T)0) {
        const cx<T> tw = cscale(w, -tj);
        for (int i = j + g.lg; i < m; i += g.G) A[i * lda + c] = cmac(A[i * lda + c], A[i * lda + j], tw);
      }
    }
    __syncthreads();
    // column j of Q: H_j e_j = e_j - tau v conj(v_j)
    const cx<T> vj = A[j * lda + j];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      cx<T> q;
      if (i < j) {
        q = mk<T>(0, 0);
      } else if (i == j) {
        q = mk<T>((T)1 - tj * abs2(vj), 0);
      } else {
        const cx<T> vi = A[i * lda + j];
        // -tau * v_i * conj(v_j)
        q = mk<T>(-tj * fma(vi.re, vj.re, vi.im * vj.im), -tj * fma(vi.im, vj.re, -vi.re * vj.im));
      }
      A[i * lda + j] = q;
    }
    __syncthreads();
  }
}

// a > b (and a == b) for non-negative values; doubles compare through their
// bit patterns (an integer compare, off the FP64 pipe)
template <class T>
__device__ __forceinline__ bool nn_gt(T a, T b) {
  return a > b;
}
template <>
__device__ __forceinline__ bool nn_gt<double>(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
template <class T>
__device__ __forceinline__ bool nn_eq(T a, T b) {
  return a == b;
}
template <>
__device__ __forceinline__ bool nn_eq<double>(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

// Plane rotation for one Jacobi pair from its Gram entries a = |x_p|^2,
// b = |x_q|^2 and g = <x_p, x_q>: the classical angle (Rutishauser: zeta =
// (b - a)/(2|g|), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2))) computed in FP32
// from exact power-of-two-scaled images of the T-precision entries, then
// normalised in T.  Returns false when the pair is left alone (a row below the
// noise floor skip2, the pair orthogonal to tolf, or a degenerate angle); else
// cc = cos and (sre, sim) = sin * g/|g|, with cc^2 + |s|^2 = 1 to T's rounding
// (normalised through rho = c^2 + |s|^2, or for small angles through c).
// The angle is kept to IEEE FP32 accuracy (not MUFU estimates): a sloppier
// angle costs extra rotations, whose rounding lifts the noise rows of
// rank-deficient matrices toward the rank rule's threshold.  `small` (when
// given) is set when the pair rotates with |g| <= 2^-32 sqrt(a b).
template <class T>
__device__ __forceinline__ bool jacobi_rotation(T a, T b, cx<T> gg, float tolf, T skip2, T& cc, T& sre, T& sim,
                                                bool* small = nullptr) {
  if (!(nn_gt(a, skip2) && nn_gt(b, skip2))) return false;
  const int sh = expo_of(nn_gt(a, b) ? a : b);
  const float af = f32_scaled(a, sh), bf = f32_scaled(b, sh);
  const float dab = f32_scaled(b - a, sh);  // difference taken in T
  const float gr = f32_scaled(gg.re, sh), gi = f32_scaled(gg.im, sh);
  const float gabs = sqrtf(fmaf(gr, gr, gi * gi));
  const float sab = sqrtf(af) * sqrtf(bf);
  if (!(gabs > tolf * sab && gabs > 0.f)) return false;
  if (small != nullptr) *small = gabs <= 2.3283064e-10f * sab;
  const float zeta = dab / (2.f * gabs);
  // small-root formula; for |zeta| > 2^60 (zeta^2 would overflow) t = 1/(2 zeta)
  const float tt = fabsf(zeta) > 1.1529215e18f ? 0.5f / zeta
                                               : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
  if (!(tt != 0.f && isfinite(tt))) return false;
  const float cf = rsqrtf(fmaf(tt, tt, 1.f));
  const float sf = cf * tt;
  sre = widen<T>(sf * (gr / gabs));
  sim = widen<T>(sf * (gi / gabs));
  if (fabsf(tt) < 3.0517578e-05f) {
    // small angle (|t| < 2^-15): keep s as rounded and take c = 1 - |s|^2/2,
    // so c^2 + |s|^2 = 1 + |s|^4/4 = 1 to T's rounding (|s|^4 < 2^-60)
    cc = fma(fma(sre, sre, sim * sim), (T)-0.5f, (T)1);
    return true;
  }
  cc = widen<T>(cf);
  const T rho = fma(cc, cc, fma(sre, sre, sim * sim));
  const T dd = rho - (T)1;
  const T f = fma(dd, fma(dd, (T)0.375f, (T)-0.5f), (T)1);
  cc *= f;
  sre *= f;
  sim *= f;
  return true;
}

// ---------------------------------------------------- one-sided Jacobi SVD
// Orthogonalise the rows of Mat (r x c, leading dim ldm) by unitary plane
// rotations J = [[c, -conj(s)], [s, c]] applied from the left (Hestenes'
// one-sided Jacobi on the rows).  Pairs follow the round-robin (circle)
// ordering so that the r/2 disjoint pairs of a round run in parallel, one
// lane group per pair.  The rotation angle is the classical one (Rutishauser:
// zeta = (b - a)/(2|g|), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2))) computed
// in FP32 from the pair's T-precision Gram entries after an exact
// power-of-two scaling, then normalised in T so that c^2 + |s|^2 = 1 to T's
// rounding.  A pair is rotated while |g| > tol sqrt(a b); pairs in which a
// row's squared norm is below `skip2` (noise far under the rank rule's
// threshold, which the truncation drops) are left alone.  U starts as the
// identity, or (u_given) as the rotation the caller already applied to Mat.
// The sweeps stop after one that rotated no pair.  (Stopping once every
// rotation of a sweep is small is not safe: within a cluster of nearly equal
// singular values a pair with a tiny off-diagonal can still turn by a large
// angle and move the other pairs' off-diagonals around at first order.)
// Returns sweeps used, or -1 if max_sweeps was exhausted.
template <class T>
__device__ int jacobi_rows(cx<T>* Mat, int r, int c, int ldm, cx<T>* U, int ldu, int max_sweeps, float tolf,
                           T skip2, bool u_given = false) {
  if (!u_given)
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
      const int a = i / r, b = i % r;
      U[a * ldu + b] = mk<T>(a == b ? (T)1 : (T)0, 0);
    }
  __syncthreads();
  if (r < 2) return 0;
  const int rp = r + (r & 1);
  const int npairs = rp / 2;
  // A pair is handled by a team of 4 quarters of Q lanes (Q a power of two,
  // 4Q <= 32).  For the Gram entries quarter 0 sums |x_p|^2, 1 |x_q|^2, 2 Re
  // and 3 Im of conj(x_p) x_q, so every lane issues few T instructions; the
  // rotation then spreads the columns of both matrices over the whole team.
  // Q: at most 8, and small enough that every real pair of a round has its
  // own team (one pass per round) while Q >= 2
  int Q = min(8, pow2_cap32(max(c, r)));
  while (Q > 2 && (int)(blockDim.x >> 5) * (32 / (4 * Q)) < r / 2) Q >>= 1;
  const int TM = 4 * Q;                 // lanes per team
  const int lane = threadIdx.x & 31;
  const int team_in_warp = lane / TM, tl = lane % TM, quarter = tl / Q, ql = tl % Q;
  const int teams = (blockDim.x >> 5) * (32 / TM);
  const int team = (threadIdx.x >> 5) * (32 / TM) + team_in_warp;
  const int base = (lane / TM) * TM;    // first lane of this team in the warp
  // with r odd, pair 0 of every round holds the padding row: teams take the
  // real pairs 1 .. npairs-1 only
  const int k0 = r & 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int t = 0; t < rp - 1; ++t) {
      for (int t0 = k0; t0 < npairs; t0 += teams) {
        const int k = t0 + team;
        int p = -1, q = -1;
        if (k < npairs) {
          if (k == 0) {
            p = rp - 1;
            q = t;
          } else {
            p = (t + k) % (rp - 1);
            q = (t - k + rp - 1) % (rp - 1);
          }
          if (p >= r || q >= r) p = q = -1;
        }
        const bool act = p >= 0;
        T part = 0;
        if (act) {
          // one instruction stream for all quarters: part += Re(conj(u) v) with
          // (u, v) = (x_p, x_p), (x_q, x_q), (x_p, x_q), (x_p, -i x_q)
          for (int j = ql; j < c; j += Q) {
            const cx<T> xp = Mat[p * ldm + j], xq = Mat[q * ldm + j];
            const cx<T> u = quarter == 1 ? xq : xp;
            const cx<T> v = quarter == 0 ? xp : (quarter == 3 ? mk<T>(xq.im, -xq.re) : xq);
            part = fma(u.re, v.re, fma(u.im, v.im, part));
          }
        }
        part = gsum(part, Q);  // within the quarter (xor offsets < Q)
        const T a = shidx(part, base), b = shidx(part, base + Q);
        cx<T> gg;
        gg.re = shidx(part, base + 2 * Q);
        gg.im = shidx(part, base + 3 * Q);
        // skip pairs with a row below the noise floor (dropped by the rank rule)
        T cc, sre, sim;
        if (act && jacobi_rotation<T>(a, b, gg, tolf, skip2, cc, sre, sim)) {
          // row p: c x_p - conj(s) x_q ; row q: c x_q + s x_p, for the c
          // columns of Mat and the r columns of U as one list of column
          // tasks: lane tl of the team owns tasks tl, tl + TM, ... and updates
          // both rows at its column (no lane reads what another writes)
          const cx<T> cq = mk<T>(sre, sim), cp = mk<T>(-sre, sim);
          for (int e = tl; e < c + r; e += TM) {
            const bool inm = e < c;
            cx<T>* rows = inm ? Mat : U;
            const int ld = inm ? ldm : ldu, j = inm ? e : e - c;
            const cx<T> xp = rows[p * ld + j], xq = rows[q * ld + j];
            rows[p * ld + j] = cmac(cscale(xp, cc), cp, xq);
            rows[q * ld + j] = cmac(cscale(xq, cc), cq, xp);
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) return sweep + 1;
  }
  return -1;
}

// LQ factorisation with row pivoting, in place, of A (r x c, r <= c, leading
// dim ld): P A H_0 H_1 ... H_{r-1} = [L 0] with L lower triangular and
// H_k = I - tau_k v_k v_k^dag acting on columns k..c-1 from the right (the
// Householder reflector of the conjugated row, so that row k becomes
// beta_k e_k).  Row k keeps u_k = conj(v_k) from column k on, beta (L's
// diagonal) and tau are returned, L's strict lower part stays in place.
// Pivot: the remaining row of largest norm over the trailing columns
// (exact FP32 images, lowest row on ties); rperm[k] = the original row now at
// position k.  rn: scratch for r norms; ctl: 1 int.
template <class T>
__device__ void lq_rows_pivoted(cx<T>* A, int r, int c, int ld, T* tau, cx<T>* beta, int* rperm, T* rn,
                                int* ctl) {
  {
    const Grp g = make_grp(pick_g(c, r));
    for (int t0 = 0; t0 < r; t0 += g.ng) {
      const int i = t0 + g.gid;
      T s2 = 0;
      if (i < r)
        for (int j = g.lg; j < c; j += g.G) s2 += abs2(A[i * ld + j]);
      s2 = gsum(s2, g.G);
      if (i < r && g.lg == 0) {
        rn[i] = s2;
        rperm[i] = i;
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      float bv = f32_scaled(rn[k], 0);
      for (int i = k + 1; i < r; ++i) {
        const float v = f32_scaled(rn[i], 0);
        if (v > bv) {
          bv = v;
          best = i;
        }
      }
      ctl[0] = best;
      if (best != k) {
        const T tn = rn[k];
        rn[k] = rn[best];
        rn[best] = tn;
        const int tp = rperm[k];
        rperm[k] = rperm[best];
        rperm[best] = tp;
      }
    }
    __syncthreads();
    const int best = ctl[0];
    if (best != k)
      for (int j = threadIdx.x; j < c; j += blockDim.x) {
        const cx<T> t = A[k * ld + j];
        A[k * ld + j] = A[best * ld + j];
        A[best * ld + j] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      // y = conj(row k) from column k: H y = b e_0 with b = -e^{i arg y_0} |y|;
      // the row becomes conj(b) e_0 and u = conj(y - b e_0) is the row with
      // its first entry less conj(b)
      const T s2 = rn[k];
      const cx<T> x0 = A[k * ld + k];
      const T a2 = abs2(x0);
      cx<T> b = mk<T>(0, 0);
      T t = 0;
      if (s2 > K<T>::tiny2()) {
        const T inv = rsqrt(s2);
        const T nrm = s2 * inv;
        cx<T> ph = mk<T>(1, 0);
        T ax0 = 0;
        if (a2 > K<T>::phase_floor() * s2) {
          const T ia = rsqrt(a2);
          ax0 = a2 * ia;
          ph = mk<T>(x0.re * ia, -x0.im * ia);  // e^{i arg y_0}, y_0 = conj(x0)
        }
        b = cscale(ph, -nrm);
        t = (T)1 / (nrm * (nrm + ax0));
        A[k * ld + k] = csub(x0, mk<T>(b.re, -b.im));
      }
      beta[k] = mk<T>(b.re, -b.im);
      tau[k] = t;
    }
    __syncthreads();
    const T tk = tau[k];
    const int ntask = r - k - 1;
    const Grp g = make_grp(pick_g(c - k, ntask));
    for (int t0 = 0; t0 < ntask; t0 += g.ng) {
      const int i = k + 1 + t0 + g.gid;
      const bool act = (t0 + g.gid) < ntask;
      cx<T> w = mk<T>(0, 0);
      if (act)
        for (int j = k + g.lg; j < c; j += g.G) w = cmacc(w, A[k * ld + j], A[i * ld + j]);
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      T s2 = 0;
      if (act) {
        const cx<T> tw = cscale(w, -tk);
        for (int j = k + g.lg; j < c; j += g.G) {
          cx<T> x = A[i * ld + j];
          if (tk != (T)0) x = cmac(x, tw, A[k * ld + j]);
          A[i * ld + j] = x;
          if (j > k) s2 += abs2(x);
        }
      }
      s2 = gsum(s2, g.G);
      if (act && g.lg == 0) rn[i] = s2;
    }
    __syncthreads();
  }
}

// Q (r x c) of lq_rows_pivoted in place over its reflector rows: row k of Q
// is e_k^T H_k H_{k-1} ... H_0, formed from the last row up (row k's
// reflector is consumed when rows k+1.. have taken H_k); columns left of k
// of row k are zero.  L must have been copied out first.
template <class T>
__device__ void lq_form_q(cx<T>* A, int r, int c, int ld, const T* tau) {
  for (int k = r - 1; k >= 0; --k) {
    const T tk = tau[k];
    const int ntask = r - k - 1;
    const Grp g = make_grp(pick_g(c - k, ntask));
    for (int t0 = 0; t0 < ntask; t0 += g.ng) {
      const int i = k + 1 + t0 + g.gid;
      const bool act = (t0 + g.gid) < ntask;
      cx<T> w = mk<T>(0, 0);
      if (act)
        for (int j = k + g.lg; j < c; j += g.G) w = cmacc(w, A[k * ld + j], A[i * ld + j]);
      w.re = gsum(w.re, g.G);
      w.im = gsum(w.im, g.G);
      if (act && tk != (T)0) {
        const cx<T> tw = cscale(w, -tk);
        for (int j = k + g.lg; j < c; j += g.G) A[i * ld + j] = cmac(A[i * ld + j], tw, A[k * ld + j]);
      }
    }
    __syncthreads();
    // row k: e_k^T - tau conj(u_0) u on columns >= k
    const cx<T> u0 = A[k * ld + k];
    const cx<T> f = cscale(mk<T>(u0.re, -u0.im), -tk);
    __syncthreads();
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
      cx<T> q = mk<T>(0, 0);
      if (j >= k) {
        q = cmul(f, A[k * ld + j]);
        if (j == k) q.re += (T)1;
      }
      A[k * ld + j] = q;
    }
    __syncthreads();
  }
}

// Mat (r x c, leading dim c) <- U (r x r, leading dim r) Mat in place: the
// block holds a chunk of columns' results in registers (at most 4 per
// thread; each output column depends on its own input column only) before
// writing them back.  Needs r <= 4 blockDim.x.
template <class T>
__device__ void rotate_rows(cx<T>* Mat, int r, int c, const cx<T>* U) {
  const int cw = max(1, (4 * (int)blockDim.x) / r);
  for (int j0 = 0; j0 < c; j0 += cw) {
    const int w = min(cw, c - j0), tot = r * w;
    cx<T> o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + u * (int)blockDim.x;
      o[u] = mk<T>(0, 0);
      if (e < tot) {
        const int i = e / w, j = j0 + e % w;
        for (int a = 0; a < r; ++a) o[u] = cmac(o[u], U[i * r + a], Mat[a * c + j]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + u * (int)blockDim.x;
      if (e < tot) Mat[(e / w) * c + j0 + e % w] = o[u];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ contraction
// MPO factor w_b(s, s') of site l (0 <= b < D) for the oracle (O) and the
// diffusion (D) operators, boundaries folded in by the caller.
// oracle:    w_0 = I, w_b = P_{bit(w_b, l)} = |x><x| (b >= 1)
// diffusion: w_0 = I, w_1 = |+><+| = 1/2 (all entries)
template <class CR>
__device__ __forceinline__ CR mpo_w(int op, int b, int l, int s, int sp, const unsigned long long* marked) {
  if (b == 0) return s == sp ? (CR)1 : (CR)0;
  if (op == 0) {
    const int x = (int)((marked[b - 1] >> l) & 1ull);
    return (s == sp && s == x) ? (CR)1 : (CR)0;
  }
  return (CR)0.5f;
}

// C = Rp * B_l, written as the (2 r) x X_right matrix W (row (i, s) = 2 i + s).
// B_l is the operator-expanded site l: an MPO contraction (op 0 oracle, 1
// diffusion; boundary vector `lbnd` of length D at site 0, all-ones at the
// right end) or a direct sum of the current MPS (coefficient cpsi at site 0)
// with `nt` product states (coefficients tcoef at site 0).  expand_elem gives
// one element C[(i, s), j]; expand_absorb writes all of W with the block.
template <class T, class S, class CR>
__device__ __forceinline__ cx<T> expand_elem(Blk<T, S>& B, int l, int i, int s, int j, int xl, int mode, int op,
                                             int D, const cx<T>* lbnd, cx<T> cpsi, int nt) {
  // The chain's own tensors are contracted in CR (the bulk contraction); the
  // operator's coefficients (MPO boundary, direct-sum product states and
  // their weights, 1/sqrt 2 of |+>) enter in T: they set every iteration's
  // rotation, and a CR rounding of them would repeat the same error each
  // iteration (a drift linear in k for the complex64 form).
  const int n = B.n;
  const int cl = B.chi[l], cr = B.chi[l + 1];
  const S* A = B.slot(l);
  const T h = K<T>::isq2();
  cx<CR> acc = mk<CR>(0, 0);  // chain part
  cx<T> acc_t = mk<T>(0, 0);  // coefficient part
  if (mode == 0) {  // ---- MPO
    if (n == 1) {
      for (int b = 0; b < D; ++b) {
        cx<CR> tb = mk<CR>(0, 0);
        for (int sp = 0; sp < 2; ++sp) {
          const CR w = mpo_w<CR>(op, b, l, s, sp, B.d->marked);
          if (w != (CR)0) tb = cmac(tb, mk<CR>(w, 0), ld<CR>(A + sp));
        }
        acc_t = cmac(acc_t, lbnd[b], cvt<T>(tb));
      }
    } else if (l == 0) {
      const int b = j / cr, jj = j % cr;
      cx<CR> tb = mk<CR>(0, 0);
      for (int sp = 0; sp < 2; ++sp) {
        const CR w = mpo_w<CR>(op, b, l, s, sp, B.d->marked);
        if (w != (CR)0) tb = cmac(tb, mk<CR>(w, 0), ld<CR>(A + sp * cr + jj));
      }
      acc_t = cmul(lbnd[b], cvt<T>(tb));
    } else {
      const bool last = (l == n - 1);
      const int b0 = last ? 0 : j / cr, b1 = last ? D : b0 + 1;
      const int jj = last ? 0 : j % cr;
      for (int b = b0; b < b1; ++b) {
        for (int sp = 0; sp < 2; ++sp) {
          const CR w = mpo_w<CR>(op, b, l, s, sp, B.d->marked);
          if (w == (CR)0) continue;
          cx<CR> t = mk<CR>(0, 0);
          for (int a = 0; a < cl; ++a)
            t = cmac(t, cvt<CR>(B.Rp[i * xl + b * cl + a]), ld<CR>(A + (a * 2 + sp) * cr + jj));
          acc = cmac(acc, mk<CR>(w, 0), t);
        }
      }
    }
  } else {  // ---- direct sum
    auto pval = [&](int t) -> T {
      if (B.tplus[t]) return h;
      return ((int)((B.tbits[t] >> l) & 1ull) == s) ? (T)1 : (T)0;
    };
    if (n == 1) {
      acc_t = cmul(cpsi, ld<T>(A + s));
      for (int t = 0; t < nt; ++t) acc_t = cmac(acc_t, B.tcoef[t], mk<T>(pval(t), 0));
      return acc_t;
    } else if (l == 0) {
      if (j < cr) return cmul(cpsi, ld<T>(A + s * cr + j));
      return cscale(B.tcoef[j - cr], pval(j - cr));
    } else if (l == n - 1) {
      for (int a = 0; a < cl; ++a) acc = cmac(acc, cvt<CR>(B.Rp[i * xl + a]), ld<CR>(A + a * 2 + s));
      acc_t = cvt<T>(acc);
      for (int t = 0; t < nt; ++t) acc_t = cmac(acc_t, B.Rp[i * xl + cl + t], mk<T>(pval(t), 0));
      return acc_t;
    } else {
      if (j < cr) {
        for (int a = 0; a < cl; ++a)
          acc = cmac(acc, cvt<CR>(B.Rp[i * xl + a]), ld<CR>(A + (a * 2 + s) * cr + j));
        return cvt<T>(acc);
      }
      return cscale(B.Rp[i * xl + cl + (j - cr)], pval(j - cr));
    }
  }
  // MPO: the chain part, or at site 0 (and for n = 1) the boundary-weighted part
  return (n == 1 || l == 0) ? acc_t : cvt<T>(acc);
}
template <class T, class S, class CR>
__device__ void expand_absorb(Blk<T, S>& B, int l, int r, int xl, int xr, int mode, int op, int D,
                              const cx<T>* lbnd, cx<T> cpsi, int nt) {
  const int total = r * 2 * xr;
  for (int e = threadIdx.x; e < total; e += blockDim.x)
    B.W[e] = expand_elem<T, S, CR>(B, l, e / (2 * xr), (e / xr) & 1, e % xr, xl, mode, op, D, lbnd, cpsi, nt);
  __syncthreads();
}

// ------------------------------------------------------------- sweeps
template <class T>
__device__ __forceinline__ void set_status(int* misc, int code) {
  if (misc[0] == 0) misc[0] = code;
}

// Relative floor of the rank rule for an m x n matrix: singular values (and
// rank-revealing QR pivots) at or below floor * sigma_0 are dropped.  Either
// max(m, n) eps (the forms whose linear algebra runs in the storage type's
// precision) or a fixed eps (the complex64 form, whose FP64 QR and SVD see
// FP32-stored tensors: its rounding noise stays far below a fixed floor while
// max(m, n) 2^-23 would reach the marked component's Schmidt values).
template <class T, class S>
__device__ __forceinline__ T rank_floor(const Blk<T, S>& B, int m, int n) {
  return B.misc[5] ? (T)max(m, n) * B.tmisc[0] : B.tmisc[0];
}

#include "gmps_tiny.cuh"

// Right environments of the product-state targets, folded site by site from
// the right while the SVD sweep finalises the sites (warp 1): E <- A_s[:, b_s, :] E
// (or (A_s[:,0,:] + A_s[:,1,:]) E / sqrt 2 for |+>^n).  A group of G lanes per
// target (G a power of two covering every bond), lane lg holding E[lg]; after
// site 0 lane 0 of each group holds <target|psi>.  Same quantity as
// chain_targets, accumulated from the other end.  Both are called with
// CR = T, the precision of the QR/SVD: these overlaps set the coefficients
// of the next Grover step (its rotation in the {|w>, |r>} plane), so the
// complex64 form reads its FP32 tensors but accumulates in FP64 (an FP32
// chain product of n sites carries ~n 2^-24 relative error into every
// iteration's rotation).
template <class T, class S, class CR>
__device__ __forceinline__ void env_fold(Blk<T, S>& B, int s, int nt, int G, cx<CR>& E) {
  const int lane = threadIdx.x & 31, lg = lane & (G - 1), base = lane & ~(G - 1);
  const int t = lane / G;
  const bool on = t < nt;
  const bool plus = on && B.tplus[t];
  const unsigned long long bits = (on && !plus) ? B.tbits[t] : 0ull;
  const int cl = B.chi[s], cr = B.chi[s + 1];
  const int b = (int)((bits >> s) & 1ull);
  const S* A = B.slot(s);
  cx<CR> nv = mk<CR>(0, 0);
  for (int j = 0; j < cr; ++j) {
    cx<CR> ej;
    ej.re = shidx(E.re, base + j);
    ej.im = shidx(E.im, base + j);
    if (lg < cl) {
      cx<CR> a = ld<CR>(A + (lg * 2 + b) * cr + j);
      if (plus) a = cadd(a, ld<CR>(A + (lg * 2 + 1) * cr + j));
      nv = cmac(nv, a, ej);
    }
  }
  E = plus ? cscale(nv, K<CR>::isq2()) : nv;
}

// Jacobi rotation cache of one instance (InstDesc::jcache): per bank (sweep
// pair of the iteration) and site, the rotations that site's SVD ended with
// (rcap^2 complex entries of 16 bytes); then per bank and site two pivot
// sequences of rcap ints: [0] the one of the QR step that made the site's left
// bond when the rotations were saved, [1] the one of the current QR sweep.
// The rows of the site's SVD matrix are that QR's reflectors in pivot order,
// so the cached rotations only fit while the pivot sequence is unchanged.
template <class T>
__device__ __forceinline__ cx<T>* jc_rot(const InstDesc& d, int bank, int l) {
  return (cx<T>*)((unsigned char*)d.jcache + ((size_t)bank * d.n + l) * d.rcap * d.rcap * 16);
}
__device__ __forceinline__ int* jc_piv(const InstDesc& d, int which, int bank, int l) {
  int* base = (int*)((unsigned char*)d.jcache + (size_t)d.jbanks * d.n * d.rcap * d.rcap * 16);
  return base + (((size_t)which * d.jbanks + bank) * d.n + l) * d.rcap;
}

// The cluster branch of a QR-sweep step (CTA 0): posts the command, factors
// W (m x xr, work area) with the other CTAs of the cluster, checks the rank
// against the capacity and stores the thin Q of the exchanged reflectors into
// the site.  Out of line so that its registers do not weigh on the sweep's
// hot path.  Returns the rank p >= 1, or 0 after recording a capacity status.
template <class T, class S>
__device__ __noinline__ int cluster_qr_step(const InstDesc& d, int n, int m, int xr, T fl, cx<T>* W, cx<T>* Rp,
                                            T* tau, int* misc, T* qcn, int* qperm, S* dst, unsigned long long key,
                                            int* piv_out) {
  const SmemPlan Pw = make_plan(n, d.M, d.xcap, d.chicap, d.rcap, sizeof(T), 0, true);
  unsigned char* work = (unsigned char*)d.work;
  const ClusterView<T> cv = cluster_view<T>(work, Pw, d.rcap);
  if (threadIdx.x == 0) {
    cv.c->op = 1;
    cv.c->m = m;
    cv.c->ncol = xr;
    cv.c->floor_rel2 = (double)(fl * fl);
    __threadfence();
  }
  __syncthreads();
  cg::this_cluster().sync();  // command posted
  cx<T>* refl = (cx<T>*)(work + Pw.off_refl);
  int p = cluster_qr<T>(W, m, xr, Rp, refl, d.rcap, cv, fl * fl, d.rcap, qcn, qperm);
  if (p < 1) p = 1;
  if (p > d.rcap) {  // the rank exceeds what R, W and the slots were sized for
    if (threadIdx.x == 0) set_status<T>(misc, kDevCapacity);
    __syncthreads();
    return 0;
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    tau[j] = __ldcg(&cv.tau[j]);
    if (piv_out != nullptr) piv_out[j] = __ldcg(&cv.piv[j]);
  }
  __syncthreads();
  qr_form_q_cluster(refl, m, p, d.rcap, tau);
  for (int e = threadIdx.x; e < m * p; e += blockDim.x)
    st_site(dst + e, ldcg_cx(refl + (e / p) * d.rcap + (e % p)), key, e);
  __syncthreads();
  return p;
}

// One contraction followed by the QR sweep and the truncated SVD sweep.  With
// env_nt > 0 (two or more warps, every bond within 16 lanes, env_nt targets
// in one warp) warp 1 also computes <target|psi> of the result for the
// env_nt targets in B.tbits/B.tplus, into B.amps, hidden under the SVD sweep.
// `bank` (0 or 1) names this sweep pair's place in the iteration for the
// per-site cache of Jacobi rotations (d.jcache).
template <class T, class S, class CR, bool kCl = false>
__device__ void sweep_pair(Blk<T, S>& B, int mode, int op, int D, const cx<T>* lbnd, cx<T> cpsi,
                           int nt, int env_nt = 0, int bank = 0) {
  const InstDesc& d = *B.d;
  B.rng = fmix64(B.rng + 0x632be59bd9b4e019ull);  // a fresh rounding key per sweep pair
  const int n = B.n;
  // expanded bond at cut l (0 < l < n)
  auto xb = [&](int l) -> int {
    if (l == 0 || l == n) return 1;
    return mode == 0 ? D * B.chi[l] : B.chi[l] + nt;
  };
  // ------------------------------------------------ QR sweep, left to right
  if (threadIdx.x == 0) {
    B.Rp[0] = mk<T>(1, 0);
    B.qb[0] = 1;
  }
  __syncthreads();
  int r = 1;
  // site whose Q warp 1 still has to form from the hand-off buffer (-1: none)
  int pend = -1;
  const bool offload = blockDim.x >= 64;
  auto flush_q = [&](int site) {
    if (threadIdx.x >= 32 && threadIdx.x < 64) {
      const int* meta = tbuf_meta<T>(B.tbuf, site & 1);
      tiny_q_store<T, S>(tbuf_regs<T>(B.tbuf, site & 1)[threadIdx.x & 31], meta[1], meta[0], B.slot(site),
                         B.key(site, 0));
    }
  };
  for (int l = 0; l < n; ++l) {
    const int xl = xb(l), xr = xb(l + 1);
    if (xr > d.xcap || xl > d.xcap) {
      if (threadIdx.x == 0) set_status<T>(B.misc, kDevCapacity);
      __syncthreads();
      return;
    }
    const int m = 2 * r;
    S* dst = B.slot(l);
    if (l < n - 1 && m <= 8 && xr <= 4) {  // register-resident step (one warp)
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x, c = lane >> 3, i = lane & 7;
        const cx<T> w0 = (c < xr && i < m)
                             ? expand_elem<T, S, CR>(B, l, i >> 1, i & 1, c, xl, mode, op, D, lbnd, cpsi, nt)
                             : mk<T>(0, 0);
        const T fl = rank_floor(B, m, xr);
        cx<T> a;
        const int pt = tiny_qr_factor<T>(w0, m, xr, fl * fl, B.Rp, a);
        if (offload) {  // warp 1 forms Q during the next step
          tbuf_regs<T>(B.tbuf, l & 1)[lane] = a;
          if (lane == 0) {
            tbuf_meta<T>(B.tbuf, l & 1)[0] = pt;
            tbuf_meta<T>(B.tbuf, l & 1)[1] = m;
          }
        } else {
          tiny_q_store<T, S>(a, m, pt, dst, B.key(l, 0));
        }
        if (threadIdx.x == 0) {
          B.qb[l + 1] = pt;
          if (d.jcache != nullptr) jc_piv(d, 1, bank, l + 1)[0] = -1;  // no pivot record: no warm start
        }
      } else if (pend >= 0) {
        flush_q(pend);
      }
      __syncthreads();
      pend = offload ? l : -1;
      r = B.qb[l + 1];
      continue;
    }
    if (pend >= 0) {  // the next step needs every thread: finish the pending Q first
      flush_q(pend);
      __syncthreads();
      pend = -1;
    }
    expand_absorb<T, S, CR>(B, l, r, xl, xr, mode, op, D, lbnd, cpsi, nt);
    if (l == n - 1) {
      for (int e = threadIdx.x; e < m; e += blockDim.x) st_site(dst + e, B.W[e], B.key(l, 0), e);
      if (threadIdx.x == 0) B.qb[n] = 1;
      __syncthreads();
      break;
    }
    int p;
    if constexpr (kCl && std::is_same<T, double>::value) {
      if (B.csize > 1 && xr >= kClusterMinCols && d.work != nullptr) {
        // the whole cluster factors W (out of line: its registers stay off this path)
        p = cluster_qr_step<T, S>(d, n, m, xr, rank_floor(B, m, xr), B.W, B.Rp, B.tau, B.misc, B.qcn, B.qperm, dst,
                                  B.key(l, 0), d.jcache != nullptr ? jc_piv(d, 1, bank, l + 1) : nullptr);
        if (p == 0) return;  // capacity status recorded
        if (threadIdx.x == 0) B.qb[l + 1] = p;
        __syncthreads();
        r = p;
        continue;
      }
    }
    {
      const T fl = rank_floor(B, m, xr);
      // the pivot sequence saved with site l+1's rotations, unless that came
      // from a register-resident QR step (no record)
      const int* pref = d.jcache != nullptr ? jc_piv(d, 0, bank, l + 1) : nullptr;
      const int npref = (pref != nullptr && d.stats->jrank[bank][l + 1] > 0 && pref[0] >= 0)
                            ? d.stats->jrank[bank][l + 1] : 0;
      p = qr_rank_revealing<T>(B.W, m, xr, xr, B.tau, B.beta, B.qperm, B.qcn, B.misc + 8, fl * fl, pref, npref);
    }
    if (p < 1) p = 1;
    if (p > d.rcap) {  // the rank exceeds what R, W and the slots were sized for
      if (threadIdx.x == 0) set_status<T>(B.misc, kDevCapacity);
      __syncthreads();
      return;
    }
    if (d.jcache != nullptr) {
      int* pv = jc_piv(d, 1, bank, l + 1);
      for (int c = threadIdx.x; c < p; c += blockDim.x) pv[c] = B.qperm[c];
    }
    // R P^T -> Rp (p x xr, ld xr): column c of the pivoted R is original column perm[c]
    for (int e = threadIdx.x; e < p * xr; e += blockDim.x) {
      const int i = e / xr, c = e % xr;
      B.Rp[i * xr + B.qperm[c]] = (c > i) ? B.W[i * xr + c] : (c == i ? B.beta[i] : mk<T>(0, 0));
    }
    __syncthreads();
    qr_form_q<T>(B.W, m, p, xr, B.tau);
    for (int e = threadIdx.x; e < m * p; e += blockDim.x)
      st_site(dst + e, B.W[(e / p) * xr + (e % p)], B.key(l, 0), e);
    if (threadIdx.x == 0) B.qb[l + 1] = p;
    __syncthreads();
    r = p;
  }
  if (n == 1) {
    // single site: renormalise only
    S* a = B.slot(0);
    if (threadIdx.x < 32) {
      T s2 = 0;
      if (threadIdx.x < 2) s2 = abs2(ld<T>(a + threadIdx.x));
      s2 = gsum(s2, 32);
      if (threadIdx.x == 0) {
        if (!(s2 > 0) || !isfinite((double)s2)) set_status<T>(B.misc, kDevNumeric);
        B.dmisc[0] += 0.5 * log((double)s2);
        B.amps[0] = mk<T>(rsqrt(s2), 0);
      }
    }
    __syncthreads();
    const T inv = B.amps[0].re;
    if (threadIdx.x < 2) st_site(a + threadIdx.x, cscale(ld<T>(a + threadIdx.x), inv), B.key(0, 1), threadIdx.x);
    __syncthreads();
    return;
  }
  // ------------------------------------------------ SVD sweep, right to left
  if (threadIdx.x == 0) B.US[0] = mk<T>(1, 0);
  __syncthreads();
  int kr = 1;  // bond to the right of the current site after truncation
  const T tol_rule = B.tmisc[1];
  // target environments (warp 1): E holds E_{folded}; sites >= folded are in
  const int envG = pow2_cap32(d.chicap);
  const bool warp1 = threadIdx.x >= 32 && threadIdx.x < 64;
  cx<T> E = mk<T>((threadIdx.x & (envG - 1)) == 0 ? (T)1 : (T)0, 0);
  int folded = n;
  for (int l = n - 1; l >= 1; --l) {
    const int rl = B.qb[l], rr = B.qb[l + 1];
    const S* A = B.slot(l);
    const int c = 2 * kr;
    if (rl <= 4 && c + rl <= 8) {  // register-resident step (one warp)
      if (threadIdx.x < 32)
        tiny_svd_step<T, S, CR>(B, l, rl, rr, kr);
      else if (env_nt > 0 && warp1 && folded == l + 2)
        env_fold<T, S, T>(B, l + 1, env_nt, envG, E);  // site l+1 is final
      __syncthreads();
      if (env_nt > 0 && folded == l + 2) folded = l + 1;
      kr = B.misc[4];
      continue;
    }
    if (env_nt > 0 && folded == l + 2) {  // the block step needs every thread
      if (warp1) env_fold<T, S, T>(B, l + 1, env_nt, envG, E);
      __syncthreads();
      folded = l + 1;
    }
    // Mat = A (rl x 2 x rr) * US (rr x kr)  -> rl x (2 kr)
    for (int e = threadIdx.x; e < rl * c; e += blockDim.x) {
      const int i = e / c, s = (e / kr) & 1, j = e % kr;
      cx<CR> acc = mk<CR>(0, 0);
      for (int a = 0; a < rr; ++a) acc = cmac(acc, ld<CR>(A + (i * 2 + s) * rr + a), cvt<CR>(B.US[a * kr + j]));
      B.Mat[e] = cvt<T>(acc);
    }
    __syncthreads();
    // noise floor for skipping rotations: (max(m,n) eps / 4)^2 times the
    // squared Frobenius norm of the matrix, which the sweep conserves up to
    // truncation -- measured once, at its first site
    if (l == n - 1 && threadIdx.x < 32) {
      T f2 = 0;
      for (int e = threadIdx.x; e < rl * c; e += 32) f2 += abs2(B.Mat[e]);
      f2 = gsum(f2, 32);
      if (threadIdx.x == 0) B.tmisc[9] = f2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const T f = rank_floor(B, rl, c) * (T)0.25f;
      B.tmisc[8] = B.tmisc[9] * f * f;
    }
    __syncthreads();
    // warm start: the rotations this site's SVD ended with in the previous
    // iteration (same sweep pair, same row count) nearly diagonalise the Gram
    // matrix again, since one Grover iteration turns the state by a small
    // angle; any unitary start gives the same SVD, so the cache only saves
    // sweeps
    cx<T>* jc = (d.jcache != nullptr && rl <= 4 * (int)blockDim.x) ? jc_rot<T>(d, bank, l) : nullptr;
    int* pv_old = jc != nullptr ? jc_piv(d, 0, bank, l) : nullptr;
    const int* pv_cur = jc != nullptr ? jc_piv(d, 1, bank, l) : nullptr;
    int fits = jc != nullptr && d.stats->jrank[bank][l] == rl;
    if (fits)
      for (int e = threadIdx.x; e < rl; e += blockDim.x) fits &= (pv_cur[e] >= 0 && pv_cur[e] == pv_old[e]);
    const bool warm = __syncthreads_and(fits);
    // without a cached start (FP64): precondition with a row-pivoted LQ,
    // P Mat = [L 0] Q, i.e. the column-pivoted QR of Mat^dag with R = L^dag,
    // and rotate the rows of X = L^dag (rl x rl, held in the U*S buffer, free
    // until this step writes its own U*S): half the columns per rotation,
    // and R's rows are graded by the pivoting (QR-preconditioned one-sided
    // Jacobi, Drmac-Veselic).  With J X = S W^dag: Mat = P^T W S (J Q), so
    // the new site is J Q and U*S = P^T (J X)^dag.  Measured: it pays from
    // about 24 rows (n = 40, M = 32: +8.5%; 17 rows: the LQ and Q's formation
    // cost more than the narrower rotations save)
    bool lq = false;
    if constexpr (std::is_same<T, double>::value)
      lq = jc == nullptr && rl >= 24 && c >= rl && rl * rl <= d.rcap * d.chicap;
    cx<T>* const Lb = B.US;
    int sw;
    if (lq) {
      lq_rows_pivoted<T>(B.Mat, rl, c, c, B.tau, B.beta, B.qperm, B.qcn, B.misc + 8);
      for (int e = threadIdx.x; e < rl * rl; e += blockDim.x) {  // X = L^dag
        const int i = e / rl, j = e % rl;
        const cx<T> x = i < j ? B.Mat[j * c + i] : (j == i ? B.beta[i] : mk<T>(0, 0));
        Lb[e] = mk<T>(x.re, -x.im);
      }
      __syncthreads();
      lq_form_q<T>(B.Mat, rl, c, c, B.tau);
      sw = jacobi_rows<T>(Lb, rl, rl, rl, B.U, rl, d.max_sweeps, K<T>::jtolf(), B.tmisc[8], false);
    } else {
      if (warm) {
        for (int e = threadIdx.x; e < rl * rl; e += blockDim.x) B.U[e] = jc[e];
        __syncthreads();
        rotate_rows<T>(B.Mat, rl, c, B.U);
      }
      sw = jacobi_rows<T>(B.Mat, rl, c, c, B.U, rl, d.max_sweeps, K<T>::jtolf(), B.tmisc[8], warm);
      if (jc != nullptr) {
        for (int e = threadIdx.x; e < rl * rl; e += blockDim.x) jc[e] = B.U[e];
        for (int e = threadIdx.x; e < rl; e += blockDim.x) pv_old[e] = pv_cur[e];
        if (threadIdx.x == 0) d.stats->jrank[bank][l] = rl;
      }
    }
    // row norms -> sigma, ranks -> perm
    {
      const cx<T>* R = lq ? Lb : B.Mat;
      const int rc = lq ? rl : c;
      const int G = pow2_cap32(rc);
      const Grp g = make_grp(G);
      for (int t0 = 0; t0 < rl; t0 += g.ng) {
        const int i = t0 + g.gid;
        T s2 = 0;
        if (i < rl)
          for (int j = g.lg; j < rc; j += G) s2 += abs2(R[i * rc + j]);
        s2 = gsum(s2, G);
        if (i < rl && g.lg == 0) B.sig[i] = s2;  // sigma_i^2 (rows are orthogonal)
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rl; i += blockDim.x) {
      const T si = B.sig[i];
      int rank = 0;
      for (int j = 0; j < rl; ++j) {
        const T sj = B.sig[j];
        rank += (sj > si) || (sj == si && j < i);
      }
      B.perm[rank] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (sw < 0) set_status<T>(B.misc, kDevNoConv);
      const int swc = sw < 0 ? d.max_sweeps : sw;
      B.misc[1] = max(B.misc[1], swc);
      B.misc[2] += swc;
      B.misc[3] += 1;
      // sigma_t > max(tol, max(m,n) eps) sigma_0, compared as squares
      const T s0 = B.sig[B.perm[0]];
      const T fr = fmax(tol_rule, rank_floor(B, rl, c));
      const T thr2 = fr * fr * s0;
      int k = 0;
      T tot = 0, kept = 0;
      for (int t = 0; t < rl; ++t) {
        const T st_ = B.sig[B.perm[t]];
        tot += st_;
        if (st_ > thr2) ++k;
      }
      if (k < 1) k = 1;
      if (k > d.chi_max) k = d.chi_max;
      if (k > d.chicap) {
        set_status<T>(B.misc, kDevCapacity);
        k = d.chicap;
      }
      for (int t = 0; t < k; ++t) kept += B.sig[B.perm[t]];
      if (tot > (T)0 && kept != tot) B.tmisc[2] += (tot - kept) / tot;
      B.misc[4] = k;
    }
    __syncthreads();
    const int k = B.misc[4];
    // new site l = rows of V^dag (k x 2 x kr); US_l = U^dag[:, perm] * sigma (rl x k)
    // 1/sigma of each kept row from one rsqrt of sigma^2 (qcn is free here)
    for (int t = threadIdx.x; t < k; t += blockDim.x) B.qcn[t] = rsqrt(B.sig[B.perm[t]]);
    S* dst = B.slot(l);
    __syncthreads();
    for (int e = threadIdx.x; e < k * c; e += blockDim.x) {
      const int t = e / c, j = e % c;
      const int pr = B.perm[t];
      cx<T> v;
      if (lq) {  // row pr of J Q (orthonormal rows)
        v = mk<T>(0, 0);
        for (int a = 0; a < rl; ++a) v = cmac(v, B.U[pr * rl + a], B.Mat[a * c + j]);
      } else {
        v = cscale(B.Mat[pr * c + j], B.qcn[t]);
      }
      st_site(dst + e, v, B.key(l, 1), e);
    }
    // U S with U = J^dag (the product of the rotations is accumulated in B.U;
    // the previous US was consumed when Mat was formed); after the LQ it is
    // P^T (J X)^dag: row rperm[ip] takes conj((J X)[pr][ip]), staged in the
    // Mat buffer (Q is consumed) because J X sits in the U*S buffer
    __syncthreads();
    if (lq) {
      for (int e = threadIdx.x; e < rl * k; e += blockDim.x) {
        const cx<T> x = Lb[B.perm[e % k] * rl + e / k];
        B.Mat[e] = mk<T>(x.re, -x.im);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < rl * k; e += blockDim.x) B.US[B.qperm[e / k] * k + e % k] = B.Mat[e];
    }
    for (int e = threadIdx.x; e < rl * k && !lq; e += blockDim.x) {
      const int i = e / k, t = e % k;
      const int pr = B.perm[t];
      const cx<T> u = B.U[pr * rl + i];
      B.US[e] = cscale(mk<T>(u.re, -u.im), B.sig[pr] * B.qcn[t]);  // sigma = sigma^2 / sigma
    }
    if (threadIdx.x == 0) B.chi[l] = k;
    __syncthreads();
    kr = k;
  }
  // ------------------------------------------------ site 0 and renormalisation
  {
    const int rr = B.qb[1];
    S* A = B.slot(0);
    const int c = 2 * kr;
    for (int e = threadIdx.x; e < c; e += blockDim.x) {
      const int s = e / kr, j = e % kr;
      cx<CR> acc = mk<CR>(0, 0);
      for (int a = 0; a < rr; ++a) acc = cmac(acc, ld<CR>(A + s * rr + a), cvt<CR>(B.US[a * kr + j]));
      B.Mat[e] = cvt<T>(acc);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      T s2 = 0;
      for (int e = threadIdx.x; e < c; e += 32) s2 += abs2(B.Mat[e]);
      s2 = gsum(s2, 32);
      if (threadIdx.x == 0) {
        if (!(s2 > 0) || !isfinite((double)s2)) set_status<T>(B.misc, kDevNumeric);
        B.dmisc[0] += 0.5 * log((double)s2);
        B.amps[0] = mk<T>(rsqrt(s2), 0);
        B.chi[0] = 1;
      }
    }
    __syncthreads();
    const T inv = B.amps[0].re;
    for (int e = threadIdx.x; e < c; e += blockDim.x) st_site(A + e, cscale(B.Mat[e], inv), B.key(0, 1), e);
    __syncthreads();
  }
  if (env_nt > 0) {  // sites folded..1 are final, site 0 just renormalised
    if (warp1) {
      for (int s = folded - 1; s >= 0; --s) env_fold<T, S, T>(B, s, env_nt, envG, E);
      const int lane = threadIdx.x & 31;
      if ((lane & (envG - 1)) == 0 && lane / envG < env_nt) B.amps[lane / envG] = cvt<T>(E);
    }
    __syncthreads();
  }
}

// <target_t|psi> for product-state targets (basis strings or |+>^n), by the
// chain v <- v A_l[:, b_l, :] (or v (A_l[:,0,:]+A_l[:,1,:])/sqrt 2); lanes
// over the right bond: a group of G lanes per target when every bond fits
// 16 lanes, else one warp per target (bonds <= 64).
template <class T, class S, class CR>
__device__ void chain_targets(Blk<T, S>& B, int nt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const CR h = K<CR>::isq2();
  const int G = pow2_cap32(B.d->chicap);  // lanes that cover any bond
  if (G <= 16) {
    // 32/G targets per warp in one instruction stream; for |+>^n the factor
    // (A_0 + A_1) v is summed first and scaled by 1/sqrt 2 once per site
    const int per = 32 / G, lg = lane & (G - 1), base = lane & ~(G - 1);
    for (int t0 = warp * per; t0 < nt; t0 += nw * per) {
      const int t = t0 + lane / G;
      const bool on = t < nt;
      const bool plus = on && B.tplus[t];
      const unsigned long long bits = (on && !plus) ? B.tbits[t] : 0ull;
      cx<CR> v = mk<CR>(lg == 0 ? (CR)1 : (CR)0, 0);
      for (int l = 0; l < B.n; ++l) {
        const int cl = B.chi[l], cr = B.chi[l + 1];
        const S* A = B.slot(l);
        const int b = (int)((bits >> l) & 1ull);
        cx<CR> nv = mk<CR>(0, 0);
        for (int i = 0; i < cl; ++i) {
          cx<CR> vi;
          vi.re = shidx(v.re, base + i);
          vi.im = shidx(v.im, base + i);
          if (lg < cr) {
            cx<CR> a = ld<CR>(A + (i * 2 + b) * cr + lg);
            if (plus) a = cadd(a, ld<CR>(A + (i * 2 + 1) * cr + lg));
            nv = cmac(nv, vi, a);
          }
        }
        v = plus ? cscale(nv, h) : nv;
      }
      if (on && lg == 0) B.amps[t] = cvt<T>(v);
    }
    __syncthreads();
    return;
  }
  for (int t = warp; t < nt; t += nw) {
    const bool plus = B.tplus[t];
    const unsigned long long bits = B.tbits[t];
    cx<CR> v0 = mk<CR>(lane == 0 ? (CR)1 : (CR)0, 0), v1 = mk<CR>(0, 0);
    for (int l = 0; l < B.n; ++l) {
      const int cl = B.chi[l], cr = B.chi[l + 1];
      const S* A = B.slot(l);
      const int b = (int)((bits >> l) & 1ull);
      cx<CR> n0 = mk<CR>(0, 0), n1 = mk<CR>(0, 0);
      for (int i = 0; i < cl; ++i) {
        const cx<CR> src = (i < 32) ? v0 : v1;
        cx<CR> vi;
        vi.re = shidx(src.re, i & 31);
        vi.im = shidx(src.im, i & 31);
        if (lane < cr) {
          cx<CR> a = plus ? cscale(cadd(ld<CR>(A + (i * 2) * cr + lane), ld<CR>(A + (i * 2 + 1) * cr + lane)), h)
                          : ld<CR>(A + (i * 2 + b) * cr + lane);
          n0 = cmac(n0, vi, a);
        }
        if (lane + 32 < cr) {
          cx<CR> a = plus ? cscale(cadd(ld<CR>(A + (i * 2) * cr + lane + 32), ld<CR>(A + (i * 2 + 1) * cr + lane + 32)), h)
                          : ld<CR>(A + (i * 2 + b) * cr + lane + 32);
          n1 = cmac(n1, vi, a);
        }
      }
      v0 = n0;
      v1 = n1;
    }
    if (lane == 0) B.amps[t] = cvt<T>(v0);
  }
  __syncthreads();
}

// ------------------------------------------------------------ block set-up
// Point a block's working state at its shared-memory plan, copy the chain in
// when it is resident, and load the instance's bond table and counters
// (log-norm reset to zero when zero_log_norm).  Ends with a block barrier.
template <class T, class S>
__device__ void blk_open(Blk<T, S>& B, const InstDesc& d, unsigned char* smem, bool zero_log_norm) {
  const int n = d.n;
  const size_t site_bytes = d.resident ? (size_t)d.site_off[n] * sizeof(S) : 0;
  const SmemPlan P = make_plan(n, d.M, d.xcap, d.chicap, d.rcap, sizeof(T), site_bytes, d.work != nullptr);
  B.d = &d;
  B.n = n;
  B.csize = 1;
  {
    int* so = (int*)(smem + P.off_soff);
    for (int l = threadIdx.x; l <= n; l += blockDim.x) so[l] = (int)d.site_off[l];
    B.off = so;
  }
  B.chi = (int*)(smem + P.off_chi);
  B.qb = (int*)(smem + P.off_qb);
  unsigned char* tb = smem + P.off_terms;
  B.tbits = (unsigned long long*)tb;
  B.tcoef = (cx<T>*)(tb + sizeof(unsigned long long) * (d.M + 2));
  B.tplus = (int*)(tb + (sizeof(unsigned long long) + 2 * sizeof(T)) * (d.M + 2));
  B.amps = (cx<T>*)(smem + P.off_amps);
  B.misc = (int*)(smem + P.off_misc);
  B.dmisc = (double*)(smem + P.off_misc + 128);
  B.tmisc = (T*)(smem + P.off_misc + 256);
  unsigned char* qbase = d.work ? (unsigned char*)d.work : smem;  // QR matrices
  B.Rp = (cx<T>*)(qbase + P.off_rprev);
  B.W = (cx<T>*)(qbase + P.off_w);
  B.tau = (T*)(smem + P.off_tau);
  B.beta = (cx<T>*)(smem + P.off_beta);
  B.Mat = (cx<T>*)(smem + P.off_mat);
  B.U = (cx<T>*)(smem + P.off_u);
  B.US = (cx<T>*)(smem + P.off_us);
  B.sig = (T*)(smem + P.off_sig);
  B.perm = (int*)(smem + P.off_perm);
  B.qperm = (int*)(smem + P.off_qperm);
  B.qcn = (T*)(smem + P.off_qcn);
  B.tbuf = smem + P.off_tbuf;
  S* gsites = (S*)d.sites;
  if (d.resident) {
    S* ssites = (S*)(smem + P.off_sites);
    for (long long e = threadIdx.x; e < d.site_off[n]; e += blockDim.x) ssites[e] = gsites[e];
    B.sites = ssites;
  } else {
    B.sites = gsites;
  }
  DevStats* ds = d.stats;
  for (int l = threadIdx.x; l <= n; l += blockDim.x) B.chi[l] = ds->chi[l];
  if (threadIdx.x == 0) {
    B.misc[0] = ds->status;
    B.misc[1] = ds->max_jacobi_sweeps;
    B.misc[2] = 0;
    B.misc[3] = 0;
    B.dmisc[0] = zero_log_norm ? 0.0 : ds->log_norm;
    B.dmisc[1] = ds->discarded;
    B.tmisc[0] = (T)d.trunc_eps;
    B.misc[5] = d.trunc_dim;
    B.tmisc[1] = (T)d.tol;
    B.tmisc[2] = (T)0;
  }
  __syncthreads();
}

// Write a block's chain (when resident), bond table and counters back.
template <class T, class S>
__device__ void blk_close(Blk<T, S>& B, const InstDesc& d) {
  __syncthreads();
  const int n = d.n;
  if (d.resident) {
    S* gsites = (S*)d.sites;
    const S* ssites = B.sites;
    for (long long e = threadIdx.x; e < d.site_off[n]; e += blockDim.x) gsites[e] = ssites[e];
  }
  DevStats* ds = d.stats;
  for (int l = threadIdx.x; l <= n; l += blockDim.x) ds->chi[l] = B.chi[l];
  if (threadIdx.x == 0) {
    ds->status = B.misc[0];
    ds->max_jacobi_sweeps = B.misc[1];
    ds->jacobi_sweeps += B.misc[2];
    ds->svd_count += B.misc[3];
    ds->log_norm = B.dmisc[0];
    ds->discarded = B.dmisc[1] + (double)B.tmisc[2];
  }
}

// ------------------------------------------------------------ the kernel
// kCl: the instance runs on a thread-block cluster (one instance, FP64 QR);
// the plain instantiation carries none of the cluster code.
template <class T, class S, class CR, bool kCl>
__global__ void __launch_bounds__(256, 1) iterate_kernel(const InstDesc* descs, int count, int* queue) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  // a single instance may run on a cluster: the first CTA runs the sweeps,
  // the others take shares of its large QR steps (cluster_worker)
  constexpr bool kClOn = kCl && std::is_same<T, double>::value;
  int csize = 1;
  if constexpr (kClOn) {
    csize = count == 1 ? (int)cg::this_cluster().num_blocks() : 1;
    if (csize > 1 && cg::this_cluster().block_rank() != 0) {
      cluster_worker<T>(descs[0], smem);
      return;
    }
  }
  for (;;) {
    if (threadIdx.x == 0) s_idx = (count == 1) ? (blockIdx.x == 0 ? 0 : count) : atomicAdd(queue, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    if (count == 1 && blockIdx.x != 0) break;
    const unsigned long long t_begin = global_ns();
    const InstDesc& d = descs[idx];
    const int n = d.n;
    Blk<T, S> B;
    B.rng = 0;
    blk_open(B, d, smem, false);
    B.csize = csize;
    DevStats* ds = d.stats;
    const int M = d.M;
    long long done = 0;
    // fused form: <w|psi> and <s|psi> for the next iteration come out of the
    // sweep (warp 1 folds the sites as the SVD sweep finalises them) when
    // the block has a second warp and the M+1 targets fit it
    const int envG = pow2_cap32(d.chicap);
    const int env_nt = (d.apply == 2 && n >= 2 && blockDim.x >= 64 && envG <= 16 && M + 1 <= 32 / envG) ? M + 1 : 0;
    bool amps_ready = false;
    const long long it0 = ds->iterations;  // iterations applied before this launch
    // rounding keys: per instance (its marked strings) and per iteration
    unsigned long long salt = fmix64(((unsigned long long)n << 8) | (unsigned long long)M);
    for (int t = 0; t < M; ++t) salt = fmix64(salt ^ d.marked[t]);
    for (long long it = 0; it < d.k; ++it) {
      if (B.misc[0] != 0) break;
      B.rng = salt + ((unsigned long long)(it0 + it) << 3);
      const long long pi = d.phase_offset + it;
      if (d.rec) {
        // record <w|psi> for every marked w and <s|psi> (adjoint recompute)
        for (int t = threadIdx.x; t <= M; t += blockDim.x) {
          B.tbits[t] = t < M ? d.marked[t] : 0ull;
          B.tplus[t] = t == M;
        }
        __syncthreads();
        if (!amps_ready) chain_targets<T, S, T>(B, M + 1);
        for (int t = threadIdx.x; t <= M; t += blockDim.x) {
          d.rec[(it * (M + 1) + t) * 2] = (double)B.amps[t].re;
          d.rec[(it * (M + 1) + t) * 2 + 1] = (double)B.amps[t].im;
        }
        __syncthreads();
      }
      // e^{i phi} - 1 and 1 - e^{i psi} in FP64 (e^{i pi} = -1 exactly for
      // the plain-Grover default), computed once and broadcast.
      if (threadIdx.x == 0) {
        double cphi = -1.0, sphi = 0.0, cpsi_ = -1.0, spsi = 0.0;
        if (d.phi) sincos(d.phi[pi], &sphi, &cphi);
        if (d.psi) sincos(d.psi[pi], &spsi, &cpsi_);
        B.tmisc[3] = (T)(cphi - 1.0);
        B.tmisc[4] = (T)sphi;
        B.tmisc[5] = (T)(1.0 - cpsi_);
        B.tmisc[6] = (T)(-spsi);
        B.tmisc[7] = (T)d.inv_sqrt_N;
      }
      __syncthreads();
      const cx<T> em1 = mk<T>(B.tmisc[3], B.tmisc[4]);   // e^{i phi} - 1
      const cx<T> opsi = mk<T>(B.tmisc[5], B.tmisc[6]);  // 1 - e^{i psi}
      if (d.apply == 0) {
        // O as an MPO of bond M+1: left boundary (1, e^{i phi}-1, ...)
        for (int a = threadIdx.x; a <= M; a += blockDim.x) B.tcoef[a] = a == 0 ? mk<T>(1, 0) : em1;
        __syncthreads();
        sweep_pair<T, S, CR, kCl>(B, 0, 0, M + 1, B.tcoef, mk<T>(1, 0), 0);
        if (B.misc[0] != 0) break;
        // D as an MPO of bond 2: left boundary (-1, 1 - e^{i psi})
        if (threadIdx.x == 0) {
          B.tcoef[0] = mk<T>(-1, 0);
          B.tcoef[1] = opsi;
        }
        __syncthreads();
        sweep_pair<T, S, CR, kCl>(B, 0, 1, 2, B.tcoef, mk<T>(1, 0), 0, 0, 1);
      } else if (d.apply == 1) {
        // O|p> = |p> + (e^{i phi}-1) sum_w p(w)|w>
        for (int t = threadIdx.x; t < M; t += blockDim.x) {
          B.tbits[t] = d.marked[t];
          B.tplus[t] = 0;
        }
        __syncthreads();
        chain_targets<T, S, T>(B, M);
        for (int t = threadIdx.x; t < M; t += blockDim.x) B.tcoef[t] = cmul(em1, B.amps[t]);
        __syncthreads();
        sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(1, 0), M);
        if (B.misc[0] != 0) break;
        // D|p> = (1 - e^{i psi}) <s|p> |s> - |p>
        if (threadIdx.x == 0) {
          B.tbits[0] = 0;
          B.tplus[0] = 1;
        }
        __syncthreads();
        chain_targets<T, S, T>(B, 1);
        if (threadIdx.x == 0) B.tcoef[0] = cmul(opsi, B.amps[0]);
        __syncthreads();
        sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(-1, 0), 1, 0, 1);
      } else {
        // G|p> = -|p> - (e^{i phi}-1) sum_w p(w)|w> + (1-e^{i psi}) <s|O p> |s>
        for (int t = threadIdx.x; t <= M; t += blockDim.x) {
          B.tbits[t] = t < M ? d.marked[t] : 0ull;
          B.tplus[t] = t == M;
        }
        __syncthreads();
        if (!amps_ready) {
          chain_targets<T, S, T>(B, M + 1);
        }
        if (threadIdx.x == 0) {
          cx<T> sum = mk<T>(0, 0);
          for (int t = 0; t < M; ++t) sum = cadd(sum, B.amps[t]);
          const cx<T> so = cadd(B.amps[M], cscale(cmul(em1, sum), B.tmisc[7]));
          B.tcoef[M] = cmul(opsi, so);
        }
        for (int t = threadIdx.x; t < M; t += blockDim.x) {
          const cx<T> c = cmul(em1, B.amps[t]);
          B.tcoef[t] = mk<T>(-c.re, -c.im);
        }
        __syncthreads();
        sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(-1, 0), M + 1, env_nt);
        amps_ready = env_nt > 0;
      }
      __syncthreads();
      if (B.misc[0] == 0) ++done;
    }
    blk_close(B, d);
    if (threadIdx.x == 0) {
      ds->iterations += done;
      ds->t_begin = t_begin;
      ds->t_end = global_ns();
      ds->sm = sm_id();
    }
    __syncthreads();
    if (count == 1) break;
  }
  if constexpr (kClOn) {
    if (csize > 1) {  // release the cluster's other CTAs
      const InstDesc& d = descs[0];
      const SmemPlan Pw = make_plan(d.n, d.M, d.xcap, d.chicap, d.rcap, sizeof(T), 0, true);
      const ClusterView<T> cv = cluster_view<T>((unsigned char*)d.work, Pw, d.rcap);
      if (threadIdx.x == 0) {
        cv.c->op = 0;
        __threadfence();
      }
      __syncthreads();
      cg::this_cluster().sync();
    }
  }
}

// ------------------------------------------------------------------ adjoint
// One costate step as two direct sums (D(-psi_k) with the |s> term, then
// O(-phi_k) with the marked terms), for arenas sized for the split form;
// gradients as in adjoint_kernel.  Leaves the targets' table set to the M
// marked strings.
template <class T, class S, class CR>
__device__ void adjoint_two_steps(Blk<T, S>& B, const double* rec, long long k, long long k_lo, const double* phi,
                                  const double* psi, double scale, double* gphi, double* gpsi) {
  const InstDesc& d = *B.d;
  const int M = d.M;
  if (threadIdx.x == 0) {
    double sp, cp, ss, cs;
    sincos(phi[k - 1], &sp, &cp);
    sincos(psi[k - 1], &ss, &cs);
    B.dmisc[2] = cp;
    B.dmisc[3] = sp;
    B.dmisc[4] = cs;
    B.dmisc[5] = ss;
    B.tbits[0] = 0ull;
    B.tplus[0] = 1;
  }
  __syncthreads();
  const double cp = B.dmisc[2], sp = B.dmisc[3], cs = B.dmisc[4], ss = B.dmisc[5];
  // <s|mu_k> of the normalised chain, scale lambda = e^{log norm}
  chain_targets<T, S, T>(B, 1);
  double smr = 0, smi = 0;  // <s|mu_k> (thread 0)
  if (threadIdx.x == 0) {
    const double lam = exp(B.dmisc[0]);
    smr = lam * (double)B.amps[0].re;
    smi = lam * (double)B.amps[0].im;
    // nu = D(-psi) mu = (1 - e^{-i psi}) <s|mu> |s> - mu
    const cx<T> c1 = mk<T>((T)(1.0 - cs), (T)ss);
    B.tcoef[0] = cmul(c1, B.amps[0]);
  }
  __syncthreads();
  sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(-1, 0), 1);
  if (B.misc[0] != 0) return;
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    B.tbits[t] = d.marked[t];
    B.tplus[t] = 0;
  }
  __syncthreads();
  chain_targets<T, S, T>(B, M);
  if (threadIdx.x == 0) {
    const double lam = exp(B.dmisc[0]);
    const double* S_ = rec + (k - 1 - k_lo) * (M + 1) * 2;
    double zr = 0, zi = 0, sr = 0, si = 0;  // sum conj(nu) psi, sum psi
    for (int t = 0; t < M; ++t) {
      const double nr = (double)B.amps[t].re, ni = (double)B.amps[t].im;
      const double pr = S_[2 * t], pim = S_[2 * t + 1];
      zr += nr * pr + ni * pim;
      zi += nr * pim - ni * pr;
      sr += pr;
      si += pim;
    }
    zr *= lam;
    zi *= lam;
    gphi[k - 1] = scale * (-2.0 * (sp * zr + cp * zi));
    const double h = d.inv_sqrt_N;
    const double er = cp - 1.0, ei = sp;
    const double sor = S_[2 * M] + h * (er * sr - ei * si);
    const double soi = S_[2 * M + 1] + h * (er * si + ei * sr);
    const double qr = smr * sor + smi * soi, qi = smr * soi - smi * sor;
    gpsi[k - 1] = scale * (2.0 * (ss * qr + cs * qi));
    // mu_{k-1} = O(-phi) nu = nu + (e^{-i phi} - 1) sum_w nu(w)|w>
    const cx<T> c2 = mk<T>((T)(cp - 1.0), (T)(-sp));
    for (int t = 0; t < M; ++t) B.tcoef[t] = cmul(c2, B.amps[t]);
  }
  __syncthreads();
  sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(1, 0), M);
}

// Reverse sweep of the phase gradient of P = sum_w |<w|psi_K>|^2 over
// iterations k_hi..k_lo+1 (1-based), on the costate chain of `descs[0]`:
//   mu_K = Pi_W psi_K  (project != 0: built from the chain itself),
//   nu_k = D(psi_k)^dag mu_k = D(-psi_k) mu_k,   mu_{k-1} = O(-phi_k) nu_k,
//   dP/dphi_k = 2 Re[ i e^{i phi_k} sum_w conj(nu_k(w)) psi_{k-1}(w) ],
//   dP/dpsi_k = 2 Re[ -i e^{i psi_k} conj(<s|mu_k>) <s|O_k psi_{k-1}> ],
//   <s|O_k psi> = <s|psi> + (e^{i phi_k} - 1) 2^{-n/2} sum_w psi(w).
// Each costate step applies G_k^dag = O(-phi_k) D(-psi_k) as one direct sum
// (mu_{k-1} = -mu_k + (1 - e^{-i psi_k}) <s|mu_k> |s> + (e^{-i phi_k} - 1)
// sum_w nu_k(w) |w>, with nu_k(w) = (1 - e^{-i psi_k}) <s|mu_k> 2^{-n/2} -
// mu_k(w)) followed by the QR and SVD sweeps (two direct sums, D then O, when
// the arena is sized for the split form); the costate's norm is carried by
// the chain's log-norm.  rec holds
// the forward chain's marked amplitudes and <s|psi_{k-1}> for k-1 = k_lo..k_hi-1.
// The gradients are written scaled by `scale` (dL/dP).  One thread block per
// costate chain: block b works on descs[b] with the arguments args[b] (a batch
// of phase vectors of one problem runs as one launch).
template <class T, class S, class CR>
__global__ void __launch_bounds__(256, 1) adjoint_kernel(const InstDesc* descs, const AdjArgs* args, long long k_lo,
                                                       long long k_hi, int project) {
  extern __shared__ __align__(16) unsigned char smem[];
  const InstDesc& d = descs[blockIdx.x];
  const AdjArgs& aa = args[blockIdx.x];
  const double* rec = aa.rec;
  const double* phi = aa.phi;
  const double* psi = aa.psi;
  const double scale = aa.scale;
  double* gphi = aa.gphi;
  double* gpsi = aa.gpsi;
  const int n = d.n, M = d.M;
  Blk<T, S> B;
  B.rng = 0x2000000000000000ull;
  blk_open(B, d, smem, project != 0);
  // targets: the marked strings (t < M) and |s> = |+>^n (t = M)
  for (int t = threadIdx.x; t <= M; t += blockDim.x) {
    B.tbits[t] = t < M ? d.marked[t] : 0ull;
    B.tplus[t] = t == M;
  }
  __syncthreads();
  // with a second warp the targets' amplitudes of each new costate come out
  // of its sweep (environments folded as the SVD sweep finalises the sites)
  // G_k^dag as one direct sum needs the expanded bond chi + M + 1 (the
  // fused and MPO arenas have it; a split-form arena gets the two steps)
  const bool fused = d.xcap >= d.chicap + M + 1;
  const int envG = pow2_cap32(d.chicap);
  const int env_nt =
      (fused && n >= 2 && blockDim.x >= 64 && envG <= 16 && M + 1 <= 32 / envG) ? M + 1 : 0;
  bool amps_ready = false;
  if (project) {
    // mu_K = sum_w psi_K(w) |w>: a direct sum without the chain's own block
    chain_targets<T, S, T>(B, M);
    for (int t = threadIdx.x; t < M; t += blockDim.x) B.tcoef[t] = B.amps[t];
    __syncthreads();
    sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(0, 0), M, env_nt);
    amps_ready = env_nt > 0;
  }
  for (long long k = k_hi; k > k_lo && B.misc[0] == 0; --k) {
    B.rng = ((unsigned long long)k << 3) | 0x4000000000000000ull;
    if (!fused) {
      adjoint_two_steps<T, S, CR>(B, rec, k, k_lo, phi, psi, scale, gphi, gpsi);
      continue;
    }
    // <w|mu_k> and <s|mu_k> of the normalised chain (scale lambda = e^{log norm})
    if (!amps_ready) chain_targets<T, S, T>(B, M + 1);
    if (threadIdx.x == 0) {
      double sp, cp, ss, cs;
      sincos(phi[k - 1], &sp, &cp);
      sincos(psi[k - 1], &ss, &cs);
      const double lam = exp(B.dmisc[0]);
      const double h = d.inv_sqrt_N;
      // nu = D(-psi) mu = (1 - e^{-i psi}) <s|mu> |s> - mu, so that
      // nu(w) = (1 - e^{-i psi}) <s|mu> 2^{-n/2} - mu(w)
      const cx<T> c1 = mk<T>((T)(1.0 - cs), (T)ss);
      const cx<T> cs_mu = cmul(c1, B.amps[M]);
      // mu_{k-1} = O(-phi) nu = (1 - e^{-i psi}) <s|mu> |s> - mu + (e^{-i phi} - 1) sum_w nu(w) |w>
      const cx<T> c2 = mk<T>((T)(cp - 1.0), (T)(-sp));
      const double* S_ = rec + (k - 1 - k_lo) * (M + 1) * 2;
      double zr = 0, zi = 0, sr = 0, si = 0;  // sum conj(nu) psi, sum psi
      for (int t = 0; t < M; ++t) {
        const cx<T> nu = csub(cscale(cs_mu, (T)h), B.amps[t]);
        const double nr = (double)nu.re, ni = (double)nu.im;
        const double pr = S_[2 * t], pim = S_[2 * t + 1];
        zr += nr * pr + ni * pim;
        zi += nr * pim - ni * pr;
        sr += pr;
        si += pim;
        B.tcoef[t] = cmul(c2, nu);
      }
      B.tcoef[M] = cs_mu;
      zr *= lam;
      zi *= lam;
      // dP/dphi = 2 Re[i e^{i phi} z] = -2 (sin(phi) zr + cos(phi) zi)
      gphi[k - 1] = scale * (-2.0 * (sp * zr + cp * zi));
      // <s|O psi> = <s|psi> + (e^{i phi} - 1) 2^{-n/2} sum_w psi(w)
      const double er = cp - 1.0, ei = sp;
      const double sor = S_[2 * M] + h * (er * sr - ei * si);
      const double soi = S_[2 * M + 1] + h * (er * si + ei * sr);
      // q = conj(<s|mu>) <s|O psi>, <s|mu> = lambda <s|mu>_normalised
      const double smr = lam * (double)B.amps[M].re, smi = lam * (double)B.amps[M].im;
      const double qr = smr * sor + smi * soi, qi = smr * soi - smi * sor;
      // dP/dpsi = 2 Re[-i e^{i psi} q] = 2 (sin(psi) qr + cos(psi) qi)
      gpsi[k - 1] = scale * (2.0 * (ss * qr + cs * qi));
    }
    __syncthreads();
    // G_k^dag mu as one direct sum: -mu plus M + 1 product states
    sweep_pair<T, S, CR>(B, 1, 0, 0, nullptr, mk<T>(-1, 0), M + 1, env_nt);
    amps_ready = env_nt > 0;
  }
  blk_close(B, d);
}

// ------------------------------------------------------------ gate-level circuit
// One-qubit gate u on site l, in place: A[i, s, j] <- sum_s' u[s][s'] A[i, s', j].
// A unitary on the physical index keeps a right-orthonormal site
// right-orthonormal, so the chain stays canonical.
template <class T, class S>
__device__ void apply_1q(Blk<T, S>& B, int l, const double* u) {
  const int cl = B.chi[l], cr = B.chi[l + 1];
  S* A = B.slot(l);
  const cx<T> u00 = mk<T>((T)u[0], (T)u[1]), u01 = mk<T>((T)u[2], (T)u[3]);
  const cx<T> u10 = mk<T>((T)u[4], (T)u[5]), u11 = mk<T>((T)u[6], (T)u[7]);
  for (int e = threadIdx.x; e < cl * cr; e += blockDim.x) {
    const int i = e / cr, j = e % cr;
    const cx<T> a0 = ld<T>(A + (i * 2) * cr + j), a1 = ld<T>(A + (i * 2 + 1) * cr + j);
    st_site(A + (i * 2) * cr + j, cmac(cmul(u00, a0), u01, a1), B.key(l, 2), (unsigned)((i * 2) * cr + j));
    st_site(A + (i * 2 + 1) * cr + j, cmac(cmul(u10, a0), u11, a1), B.key(l, 2), (unsigned)((i * 2 + 1) * cr + j));
  }
  __syncthreads();
}

// Gate-level simulation of one instance (one thread block): `repeat` passes
// over `count` gates.  A one-qubit gate updates its site tensor in place; a
// multi-controlled phase I - (1 - e^{i phase}) |1...1><1...1| is the MPO of
// bond 2 diag(I, |1><1|) with left boundary (1, e^{i phase} - 1) -- the
// oracle MPO of the all-ones string, d.marked[0] -- contracted into the sites
// and recompressed by the QR and truncated SVD sweeps.
template <class T, class S, class CR>
__global__ void __launch_bounds__(256, 1) circuit_kernel(const InstDesc* descs, const GateOp* gates, long long count,
                                                       long long repeat) {
  extern __shared__ __align__(16) unsigned char smem[];
  const InstDesc& d = descs[0];
  Blk<T, S> B;
  B.rng = 0x1000000000000000ull;
  blk_open(B, d, smem, false);
  for (long long r = 0; r < repeat && B.misc[0] == 0; ++r) {
    for (long long g = 0; g < count && B.misc[0] == 0; ++g) {
      const GateOp& op = gates[g];
      B.rng = fmix64(B.rng + 0x9e3779b97f4a7c15ull);
      if (op.kind == 0) {
        apply_1q(B, op.site, op.u);
      } else {
        if (threadIdx.x == 0) {
          double sp, cp;
          sincos(op.u[0], &sp, &cp);
          B.tcoef[0] = mk<T>(1, 0);
          B.tcoef[1] = mk<T>((T)(cp - 1.0), (T)sp);
        }
        __syncthreads();
        sweep_pair<T, S, CR>(B, 0, 0, 2, B.tcoef, mk<T>(1, 0), 0);
      }
    }
  }
  blk_close(B, d);
}

// ------------------------------------------------------------------ init
template <class S>
__global__ void init_kernel(const InstDesc* descs, int count) {
  const int idx = blockIdx.x;
  if (idx >= count) return;
  const InstDesc& d = descs[idx];
  S* sites = (S*)d.sites;
  const double h = 0.70710678118654752440;
  for (int l = threadIdx.x; l < d.n; l += blockDim.x) {
    S* a = sites + d.site_off[l];
    st(a, mk<double>(h, 0.0));
    st(a + 1, mk<double>(h, 0.0));
  }
  DevStats* ds = d.stats;
  for (int l = threadIdx.x; l <= d.n; l += blockDim.x) {
    ds->chi[l] = 1;
    ds->jrank[0][l] = 0;
    ds->jrank[1][l] = 0;
  }
  if (threadIdx.x == 0) {
    ds->iterations = 0;
    ds->jacobi_sweeps = 0;
    ds->svd_count = 0;
    ds->max_jacobi_sweeps = 0;
    ds->status = 0;
    ds->log_norm = 0.0;
    ds->discarded = 0.0;
  }
}

// ------------------------------------------------------------ amplitudes
// <x|psi> = prod_l A_l[:, x_l, :]: one warp per bitstring.
template <class S>
__global__ void amplitude_kernel(const InstDesc* descs, int inst, const unsigned long long* bits,
                                 int nbits, double* out) {
  const InstDesc& d = descs[inst];
  const S* sites = (const S*)d.sites;
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nbits) return;
  const unsigned long long x = bits[w];
  const int* chi = d.stats->chi;
  cx<double> v0 = mk<double>(lane == 0 ? 1.0 : 0.0, 0.0), v1 = mk<double>(0, 0);
  for (int l = 0; l < d.n; ++l) {
    const int cl = chi[l], cr = chi[l + 1];
    const S* A = sites + d.site_off[l];
    const int b = (int)((x >> l) & 1ull);
    cx<double> n0 = mk<double>(0, 0), n1 = mk<double>(0, 0);
    for (int i = 0; i < cl; ++i) {
      const cx<double> src = (i < 32) ? v0 : v1;
      cx<double> vi;
      vi.re = __shfl_sync(0xffffffffu, src.re, i & 31);
      vi.im = __shfl_sync(0xffffffffu, src.im, i & 31);
      if (lane < cr) n0 = cmac(n0, vi, ld<double>(A + (i * 2 + b) * cr + lane));
      if (lane + 32 < cr) n1 = cmac(n1, vi, ld<double>(A + (i * 2 + b) * cr + lane + 32));
    }
    v0 = n0;
    v1 = n1;
  }
  if (lane == 0) {
    out[2 * w] = v0.re;
    out[2 * w + 1] = v0.im;
  }
}

// P_marked of every instance of a batch: one block per instance, one warp
// per marked string, chain products as above.
template <class S>
__global__ void batch_prob_kernel(const InstDesc* descs, int count, double* out) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  const InstDesc& d = descs[inst];
  const S* sites = (const S*)d.sites;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double part[32];
  double acc = 0.0;
  const int* chi = d.stats->chi;
  for (int t = warp; t < d.M; t += nw) {
    const unsigned long long x = d.marked[t];
    cx<double> v0 = mk<double>(lane == 0 ? 1.0 : 0.0, 0.0), v1 = mk<double>(0, 0);
    for (int l = 0; l < d.n; ++l) {
      const int cl = chi[l], cr = chi[l + 1];
      const S* A = sites + d.site_off[l];
      const int b = (int)((x >> l) & 1ull);
      cx<double> n0 = mk<double>(0, 0), n1 = mk<double>(0, 0);
      for (int i = 0; i < cl; ++i) {
        const cx<double> src = (i < 32) ? v0 : v1;
        cx<double> vi;
        vi.re = __shfl_sync(0xffffffffu, src.re, i & 31);
        vi.im = __shfl_sync(0xffffffffu, src.im, i & 31);
        if (lane < cr) n0 = cmac(n0, vi, ld<double>(A + (i * 2 + b) * cr + lane));
        if (lane + 32 < cr) n1 = cmac(n1, vi, ld<double>(A + (i * 2 + b) * cr + lane + 32));
      }
      v0 = n0;
      v1 = n1;
    }
    if (lane == 0) acc += abs2(v0);
  }
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += part[w];
    out[inst] = s;
  }
}

// ------------------------------------------------------------ sampling
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of
// (x0,x1,x2,x3) <- (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1,
// lo(M0 x0)) with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Perfect sampling on the right-canonical chain: one thread per shot, the
// conditional probabilities p_b = |v A_l[:, b, :]|^2 in FP64.
template <class S, int CH>
__global__ void sample_kernel(const InstDesc* descs, int inst, long long shots, unsigned long long seed,
                              unsigned long long* out, double* margin) {
  const long long shot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (shot >= shots) return;
  const InstDesc& d = descs[inst];
  const S* sites = (const S*)d.sites;
  const int* chi = d.stats->chi;
  cx<double> v[CH], w0[CH], w1[CH];
  v[0] = mk<double>(1.0, 0.0);
  unsigned long long bits = 0;
  double mg = 1e300;
  for (int l = 0; l < d.n; ++l) {
    const int cl = chi[l], cr = chi[l + 1];
    const S* A = sites + d.site_off[l];
    double p0 = 0.0, p1 = 0.0;
    for (int j = 0; j < cr; ++j) {
      cx<double> a0 = mk<double>(0, 0), a1 = mk<double>(0, 0);
      for (int i = 0; i < cl; ++i) {
        a0 = cmac(a0, v[i], ld<double>(A + (i * 2) * cr + j));
        a1 = cmac(a1, v[i], ld<double>(A + (i * 2 + 1) * cr + j));
      }
      w0[j] = a0;
      w1[j] = a1;
      p0 += abs2(a0);
      p1 += abs2(a1);
    }
    unsigned long long c[4] = {(unsigned long long)shot, (unsigned long long)l, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
    const double u = (double)(c[0] >> 11) * 0x1.0p-53;
    const double tot = p0 + p1;
    const int b = (u * tot >= p0) ? 1 : 0;
    if (margin) mg = fmin(mg, fabs(u - p0 / tot));
    bits |= (unsigned long long)b << l;
    const double inv = rsqrt(b ? p1 : p0);
    for (int j = 0; j < cr; ++j) v[j] = cscale(b ? w1[j] : w0[j], inv);
  }
  out[shot] = bits;
  if (margin) margin[shot] = mg;
}

// Copy the chain of instance src[i] into the slab of dst[i] (checkpoints),
// i = blockIdx.y.
template <class S>
__global__ void copy_sites_kernel(const InstDesc* srcs, const InstDesc* dsts) {
  const InstDesc* src = srcs + blockIdx.y;
  const InstDesc* dst = dsts + blockIdx.y;
  const long long total = src->site_off[src->n];
  const S* a = (const S*)src->sites;
  S* b = (S*)dst->sites;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = a[e];
  if (blockIdx.x == 0) {
    const int* c0 = src->stats->chi;
    int* c1 = dst->stats->chi;
    for (int l = threadIdx.x; l <= src->n; l += blockDim.x) {
      c1[l] = c0[l];
      dst->stats->jrank[0][l] = 0;  // the copy starts without cached rotations
      dst->stats->jrank[1][l] = 0;
    }
    if (threadIdx.x == 0) {
      dst->stats->status = src->stats->status;
      dst->stats->log_norm = src->stats->log_norm;
    }
  }
}

// ------------------------------------------------------------ launchers
template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::init(const InstDesc* d_desc, int count, cudaStream_t stream) {
  init_kernel<S><<<count, 64, 0, stream>>>(d_desc, count);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::iterate(const InstDesc* d_desc, int count, int* d_queue, int threads, size_t smem,
                                          int grid, cudaStream_t stream, int cluster) {
  if constexpr (std::is_same<T, double>::value) {
    if (cluster > 1 && count == 1) {
      // one instance on a cluster of `cluster` CTAs (one per SM)
      auto kc = iterate_kernel<T, S, CR, true>;
      cudaError_t e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cluster, 1, 1);
      cfg.blockDim = dim3(threads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, kc, d_desc, count, d_queue);
      if (e != cudaSuccess) return e;
      count_launch(1);
      return cudaGetLastError();
    }
  }
  auto k = iterate_kernel<T, S, CR, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, stream>>>(d_desc, count, d_queue);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::adjoint(const InstDesc* d_mu, const AdjArgs* d_args, int count, int threads,
                                          size_t smem, long long k_lo, long long k_hi, int project,
                                          cudaStream_t stream) {
  auto k = adjoint_kernel<T, S, CR>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<count, threads, smem, stream>>>(d_mu, d_args, k_lo, k_hi, project);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::amplitudes(const InstDesc* d_desc, int inst, const unsigned long long* d_bits,
                                             int nbits, double* d_out, cudaStream_t stream) {
  const int warps = 4;
  const int grid = (nbits + warps - 1) / warps;
  amplitude_kernel<S><<<grid, 32 * warps, 0, stream>>>(d_desc, inst, d_bits, nbits, d_out);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::batch_prob(const InstDesc* d_desc, int count, double* d_p, cudaStream_t stream) {
  batch_prob_kernel<S><<<count, 128, 0, stream>>>(d_desc, count, d_p);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::sample(const InstDesc* d_desc, int inst, int chmax, long long shots,
                                         unsigned long long seed, unsigned long long* d_bits, double* d_margin,
                                         cudaStream_t stream) {
  const int threads = 128;
  const long long grid = (shots + threads - 1) / threads;
  if (chmax <= 4)
    sample_kernel<S, 4><<<(unsigned)grid, threads, 0, stream>>>(d_desc, inst, shots, seed, d_bits, d_margin);
  else if (chmax <= 16)
    sample_kernel<S, 16><<<(unsigned)grid, threads, 0, stream>>>(d_desc, inst, shots, seed, d_bits, d_margin);
  else if (chmax <= 64)
    sample_kernel<S, 64><<<(unsigned)grid, threads, 0, stream>>>(d_desc, inst, shots, seed, d_bits, d_margin);
  else
    return cudaErrorInvalidValue;
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::circuit(const InstDesc* d_desc, const GateOp* d_gates, long long count,
                                          long long repeat, int threads, size_t smem, cudaStream_t stream) {
  auto k = circuit_kernel<T, S, CR>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<1, threads, smem, stream>>>(d_desc, d_gates, count, repeat);
  count_launch(1);
  return cudaGetLastError();
}

template <class T, class S, class CR>
cudaError_t FormLaunch<T, S, CR>::copy_sites(const InstDesc* d_src, const InstDesc* d_dst, int count,
                                             cudaStream_t stream) {
  copy_sites_kernel<S><<<dim3(count > 1 ? 4 : 32, count), 256, 0, stream>>>(d_src, d_dst);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace gmps
