// Iterative Grover on a dense statevector (include/grover_sv.h): the
// statevector backend of Sec. III-B-1 running the iterative method of
// Sec. III-A.  One streaming pass per iteration over the 2^n amplitudes.
//
// With u = O(phi) v and S(u) = sum_x u(x), the diffusion D(psi) = (1 -
// e^{i psi})|s><s| - I gives v'(x) = c - u(x), c = (1 - e^{i psi}) S(u) / N,
// and S(u) = S(v) + (e^{i phi} - 1) sum_w v(w).  A pass therefore needs only
// the previous pass's total S(v) and the M marked amplitudes v(w): every
// block computes c from them, streams v'(x) = c - v(x) over its part of the
// vector (the unmarked update, which is also right for every index until the
// marked ones are patched) and accumulates sum_x v'(x).  The last block to
// finish (an atomic ticket, no waiting) folds the per-block partial sums in a
// fixed order, patches the marked entries to c - e^{i phi} v(w), adds their
// correction (1 - e^{i phi}) v(w) to the total, and records the new total,
// the new marked amplitudes (double-buffered by iteration parity) and the
// iteration count for the next pass.  The iteration index lives in device
// memory, so every launch is identical and k launches replay from a CUDA
// graph.  Coefficients, block sums and totals are FP64.
//
// On this part the FP64 pipe (measured 1.06 TFLOP/s for the chip) would bind
// a pass that spends four FP64 additions per amplitude (the update and the
// running sum): 32 bytes per 4 DADDs is ~4.2 TB/s.  So each thread keeps its
// running sum on the FP32 pipes instead: every FP64 value is split exactly by
// bit manipulation into a truncated FP32 head (24 significant bits) and the
// round-to-nearest FP32 value of the remainder (error below 2^-48 |v|,
// unbiased); heads accumulate with Knuth's TwoSum (error-free), remainders
// with plain FP32 adds, and the thread's three FP32 partials are added in
// FP64 once at the end.  The complex128 update c - v stays FP64 (two DADDs
// per amplitude); the complex64 form updates in FP32 with c as a double-word
// pair (c_hi + c_lo), one rounding per stored value, and never touches the
// FP64 pipe in its loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/grover_sv.h"
#include "gmps_internal.h"

namespace gmps {
void set_last_error(const std::string& msg);
}

namespace {

using gmps::count_launch;

constexpr int kSvThreads = 256;
constexpr int kSvUnroll = 4;   // independent loads in flight per thread
constexpr int kGraphLaunches = 64;

// Device-side state of one statevector besides the amplitudes.
struct SvState {
  unsigned long long* marked;  // M strings
  double2* mk;                 // [2][M] marked amplitudes, indexed by iteration parity
  double2* total;              // [2] sum_x v(x), indexed by iteration parity
  double2* part;               // [grid] per-block partial sums of the current pass
  unsigned int* ticket;        // blocks finished in the current pass
  long long* iter;             // iterations applied since reset
  const double* const* phase;  // [2]: this call's phi, psi arrays (or null = pi)
  long long* phase_base;       // iteration index of this call's first phase
  long long N;
  int M;
  int grid;
};

__device__ __forceinline__ double2 ld_amp(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_amp(const float2* p) {
  const float2 v = __ldcs(p);
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ void st_amp(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_amp(float2* p, double2 v) { __stcs(p, make_float2((float)v.x, (float)v.y)); }
// a stored value as FP64, and an FP64 value known to be a stored value back
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 narrow(double2 v, const double2*) { return v; }
__device__ __forceinline__ float2 narrow(double2 v, const float2*) { return make_float2((float)v.x, (float)v.y); }
// the value as stored (rounded to the storage type)
__device__ __forceinline__ double2 as_stored(double2 v, const double2*) { return v; }
__device__ __forceinline__ double2 as_stored(double2 v, const float2*) {
  return make_double2((double)(float)v.x, (double)(float)v.y);
}

__device__ __forceinline__ void phases_of(const SvState& s, long long it, double& cphi, double& sphi, double& cpsi,
                                          double& spsi) {
  cphi = -1.0, sphi = 0.0, cpsi = -1.0, spsi = 0.0;
  const long long j = it - *s.phase_base;
  if (s.phase[0]) sincos(s.phase[0][j], &sphi, &cphi);
  if (s.phase[1]) sincos(s.phase[1][j], &spsi, &cpsi);
}

// FP32 running sum of FP64 values (see the file comment): TwoSum of the heads,
// plain sum of the remainders.
struct Acc32 {
  float s = 0.f, e = 0.f, r = 0.f;
  __device__ __forceinline__ void add_f32(float v) {
    const float t = __fadd_rn(s, v);
    const float z = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(v, z)));
    s = t;
  }
  __device__ __forceinline__ void add(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned E = (hi >> 20) & 0x7ffu;
    if (E < 1023u - 100u) return;  // |x| < 2^-100: below every sum this pass forms
    // head: the top 24 significant bits, exactly an FP32 value
    const unsigned m = ((hi & 0xfffffu) << 3) | ((unsigned)b >> 29);
    add_f32(__uint_as_float((hi & 0x80000000u) | ((E - 1023u + 127u) << 23) | m));
    // remainder: the low 29 bits times 2^(E-1075), rounded to nearest FP32
    const float low = __uint2float_rn((unsigned)b & 0x1fffffffu);
    const int ex = (int)E - 1075;  // >= -198: scale in two exact steps
    const float sc1 = __uint_as_float((unsigned)(ex / 2 + 127) << 23);
    const float sc2 = __uint_as_float((unsigned)(ex - ex / 2 + 127) << 23);
    const float rv = __fmul_rn(__fmul_rn(low, sc1), sc2);
    r = __fadd_rn(r, (hi & 0x80000000u) ? -rv : rv);
  }
  __device__ __forceinline__ double value() const { return ((double)s + (double)e) + (double)r; }
};

// Block-wide FP64 complex sum in a fixed order (warp shuffles, then warp 0).
__device__ __forceinline__ double2 block_sum(double2 a, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = a;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : make_double2(0.0, 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
      r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
    }
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// v -> c - v in the storage type: FP64 for complex128; for complex64 in FP32
// with c = c_hi + c_lo (double-word), rounded once.
template <class S>
struct Upd;
template <>
struct Upd<double2> {
  double2 c;
  __device__ explicit Upd(double2 c_) : c(c_) {}
  __device__ __forceinline__ double2 operator()(double2 x) const { return make_double2(c.x - x.x, c.y - x.y); }
};
template <>
struct Upd<float2> {
  float hr, lr, hi_, li;
  __device__ explicit Upd(double2 c) {
    hr = (float)c.x;
    lr = (float)(c.x - (double)hr);
    hi_ = (float)c.y;
    li = (float)(c.y - (double)hi_);
  }
  __device__ __forceinline__ float2 operator()(float2 x) const {
    return make_float2(__fadd_rn(__fsub_rn(hr, x.x), lr), __fadd_rn(__fsub_rn(hi_, x.y), li));
  }
};
__device__ __forceinline__ void acc_add(Acc32& ar, Acc32& ai, double2 y) {
  ar.add(y.x);
  ai.add(y.y);
}
__device__ __forceinline__ void acc_add(Acc32& ar, Acc32& ai, float2 y) {
  ar.add_f32(y.x);
  ai.add_f32(y.y);
}

template <class S>
__global__ void __launch_bounds__(kSvThreads) sv_pass(S* v, SvState s) {
  __shared__ double2 sh[32];
  __shared__ double2 c_sh;
  __shared__ int last_sh;
  const long long it = *s.iter;
  const int par = (int)(it & 1);
  if (threadIdx.x == 0) {
    double cphi, sphi, cpsi, spsi;
    phases_of(s, it, cphi, sphi, cpsi, spsi);
    // S(u) = S(v) + (e^{i phi} - 1) sum_w v(w)
    double wr = 0.0, wi = 0.0;
    const double2* mk = s.mk + par * s.M;
    for (int t = 0; t < s.M; ++t) {
      wr += mk[t].x;
      wi += mk[t].y;
    }
    const double er = cphi - 1.0, ei = sphi;
    const double2 tot = s.total[par];
    const double ur = tot.x + er * wr - ei * wi, ui = tot.y + er * wi + ei * wr;
    // c = (1 - e^{i psi}) S(u) / N
    const double fr = 1.0 - cpsi, fi = -spsi, invN = 1.0 / (double)s.N;
    c_sh = make_double2((fr * ur - fi * ui) * invN, (fr * ui + fi * ur) * invN);
  }
  __syncthreads();
  const double2 c = c_sh;
  // stream v(x) <- c - v(x), summing the stored values on the FP32 pipes
  Acc32 ar, ai;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Upd<S> up(c);
  for (; i + (kSvUnroll - 1) * stride < s.N; i += kSvUnroll * stride) {
    S x[kSvUnroll];
#pragma unroll
    for (int u = 0; u < kSvUnroll; ++u) x[u] = __ldcs(v + i + u * stride);
#pragma unroll
    for (int u = 0; u < kSvUnroll; ++u) {
      const S y = up(x[u]);
      __stcs(v + i + u * stride, y);
      acc_add(ar, ai, y);
    }
  }
  for (; i < s.N; i += stride) {
    const S y = up(__ldcs(v + i));
    __stcs(v + i, y);
    acc_add(ar, ai, y);
  }
  const double2 acc = make_double2(ar.value(), ai.value());
  const double2 bs = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    s.part[blockIdx.x] = bs;
    __threadfence();
    last_sh = atomicAdd(s.ticket, 1u) == (unsigned)(gridDim.x - 1);
  }
  __syncthreads();
  if (!last_sh) return;
  // ---- last block: fold the partial sums in block order, patch the marked entries
  __threadfence();
  double2 a = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double2 p = __ldcg(s.part + b);
    a.x += p.x;
    a.y += p.y;
  }
  const double2 tot = block_sum(a, sh);
  if (threadIdx.x == 0) {
    double cphi, sphi, cpsi, spsi;
    phases_of(s, it, cphi, sphi, cpsi, spsi);
    double tr = tot.x, ti = tot.y;
    const double2* mk = s.mk + par * s.M;
    double2* mk_next = s.mk + (par ^ 1) * s.M;
    for (int t = 0; t < s.M; ++t) {
      const double2 w = mk[t];
      // v'(w) = c - e^{i phi} v(w); the pass wrote c - v(w)
      const double2 y = make_double2(c.x - (cphi * w.x - sphi * w.y), c.y - (cphi * w.y + sphi * w.x));
      S* dst = v + s.marked[t];
      const double2 old = widen(up(narrow(w, v)));  // exactly what the pass stored there
      st_amp(dst, y);
      const double2 ys = as_stored(y, v);
      mk_next[t] = ys;
      tr += ys.x - old.x;
      ti += ys.y - old.y;
    }
    s.total[par ^ 1] = make_double2(tr, ti);
    *s.iter = it + 1;
    *s.ticket = 0u;
    __threadfence();
  }
}

template <class S>
__global__ void sv_init(S* v, SvState s) {
  const double a = rsqrt((double)s.N);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.N; i += stride)
    st_amp(v + i, make_double2(a, 0.0));
  if (blockIdx.x == 0) {
    const double2 as = as_stored(make_double2(a, 0.0), v);
    for (int t = threadIdx.x; t < s.M; t += blockDim.x) s.mk[t] = as;
    if (threadIdx.x == 0) {
      s.total[0] = make_double2(as.x * (double)s.N, 0.0);
      *s.iter = 0;
      *s.ticket = 0u;
      *s.phase_base = 0;
    }
  }
}

template <class S>
__global__ void sv_gather(const S* v, const unsigned long long* idx, int cnt, double2* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cnt) out[t] = ld_amp(v + idx[t]);
}

gmps_status fail(gmps_status st, const std::string& msg) {
  gmps::set_last_error(msg);
  return st;
}
gmps_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GMPS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define SV_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct gsv_ctx {
  int n = 0, M = 0, dtype = 0;
  long long N = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* amps = nullptr;
  char* aux = nullptr;
  SvState s{};
  const double** d_phase = nullptr;  // device [2]
  double* d_ph = nullptr;            // device phases of the current call
  size_t ph_cap = 0;
  double2* d_gather = nullptr;       // M + 1
  unsigned long long* d_q = nullptr; // M + 1 query indices
  cudaGraphExec_t graph = nullptr;
  long long applied = 0;
};

static size_t elem_bytes(int dtype) { return dtype == GMPS_C64_F64SVD ? sizeof(float2) : sizeof(double2); }

static cudaError_t sv_launch_pass(gsv_ctx* h) {
  if (h->dtype == GMPS_C64_F64SVD)
    sv_pass<float2><<<h->s.grid, kSvThreads, 0, h->stream>>>((float2*)h->amps, h->s);
  else
    sv_pass<double2><<<h->s.grid, kSvThreads, 0, h->stream>>>((double2*)h->amps, h->s);
  count_launch(1);
  return cudaGetLastError();
}

extern "C" {

gmps_status grover_sv_bytes(int n, int dtype, size_t* bytes) {
  if (!bytes) return fail(GMPS_ERR_ARG, "bytes is NULL");
  if (n < 1 || n > 36) return fail(GMPS_ERR_ARG, "n must be in [1, 36]");
  if (dtype != GMPS_C128 && dtype != GMPS_C64_F64SVD) return fail(GMPS_ERR_ARG, "dtype must be C128 or C64");
  *bytes = a256(elem_bytes(dtype) << n);
  return GMPS_OK;
}

gmps_status grover_sv_create(int n, const uint64_t* marked, int M, int dtype, void* cuda_stream, gsv_handle* out) {
  if (!out) return fail(GMPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 36) return fail(GMPS_ERR_ARG, "n must be in [1, 36]");
  if (M < 1 || M > 64) return fail(GMPS_ERR_ARG, "M must be in [1, 64]");
  if ((uint64_t)M >= (1ull << n)) return fail(GMPS_ERR_ARG, "M must be < 2^n");
  if (!marked) return fail(GMPS_ERR_ARG, "marked is NULL");
  if (dtype != GMPS_C128 && dtype != GMPS_C64_F64SVD) return fail(GMPS_ERR_ARG, "dtype must be C128 or C64");
  uint64_t sorted[64];
  for (int i = 0; i < M; ++i) {
    if (marked[i] >> n) return fail(GMPS_ERR_ARG, "marked string has bits >= n");
    sorted[i] = marked[i];
  }
  std::sort(sorted, sorted + M);
  for (int i = 1; i < M; ++i)
    if (sorted[i] == sorted[i - 1]) return fail(GMPS_ERR_ARG, "duplicate marked string");
  gsv_ctx* h = new gsv_ctx();
  h->n = n;
  h->M = M;
  h->dtype = dtype;
  h->N = 1ll << n;
  h->stream = (cudaStream_t)cuda_stream;
  if (!h->stream) {
    if (cudaStreamCreate(&h->stream) != cudaSuccess) {
      delete h;
      return fail(GMPS_ERR_CUDA, "stream creation failed");
    }
    h->own_stream = true;  // graph capture needs a non-legacy stream
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // 8 blocks of 256 threads per SM, fewer when the vector is small
  const long long per_block = (long long)kSvThreads * kSvUnroll * 2;
  h->s.grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8, (h->N + per_block - 1) / per_block));
  h->s.N = h->N;
  h->s.M = M;
  const size_t vb = a256(elem_bytes(dtype) * (size_t)h->N);
  cudaError_t e = gmps::dev_malloc((void**)&h->amps, vb);
  if (e != cudaSuccess) {
    grover_sv_destroy(h);
    return fail(GMPS_ERR_OOM, std::string("statevector allocation: ") + cudaGetErrorString(e));
  }
  const size_t aux = a256(sizeof(unsigned long long) * M) + a256(sizeof(double2) * 2 * M) +
                     a256(sizeof(double2) * 2) + a256(sizeof(double2) * h->s.grid) + a256(sizeof(unsigned)) +
                     a256(sizeof(long long)) + a256(sizeof(double*) * 2) + a256(sizeof(long long)) +
                     a256(sizeof(double2) * (M + 1)) + a256(sizeof(unsigned long long) * (M + 1));
  e = gmps::dev_malloc((void**)&h->aux, aux);
  if (e != cudaSuccess) {
    grover_sv_destroy(h);
    return fail(GMPS_ERR_OOM, "statevector scratch");
  }
  char* p = h->aux;
  h->s.marked = (unsigned long long*)p;  p += a256(sizeof(unsigned long long) * M);
  h->s.mk = (double2*)p;                 p += a256(sizeof(double2) * 2 * M);
  h->s.total = (double2*)p;              p += a256(sizeof(double2) * 2);
  h->s.part = (double2*)p;               p += a256(sizeof(double2) * h->s.grid);
  h->s.ticket = (unsigned*)p;            p += a256(sizeof(unsigned));
  h->s.iter = (long long*)p;             p += a256(sizeof(long long));
  h->d_phase = (const double**)p;        p += a256(sizeof(double*) * 2);
  h->s.phase = h->d_phase;
  h->s.phase_base = (long long*)p;       p += a256(sizeof(long long));
  h->d_gather = (double2*)p;             p += a256(sizeof(double2) * (M + 1));
  h->d_q = (unsigned long long*)p;
  e = cudaMemcpyAsync(h->s.marked, marked, sizeof(uint64_t) * M, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q, marked, sizeof(uint64_t) * M, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    grover_sv_destroy(h);
    return cuda_fail(e, "upload marked");
  }
  gmps_status st = grover_sv_reset(h);
  if (st) {
    grover_sv_destroy(h);
    return st;
  }
  *out = h;
  return GMPS_OK;
}

gmps_status grover_sv_reset(gsv_handle h) {
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  const double* none[2] = {nullptr, nullptr};
  SV_TRY(cudaMemcpyAsync((void*)h->d_phase, none, sizeof(none), cudaMemcpyHostToDevice, h->stream));
  const int grid = std::min(h->s.grid, 1024);
  if (h->dtype == GMPS_C64_F64SVD)
    sv_init<float2><<<grid, kSvThreads, 0, h->stream>>>((float2*)h->amps, h->s);
  else
    sv_init<double2><<<grid, kSvThreads, 0, h->stream>>>((double2*)h->amps, h->s);
  count_launch(1);
  SV_TRY(cudaGetLastError());
  SV_TRY(cudaStreamSynchronize(h->stream));
  h->applied = 0;
  return GMPS_OK;
}

gmps_status grover_sv_iterate(gsv_handle h, int64_t k, const double* host_phi, const double* host_psi) {
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  if (k < 0) return fail(GMPS_ERR_ARG, "k must be >= 0");
  if (k == 0) return GMPS_OK;
  for (int64_t i = 0; host_phi && i < k; ++i)
    if (!std::isfinite(host_phi[i])) return fail(GMPS_ERR_ARG, "non-finite phase");
  for (int64_t i = 0; host_psi && i < k; ++i)
    if (!std::isfinite(host_psi[i])) return fail(GMPS_ERR_ARG, "non-finite phase");
  const double* dp[2] = {nullptr, nullptr};
  if (host_phi || host_psi) {
    if (h->ph_cap < (size_t)k) {
      if (h->d_ph) cudaFree(h->d_ph);
      h->d_ph = nullptr;
      h->ph_cap = 0;
      if (gmps::dev_malloc((void**)&h->d_ph, sizeof(double) * 2 * k) != cudaSuccess)
        return fail(GMPS_ERR_OOM, "phase buffer");
      h->ph_cap = k;
    }
    if (host_phi) {
      SV_TRY(cudaMemcpyAsync(h->d_ph, host_phi, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
      dp[0] = h->d_ph;
    }
    if (host_psi) {
      SV_TRY(cudaMemcpyAsync(h->d_ph + h->ph_cap, host_psi, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
      dp[1] = h->d_ph + h->ph_cap;
    }
  }
  const long long base = h->applied;
  SV_TRY(cudaMemcpyAsync((void*)h->d_phase, dp, sizeof(dp), cudaMemcpyHostToDevice, h->stream));
  SV_TRY(cudaMemcpyAsync(h->s.phase_base, &base, sizeof(base), cudaMemcpyHostToDevice, h->stream));
  int64_t left = k;
  if (k >= kGraphLaunches) {
    if (!h->graph) {
      cudaGraph_t g;
      SV_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = cudaSuccess;
      for (int i = 0; i < kGraphLaunches && le == cudaSuccess; ++i) le = sv_launch_pass(h);
      cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
      if (le != cudaSuccess) return cuda_fail(le, "statevector pass");
      if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
      count_launch(-kGraphLaunches);  // counted on replay
      ce = cudaGraphInstantiate(&h->graph, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    }
    while (left >= kGraphLaunches) {
      SV_TRY(cudaGraphLaunch(h->graph, h->stream));
      count_launch(kGraphLaunches);
      left -= kGraphLaunches;
    }
  }
  for (; left > 0; --left) SV_TRY(sv_launch_pass(h));
  h->applied += k;
  SV_TRY(cudaStreamSynchronize(h->stream));
  return GMPS_OK;
}

static gmps_status sv_gather_host(gsv_handle h, int cnt, double2* out) {
  if (h->dtype == GMPS_C64_F64SVD)
    sv_gather<float2><<<1, 128, 0, h->stream>>>((const float2*)h->amps, h->d_q, cnt, h->d_gather);
  else
    sv_gather<double2><<<1, 128, 0, h->stream>>>((const double2*)h->amps, h->d_q, cnt, h->d_gather);
  count_launch(1);
  SV_TRY(cudaGetLastError());
  SV_TRY(cudaMemcpyAsync(out, h->d_gather, sizeof(double2) * cnt, cudaMemcpyDeviceToHost, h->stream));
  SV_TRY(cudaStreamSynchronize(h->stream));
  return GMPS_OK;
}

gmps_status grover_sv_amplitude(gsv_handle h, uint64_t bits, double* re, double* im) {
  if (!h || !re || !im) return fail(GMPS_ERR_ARG, "NULL argument");
  if (bits >> h->n) return fail(GMPS_ERR_ARG, "bits >= 2^n");
  // the query slot after the M marked strings
  SV_TRY(cudaMemcpyAsync(h->d_q + h->M, &bits, sizeof(bits), cudaMemcpyHostToDevice, h->stream));
  double2 o[65];
  if (h->dtype == GMPS_C64_F64SVD)
    sv_gather<float2><<<1, 32, 0, h->stream>>>((const float2*)h->amps, h->d_q + h->M, 1, h->d_gather);
  else
    sv_gather<double2><<<1, 32, 0, h->stream>>>((const double2*)h->amps, h->d_q + h->M, 1, h->d_gather);
  count_launch(1);
  SV_TRY(cudaGetLastError());
  SV_TRY(cudaMemcpyAsync(o, h->d_gather, sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  SV_TRY(cudaStreamSynchronize(h->stream));
  *re = o[0].x;
  *im = o[0].y;
  return GMPS_OK;
}

gmps_status grover_sv_prob_marked(gsv_handle h, double* p) {
  if (!h || !p) return fail(GMPS_ERR_ARG, "NULL argument");
  double2 o[64];
  gmps_status st = sv_gather_host(h, h->M, o);
  if (st) return st;
  double acc = 0.0;
  for (int t = 0; t < h->M; ++t) acc += o[t].x * o[t].x + o[t].y * o[t].y;
  *p = acc;
  return GMPS_OK;
}

gmps_status grover_sv_export(gsv_handle h, double* host_out, size_t capacity) {
  if (!h || !host_out) return fail(GMPS_ERR_ARG, "NULL argument");
  if (capacity < 2 * (size_t)h->N) return fail(GMPS_ERR_ARG, "export buffer too small");
  if (h->dtype == GMPS_C64_F64SVD) {
    std::vector<float2> tmp(h->N);
    SV_TRY(cudaMemcpyAsync(tmp.data(), h->amps, sizeof(float2) * h->N, cudaMemcpyDeviceToHost, h->stream));
    SV_TRY(cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < h->N; ++i) {
      host_out[2 * i] = tmp[i].x;
      host_out[2 * i + 1] = tmp[i].y;
    }
  } else {
    SV_TRY(cudaMemcpyAsync(host_out, h->amps, sizeof(double2) * h->N, cudaMemcpyDeviceToHost, h->stream));
    SV_TRY(cudaStreamSynchronize(h->stream));
  }
  return GMPS_OK;
}

gmps_status grover_sv_destroy(gsv_handle h) {
  if (!h) return GMPS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->amps) cudaFree(h->amps);
  if (h->aux) cudaFree(h->aux);
  if (h->d_ph) cudaFree(h->d_ph);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return GMPS_OK;
}

}  // extern "C"
