// C ABI of libgrover_mps.so (declared in include/grover_mps.h): argument
// validation, the per-handle device arena, launch configuration and status
// propagation.  All compute runs in gmps_kernels.cu.
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/grover_mps.h"
#include "gmps_internal.h"

using namespace gmps;

namespace gmps {
long long launches_so_far();
}

static thread_local std::string g_err;

namespace gmps {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace gmps

static gmps_status fail(gmps_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
static gmps_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GMPS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CUDA_TRY(x)                                   \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);  \
  } while (0)

static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// Rank rule sigma_i > max(tol, floor) sigma_0 (and the rank-revealing QR's
// stop), with the floor set above the rounding noise that a contraction + QR
// + Jacobi chain leaves in a rank-deficient direction, so that the noise is
// never kept as a Schmidt direction:
//  * FP64: max(m, n) times four units (2^-50) -- a noise row of 2.7 units was
//    measured on a 2 x 2 step, whose max(m, n) = 2 would otherwise put the
//    floor at 2 units;
//  * double-word: max(m, n) 2^-42;
//  * complex64 with FP64 QR/SVD: a fixed 2^-22.  Its noise is the FP32
//    storage and contraction seen by FP64 linear algebra; rounding-noise
//    singular values reached 2^-26.4 sigma_0 over 1500 iterations of an
//    n = 36, M = 16 instance, while the marked component's Schmidt values
//    start near 2^{1-n/2} (2^-17 at n = 36).  The storage-unit rule
//    max(m, n) 2^-23 reached those values and truncated the marked component
//    away at n = 36.
struct RankRule {
  double eps;
  int dim;  // 1: floor = max(m, n) eps
};
static RankRule rank_rule_for(int dtype) {
  if (dtype == GMPS_C64_F64SVD) return {2.384185791015625e-07, 0};
  if (dtype == GMPS_DW) return {2.2737367544323206e-13, 1};
  return {8.881784197001252e-16, 1};
}

// ---------------------------------------------------------------- sizing
// Launch and storage plan of one instance (host only; fixed size, so that
// planning allocates nothing).
struct Plan {
  int chicap, xcap, rcap, threads, resident;
  int cluster;               // CTAs sharing a single instance's large QR steps (1: none)
  size_t smem, site_elems, elem_bytes;
  size_t work_bytes;         // device work area for the QR matrices (0: in shared memory)
  size_t jc_bytes;           // per-site cache of Jacobi rotations (InstDesc::jcache), 0: none
  int jbanks;                // its banks (sweep pairs per iteration)
  long long off[kMaxN + 1];  // slot offsets, n+1 used
};

static int xcap_for(int apply, int M, int chicap) {
  if (apply == GMPS_APPLY_MPO) return (M + 1) * chicap;
  if (apply == GMPS_APPLY_GATES) return 2 * chicap;
  if (apply == GMPS_APPLY_SPLIT) return chicap + M;
  return chicap + M + 1;
}

// Rank capacity of a QR-sweep bond: the Schmidt rank of the state a QR step
// factors.  O|psi> = |psi> + sum_w c_w |w> has rank <= chi + M and the
// diffusion MPO of bond 2 at most doubles it, plus two for rounding-noise
// directions at the rank-revealing QR's floor; the direct sums are bounded by
// their expanded bond.  A rank above it raises GMPS_ERR_CAPACITY.
static int rcap_for(int apply, int M, int chicap, int xcap) {
  if (apply == GMPS_APPLY_MPO) return std::min(xcap, std::max(chicap + M, 2 * chicap) + 2);
  return xcap;
}

// CTA size from the expanded bond; at least two warps, so that the small
// register-resident QR steps hand their Q formation to warp 1
static int auto_threads(int xcap) {
  if (xcap <= 16) return 64;
  if (xcap <= 32) return 128;
  return 256;
}

static gmps_status validate(const gmps_config* c) {
  if (!c) return fail(GMPS_ERR_ARG, "config is NULL");
  if (c->n < 1 || c->n > 64) return fail(GMPS_ERR_ARG, "n must be in [1, 64]");
  if (c->M < 1) return fail(GMPS_ERR_ARG, "M must be >= 1");
  if (c->n < 64 && (uint64_t)c->M >= (1ull << c->n)) return fail(GMPS_ERR_ARG, "M must be < 2^n");
  if (c->M > kMaxMarked) return fail(GMPS_ERR_UNSUPPORTED, "M above the built maximum (64)");
  if (!c->marked) return fail(GMPS_ERR_ARG, "marked is NULL");
  uint64_t sorted[kMaxMarked];
  for (int i = 0; i < c->M; ++i) {
    uint64_t w = c->marked[i];
    if (c->n < 64 && (w >> c->n) != 0) return fail(GMPS_ERR_ARG, "marked string has bits >= n");
    sorted[i] = w;
  }
  std::sort(sorted, sorted + c->M);
  for (int i = 1; i < c->M; ++i)
    if (sorted[i] == sorted[i - 1]) return fail(GMPS_ERR_ARG, "duplicate marked string");
  if (c->chi_max < 1) return fail(GMPS_ERR_ARG, "chi_max must be >= 1");
  if (!(c->tol >= 0.0) || !std::isfinite(c->tol)) return fail(GMPS_ERR_ARG, "tol must be finite and >= 0");
  if (c->dtype != GMPS_C128 && c->dtype != GMPS_C64_F64SVD && c->dtype != GMPS_DW)
    return fail(GMPS_ERR_ARG, "unknown dtype");
  if (c->apply < 0 || c->apply > 3) return fail(GMPS_ERR_ARG, "apply must be 0, 1, 2 or 3");
  if (c->threads != 0 && (c->threads % 32 != 0 || c->threads < 32 || c->threads > 256))
    return fail(GMPS_ERR_ARG, "threads must be a multiple of 32 in [32, 256]");
  if (c->max_sweeps < 0) return fail(GMPS_ERR_ARG, "max_sweeps must be >= 0");
  return GMPS_OK;
}

static gmps_status make_plan_for(const gmps_config* c, bool allow_resident, Plan* P) {
  const int smax = max_smem_optin();
  const size_t eb = storage_bytes(c->dtype), rb = linalg_real_bytes(c->dtype);
  // bond capacity: the exact rank bound M+1 plus headroom for rounding-noise
  // singular values above the rank rule (larger for complex64's FP32 noise)
  const int slacks[3] = {c->dtype == GMPS_C64_F64SVD ? c->M + 1 : 2, 2, 0};
  for (int si = 0; si < 3; ++si) {
    const int slack = slacks[si];
    // Grover states have Schmidt rank <= M + 1; gate-level circuits take chi_max
    int chicap = c->apply == GMPS_APPLY_GATES ? c->chi_max : std::min(c->chi_max, c->M + 1 + slack);
    // a bond never exceeds 2^floor(n/2)
    long long half = 1;
    for (int i = 0; i < c->n / 2 && half < chicap; ++i) half *= 2;
    chicap = (int)std::min<long long>(chicap, half);
    const int xcap = xcap_for(c->apply, c->M, chicap);
    const int rcap = rcap_for(c->apply, c->M, chicap, xcap);
    P->chicap = chicap;
    P->xcap = xcap;
    P->rcap = rcap;
    P->off[0] = 0;
    for (int l = 0; l < c->n; ++l) P->off[l + 1] = P->off[l] + slot_elems(l, c->n, rcap);
    P->site_elems = P->off[c->n];
    P->elem_bytes = eb;
    // the QR matrices in shared memory, else in a device work area
    bool work = false;
    SmemPlan sp = make_plan(c->n, c->M, xcap, chicap, rcap, rb, 0, false);
    if (sp.total > (size_t)smax) {
      sp = make_plan(c->n, c->M, xcap, chicap, rcap, rb, 0, true);
      if (sp.total > (size_t)smax) continue;
      work = true;
    }
    P->work_bytes = work ? sp.work_bytes : 0;
    // the precision forms keep each site's last Jacobi rotations, one bank
    // per sweep pair of an iteration (the fused and gate-level forms sweep
    // once per operator); the plain FP64 form always starts from the identity
    const int banks = (c->apply == GMPS_APPLY_FUSED || c->apply == GMPS_APPLY_GATES) ? 1 : 2;
    P->jbanks = banks;
    P->jc_bytes = (rcap > 2 && c->dtype != GMPS_C128)
                      ? (size_t)banks * c->n * ((size_t)rcap * rcap * 16 + 2 * sizeof(int) * rcap)
                      : 0;
    // a generic MPO with an expanded bond in the hundreds: its QR steps are
    // split over a cluster of CTAs when the instance runs alone (FP64 QR)
    P->cluster = (work && c->apply == GMPS_APPLY_MPO && c->dtype != GMPS_DW && xcap >= kClusterMinCols) ? kMaxCluster : 1;
    P->resident = 0;
    P->smem = sp.total;
    if (allow_resident) {
      SmemPlan sr = make_plan(c->n, c->M, xcap, chicap, rcap, rb, P->site_elems * eb, work);
      if (sr.total <= (size_t)smax) {
        P->resident = 1;
        P->smem = sr.total;
      }
    }
    P->threads = c->threads ? c->threads : auto_threads(xcap);
    return GMPS_OK;
  }
  return fail(GMPS_ERR_UNSUPPORTED, "working set exceeds shared memory for this (M, chi_max)");
}

// ---------------------------------------------------------------- handle
struct Slab {  // one chain + its descriptor, statistics and work area, carved from an arena
  InstDesc* d_desc = nullptr;
  long long* d_off = nullptr;
  DevStats* d_stats = nullptr;
  void* d_sites = nullptr;
  void* d_work = nullptr;
  void* d_jc = nullptr;  // Jacobi rotation cache (the handle's main chain only)
};

struct gmps_ctx {
  gmps_config cfg{};
  std::vector<uint64_t> marked;
  cudaStream_t stream = nullptr;
  int device = 0;
  Plan plan;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  InstDesc h{};
  Slab main;
  unsigned long long* d_marked = nullptr;
  unsigned long long* d_qbits = nullptr;  // M+1 query strings
  double* d_qout = nullptr;               // 2(M+1)
  InstDesc* d_cdesc = nullptr;            // gate-level circuits: the chain with the all-ones string
  unsigned long long* d_ones = nullptr;
  unsigned char* d_canary = nullptr;  // the arena's closing canary (last kCanaryBytes)
  GateOp* d_gates = nullptr;
  size_t gate_cap = 0;
  double* d_phase = nullptr;
  size_t phase_cap = 0;
  unsigned long long* d_sample = nullptr;
  double* d_margin = nullptr;
  size_t sample_cap = 0;
  int error = 0;
  long long iterations = 0;
  // differentiable form
  std::vector<double> phi_hist, psi_hist;
  std::vector<Slab> ckpt;          // ckpt[j] holds the state after j*every iterations
  Slab work;                       // segment recompute
  Slab costate;                    // adjoint chain
  int every = 8;
  int max_iters = 0;
  double* d_rec = nullptr;         // every * (M+1) complex
  double* d_grad = nullptr;        // 2 * max_iters
  double* d_ph_all = nullptr;      // 2 * max_iters
  AdjArgs* d_args = nullptr;       // [0] projection step, [1] segment steps
  char* diff_mem = nullptr;
  bool all_phases_explicit = true;
};

// forced device-allocation failures left (grover_mps_debug_fail_allocations)
static std::atomic<int> g_fail_allocs{0};

cudaError_t gmps::dev_malloc(void** p, size_t bytes) {
  int c = g_fail_allocs.load();
  while (c > 0 && !g_fail_allocs.compare_exchange_weak(c, c - 1)) {
  }
  if (c > 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

// A canary of 32 distinct 64-bit words closes every handle's arena; it is
// written at creation and compared after every call that synchronises, so a
// kernel writing past the instance's slabs shows as GMPS_ERR_STATE.
static constexpr size_t kCanaryBytes = 256;
static const unsigned long long* canary_words() {
  static unsigned long long w[kCanaryBytes / 8];
  static std::once_flag once;
  std::call_once(once, [] {
    for (size_t i = 0; i < kCanaryBytes / 8; ++i) w[i] = 0x9e3779b97f4a7c15ull * (i + 1) ^ 0xc0ffee0ddba11ull;
  });
  return w;
}

// NVTX range over one C-ABI call (visible to profilers; no cost otherwise)
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
};

static size_t slab_bytes(const gmps_config* c, const Plan& P) {
  return a256(sizeof(InstDesc)) + a256(sizeof(long long) * (c->n + 1)) + a256(sizeof(DevStats)) +
         a256(P.site_elems * P.elem_bytes) + a256(P.work_bytes);
}

static char* carve_slab(char* p, const gmps_config* c, const Plan& P, Slab* s) {
  s->d_desc = (InstDesc*)p;
  p += a256(sizeof(InstDesc));
  s->d_off = (long long*)p;
  p += a256(sizeof(long long) * (c->n + 1));
  s->d_stats = (DevStats*)p;
  p += a256(sizeof(DevStats));
  s->d_sites = p;
  p += a256(P.site_elems * P.elem_bytes);
  s->d_work = P.work_bytes ? p : nullptr;
  p += a256(P.work_bytes);
  return p;
}

static size_t arena_size(const gmps_config* c, const Plan& P) {
  return slab_bytes(c, P) + a256(P.jc_bytes) + kCanaryBytes + a256(sizeof(unsigned long long) * c->M) +
         a256(sizeof(unsigned long long) * (c->M + 1)) + a256(sizeof(double) * 2 * (c->M + 1)) +
         a256(sizeof(InstDesc)) + a256(sizeof(unsigned long long));
}

static InstDesc base_desc(const gmps_ctx* h, const Slab& s) {
  InstDesc d{};
  d.n = h->cfg.n;
  d.M = h->cfg.M;
  d.apply = h->cfg.apply;
  d.chi_max = h->cfg.chi_max;
  d.chicap = h->plan.chicap;
  d.xcap = h->plan.xcap;
  d.rcap = h->plan.rcap;
  d.work = s.d_work;
  d.jcache = s.d_jc;
  d.jbanks = h->plan.jbanks;
  d.cluster = h->plan.cluster;
  d.max_sweeps = h->cfg.max_sweeps ? h->cfg.max_sweeps : kDefaultMaxSweeps;
  d.resident = h->plan.resident;
  d.tol = h->cfg.tol;
  d.trunc_eps = rank_rule_for(h->cfg.dtype).eps;
  d.trunc_dim = rank_rule_for(h->cfg.dtype).dim;
  d.inv_sqrt_N = std::ldexp(1.0, -h->cfg.n / 2) * ((h->cfg.n & 1) ? std::sqrt(0.5) : 1.0);
  d.marked = h->d_marked;
  d.sites = s.d_sites;
  d.site_off = s.d_off;
  d.stats = s.d_stats;
  return d;
}

static gmps_status upload_slab(gmps_ctx* h, const Slab& s) {
  InstDesc d = base_desc(h, s);
  CUDA_TRY(cudaMemcpyAsync(s.d_off, h->plan.off, sizeof(long long) * (h->cfg.n + 1),
                           cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(s.d_desc, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(launch_init(s.d_desc, 1, h->cfg.dtype, 64, h->stream));
  return GMPS_OK;
}

static gmps_status check_device(gmps_ctx* h) {
  DevStats ds;
  unsigned long long can[kCanaryBytes / 8];
  CUDA_TRY(cudaMemcpyAsync(&ds, h->main.d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(can, h->d_canary, kCanaryBytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (memcmp(can, canary_words(), kCanaryBytes) != 0) {
    h->error = GMPS_ERR_STATE;
    return fail(GMPS_ERR_STATE, "arena canary overwritten: a write went past the instance's arena");
  }
  if (ds.status != 0) {
    h->error = ds.status;
    const char* what = ds.status == kDevNoConv   ? "Jacobi SVD did not converge"
                       : ds.status == kDevNumeric ? "non-finite or zero norm"
                       : ds.status == kDevCapacity ? "bond exceeded arena capacity"
                                                   : "device error";
    return fail((gmps_status)ds.status, what);
  }
  return GMPS_OK;
}

extern "C" {

const char* grover_mps_last_error(void) { return g_err.c_str(); }

gmps_status grover_mps_debug_fail_allocations(int count) {
  if (count < 0) return fail(GMPS_ERR_ARG, "count must be >= 0");
  g_fail_allocs.store(count);
  return GMPS_OK;
}

int64_t grover_mps_launch_count(void) { return gmps::launches_so_far(); }

gmps_status grover_mps_arena_bytes(const gmps_config* cfg, size_t* bytes) {
  gmps_status s = validate(cfg);
  if (s) return s;
  if (!bytes) return fail(GMPS_ERR_ARG, "bytes is NULL");
  Plan P;
  if ((s = make_plan_for(cfg, true, &P))) return s;
  *bytes = arena_size(cfg, P);
  return GMPS_OK;
}

gmps_status grover_mps_create_ex(const gmps_config* cfg, void* cuda_stream, gmps_handle* out) {
  CallRange range_("grover_mps_create_ex");
  if (!out) return fail(GMPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  gmps_status s = validate(cfg);
  if (s) return s;
  gmps_ctx* h = new gmps_ctx();
  h->cfg = *cfg;
  h->marked.assign(cfg->marked, cfg->marked + cfg->M);
  h->cfg.marked = h->marked.data();
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);
  if ((s = make_plan_for(&h->cfg, true, &h->plan))) {
    delete h;
    return s;
  }
  h->arena_bytes = arena_size(&h->cfg, h->plan);
  if (cfg->arena) {
    if (cfg->arena_bytes < h->arena_bytes) {
      delete h;
      return fail(GMPS_ERR_ARG, "caller arena smaller than grover_mps_arena_bytes");
    }
    if (((uintptr_t)cfg->arena) % 256 != 0) {
      delete h;
      return fail(GMPS_ERR_ARG, "caller arena must be 256-byte aligned");
    }
    h->arena = (char*)cfg->arena;
  } else {
    cudaError_t e = dev_malloc((void**)&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
      delete h;
      return fail(GMPS_ERR_OOM, std::string("arena allocation: ") + cudaGetErrorString(e));
    }
    h->own_arena = true;
  }
  char* p = carve_slab(h->arena, &h->cfg, h->plan, &h->main);
  h->main.d_jc = h->plan.jc_bytes ? p : nullptr;
  p += a256(h->plan.jc_bytes);
  h->d_marked = (unsigned long long*)p;
  p += a256(sizeof(unsigned long long) * cfg->M);
  h->d_qbits = (unsigned long long*)p;
  p += a256(sizeof(unsigned long long) * (cfg->M + 1));
  h->d_qout = (double*)p;
  p += a256(sizeof(double) * 2 * (cfg->M + 1));
  h->d_cdesc = (InstDesc*)p;
  p += a256(sizeof(InstDesc));
  h->d_ones = (unsigned long long*)p;
  h->d_canary = (unsigned char*)h->arena + h->arena_bytes - kCanaryBytes;
  cudaError_t e = cudaMemcpyAsync(h->d_canary, canary_words(), kCanaryBytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_marked, h->marked.data(), sizeof(uint64_t) * cfg->M, cudaMemcpyHostToDevice,
                        h->stream);
  if (e != cudaSuccess) {
    grover_mps_destroy(h);
    return cuda_fail(e, "upload marked");
  }
  h->h = base_desc(h, h->main);
  if ((s = upload_slab(h, h->main))) {
    grover_mps_destroy(h);
    return s;
  }
  if (cfg->differentiable) {
    h->every = cfg->checkpoint_every > 0 ? cfg->checkpoint_every : 8;
    h->max_iters = cfg->max_iters;
    if (h->max_iters < 1) {
      grover_mps_destroy(h);
      return fail(GMPS_ERR_ARG, "differentiable handles need max_iters >= 1");
    }
    const int nck = h->max_iters / h->every + 1;
    const size_t sb = slab_bytes(&h->cfg, h->plan);
    const size_t bytes = sb * (nck + 2) + a256(sizeof(double) * 2 * (cfg->M + 1) * h->every) +
                         2 * a256(sizeof(double) * 2 * h->max_iters) + a256(sizeof(AdjArgs) * 2);
    cudaError_t e2 = dev_malloc((void**)&h->diff_mem, bytes);
    if (e2 != cudaSuccess) {
      grover_mps_destroy(h);
      return fail(GMPS_ERR_OOM, "checkpoint storage");
    }
    char* q = h->diff_mem;
    h->ckpt.resize(nck);
    for (int j = 0; j < nck; ++j) q = carve_slab(q, &h->cfg, h->plan, &h->ckpt[j]);
    q = carve_slab(q, &h->cfg, h->plan, &h->work);
    q = carve_slab(q, &h->cfg, h->plan, &h->costate);
    h->d_rec = (double*)q;
    q += a256(sizeof(double) * 2 * (cfg->M + 1) * h->every);
    h->d_grad = (double*)q;
    q += a256(sizeof(double) * 2 * h->max_iters);
    h->d_ph_all = (double*)q;
    q += a256(sizeof(double) * 2 * h->max_iters);
    h->d_args = (AdjArgs*)q;
    for (int j = 0; j < nck && !s; ++j) s = upload_slab(h, h->ckpt[j]);
    if (!s) s = upload_slab(h, h->work);
    if (!s) s = upload_slab(h, h->costate);
    if (s) {
      grover_mps_destroy(h);
      return s;
    }
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    grover_mps_destroy(h);
    return cuda_fail(e, "create");
  }
  *out = h;
  return GMPS_OK;
}

gmps_status grover_mps_create(int n, const uint64_t* marked, int M, int dtype, int chi_max, double tol,
                              void* cuda_stream, gmps_handle* out) {
  gmps_config c{};
  c.n = n;
  c.M = M;
  c.marked = marked;
  c.dtype = dtype;
  c.apply = GMPS_APPLY_MPO;
  c.chi_max = chi_max;
  c.tol = tol;
  return grover_mps_create_ex(&c, cuda_stream, out);
}

gmps_status grover_mps_reset(gmps_handle h) {
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  h->error = 0;
  h->iterations = 0;
  h->phi_hist.clear();
  h->psi_hist.clear();
  h->all_phases_explicit = true;
  gmps_status s = upload_slab(h, h->main);
  if (s) return s;
  return GMPS_OK;
}

static gmps_status ensure_phase(gmps_ctx* h, size_t need) {
  if (h->phase_cap >= need) return GMPS_OK;
  if (h->d_phase) cudaFree(h->d_phase);
  h->d_phase = nullptr;
  size_t cap = std::max<size_t>(need, 1024);
  cudaError_t e = dev_malloc((void**)&h->d_phase, sizeof(double) * 2 * cap);
  if (e != cudaSuccess) return fail(GMPS_ERR_OOM, "phase buffer");
  h->phase_cap = cap;
  return GMPS_OK;
}

static gmps_status enqueue_iterate(gmps_ctx* h, int64_t k, const double* dphi, const double* dpsi,
                                   const Slab& slab, double* rec = nullptr) {
  InstDesc d = base_desc(h, slab);
  d.k = k;
  d.phase_offset = 0;
  d.phi = dphi;
  d.psi = dpsi;
  d.rec = rec;
  CUDA_TRY(cudaMemcpyAsync(slab.d_desc, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(launch_iterate(slab.d_desc, 1, nullptr, h->cfg.dtype, h->plan.threads, h->plan.smem, 1, h->stream,
                          h->plan.cluster));
  return GMPS_OK;
}

gmps_status grover_mps_iterate_device(gmps_handle h, int64_t k, const double* dev_phi, const double* dev_psi) {
  CallRange range_("grover_mps_iterate_device");
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  if (h->cfg.apply == GMPS_APPLY_GATES)
    return fail(GMPS_ERR_UNSUPPORTED, "a gate-level handle takes circuits (grover_mps_apply_circuit)");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (k < 0) return fail(GMPS_ERR_ARG, "k must be >= 0");
  if (k == 0) return GMPS_OK;
  if (h->cfg.differentiable)
    return fail(GMPS_ERR_UNSUPPORTED, "differentiable handles take host phases (grover_mps_iterate)");
  gmps_status s = enqueue_iterate(h, k, dev_phi, dev_psi, h->main);
  if (s) return s;
  h->iterations += k;
  h->all_phases_explicit = false;
  return GMPS_OK;
}

gmps_status grover_mps_iterate(gmps_handle h, int64_t k, const double* host_phi, const double* host_psi) {
  CallRange range_("grover_mps_iterate");
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  if (h->cfg.apply == GMPS_APPLY_GATES)
    return fail(GMPS_ERR_UNSUPPORTED, "a gate-level handle takes circuits (grover_mps_apply_circuit)");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (k < 0) return fail(GMPS_ERR_ARG, "k must be >= 0");
  if (k == 0) return GMPS_OK;
  gmps_status s;
  const double* dphi = nullptr;
  const double* dpsi = nullptr;
  if (host_phi || host_psi) {
    if ((s = ensure_phase(h, (size_t)k))) return s;
    if (host_phi) {
      for (int64_t i = 0; i < k; ++i)
        if (!std::isfinite(host_phi[i])) return fail(GMPS_ERR_ARG, "non-finite phase");
      CUDA_TRY(cudaMemcpyAsync(h->d_phase, host_phi, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
      dphi = h->d_phase;
    }
    if (host_psi) {
      for (int64_t i = 0; i < k; ++i)
        if (!std::isfinite(host_psi[i])) return fail(GMPS_ERR_ARG, "non-finite phase");
      CUDA_TRY(cudaMemcpyAsync(h->d_phase + h->phase_cap, host_psi, sizeof(double) * k,
                               cudaMemcpyHostToDevice, h->stream));
      dpsi = h->d_phase + h->phase_cap;
    }
  }
  if (h->cfg.differentiable) {
    if (h->iterations + k > h->max_iters) return fail(GMPS_ERR_ARG, "iterations would exceed max_iters");
    int64_t done = 0;
    while (done < k) {
      const int64_t pos = h->iterations + done;
      const int64_t chunk = std::min<int64_t>(k - done, h->every - pos % h->every);
      if ((s = enqueue_iterate(h, chunk, dphi ? dphi + done : nullptr, dpsi ? dpsi + done : nullptr, h->main)))
        return s;
      done += chunk;
      if ((pos + chunk) % h->every == 0)
        CUDA_TRY(launch_copy_sites(h->main.d_desc, h->ckpt[(pos + chunk) / h->every].d_desc, 1, h->cfg.dtype,
                                   h->stream));
    }
  } else if ((s = enqueue_iterate(h, k, dphi, dpsi, h->main))) {
    return s;
  }
  h->iterations += k;
  for (int64_t i = 0; i < k; ++i) {
    h->phi_hist.push_back(host_phi ? host_phi[i] : M_PI);
    h->psi_hist.push_back(host_psi ? host_psi[i] : M_PI);
  }
  return check_device(h);
}

gmps_status grover_mps_sync(gmps_handle h) {
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  return check_device(h);
}

static gmps_status query_amps(gmps_ctx* h, const unsigned long long* d_bits, int nb, std::vector<double>* out) {
  CUDA_TRY(launch_amplitudes(h->main.d_desc, 0, h->cfg.dtype, d_bits, nb, h->d_qout, h->stream));
  out->resize(2 * nb);
  CUDA_TRY(cudaMemcpyAsync(out->data(), h->d_qout, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, h->stream));
  return check_device(h);
}

gmps_status grover_mps_amplitude(gmps_handle h, uint64_t bits, double* re, double* im) {
  if (!h || !re || !im) return fail(GMPS_ERR_ARG, "NULL argument");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (h->cfg.n < 64 && (bits >> h->cfg.n)) return fail(GMPS_ERR_ARG, "bits >= 2^n");
  CUDA_TRY(cudaMemcpyAsync(h->d_qbits, &bits, sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
  std::vector<double> o;
  gmps_status s = query_amps(h, h->d_qbits, 1, &o);
  if (s) return s;
  *re = o[0];
  *im = o[1];
  return GMPS_OK;
}

gmps_status grover_mps_prob_marked(gmps_handle h, double* p) {
  if (!h || !p) return fail(GMPS_ERR_ARG, "NULL argument");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  std::vector<double> o;
  gmps_status s = query_amps(h, h->d_marked, h->cfg.M, &o);
  if (s) return s;
  double acc = 0.0;
  for (int i = 0; i < h->cfg.M; ++i) acc += o[2 * i] * o[2 * i] + o[2 * i + 1] * o[2 * i + 1];
  *p = acc;
  return GMPS_OK;
}

gmps_status grover_mps_sample_device(gmps_handle h, int64_t shots, uint64_t seed, uint64_t* dev_bits,
                                     double* dev_margin) {
  if (!h || (!dev_bits && shots > 0)) return fail(GMPS_ERR_ARG, "NULL argument");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (shots < 0) return fail(GMPS_ERR_ARG, "shots must be >= 0");
  if (shots == 0) return GMPS_OK;
  if (h->plan.chicap > 64) return fail(GMPS_ERR_UNSUPPORTED, "sampling needs chi <= 64");
  CUDA_TRY(launch_sample(h->main.d_desc, 0, h->cfg.dtype, h->plan.chicap, shots, seed,
                         (unsigned long long*)dev_bits, dev_margin, h->stream));
  return GMPS_OK;
}

gmps_status grover_mps_sample(gmps_handle h, int64_t shots, uint64_t seed, uint64_t* out_bits) {
  CallRange range_("grover_mps_sample");
  if (!h || (!out_bits && shots > 0)) return fail(GMPS_ERR_ARG, "NULL argument");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (shots < 0) return fail(GMPS_ERR_ARG, "shots must be >= 0");
  if (shots == 0) return GMPS_OK;
  if ((size_t)shots > h->sample_cap) {
    if (h->d_sample) cudaFree(h->d_sample);
    h->d_sample = nullptr;
    cudaError_t e = dev_malloc((void**)&h->d_sample, sizeof(uint64_t) * shots);
    if (e != cudaSuccess) return fail(GMPS_ERR_OOM, "sample buffer");
    h->sample_cap = shots;
  }
  gmps_status s = grover_mps_sample_device(h, shots, seed, (uint64_t*)h->d_sample, nullptr);
  if (s) return s;
  CUDA_TRY(cudaMemcpyAsync(out_bits, h->d_sample, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, h->stream));
  return check_device(h);
}

static void fill_stats(const DevStats& ds, int n, int ctas, gmps_stats* out) {
  memset(out, 0, sizeof(*out));
  out->iterations = ds.iterations;
  out->n = n;
  int mb = 1;
  for (int l = 0; l <= n; ++l) {
    out->chi[l] = ds.chi[l];
    mb = std::max(mb, ds.chi[l]);
  }
  out->max_bond = mb;
  out->log_norm = ds.log_norm;
  out->discarded_weight = ds.discarded;
  out->max_jacobi_sweeps = ds.max_jacobi_sweeps;
  out->jacobi_sweeps = ds.jacobi_sweeps;
  out->svd_count = ds.svd_count;
  out->device_status = ds.status;
  out->sm_id = ds.sm;
  out->t_begin_ns = (int64_t)ds.t_begin;
  out->t_end_ns = (int64_t)ds.t_end;
  out->ctas = ctas;
}

gmps_status grover_mps_stats(gmps_handle h, gmps_stats* out) {
  if (!h || !out) return fail(GMPS_ERR_ARG, "NULL argument");
  DevStats ds;
  CUDA_TRY(cudaMemcpyAsync(&ds, h->main.d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  fill_stats(ds, h->cfg.n, std::max(1, h->plan.cluster), out);
  return GMPS_OK;
}

gmps_status grover_mps_export(gmps_handle h, double* host_out, size_t capacity, size_t* needed) {
  if (!h || !needed) return fail(GMPS_ERR_ARG, "NULL argument");
  DevStats ds;
  CUDA_TRY(cudaMemcpyAsync(&ds, h->main.d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  size_t need = 0;
  for (int l = 0; l < h->cfg.n; ++l) need += 2ull * 2 * ds.chi[l] * ds.chi[l + 1];
  *needed = need;
  if (!host_out) return GMPS_OK;
  if (capacity < need) return fail(GMPS_ERR_ARG, "export buffer too small");
  const size_t eb = h->plan.elem_bytes;
  std::vector<char> raw(h->plan.site_elems * eb);
  CUDA_TRY(cudaMemcpyAsync(raw.data(), h->main.d_sites, raw.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  size_t o = 0;
  for (int l = 0; l < h->cfg.n; ++l) {
    const size_t cnt = 2ull * ds.chi[l] * ds.chi[l + 1];
    const char* base = raw.data() + h->plan.off[l] * eb;
    for (size_t e = 0; e < cnt; ++e) {
      if (h->cfg.dtype == GMPS_DW) {
        const float* v = (const float*)(base + e * eb);
        host_out[o++] = (double)v[0] + (double)v[1];
        host_out[o++] = (double)v[2] + (double)v[3];
      } else if (eb == sizeof(double2)) {
        const double* v = (const double*)(base + e * eb);
        host_out[o++] = v[0];
        host_out[o++] = v[1];
      } else {
        const float* v = (const float*)(base + e * eb);
        host_out[o++] = v[0];
        host_out[o++] = v[1];
      }
    }
  }
  return GMPS_OK;
}

static gmps_status check_slab(gmps_ctx* h, const Slab& sl, const char* what) {
  int st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, (char*)sl.d_stats + offsetof(DevStats, status), sizeof(int),
                           cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (st) return fail((gmps_status)st, std::string(what) + ": device reported an error");
  return GMPS_OK;
}

gmps_status grover_mps_backward(gmps_handle h, double dL_dP, double* grad_phi, double* grad_psi) {
  CallRange range_("grover_mps_backward");
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  if (!h->cfg.differentiable) return fail(GMPS_ERR_STATE, "handle was not created differentiable");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  const int64_t K = h->iterations;
  if (K == 0) return GMPS_OK;
  if (!grad_phi || !grad_psi) return fail(GMPS_ERR_ARG, "gradient outputs are NULL");
  const int mi = h->max_iters;
  CUDA_TRY(cudaMemcpyAsync(h->d_ph_all, h->phi_hist.data(), sizeof(double) * K, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_ph_all + mi, h->psi_hist.data(), sizeof(double) * K, cudaMemcpyHostToDevice,
                           h->stream));
  AdjArgs args[2];
  args[0] = AdjArgs{nullptr, h->d_ph_all, h->d_ph_all + mi, h->d_grad, h->d_grad + mi, dL_dP};
  args[1] = args[0];
  args[1].rec = h->d_rec;
  CUDA_TRY(cudaMemcpyAsync(h->d_args, args, sizeof(args), cudaMemcpyHostToDevice, h->stream));
  // mu_K = Pi_W psi_K on the costate chain
  CUDA_TRY(launch_copy_sites(h->main.d_desc, h->costate.d_desc, 1, h->cfg.dtype, h->stream));
  CUDA_TRY(launch_adjoint(h->costate.d_desc, h->d_args, 1, h->cfg.dtype, h->plan.threads, h->plan.smem, K, K, 1,
                          h->stream));
  for (int64_t j = (K - 1) / h->every; j >= 0; --j) {
    const int64_t k_lo = j * h->every, k_hi = std::min<int64_t>(K, k_lo + h->every);
    // recompute the segment from its checkpoint, recording <w|psi> and <s|psi>
    CUDA_TRY(launch_copy_sites(h->ckpt[j].d_desc, h->work.d_desc, 1, h->cfg.dtype, h->stream));
    gmps_status s = enqueue_iterate(h, k_hi - k_lo, h->d_ph_all + k_lo, h->d_ph_all + mi + k_lo, h->work, h->d_rec);
    if (s) return s;
    CUDA_TRY(launch_adjoint(h->costate.d_desc, h->d_args + 1, 1, h->cfg.dtype, h->plan.threads, h->plan.smem, k_lo,
                            k_hi, 0, h->stream));
  }
  CUDA_TRY(cudaMemcpyAsync(grad_phi, h->d_grad, sizeof(double) * K, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(grad_psi, h->d_grad + mi, sizeof(double) * K, cudaMemcpyDeviceToHost, h->stream));
  gmps_status s = check_slab(h, h->work, "segment recompute");
  if (!s) s = check_slab(h, h->costate, "adjoint");
  return s;
}

static_assert(sizeof(gmps_gate) == sizeof(GateOp), "gmps_gate and GateOp must share their layout");

gmps_status grover_mps_apply_circuit(gmps_handle h, const gmps_gate* gates, int64_t count, int64_t repeat) {
  CallRange range_("grover_mps_apply_circuit");
  if (!h) return fail(GMPS_ERR_ARG, "handle is NULL");
  if (h->error) return fail(GMPS_ERR_STATE, "handle is in an error state");
  if (count < 0 || repeat < 0) return fail(GMPS_ERR_ARG, "count and repeat must be >= 0");
  if (count == 0 || repeat == 0) return GMPS_OK;
  if (!gates) return fail(GMPS_ERR_ARG, "gates is NULL");
  if (h->cfg.differentiable) return fail(GMPS_ERR_UNSUPPORTED, "circuits on differentiable handles are not built");
  if (h->plan.xcap < 2 * h->plan.chicap)
    return fail(GMPS_ERR_UNSUPPORTED, "circuits need a handle created with apply = GMPS_APPLY_GATES or MPO");
  for (int64_t g = 0; g < count; ++g) {
    const gmps_gate& x = gates[g];
    if (x.kind == GMPS_GATE_1Q) {
      if (x.site < 0 || x.site >= h->cfg.n) return fail(GMPS_ERR_ARG, "gate site out of range");
    } else if (x.kind != GMPS_GATE_MCPHASE) {
      return fail(GMPS_ERR_ARG, "unknown gate kind");
    }
    for (int q = 0; q < 8; ++q)
      if (!std::isfinite(x.u[q])) return fail(GMPS_ERR_ARG, "non-finite gate entry");
  }
  if (h->gate_cap < (size_t)count) {
    if (h->d_gates) cudaFree(h->d_gates);
    h->d_gates = nullptr;
    h->gate_cap = 0;
    if (dev_malloc((void**)&h->d_gates, sizeof(GateOp) * count) != cudaSuccess) return fail(GMPS_ERR_OOM, "gate list");
    h->gate_cap = count;
  }
  InstDesc d = base_desc(h, h->main);
  d.M = 1;
  d.apply = GMPS_APPLY_MPO;
  d.marked = h->d_ones;
  const unsigned long long ones = h->cfg.n == 64 ? ~0ull : ((1ull << h->cfg.n) - 1ull);
  CUDA_TRY(cudaMemcpyAsync(h->d_ones, &ones, sizeof(ones), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_cdesc, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->d_gates, gates, sizeof(GateOp) * count, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(launch_circuit(h->d_cdesc, h->d_gates, count, repeat, h->cfg.dtype, h->plan.threads, h->plan.smem,
                          h->stream));
  h->all_phases_explicit = false;
  return check_device(h);
}

gmps_status grover_mps_grover_gates(int n, const uint64_t* marked, int M, int64_t iterations, gmps_gate* out,
                                    int64_t capacity, int64_t* count) {
  if (!count) return fail(GMPS_ERR_ARG, "count is NULL");
  if (n < 1 || n > 64) return fail(GMPS_ERR_ARG, "n must be in [1, 64]");
  if (M < 1 || !marked) return fail(GMPS_ERR_ARG, "need M >= 1 marked strings");
  if (iterations < 0) return fail(GMPS_ERR_ARG, "iterations must be >= 0");
  int64_t per = 4 * (int64_t)n + 1;  // diffusion
  for (int i = 0; i < M; ++i) {
    if (n < 64 && (marked[i] >> n)) return fail(GMPS_ERR_ARG, "marked string has bits >= n");
    int zeros = 0;
    for (int l = 0; l < n; ++l) zeros += !((marked[i] >> l) & 1ull);
    per += 2 * zeros + 1;
  }
  *count = per * iterations;
  if (!out) return GMPS_OK;
  if (capacity < *count) return fail(GMPS_ERR_ARG, "gate buffer too small");
  const double r = 0.70710678118654752440;
  auto one = [](gmps_gate* g, int site, double a, double b, double c, double d) {
    g->kind = GMPS_GATE_1Q;
    g->site = site;
    const double u[8] = {a, 0.0, b, 0.0, c, 0.0, d, 0.0};
    for (int q = 0; q < 8; ++q) g->u[q] = u[q];
  };
  auto mcz = [](gmps_gate* g) {
    g->kind = GMPS_GATE_MCPHASE;
    g->site = 0;
    for (int q = 0; q < 8; ++q) g->u[q] = 0.0;
    g->u[0] = M_PI;
  };
  gmps_gate* g = out;
  for (int64_t it = 0; it < iterations; ++it) {
    for (int i = 0; i < M; ++i) {  // oracle of w: X on its zeros, MCZ, X on its zeros
      for (int l = 0; l < n; ++l)
        if (!((marked[i] >> l) & 1ull)) one(g++, l, 0, 1, 1, 0);
      mcz(g++);
      for (int l = 0; l < n; ++l)
        if (!((marked[i] >> l) & 1ull)) one(g++, l, 0, 1, 1, 0);
    }
    for (int l = 0; l < n; ++l) one(g++, l, r, r, r, -r);  // H
    for (int l = 0; l < n; ++l) one(g++, l, 0, 1, 1, 0);   // X
    mcz(g++);
    for (int l = 0; l < n; ++l) one(g++, l, 0, 1, 1, 0);
    for (int l = 0; l < n; ++l) one(g++, l, r, r, r, -r);
  }
  return GMPS_OK;
}

gmps_status grover_mps_destroy(gmps_handle h) {
  if (!h) return GMPS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->own_arena && h->arena) cudaFree(h->arena);
  if (h->d_phase) cudaFree(h->d_phase);
  if (h->d_sample) cudaFree(h->d_sample);
  if (h->diff_mem) cudaFree(h->diff_mem);
  if (h->d_gates) cudaFree(h->d_gates);
  delete h;
  return GMPS_OK;
}

}  // extern "C"

// ================================================================ batched
struct gmps_batch_ctx {
  int count = 0;
  int dtype = 0;
  cudaStream_t stream = nullptr;
  std::vector<gmps_config> cfgs;
  std::vector<std::vector<uint64_t>> marked;
  std::vector<Plan> plans;
  std::vector<InstDesc> h;   // in queue order
  std::vector<int> order;    // queue position -> instance index
  std::vector<int> pos;      // instance index -> queue position
  char* mem = nullptr;
  InstDesc* d_desc = nullptr;
  int* d_queue = nullptr;
  double* d_p = nullptr;
  unsigned long long* d_q = nullptr;
  double* d_qout = nullptr;
  int threads = 0;
  size_t smem = 0;
  int grid = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_threads = -1;
  bool own_stream = false;  // graph capture needs a non-legacy stream
};

static gmps_status batch_enqueue(gmps_batch_ctx* b) {
  CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(int), b->stream));
  CUDA_TRY(launch_init(b->d_desc, b->count, b->dtype, 64, b->stream));
  CUDA_TRY(launch_iterate(b->d_desc, b->count, b->d_queue, b->dtype, b->threads, b->smem, b->grid, b->stream));
  return GMPS_OK;
}

extern "C" {

gmps_status grover_mps_batch_create(int count, const gmps_config* cfgs, const int64_t* ks,
                                    const double* const* host_phi, const double* const* host_psi,
                                    void* cuda_stream, gmps_batch_handle* out) {
  CallRange range_("grover_mps_batch_create");
  if (!out || !cfgs || !ks || count < 1) return fail(GMPS_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  gmps_batch_ctx* b = new gmps_batch_ctx();
  b->count = count;
  b->stream = (cudaStream_t)cuda_stream;
  if (!b->stream) {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      delete b;
      return fail(GMPS_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  b->dtype = cfgs[0].dtype;
  b->cfgs.assign(cfgs, cfgs + count);
  b->marked.resize(count);
  b->plans.resize(count);
  gmps_status s;
  size_t total = 0, smem = 0;
  int maxx = 1;
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i) {
    if ((s = validate(&cfgs[i]))) {
      grover_mps_batch_destroy(b);  // also the stream it created
      return s;
    }
    if (cfgs[i].dtype != b->dtype) {
      grover_mps_batch_destroy(b);  // also the stream it created
      return fail(GMPS_ERR_ARG, "all batch instances must share dtype");
    }
    if (ks[i] < 0) {
      grover_mps_batch_destroy(b);  // also the stream it created
      return fail(GMPS_ERR_ARG, "k must be >= 0");
    }
    b->marked[i].assign(cfgs[i].marked, cfgs[i].marked + cfgs[i].M);
    b->cfgs[i].marked = b->marked[i].data();
    if ((s = make_plan_for(&b->cfgs[i], false, &b->plans[i]))) {
      grover_mps_batch_destroy(b);  // also the stream it created
      return s;
    }
    const Plan& P = b->plans[i];
    total += a256(sizeof(long long) * (cfgs[i].n + 1)) + a256(sizeof(DevStats)) +
             a256(P.site_elems * P.elem_bytes) + a256(P.work_bytes) + a256(P.jc_bytes) +
             a256(sizeof(unsigned long long) * cfgs[i].M) + a256(sizeof(double) * 2 * ks[i]);
    smem = std::max(smem, P.smem);
    maxx = std::max(maxx, P.xcap);
    cost[i] = (double)ks[i] * cfgs[i].n * std::pow((double)P.xcap, 3.0);
  }
  total += a256(sizeof(InstDesc) * count) + a256(sizeof(int)) + a256(sizeof(double) * count) +
           a256(sizeof(unsigned long long) * 64) + a256(sizeof(double) * 128);
  cudaError_t e = dev_malloc((void**)&b->mem, total);
  if (e != cudaSuccess) {
    grover_mps_batch_destroy(b);  // also the stream it created
    return fail(GMPS_ERR_OOM, "batch arena");
  }
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->pos.resize(count);
  for (int q = 0; q < count; ++q) b->pos[b->order[q]] = q;
  char* p = b->mem;
  b->d_desc = (InstDesc*)p;
  p += a256(sizeof(InstDesc) * count);
  b->d_queue = (int*)p;
  p += a256(sizeof(int));
  b->d_p = (double*)p;
  p += a256(sizeof(double) * count);
  b->d_q = (unsigned long long*)p;
  p += a256(sizeof(unsigned long long) * 64);
  b->d_qout = (double*)p;
  p += a256(sizeof(double) * 128);
  b->h.resize(count);
  for (int q = 0; q < count; ++q) {
    const int i = b->order[q];
    const gmps_config& c = b->cfgs[i];
    const Plan& P = b->plans[i];
    InstDesc d{};
    d.n = c.n;
    d.M = c.M;
    d.apply = c.apply;
    d.chi_max = c.chi_max;
    d.chicap = P.chicap;
    d.xcap = P.xcap;
    d.rcap = P.rcap;
    d.max_sweeps = c.max_sweeps ? c.max_sweeps : kDefaultMaxSweeps;
    d.resident = 0;
    d.k = ks[i];
    d.tol = c.tol;
    d.trunc_eps = rank_rule_for(c.dtype).eps;
    d.trunc_dim = rank_rule_for(c.dtype).dim;
    d.inv_sqrt_N = std::ldexp(1.0, -c.n / 2) * ((c.n & 1) ? std::sqrt(0.5) : 1.0);
    long long* off = (long long*)p;
    p += a256(sizeof(long long) * (c.n + 1));
    d.site_off = off;
    d.stats = (DevStats*)p;
    p += a256(sizeof(DevStats));
    d.sites = p;
    p += a256(P.site_elems * P.elem_bytes);
    d.work = P.work_bytes ? p : nullptr;
    p += a256(P.work_bytes);
    d.jcache = P.jc_bytes ? p : nullptr;
    d.jbanks = P.jbanks;
    p += a256(P.jc_bytes);
    unsigned long long* mk_ = (unsigned long long*)p;
    p += a256(sizeof(unsigned long long) * c.M);
    d.marked = mk_;
    double* ph = (double*)p;
    p += a256(sizeof(double) * 2 * ks[i]);
    e = cudaMemcpyAsync(off, P.off, sizeof(long long) * (c.n + 1), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(mk_, c.marked, sizeof(uint64_t) * c.M, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && host_phi && host_phi[i]) {
      e = cudaMemcpyAsync(ph, host_phi[i], sizeof(double) * ks[i], cudaMemcpyHostToDevice, b->stream);
      d.phi = ph;
    }
    if (e == cudaSuccess && host_psi && host_psi[i]) {
      e = cudaMemcpyAsync(ph + ks[i], host_psi[i], sizeof(double) * ks[i], cudaMemcpyHostToDevice, b->stream);
      d.psi = ph + ks[i];
    }
    if (e != cudaSuccess) {
      grover_mps_batch_destroy(b);
      return cuda_fail(e, "batch upload");
    }
    b->h[q] = d;
  }
  e = cudaMemcpyAsync(b->d_desc, b->h.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    grover_mps_batch_destroy(b);
    return cuda_fail(e, "batch create");
  }
  b->smem = smem;
  b->threads = auto_threads(maxx);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  b->grid = nsm;  // refined at run time from the occupancy of the chosen CTA size
  *out = b;
  return GMPS_OK;
}

gmps_status grover_mps_batch_set_threads(gmps_batch_handle b, int threads) {
  if (!b) return fail(GMPS_ERR_ARG, "NULL handle");
  if (threads != 0 && (threads % 32 || threads < 32 || threads > 256))
    return fail(GMPS_ERR_ARG, "threads must be a multiple of 32 in [32, 256]");
  int maxx = 1;
  for (auto& P : b->plans) maxx = std::max(maxx, P.xcap);
  b->threads = threads ? threads : auto_threads(maxx);
  return GMPS_OK;
}

gmps_status grover_mps_batch_run(gmps_batch_handle b, int use_graph) {
  CallRange range_("grover_mps_batch_run");
  if (!b) return fail(GMPS_ERR_ARG, "NULL handle");
  // blocks resident per SM for this CTA size and shared-memory footprint
  int dev = 0, nsm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = std::max(1, (int)(smem_sm / std::max<size_t>(b->smem + 1024, 1)));
  per_sm = std::min(per_sm, std::max(1, 2048 / b->threads));
  b->grid = std::min(b->count, nsm * per_sm);
  if (!use_graph) return batch_enqueue(b);
  if (!b->gexec || b->graph_threads != b->threads) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    gmps_status s = batch_enqueue(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graph_threads = b->threads;
  }
  CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
  count_launch(2);
  return GMPS_OK;
}

gmps_status grover_mps_batch_result(gmps_batch_handle b, double* host_p, int* host_status) {
  if (!b) return fail(GMPS_ERR_ARG, "NULL handle");
  CUDA_TRY(launch_batch_prob(b->d_desc, b->count, b->dtype, b->d_p, b->stream));
  std::vector<double> p(b->count);
  CUDA_TRY(cudaMemcpyAsync(p.data(), b->d_p, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
  std::vector<DevStats> st(b->count);
  for (int q = 0; q < b->count; ++q)
    CUDA_TRY(cudaMemcpyAsync(&st[q], b->h[q].stats, sizeof(DevStats), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  gmps_status worst = GMPS_OK;
  for (int i = 0; i < b->count; ++i) {
    const int q = b->pos[i];
    if (host_p) host_p[i] = p[q];
    if (host_status) host_status[i] = st[q].status;
    if (st[q].status && !worst) worst = (gmps_status)st[q].status;
  }
  if (worst) return fail(worst, "an instance reported a device error");
  return GMPS_OK;
}

gmps_status grover_mps_batch_amplitude(gmps_batch_handle b, int i, uint64_t bits, double* re, double* im) {
  if (!b || !re || !im || i < 0 || i >= b->count) return fail(GMPS_ERR_ARG, "bad argument");
  const int q = b->pos[i];
  CUDA_TRY(cudaMemcpyAsync(b->d_q, &bits, sizeof(uint64_t), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(launch_amplitudes(b->d_desc, q, b->dtype, b->d_q, 1, b->d_qout, b->stream));
  double o[2];
  CUDA_TRY(cudaMemcpyAsync(o, b->d_qout, sizeof(o), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  *re = o[0];
  *im = o[1];
  return GMPS_OK;
}

gmps_status grover_mps_batch_stats(gmps_batch_handle b, int i, gmps_stats* out) {
  if (!b || !out || i < 0 || i >= b->count) return fail(GMPS_ERR_ARG, "bad argument");
  const int q = b->pos[i];
  DevStats ds;
  CUDA_TRY(cudaMemcpyAsync(&ds, b->h[q].stats, sizeof(DevStats), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  fill_stats(ds, b->cfgs[i].n, 1, out);
  return GMPS_OK;
}

gmps_status grover_mps_batch_destroy(gmps_batch_handle b) {
  if (!b) return GMPS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->mem) cudaFree(b->mem);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return GMPS_OK;
}

}  // extern "C"

// ================================================================ differentiable batch
// Every phase vector b has its chain (main), checkpoints, recompute chain
// (work) and costate chain; descriptors of each role are contiguous arrays so
// that one launch serves all vectors (iterate_kernel takes them from its work
// queue, adjoint_kernel and copy_sites_kernel one block per vector).
struct gmps_diff_batch_ctx {
  gmps_config cfg{};
  std::vector<uint64_t> marked;
  Plan plan;
  int count = 0, K = 0, every = 8, nseg = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* mem = nullptr;
  InstDesc* d_main = nullptr;   // count
  InstDesc* d_work = nullptr;   // count
  InstDesc* d_cost = nullptr;   // count
  InstDesc* d_ckpt = nullptr;   // (nseg + 1) * count, checkpoint j of vector b at j * count + b
  std::vector<InstDesc> h_main, h_work, h_cost, h_ckpt;
  AdjArgs* d_args = nullptr;    // [0, count): projection, [count, 2 count): segments
  DevStats* d_stats = nullptr;  // main, work, cost: 3 * count (checkpoint stats follow)
  double* d_ph = nullptr;       // phi then psi, count x K each
  double* d_grad = nullptr;     // dphi then dpsi, count x K each
  double* d_rec = nullptr;      // count x every x (M + 1) complex
  double* d_p = nullptr;        // count
  int* d_queue = nullptr;
  int grid = 1;
};

static gmps_status diff_launch_iterate(gmps_diff_batch_ctx* b, InstDesc* d_desc, std::vector<InstDesc>& h,
                                       long long k, long long offset, bool record) {
  const int M = b->cfg.M;
  for (int i = 0; i < b->count; ++i) {
    h[i].k = k;
    h[i].phase_offset = offset;
    h[i].rec = record ? b->d_rec + (size_t)i * b->every * (M + 1) * 2 : nullptr;
  }
  CUDA_TRY(cudaMemcpyAsync(d_desc, h.data(), sizeof(InstDesc) * b->count, cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(int), b->stream));
  CUDA_TRY(launch_iterate(d_desc, b->count, b->d_queue, b->cfg.dtype, b->plan.threads, b->plan.smem, b->grid,
                          b->stream));
  return GMPS_OK;
}

extern "C" {

gmps_status grover_mps_diff_batch_create(const gmps_config* cfg, int count, int K, void* cuda_stream,
                                         gmps_diff_batch_handle* out) {
  CallRange range_("grover_mps_diff_batch_create");
  if (!out) return fail(GMPS_ERR_ARG, "out is NULL");
  *out = nullptr;
  gmps_status s = validate(cfg);
  if (s) return s;
  if (count < 1 || K < 1) return fail(GMPS_ERR_ARG, "count and K must be >= 1");
  gmps_diff_batch_ctx* b = new gmps_diff_batch_ctx();
  b->cfg = *cfg;
  b->marked.assign(cfg->marked, cfg->marked + cfg->M);
  b->cfg.marked = b->marked.data();
  b->count = count;
  b->K = K;
  b->every = cfg->checkpoint_every > 0 ? cfg->checkpoint_every : 8;
  b->nseg = (K + b->every - 1) / b->every;
  b->stream = (cudaStream_t)cuda_stream;
  if (!b->stream) {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      delete b;
      return fail(GMPS_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  if ((s = make_plan_for(&b->cfg, true, &b->plan))) {
    grover_mps_diff_batch_destroy(b);
    return s;
  }
  const int M = cfg->M, n = cfg->n;
  const int nslab = (3 + b->nseg + 1) * count;
  const size_t site_b = a256(b->plan.site_elems * b->plan.elem_bytes);
  const size_t bytes = a256(sizeof(long long) * (n + 1)) + a256(sizeof(unsigned long long) * M) +
                       4 * a256(sizeof(InstDesc) * count) + a256(sizeof(InstDesc) * count * (b->nseg + 1)) +
                       a256(sizeof(AdjArgs) * 2 * count) + a256(sizeof(DevStats) * nslab) +
                       2 * a256(sizeof(double) * 2 * (size_t)count * K) +
                       a256(sizeof(double) * 2 * (size_t)count * b->every * (M + 1)) +
                       a256(sizeof(double) * count) + a256(sizeof(int)) + site_b * nslab +
                       a256(b->plan.work_bytes) * 3 * count + a256(b->plan.jc_bytes) * count;
  cudaError_t e = dev_malloc((void**)&b->mem, bytes);
  if (e != cudaSuccess) {
    grover_mps_diff_batch_destroy(b);
    return fail(GMPS_ERR_OOM, std::string("differentiable batch: ") + cudaGetErrorString(e));
  }
  char* p = b->mem;
  long long* d_off = (long long*)p;          p += a256(sizeof(long long) * (n + 1));
  unsigned long long* d_marked = (unsigned long long*)p;  p += a256(sizeof(unsigned long long) * M);
  b->d_main = (InstDesc*)p;                   p += a256(sizeof(InstDesc) * count);
  b->d_work = (InstDesc*)p;                   p += a256(sizeof(InstDesc) * count);
  b->d_cost = (InstDesc*)p;                   p += a256(sizeof(InstDesc) * count);
  p += a256(sizeof(InstDesc) * count);        // spare
  b->d_ckpt = (InstDesc*)p;                   p += a256(sizeof(InstDesc) * count * (b->nseg + 1));
  b->d_args = (AdjArgs*)p;                    p += a256(sizeof(AdjArgs) * 2 * count);
  b->d_stats = (DevStats*)p;                  p += a256(sizeof(DevStats) * nslab);
  b->d_ph = (double*)p;                       p += a256(sizeof(double) * 2 * (size_t)count * K);
  b->d_grad = (double*)p;                     p += a256(sizeof(double) * 2 * (size_t)count * K);
  b->d_rec = (double*)p;                      p += a256(sizeof(double) * 2 * (size_t)count * b->every * (M + 1));
  b->d_p = (double*)p;                        p += a256(sizeof(double) * count);
  b->d_queue = (int*)p;                       p += a256(sizeof(int));
  char* works = p;                            p += a256(b->plan.work_bytes) * 3 * count;
  char* jcs = p;                              p += a256(b->plan.jc_bytes) * count;
  char* sites = p;
  const RankRule rr = rank_rule_for(cfg->dtype);
  auto desc = [&](int slab) {
    InstDesc d{};
    d.n = n;
    d.M = M;
    d.apply = cfg->apply;
    d.chi_max = cfg->chi_max;
    d.chicap = b->plan.chicap;
    d.xcap = b->plan.xcap;
    d.rcap = b->plan.rcap;
    // main, recompute and costate chains run kernels: each gets a work area
    d.work = (b->plan.work_bytes && slab < 3 * count) ? works + a256(b->plan.work_bytes) * slab : nullptr;
    d.max_sweeps = cfg->max_sweeps ? cfg->max_sweeps : kDefaultMaxSweeps;
    d.resident = b->plan.resident;
    d.tol = cfg->tol;
    d.trunc_eps = rr.eps;
    d.trunc_dim = rr.dim;
    d.inv_sqrt_N = std::ldexp(1.0, -n / 2) * ((n & 1) ? std::sqrt(0.5) : 1.0);
    d.marked = d_marked;
    d.site_off = d_off;
    d.stats = b->d_stats + slab;
    d.sites = sites + site_b * slab;
    return d;
  };
  b->h_main.resize(count);
  b->h_work.resize(count);
  b->h_cost.resize(count);
  b->h_ckpt.resize((size_t)count * (b->nseg + 1));
  for (int i = 0; i < count; ++i) {
    b->h_main[i] = desc(i);
    // the forward chains cache their Jacobi rotations like a handle's main chain
    b->h_main[i].jcache = b->plan.jc_bytes ? jcs + a256(b->plan.jc_bytes) * i : nullptr;
    b->h_main[i].jbanks = b->plan.jbanks;
    b->h_main[i].phi = b->d_ph + (size_t)i * K;
    b->h_main[i].psi = b->d_ph + (size_t)(count + i) * K;
    b->h_work[i] = desc(count + i);
    b->h_work[i].phi = b->h_main[i].phi;
    b->h_work[i].psi = b->h_main[i].psi;
    b->h_cost[i] = desc(2 * count + i);
  }
  for (int j = 0; j <= b->nseg; ++j)
    for (int i = 0; i < count; ++i) b->h_ckpt[(size_t)j * count + i] = desc(3 * count + j * count + i);
  std::vector<AdjArgs> args(2 * count);
  for (int i = 0; i < count; ++i) {
    args[i] = AdjArgs{nullptr, b->h_main[i].phi, b->h_main[i].psi, b->d_grad + (size_t)i * K,
                      b->d_grad + (size_t)(count + i) * K, -1.0};
    args[count + i] = args[i];
    args[count + i].rec = b->d_rec + (size_t)i * b->every * (M + 1) * 2;
  }
  e = cudaMemcpyAsync(d_off, b->plan.off, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_marked, b->marked.data(), sizeof(uint64_t) * M, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_args, args.data(), sizeof(AdjArgs) * 2 * count, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_work, b->h_work.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_cost, b->h_cost.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_ckpt, b->h_ckpt.data(), sizeof(InstDesc) * count * (b->nseg + 1),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_main, b->h_main.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    grover_mps_diff_batch_destroy(b);
    return cuda_fail(e, "differentiable batch upload");
  }
  int dev = 0, nsm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = std::max(1, (int)(smem_sm / (b->plan.smem + 1024)));
  per_sm = std::min(per_sm, std::max(1, 2048 / b->plan.threads));
  b->grid = std::min(count, nsm * per_sm);
  *out = b;
  return GMPS_OK;
}

gmps_status grover_mps_diff_batch_run(gmps_diff_batch_handle b, const double* host_phi, const double* host_psi,
                                      double* host_loss, double* host_gphi, double* host_gpsi) {
  CallRange range_("grover_mps_diff_batch_run");
  if (!b || !host_phi || !host_psi || !host_loss || !host_gphi || !host_gpsi)
    return fail(GMPS_ERR_ARG, "NULL argument");
  const size_t ck = (size_t)b->count * b->K;
  for (size_t i = 0; i < ck; ++i)
    if (!std::isfinite(host_phi[i]) || !std::isfinite(host_psi[i])) return fail(GMPS_ERR_ARG, "non-finite phase");
  const int c = b->count, dt = b->cfg.dtype;
  CUDA_TRY(cudaMemcpyAsync(b->d_ph, host_phi, sizeof(double) * ck, cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->d_ph + ck, host_psi, sizeof(double) * ck, cudaMemcpyHostToDevice, b->stream));
  // forward: |s> on every chain and checkpoint 0, then segment by segment
  CUDA_TRY(launch_init(b->d_main, c, dt, 64, b->stream));
  CUDA_TRY(launch_init(b->d_ckpt, c, dt, 64, b->stream));
  CUDA_TRY(launch_init(b->d_work, c, dt, 64, b->stream));
  CUDA_TRY(launch_init(b->d_cost, c, dt, 64, b->stream));
  gmps_status s;
  for (int j = 0; j < b->nseg; ++j) {
    const long long lo = (long long)j * b->every, hi = std::min<long long>(b->K, lo + b->every);
    if ((s = diff_launch_iterate(b, b->d_main, b->h_main, hi - lo, lo, false))) return s;
    if (j + 1 < b->nseg)
      CUDA_TRY(launch_copy_sites(b->d_main, b->d_ckpt + (size_t)(j + 1) * c, c, dt, b->stream));
  }
  CUDA_TRY(launch_batch_prob(b->d_main, c, dt, b->d_p, b->stream));
  // reverse: mu_K = Pi_W psi_K, then the segments last to first
  CUDA_TRY(launch_copy_sites(b->d_main, b->d_cost, c, dt, b->stream));
  CUDA_TRY(launch_adjoint(b->d_cost, b->d_args, c, dt, b->plan.threads, b->plan.smem, b->K, b->K, 1, b->stream));
  for (int j = b->nseg - 1; j >= 0; --j) {
    const long long lo = (long long)j * b->every, hi = std::min<long long>(b->K, lo + b->every);
    CUDA_TRY(launch_copy_sites(b->d_ckpt + (size_t)j * c, b->d_work, c, dt, b->stream));
    if ((s = diff_launch_iterate(b, b->d_work, b->h_work, hi - lo, lo, true))) return s;
    CUDA_TRY(launch_adjoint(b->d_cost, b->d_args + c, c, dt, b->plan.threads, b->plan.smem, lo, hi, 0, b->stream));
  }
  std::vector<double> p(c);
  std::vector<DevStats> st(3 * c);
  CUDA_TRY(cudaMemcpyAsync(p.data(), b->d_p, sizeof(double) * c, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaMemcpyAsync(host_gphi, b->d_grad, sizeof(double) * ck, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaMemcpyAsync(host_gpsi, b->d_grad + ck, sizeof(double) * ck, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaMemcpyAsync(st.data(), b->d_stats, sizeof(DevStats) * 3 * c, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < c; ++i) host_loss[i] = 1.0 - p[i];
  for (int i = 0; i < 3 * c; ++i)
    if (st[i].status) return fail((gmps_status)st[i].status, "a chain of the differentiable batch reported an error");
  return GMPS_OK;
}

gmps_status grover_mps_diff_batch_destroy(gmps_diff_batch_handle b) {
  if (!b) return GMPS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->mem) cudaFree(b->mem);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return GMPS_OK;
}

}  // extern "C"

// =====================================================================
// Allocation-free entry point (grover_mps_run_noalloc).
//
// Some callers cannot allocate device memory at all: code running inside a
// host process that forbids cudaMalloc after start-up (real-time or
// certified services that size every buffer up front), plugins loaded into a
// process whose allocator they must not touch, or callers that run while the
// device heap is deliberately exhausted.  For them this entry point runs a
// whole instance (init, k iterations, marked amplitudes, bond table) in a
// fixed file-scope device array instead of a handle's arena.  It calls no
// cudaMalloc, cudaFree or other allocating routine.  It plans, validates and
// truncates exactly as grover_mps_create_ex does for a complex128 instance
// (same validate, make_plan_for and rank rule), so both give the same bonds.
//
// The array below is a device symbol: in host code its name is only a
// host-side stand-in, never a device address.  Its address is fetched with
// cudaGetSymbolAddress once per device (with that device current) by the
// first call on that device; that first call should therefore come before
// any stream capture.  Every GPU that loads this library holds the array
// (kNoAllocScratchBytes) until the process exits.  All calls share it and
// it keeps the last call's contents; each call re-initialises everything it
// reads (descriptor, offsets, statistics, chain).  Calls whose GPU work
// overlaps (different streams or threads without ordering) race on it.
// =====================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = 2u << 20;  // 2 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];
bool g_noalloc_ready[64];

// Device address of g_noalloc_scratch on the current device (set-up on the
// first call per device).
cudaError_t noalloc_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
    g_noalloc_ready[dev] = true;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gmps_status grover_mps_run_noalloc(int n, const uint64_t* marked, int M, int apply, int chi_max,
                                              double tol, int64_t k, const double* dev_phi,
                                              const double* dev_psi, void* cuda_stream, double* p_marked,
                                              double* amp_marked, int* chi_out) {
  CallRange range_("grover_mps_run_noalloc");
  gmps_config c{};
  c.n = n;
  c.M = M;
  c.marked = marked;
  c.dtype = GMPS_C128;
  c.apply = apply;
  c.chi_max = chi_max;
  c.tol = tol;
  gmps_status s = validate(&c);
  if (s) return s;
  if (apply == GMPS_APPLY_GATES) return fail(GMPS_ERR_UNSUPPORTED, "grover_mps_run_noalloc runs Grover iterations");
  if (!p_marked) return fail(GMPS_ERR_ARG, "p_marked is NULL");
  if (k < 0) return fail(GMPS_ERR_ARG, "k must be >= 0");
  Plan P;
  if ((s = make_plan_for(&c, true, &P))) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // carve the static array like a handle's slab
  const size_t site_bytes = P.site_elems * P.elem_bytes;
  const size_t o_desc = 0, o_off = a256(sizeof(InstDesc));
  const size_t o_stats = o_off + a256(sizeof(long long) * (n + 1));
  const size_t o_marked = o_stats + a256(sizeof(DevStats));
  const size_t o_amp = o_marked + a256(sizeof(uint64_t) * M);
  const size_t o_sites = o_amp + a256(sizeof(double) * 2 * M);
  const size_t o_work = o_sites + a256(site_bytes);
  const size_t need = o_work + a256(P.work_bytes);
  if (need > kNoAllocScratchBytes)
    return fail(GMPS_ERR_CAPACITY, "instance needs " + std::to_string(need) +
                                       " bytes of static scratch; grover_mps_run_noalloc holds " +
                                       std::to_string(kNoAllocScratchBytes));
  void* base = nullptr;
  cudaError_t e = noalloc_scratch_address(&base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
  unsigned char* b = (unsigned char*)base;
  const RankRule rr = rank_rule_for(GMPS_C128);
  InstDesc d{};
  d.n = n;
  d.M = M;
  d.apply = apply;
  d.chi_max = chi_max;
  d.chicap = P.chicap;
  d.xcap = P.xcap;
  d.rcap = P.rcap;
  d.max_sweeps = kDefaultMaxSweeps;
  d.resident = P.resident;
  d.k = k;
  d.phase_offset = 0;
  d.tol = tol;
  d.trunc_eps = rr.eps;
  d.trunc_dim = rr.dim;
  d.inv_sqrt_N = std::ldexp(1.0, -n / 2) * ((n & 1) ? std::sqrt(0.5) : 1.0);
  d.marked = (const unsigned long long*)(b + o_marked);
  d.phi = dev_phi;
  d.psi = dev_psi;
  d.sites = b + o_sites;
  d.work = P.work_bytes ? (void*)(b + o_work) : nullptr;
  d.site_off = (const long long*)(b + o_off);
  d.stats = (DevStats*)(b + o_stats);
  const InstDesc* d_desc = (const InstDesc*)(b + o_desc);
  double* d_amp = (double*)(b + o_amp);
  // everything the kernels read is rewritten here: the array keeps the
  // previous call's contents
  CUDA_TRY(cudaMemcpyAsync(b + o_desc, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(b + o_off, P.off, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(b + o_marked, marked, sizeof(uint64_t) * M, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(launch_init(d_desc, 1, GMPS_C128, 64, stream));  // statistics and the |+>^n chain
  if (k > 0) CUDA_TRY(launch_iterate(d_desc, 1, nullptr, GMPS_C128, P.threads, P.smem, 1, stream, P.cluster));
  CUDA_TRY(launch_amplitudes(d_desc, 0, GMPS_C128, (const unsigned long long*)(b + o_marked), M, d_amp, stream));
  double amps[2 * kMaxMarked];
  DevStats ds;
  CUDA_TRY(cudaMemcpyAsync(amps, d_amp, sizeof(double) * 2 * M, cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaMemcpyAsync(&ds, b + o_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (ds.status != 0)
    return fail((gmps_status)ds.status, "device reported an error (status " + std::to_string(ds.status) + ")");
  double p = 0.0;
  for (int i = 0; i < M; ++i) p += amps[2 * i] * amps[2 * i] + amps[2 * i + 1] * amps[2 * i + 1];
  *p_marked = p;
  if (amp_marked)
    for (int i = 0; i < 2 * M; ++i) amp_marked[i] = amps[i];
  if (chi_out)
    for (int l = 0; l <= n; ++l) chi_out[l] = ds.chi[l];
  return GMPS_OK;
}
