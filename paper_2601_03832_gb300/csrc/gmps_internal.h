// Internal types shared by the C-ABI layer (gmps_capi.cu) and the kernels
// (gmps_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#define GMPS_HD __host__ __device__ __forceinline__

namespace gmps {

constexpr int kMaxN = 64;
constexpr int kMaxMarked = 64;        // direct-sum terms per operator
constexpr int kDefaultMaxSweeps = 40;
constexpr int kMaxCluster = 8;           // CTAs of a cluster sharing one instance's large QR steps
constexpr int kClusterMinCols = 256;     // expanded bonds from which the QR is split over the cluster
constexpr size_t kClusterCtlBytes = 256 + 16 * kMaxCluster;

enum DevStatusBits {
  kDevOK = 0,
  kDevNoConv = 5,
  kDevNumeric = 6,
  kDevCapacity = 8,
};

// Counters written by the device; one block per instance.
struct DevStats {
  long long iterations;     // iterations applied
  long long jacobi_sweeps;  // summed over SVDs
  long long svd_count;
  int max_jacobi_sweeps;
  int status;               // first error (DevStatusBits), 0 if none
  double log_norm;
  double discarded;
  int chi[kMaxN + 1];       // bond table after the last sweep pair
  unsigned long long t_begin, t_end;  // device clock (ns) when the last launch began and ended this instance
  int sm;                   // SM that ran it
  int jrank[2][kMaxN + 1];  // rows of the Jacobi rotations cached per sweep pair and site (0: none)
};

// Everything one persistent block needs for one instance.  Lives in device
// memory (array of descriptors for a batch).
struct InstDesc {
  int n;
  int M;
  int apply;                // gmps_apply
  int chi_max;              // user cap
  int chicap;               // storage capacity of a bond after truncation
  int xcap;                 // capacity of an expanded bond
  int rcap;                 // capacity of a QR-sweep bond (the rank after rank-revealing QR)
  int max_sweeps;
  int resident;             // copy the chain into shared memory for the launch
  long long k;              // iterations to apply in this launch
  long long phase_offset;   // index of this launch's first phase in phi/psi
  double tol;
  double trunc_eps;         // eps of the rank rule (see trunc_dim)
  int trunc_dim;            // 1: the rank floor is max(m, n) * trunc_eps; 0: trunc_eps itself
  double inv_sqrt_N;        // 2^{-n/2}
  const unsigned long long* marked;  // device, M strings
  const double* phi;        // device, or null = pi
  const double* psi;
  void* sites;              // device slab
  const long long* site_off;  // n+1 offsets (elements of the storage type)
  DevStats* stats;          // device
  void* work;               // device work area for the QR matrices when they exceed shared memory, else null
  int cluster;              // CTAs that share this instance's large QR steps (thread-block cluster), 1 = none
  void* jcache;             // device: each site's last Jacobi rotations per sweep pair (the next
                            // iteration's starting point) and QR pivot sequences; null = none
  int jbanks;               // sweep pairs per iteration with a cache bank (1 or 2)
  double* rec;              // optional: before each iteration, the marked amplitudes and
                            // <s|psi> of the chain, (M+1) complex per iteration
};

// One gate of a gate-level circuit (same layout as the public gmps_gate).
struct GateOp {
  int kind;      // 0: 2x2 unitary u on qubit `site`; 1: multi-controlled phase on all n qubits
  int site;
  double u[8];   // kind 0: u00, u01, u10, u11 as (re, im); kind 1: u[0] = phase
};

// Per-chain arguments of the adjoint kernel (one entry per costate chain).
struct AdjArgs {
  const double* rec;   // forward chain's marked amplitudes and <s|psi> of the segment
  const double* phi;   // all K phases of the chain's phase vector
  const double* psi;
  double* gphi;        // K gradient entries each
  double* gpsi;
  double scale;        // dL/dP
};

// Shared-memory plan of one block (bytes), identical on host and device.
// The QR sweep's matrices (R carried along the sweep, rank x expanded bond,
// and the (2 rank) x expanded-bond work matrix) sit in shared memory, aliased
// with the SVD sweep's working set, or -- when they do not fit, e.g. a
// generic MPO with an expanded bond in the thousands -- in a per-instance
// device work area (work_bytes, offsets from its base).
struct SmemPlan {
  size_t off_chi, off_qb, off_soff, off_terms, off_amps, off_misc, off_qperm, off_qcn, off_tbuf;
  size_t off_tau, off_beta;                          // QR reflector scalars (shared memory)
  size_t off_rprev, off_w;                           // QR matrices (shared memory or the work area)
  size_t off_refl, off_ctl;                          // work area only: reflectors and the cluster QR's control block
  size_t off_mat, off_u, off_us, off_sig, off_perm;  // SVD sweep (shared memory)
  size_t off_sites;
  size_t total;       // shared-memory bytes
  size_t work_bytes;  // work-area bytes, 0 when the QR matrices are in shared memory
};

GMPS_HD size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// rb = bytes of one real of the linear-algebra type (complex = 2*rb).
GMPS_HD SmemPlan make_plan(int n, int M, int xcap, int chicap, int rcap, size_t rb,
                           size_t site_bytes_resident, bool work_global) {
  SmemPlan p{};
  size_t cb = 2 * rb;
  size_t o = 0;
  p.off_chi = o;   o = align_up(o + sizeof(int) * (kMaxN + 2), 16);
  p.off_qb = o;    o = align_up(o + sizeof(int) * (kMaxN + 2), 16);
  p.off_soff = o;  o = align_up(o + sizeof(int) * (kMaxN + 2), 16);   // slot offsets
  p.off_terms = o; o = align_up(o + (sizeof(unsigned long long) + sizeof(int) + cb + 8) * (M + 2), 16);
  p.off_amps = o;  o = align_up(o + cb * (M + 2), 16);
  p.off_misc = o;  o = align_up(o + 512, 16);
  p.off_qperm = o; o = align_up(o + sizeof(int) * (size_t)xcap, 16);   // QR pivots
  p.off_qcn = o;   o = align_up(o + rb * (size_t)xcap, 16);            // QR column norms
  p.off_tbuf = o;  o = align_up(o + (cb * 32 + 16) * 2, 16);           // reflectors handed between warps
  p.off_tau = o;   o = align_up(o + rb * (size_t)xcap, 16);
  p.off_beta = o;  o = align_up(o + cb * (size_t)xcap, 16);
  const size_t base = o;
  // QR-sweep matrices
  size_t q = work_global ? 0 : base;
  p.off_rprev = q; q = align_up(q + cb * (size_t)rcap * xcap, 16);
  p.off_w = q;     q = align_up(q + cb * (size_t)(2 * rcap) * xcap, 16);
  if (work_global) {
    // a QR split over the CTAs of a cluster exchanges its reflectors and
    // pivot candidates here
    p.off_refl = q;  q = align_up(q + cb * (size_t)(2 * rcap) * rcap, 16);
    p.off_ctl = q;
    q = align_up(q + kClusterCtlBytes + align_up(sizeof(int) * (size_t)rcap, 16) + align_up(rb * (size_t)rcap, 16) +
                     cb * (size_t)rcap, 16);
  }
  p.work_bytes = work_global ? q : 0;
  // SVD-sweep working set (aliases the QR matrices when those are here)
  size_t s = base;
  p.off_mat = s;   s = align_up(s + cb * (size_t)rcap * (2 * chicap), 16);
  p.off_u = s;     s = align_up(s + cb * (size_t)rcap * rcap, 16);         // accumulated rotations
  p.off_us = s;    s = align_up(s + cb * (size_t)rcap * chicap, 16);
  p.off_sig = s;   s = align_up(s + rb * (size_t)rcap, 16);
  p.off_perm = s;  s = align_up(s + sizeof(int) * (size_t)rcap, 16);
  o = work_global ? s : (q > s ? q : s);
  p.off_sites = o;
  o = align_up(o + site_bytes_resident, 16);
  p.total = o;
  return p;
}

// Largest left/right dims a slot ever holds: QR-sweep bonds are bounded by
// 2^l from the left and by the rank capacity rcap.
GMPS_HD long long bond_cap(int l, int n, int rcap) {
  (void)n;
  long long c = 1;
  for (int i = 0; i < l && c < rcap; ++i) c *= 2;
  return c < rcap ? c : rcap;
}
GMPS_HD long long slot_elems(int l, int n, int rcap) {
  long long left = bond_cap(l, n, rcap);
  long long right = (l == n - 1) ? 1 : bond_cap(l + 1, n, rcap);
  return left * 2 * right;
}

// Device allocation of the C API: cudaMalloc, or cudaErrorMemoryAllocation
// while grover_mps_debug_fail_allocations has failures left to force.
cudaError_t dev_malloc(void** p, size_t bytes);

// Launchers (gmps_kernels.cu).  dtype: gmps_dtype.  All enqueue on `stream`.
cudaError_t launch_init(const InstDesc* d_desc, int count, int dtype, int threads,
                        cudaStream_t stream);
cudaError_t launch_iterate(const InstDesc* d_desc, int count, int* d_queue, int dtype,
                           int threads, size_t smem, int grid, cudaStream_t stream, int cluster = 1);
cudaError_t launch_amplitudes(const InstDesc* d_desc, int inst, int dtype,
                              const unsigned long long* d_bits, int nbits,
                              double* d_out /* 2*nbits */, cudaStream_t stream);
cudaError_t launch_sample(const InstDesc* d_desc, int inst, int dtype, int chmax, long long shots,
                          unsigned long long seed, unsigned long long* d_bits,
                          double* d_margin, cudaStream_t stream);
cudaError_t launch_copy_sites(const InstDesc* d_src, const InstDesc* d_dst, int count, int dtype,
                              cudaStream_t stream);
cudaError_t launch_adjoint(const InstDesc* d_mu, const AdjArgs* d_args, int count, int dtype, int threads,
                           size_t smem, long long k_lo, long long k_hi, int project, cudaStream_t stream);
cudaError_t launch_batch_prob(const InstDesc* d_desc, int count, int dtype, double* d_p,
                              cudaStream_t stream);
cudaError_t launch_circuit(const InstDesc* d_desc, const GateOp* d_gates, long long count, long long repeat,
                           int dtype, int threads, size_t smem, cudaStream_t stream);
size_t storage_bytes(int dtype);      // bytes of one complex site element
size_t linalg_real_bytes(int dtype);  // bytes of one linear-algebra real
int max_smem_optin();
void count_launch(long long n);

}  // namespace gmps
