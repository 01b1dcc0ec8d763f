/*
 * grover_mps.h -- C ABI of the GB300 iterative-Grover MPS library
 * (libgrover_mps.so).
 *
 * The library simulates the iterative method of "Iterative Matrix Product
 * State Simulation for Scalable Grover's Algorithm" (Sec. III-A): an n-qubit
 * state held as a matrix product state (MPS, Sec. III-B-2) is replaced by
 * G|state> once per iteration, G = D O (Sec. II, Eq. 3) in the
 * phase-generalised form
 *
 *     O(phi) = I - (1 - e^{i phi}) sum_{w in W} |w><w|     (oracle)
 *     D(psi) = (1 - e^{i psi}) |s><s| - I                  (diffusion)
 *
 * phi = psi = pi is plain Grover.  Every iteration contracts the operator
 * into the site tensors and recompresses with a canonicalising QR sweep
 * (left to right) and a truncated one-sided-Jacobi SVD sweep (right to
 * left), which leaves the MPS right-canonical with site 0 normalised.
 *
 * Conventions shared by every entry point
 *  - Qubit / site l is bit l of a uint64_t bitstring (LSB = site 0);
 *    1 <= n <= 64.
 *  - Site tensors are complex, index order [left bond][physical][right
 *    bond], row-major.
 *  - All pointers named host_* or documented as "host" are host memory,
 *    copied synchronously during the call; the caller keeps ownership.
 *    Pointers documented as "device" must be device memory of the GPU the
 *    handle was created on, valid until the call returns (stream-ordered).
 *  - A handle owns its device arena unless the caller supplied one
 *    (gmps_config.arena), in which case the caller keeps ownership of that
 *    memory and must keep it alive until grover_mps_destroy.
 *  - The optional CUDA stream is borrowed; all work of the handle is
 *    enqueued on it.  NULL means the legacy default stream.
 *  - No exceptions cross the ABI.  Every call returns a gmps_status; a
 *    thread-local message for the last failure is returned by
 *    grover_mps_last_error().  A handle whose device work reported an error
 *    (non-convergence, non-finite norm, capacity overflow) enters an error
 *    state: every later call except stats/destroy returns GMPS_ERR_STATE.
 *    The arena ends in a canary that every synchronising call compares; a
 *    write past the instance's memory makes that call return GMPS_ERR_STATE
 *    and puts the handle in the error state.
 *  - Calls on one handle are not thread-safe; different handles are
 *    independent.
 */
#ifndef GROVER_MPS_H
#define GROVER_MPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmps_ctx* gmps_handle;
typedef struct gmps_batch_ctx* gmps_batch_handle;

typedef enum {
  GMPS_OK = 0,
  GMPS_ERR_ARG = 1,         /* invalid argument (sizes, duplicates, NULL) */
  GMPS_ERR_OOM = 2,         /* device allocation failed */
  GMPS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  GMPS_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
  GMPS_ERR_NOCONV = 5,      /* Jacobi SVD did not converge in max_sweeps */
  GMPS_ERR_NUMERIC = 6,     /* non-finite or zero norm met */
  GMPS_ERR_STATE = 7,       /* handle is in an error state / wrong order */
  GMPS_ERR_CAPACITY = 8,    /* a bond exceeded the arena's capacity */
  GMPS_ERR_UNSUPPORTED = 9  /* option combination not built */
} gmps_status;

/* Arithmetic forms (what the path computes in). */
typedef enum {
  /* complex128 site tensors; contraction, QR and SVD in IEEE FP64. */
  GMPS_C128 = 0,
  /* complex64 site tensors and complex64 contractions (MPO apply, R and
   * U*S absorption, sampling reads); QR, SVD, renormalisation and all
   * scalar bookkeeping in IEEE FP64 (the precision form). */
  GMPS_C64_F64SVD = 1,
  /* double-word FP32 ("float-float", ~48-bit significand) for contraction,
   * QR and SVD, run on the FP32 pipes; stored exactly as FP64. */
  GMPS_DW = 2
} gmps_dtype;

/* How an operator is contracted into the site tensors. */
typedef enum {
  /* O as an MPO of bond M+1, QR+SVD sweeps; D as an MPO of bond 2,
   * QR+SVD sweeps (two sweep pairs per iteration). */
  GMPS_APPLY_MPO = 0,
  /* The same two steps, each written as the direct sum of the current MPS
   * with product states: O|p> = |p> + (e^{i phi}-1) sum_w p(w)|w>
   * (bond chi+M), D|p> = (1-e^{i psi})<s|p>|s> - |p> (bond chi+1). */
  GMPS_APPLY_SPLIT = 1,
  /* G = D O as one direct sum of bond chi+M+1: one sweep pair per
   * iteration. */
  GMPS_APPLY_FUSED = 2,
  /* Gate-level circuits only (grover_mps_apply_circuit): bonds up to
   * min(chi_max, 2^floor(n/2)) for general states, expanded bond 2 chi for
   * the multi-controlled phases; grover_mps_iterate is refused. */
  GMPS_APPLY_GATES = 3
} gmps_apply;

typedef struct gmps_config {
  int n;                    /* qubits / sites, 1..64 */
  int M;                    /* number of marked strings, 1 <= M < 2^n */
  const uint64_t* marked;   /* host, M distinct strings < 2^n */
  int dtype;                /* gmps_dtype */
  int apply;                /* gmps_apply */
  int chi_max;              /* bond cap, >= 1 */
  double tol;               /* relative SVD truncation tolerance, >= 0 */
  int max_sweeps;           /* Jacobi sweep limit per SVD; 0 = default 40 */
  int threads;              /* CTA size (multiple of 32, <= 256); 0 = auto */
  int differentiable;       /* keep checkpoints for grover_mps_backward */
  int checkpoint_every;     /* iterations between checkpoints; 0 = 8 */
  int max_iters;            /* differentiable: max total iterations kept */
  void* arena;              /* optional device memory owned by the caller */
  size_t arena_bytes;       /* its size; see grover_mps_arena_bytes */
} gmps_config;

typedef struct gmps_stats {
  int64_t iterations;       /* Grover iterations applied since create/reset */
  int n;
  int chi[65];              /* bond dimensions chi_0..chi_n (chi_0=chi_n=1) */
  int max_bond;             /* largest bond after the last iteration */
  double log_norm;          /* sum of log(norm) removed by renormalisation */
  double discarded_weight;  /* sum over SVDs of dropped sigma^2 / sum sigma^2 */
  int max_jacobi_sweeps;    /* most sweeps any SVD needed */
  int64_t jacobi_sweeps;    /* sweeps summed over all SVDs */
  int64_t svd_count;        /* SVDs performed */
  int device_status;        /* gmps_status reported by the device */
  int sm_id;                /* SM that ran the instance's last iterate launch */
  int64_t t_begin_ns;       /* device clock (ns) when that launch began ... */
  int64_t t_end_ns;         /* ... and finished this instance */
  int ctas;                 /* CTAs (one SM each) that run one iterate launch of
                               the instance: 1, or the thread-block cluster whose
                               CTAs share the QR steps of a generic MPO with an
                               expanded bond of 256 or more (FP64, complex64) */
} gmps_stats;

/* ------------------------------------------------------------------ */
/* Single instance.                                                    */
/* ------------------------------------------------------------------ */

/* Device bytes the handle needs for `cfg` (arena sizing for callers that
 * allocate it themselves, e.g. from a PyTorch tensor; 256-byte aligned).
 * Includes the closing canary (256 bytes) and, for the precision forms, the
 * per-site cache of Jacobi rotations (about n * rcap^2 * 16 bytes per sweep
 * pair of an iteration). */
gmps_status grover_mps_arena_bytes(const gmps_config* cfg, size_t* bytes);

/* Create a handle holding |s> = |+>^{(x)n} (Sec. II, Eq. 2) as a bond-1
 * MPS (init of the iterative method, Sec. III-A).  `cuda_stream` is a
 * cudaStream_t (borrowed) or NULL.  Validates: 1<=n<=64, 1<=M<2^n, marked
 * strings distinct and < 2^n, chi_max>=1, tol>=0.  Uses apply =
 * GMPS_APPLY_MPO and default options. */
gmps_status grover_mps_create(int n, const uint64_t* marked, int M, int dtype,
                              int chi_max, double tol, void* cuda_stream,
                              gmps_handle* out);

/* As grover_mps_create with every option of gmps_config. */
gmps_status grover_mps_create_ex(const gmps_config* cfg, void* cuda_stream,
                                 gmps_handle* out);

/* Back to |+>^{(x)n}; clears statistics and checkpoints. */
gmps_status grover_mps_reset(gmps_handle h);

/* Apply k Grover iterations (Sec. III-A, iterative method) in one
 * persistent launch.  host_phi / host_psi: host arrays of k phases
 * (phi_j, psi_j) for iteration j, or NULL for pi (plain Grover).  Returns
 * after enqueueing and then synchronising the stream (so that device
 * status is checked). */
gmps_status grover_mps_iterate(gmps_handle h, int64_t k, const double* host_phi,
                               const double* host_psi);

/* As grover_mps_iterate with device phase arrays (or NULL) and no stream
 * synchronisation: device status is checked at the next synchronising
 * call (amplitude, prob_marked, sample, stats, sync). */
gmps_status grover_mps_iterate_device(gmps_handle h, int64_t k,
                                      const double* dev_phi,
                                      const double* dev_psi);

/* Wait for the handle's stream and check device status. */
gmps_status grover_mps_sync(gmps_handle h);

/* <bits|psi> = prod_l A_l[:, b_l, :] (chain product; the amplitude whose
 * closed form is Sec. II, Eq. 5). Output: host doubles. */
gmps_status grover_mps_amplitude(gmps_handle h, uint64_t bits, double* re,
                                 double* im);

/* P_marked = sum_{w in W} |<w|psi>|^2 (success probability, Eq. 6). */
gmps_status grover_mps_prob_marked(gmps_handle h, double* p);

/* Perfect sampling of `shots` bitstrings (Sec. IV-3 measures by shots):
 * site 0 first, p_b = |v A_l[:,b,:]|^2, bit = 1 iff u*(p0+p1) >= p0 with u
 * from Philox4x64-10 keyed (seed, 0) at counter (shot, site, 0, 0),
 * u = (word0 >> 11) * 2^-53.  out_bits: host array of `shots` uint64. */
gmps_status grover_mps_sample(gmps_handle h, int64_t shots, uint64_t seed,
                              uint64_t* out_bits);

/* As grover_mps_sample into a device array; optionally also writes, per
 * shot, the smallest |u - p0/(p0+p1)| met (device, may be NULL). */
gmps_status grover_mps_sample_device(gmps_handle h, int64_t shots, uint64_t seed,
                                     uint64_t* dev_bits, double* dev_margin);

/* Reverse-mode gradient of L = 1 - P_marked(psi_K) with respect to the
 * phases of every iteration since the last reset (differentiable handles
 * only; requires the iterations to have been applied with explicit phase
 * arrays).  dL_dP is the upstream scale (host double; the gradient is
 * dL_dP * dP/dtheta -- pass -1 for dL with L = 1 - P).  grad_phi,
 * grad_psi: host arrays of K doubles. */
gmps_status grover_mps_backward(gmps_handle h, double dL_dP, double* grad_phi,
                                double* grad_psi);

/* Statistics (synchronises). */
gmps_status grover_mps_stats(gmps_handle h, gmps_stats* out);

/* Copy site tensors to the host as complex128 (interleaved re, im) in
 * [chi_l][2][chi_{l+1}] order, sites concatenated; `capacity` is the number
 * of doubles available at host_out; *needed receives the count. */
gmps_status grover_mps_export(gmps_handle h, double* host_out, size_t capacity,
                              size_t* needed);

gmps_status grover_mps_destroy(gmps_handle h);

/* Thread-local message describing the last failing call on this thread. */
const char* grover_mps_last_error(void);

/* Fault injection for tests: the next `count` device allocations of this
 * library (handles, batches, statevectors, their buffers) fail as if the
 * device were out of memory, so that the caller sees GMPS_ERR_OOM and
 * nothing half-built is left behind.  0 clears it.  count < 0:
 * GMPS_ERR_ARG.  Process-wide; no CUDA call. */
gmps_status grover_mps_debug_fail_allocations(int count);

/* ------------------------------------------------------------------ */
/* Batched: many independent instances in one persistent launch.        */
/* ------------------------------------------------------------------ */

/* `count` instances, each described by cfgs[i] (arena fields ignored) and
 * iterated ks[i] times by grover_mps_batch_run.  Phases: plain Grover
 * unless host_phi/host_psi (arrays of pointers, each to ks[i] doubles, or
 * NULL entries) are given. */
gmps_status grover_mps_batch_create(int count, const gmps_config* cfgs,
                                    const int64_t* ks,
                                    const double* const* host_phi,
                                    const double* const* host_psi,
                                    void* cuda_stream, gmps_batch_handle* out);

/* Reset every instance to |+>^n and run all ks[i] iterations in one
 * persistent launch (work queue ordered by estimated cost).  If
 * use_graph != 0 the reset+run sequence is captured once into a CUDA graph
 * and replayed on later calls. Does not synchronise. */
gmps_status grover_mps_batch_run(gmps_batch_handle b, int use_graph);

/* Synchronise and copy back per-instance P_marked (host array of count
 * doubles) and device status (host ints, may be NULL). */
gmps_status grover_mps_batch_result(gmps_batch_handle b, double* host_p,
                                    int* host_status);

/* Amplitude <bits|psi_i> of instance i (synchronises). */
gmps_status grover_mps_batch_amplitude(gmps_batch_handle b, int i, uint64_t bits,
                                       double* re, double* im);

/* Statistics of instance i of the batch (synchronises): bond table,
 * discarded weight, Jacobi counters, device status, and the SM and device
 * clock interval that ran it in the last grover_mps_batch_run. */
gmps_status grover_mps_batch_stats(gmps_batch_handle b, int i, gmps_stats* out);

/* Override the CTA size of the batched launch (autotuner hook); 0 = auto. */
gmps_status grover_mps_batch_set_threads(gmps_batch_handle b, int threads);

gmps_status grover_mps_batch_destroy(gmps_batch_handle b);

/* ------------------------------------------------------------------ */
/* Gate-level circuits (Sec. III-A, Fig. 1A: Common and Iterative).    */
/* ------------------------------------------------------------------ */

enum {
  GMPS_GATE_1Q = 0,       /* 2x2 unitary u (row-major, re/im interleaved) on qubit `site` */
  GMPS_GATE_MCPHASE = 1   /* I - (1 - e^{i u[0]}) |1...1><1...1| on all n qubits (u[0] = pi: the
                             multi-controlled Z) */
};

typedef struct gmps_gate {
  int kind;
  int site;
  double u[8];
} gmps_gate;

/* Apply `count` gates (host array) `repeat` times to the handle's MPS, gate
 * by gate, in one persistent launch: a one-qubit gate acts on its site
 * tensor in place (the chain stays canonical); a multi-controlled phase is
 * contracted as an MPO of bond 2 and recompressed by the QR and truncated
 * SVD sweeps.  The paper's "Iterative" method passes the gates of one Grover
 * iteration with repeat = k, its "Common" method the k-iteration circuit with
 * repeat = 1.  Needs a handle whose expanded bond holds a bond-2 MPO: apply =
 * GMPS_APPLY_GATES (bonds up to chi_max, any circuit) or GMPS_APPLY_MPO
 * (bonds sized for Grover states of the handle's M).  Synchronises. */
gmps_status grover_mps_apply_circuit(gmps_handle h, const gmps_gate* gates, int64_t count, int64_t repeat);

/* The gates of `iterations` Grover iterations as in Fig. 1A: for each marked
 * string w, X on the qubits where w is 0, the multi-controlled Z, the same
 * X's (the oracle I - 2|w><w|); then H and X on every qubit, the
 * multi-controlled Z, X and H on every qubit (the diffusion I - 2|s><s|).
 * Their product is -G of Sec. II, Eq. 3 (same probabilities).  Writes
 * *count; with out != NULL also the gates, which need capacity >= *count. */
gmps_status grover_mps_grover_gates(int n, const uint64_t* marked, int M, int64_t iterations, gmps_gate* out,
                                    int64_t capacity, int64_t* count);

/* ------------------------------------------------------------------ */
/* Differentiable batch: many phase vectors of one problem at once.    */
/* ------------------------------------------------------------------ */

typedef struct gmps_diff_batch_ctx* gmps_diff_batch_handle;

/* `count` phase vectors (phi_b, psi_b), b < count, of K iterations each for
 * the problem in `cfg` (n, marked, dtype, apply, chi_max, tol, max_sweeps,
 * threads, checkpoint_every as for a differentiable handle; its
 * differentiable, max_iters and arena fields are ignored).  The loss is
 * L_b = 1 - P_marked(G_K ... G_1 |s>) with G_j = D(psi_b,j) O(phi_b,j)
 * (Sec. II, Eq. 3, phases generalised).  Allocates every vector's chain,
 * checkpoints (every checkpoint_every iterations), segment-recompute chain
 * and costate chain. */
gmps_status grover_mps_diff_batch_create(const gmps_config* cfg, int count, int K, void* cuda_stream,
                                         gmps_diff_batch_handle* out);

/* Forward and reverse sweep of all phase vectors: host_phi, host_psi are
 * count x K row-major host arrays; outputs host_loss (count values of L_b)
 * and host_gphi, host_gpsi (count x K, dL_b / dphi_b,j and dL_b / dpsi_b,j).
 * Every stage runs as one launch over all vectors (one thread block per
 * vector): the forward segments between checkpoints, the checkpoint copies,
 * the projection mu_K = Pi_W psi_K, and for each segment (last first) the
 * recompute from its checkpoint and the costate sweep.  Synchronises. */
gmps_status grover_mps_diff_batch_run(gmps_diff_batch_handle b, const double* host_phi, const double* host_psi,
                                      double* host_loss, double* host_gphi, double* host_gpsi);

gmps_status grover_mps_diff_batch_destroy(gmps_diff_batch_handle b);

/* Number of kernel launches this library has enqueued on any stream since
 * load (counts every <<<>>> launch and graph kernel node replay). */
int64_t grover_mps_launch_count(void);

/* ------------------------------------------------------------------ */
/* Allocation-free run (no counterpart in the paper).                   */
/* ------------------------------------------------------------------ */

/* For callers that must not allocate device memory (no cudaMalloc/cudaFree
 * after start-up, or an allocator they may not touch): runs one FP64
 * (complex128) instance -- |+>^n, k iterations, the marked amplitudes and
 * the bond table -- entirely inside a fixed 2 MiB device array compiled into
 * the library, with no handle and no device allocation of any kind.  Inputs
 * are validated, planned and truncated exactly as grover_mps_create_ex does
 * for dtype GMPS_C128 with the same apply, chi_max and tol (same statuses,
 * same bonds).
 *   marked      host, M distinct strings < 2^n (copied during the call)
 *   apply       gmps_apply; chi_max, tol as in gmps_config
 *   dev_phi/psi device arrays of k phases, or NULL for pi
 *   p_marked    host output: sum_w |<w|psi>|^2
 *   amp_marked  host output, 2M doubles (re, im per marked string) or NULL
 *   chi_out     host output, n+1 ints (bond dimensions chi_0..chi_n) or NULL
 * The call synchronises `cuda_stream`.  Instances whose chain needs more
 * than the array's 2 MiB return GMPS_ERR_CAPACITY.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture.  All calls share the one array:
 * calls whose GPU work overlaps (unordered streams or threads) race. */
gmps_status grover_mps_run_noalloc(int n, const uint64_t* marked, int M, int apply, int chi_max,
                                   double tol, int64_t k, const double* dev_phi,
                                   const double* dev_psi, void* cuda_stream, double* p_marked,
                                   double* amp_marked, int* chi_out);

#ifdef __cplusplus
}
#endif
#endif /* GROVER_MPS_H */
