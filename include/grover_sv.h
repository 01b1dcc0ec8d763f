/*
 * grover_sv.h -- iterative Grover on a dense statevector (libgrover_mps.so).
 *
 * The paper's iterative method (Sec. III-A) on the statevector backend that
 * Sec. III-B-1 describes: the full 2^n amplitude vector is kept in device
 * memory and replaced by G|state> once per iteration, G = D(psi) O(phi)
 * (Sec. II, Eq. 3, in the phase-generalised form of grover_mps.h):
 *
 *     u = O v:   u(w) = e^{i phi} v(w) for w in W, u(x) = v(x) otherwise
 *     v' = D u:  v'(x) = (1 - e^{i psi}) (sum_y u(y)) / N - u(x)
 *
 * Each iteration is one streaming pass over the vector (read v, write v')
 * that also accumulates sum_x v'(x) for the next iteration; the last block of
 * the pass adds the marked entries' correction.  This is the memory-bound
 * baseline against which the MPS path is compared (the crossover in n of
 * Sec. IV-1).
 *
 * Conventions as in grover_mps.h: basis index x = sum_l b_l 2^l; statuses are
 * gmps_status; host pointers are copied synchronously; the CUDA stream is
 * borrowed.  Storage: complex128 (dtype GMPS_C128) or complex64 (dtype
 * GMPS_C64_F64SVD: complex64 amplitudes, FP64 sums and coefficients).
 */
#ifndef GROVER_SV_H
#define GROVER_SV_H

#include <stddef.h>
#include <stdint.h>

#include "grover_mps.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsv_ctx* gsv_handle;

/* Device bytes a handle of n qubits in `dtype` allocates. */
gmps_status grover_sv_bytes(int n, int dtype, size_t* bytes);

/* Create a statevector holding |s> = N^{-1/2} sum_x |x> (Eq. 2).  Validates
 * 1 <= n <= 36, 1 <= M <= 64, M < 2^n, marked distinct and < 2^n; dtype
 * GMPS_C128 or GMPS_C64_F64SVD.  Allocates 2^n amplitudes (16 or 8 bytes
 * each) plus O(SMs) scratch. */
gmps_status grover_sv_create(int n, const uint64_t* marked, int M, int dtype, void* cuda_stream,
                             gsv_handle* out);

/* Back to |s>. */
gmps_status grover_sv_reset(gsv_handle h);

/* k iterations G_j = D(psi_j) O(phi_j); host_phi / host_psi: k phases each
 * or NULL for pi.  One launch per iteration (replayed from CUDA graphs of up
 * to 64 launches).  Synchronises the stream. */
gmps_status grover_sv_iterate(gsv_handle h, int64_t k, const double* host_phi, const double* host_psi);

/* <bits|psi> (host doubles). */
gmps_status grover_sv_amplitude(gsv_handle h, uint64_t bits, double* re, double* im);

/* sum_{w in W} |<w|psi>|^2. */
gmps_status grover_sv_prob_marked(gsv_handle h, double* p);

/* Copy the whole vector to the host as complex128 (interleaved re, im);
 * capacity in doubles, at least 2^(n+1). */
gmps_status grover_sv_export(gsv_handle h, double* host_out, size_t capacity);

gmps_status grover_sv_destroy(gsv_handle h);

#ifdef __cplusplus
}
#endif
#endif /* GROVER_SV_H */
