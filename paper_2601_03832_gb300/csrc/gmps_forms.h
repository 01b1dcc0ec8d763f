// The three arithmetic forms of the engine as one launcher family each.
// gmps_device.cuh defines the members; gmps_form_c128.cu, gmps_form_c64.cu and
// gmps_form_dw.cu each instantiate one form (so the forms compile in
// parallel); gmps_launch.cu dispatches on gmps_dtype.
#pragma once
#include <cuda_runtime.h>

#include "gmps_dw.cuh"
#include "gmps_internal.h"

namespace gmps {

// T = real type of the QR/SVD and scalar bookkeeping, S = storage type of a
// complex site element, CR = real type of the contractions.
template <class T, class S, class CR>
struct FormLaunch {
  static cudaError_t init(const InstDesc* d_desc, int count, cudaStream_t stream);
  static cudaError_t iterate(const InstDesc* d_desc, int count, int* d_queue, int threads, size_t smem, int grid,
                             cudaStream_t stream, int cluster);
  static cudaError_t adjoint(const InstDesc* d_mu, const AdjArgs* d_args, int count, int threads, size_t smem,
                             long long k_lo, long long k_hi, int project, cudaStream_t stream);
  static cudaError_t amplitudes(const InstDesc* d_desc, int inst, const unsigned long long* d_bits, int nbits,
                                double* d_out, cudaStream_t stream);
  static cudaError_t batch_prob(const InstDesc* d_desc, int count, double* d_p, cudaStream_t stream);
  static cudaError_t sample(const InstDesc* d_desc, int inst, int chmax, long long shots, unsigned long long seed,
                            unsigned long long* d_bits, double* d_margin, cudaStream_t stream);
  static cudaError_t copy_sites(const InstDesc* d_src, const InstDesc* d_dst, int count, cudaStream_t stream);
  static cudaError_t circuit(const InstDesc* d_desc, const GateOp* d_gates, long long count, long long repeat,
                             int threads, size_t smem, cudaStream_t stream);
};

using FormC128 = FormLaunch<double, double2, double>;  // GMPS_C128
using FormC64 = FormLaunch<double, float2, float>;     // GMPS_C64_F64SVD
using FormDW = FormLaunch<dw, dw2, dw>;                 // GMPS_DW

}  // namespace gmps
