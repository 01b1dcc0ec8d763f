// Launch dispatch of the engine on gmps_dtype, and the host-side helpers the
// C ABI layer shares with the kernels (launch counter, storage sizes).
#include <cuda_runtime.h>

#include <atomic>

#include "gmps_forms.h"

namespace gmps {

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches += n; }
long long launches_so_far() { return g_launches.load(); }

size_t storage_bytes(int dtype) { return dtype == 1 ? sizeof(float2) : (dtype == 2 ? sizeof(dw2) : sizeof(double2)); }
size_t linalg_real_bytes(int dtype) { return dtype == 2 ? sizeof(dw) : sizeof(double); }

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

#define GMPS_DISPATCH(dtype, call) \
  ((dtype) == 1 ? FormC64::call : ((dtype) == 2 ? FormDW::call : FormC128::call))

cudaError_t launch_init(const InstDesc* d_desc, int count, int dtype, int threads, cudaStream_t stream) {
  (void)threads;
  return GMPS_DISPATCH(dtype, init(d_desc, count, stream));
}

cudaError_t launch_iterate(const InstDesc* d_desc, int count, int* d_queue, int dtype, int threads, size_t smem,
                           int grid, cudaStream_t stream, int cluster) {
  return GMPS_DISPATCH(dtype, iterate(d_desc, count, d_queue, threads, smem, grid, stream, cluster));
}

cudaError_t launch_adjoint(const InstDesc* d_mu, const AdjArgs* d_args, int count, int dtype, int threads,
                           size_t smem, long long k_lo, long long k_hi, int project, cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, adjoint(d_mu, d_args, count, threads, smem, k_lo, k_hi, project, stream));
}

cudaError_t launch_amplitudes(const InstDesc* d_desc, int inst, int dtype, const unsigned long long* d_bits,
                              int nbits, double* d_out, cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, amplitudes(d_desc, inst, d_bits, nbits, d_out, stream));
}

cudaError_t launch_batch_prob(const InstDesc* d_desc, int count, int dtype, double* d_p, cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, batch_prob(d_desc, count, d_p, stream));
}

cudaError_t launch_sample(const InstDesc* d_desc, int inst, int dtype, int chmax, long long shots,
                          unsigned long long seed, unsigned long long* d_bits, double* d_margin,
                          cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, sample(d_desc, inst, chmax, shots, seed, d_bits, d_margin, stream));
}

cudaError_t launch_copy_sites(const InstDesc* d_src, const InstDesc* d_dst, int count, int dtype,
                              cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, copy_sites(d_src, d_dst, count, stream));
}

cudaError_t launch_circuit(const InstDesc* d_desc, const GateOp* d_gates, long long count, long long repeat,
                           int dtype, int threads, size_t smem, cudaStream_t stream) {
  return GMPS_DISPATCH(dtype, circuit(d_desc, d_gates, count, repeat, threads, smem, stream));
}

}  // namespace gmps
