// Instantiation of the engine's kernels and launchers for one arithmetic
// form: complex64 tensors and contractions, FP64 QR, SVD and bookkeeping.
#include "gmps_device.cuh"

namespace gmps {
template struct FormLaunch<double, float2, float>;
}  // namespace gmps
