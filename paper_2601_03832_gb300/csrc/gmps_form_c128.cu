// Instantiation of the engine's kernels and launchers for one arithmetic
// form: complex128 tensors, FP64 contraction, QR and SVD.
#include "gmps_device.cuh"

namespace gmps {
template struct FormLaunch<double, double2, double>;
}  // namespace gmps
