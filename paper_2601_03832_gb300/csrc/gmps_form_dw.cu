// Instantiation of the engine's kernels and launchers for one arithmetic
// form: double-word FP32 tensors and arithmetic.
#include "gmps_device.cuh"

namespace gmps {
template struct FormLaunch<dw, dw2, dw>;
}  // namespace gmps
