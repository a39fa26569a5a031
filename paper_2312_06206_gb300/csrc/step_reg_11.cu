// step_reg_11.cu -- explicit instantiation of the register-FFT step kernels at
// FFT length 2^11 (the dense-inverse form's FFT part).
#include "step_reg.cuh"

namespace sadi {
namespace regk {
template cudaError_t launch_reg_impl<11>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
}  // namespace regk
}  // namespace sadi
