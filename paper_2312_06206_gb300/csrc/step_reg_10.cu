// step_reg_10.cu -- explicit instantiations of the register-FFT step kernels (FFT length 2^10).
#include "step_reg.cuh"

namespace sadi {
namespace regk {
template cudaError_t launch_reg_impl<10>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
}  // namespace regk
}  // namespace sadi
