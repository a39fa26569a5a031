// step_reg_8.cu -- explicit instantiations of the register-FFT step kernels (FFT length 2^8).
#include "step_reg.cuh"

namespace sadi {
namespace regk {
template cudaError_t launch_reg_impl<8>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
}  // namespace regk
}  // namespace sadi
