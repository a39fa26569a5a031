// step_reg_small.cu -- explicit instantiations of the register-FFT step kernels (FFT length 2^3,4,5,6,7).
#include "step_reg.cuh"

namespace sadi {
namespace regk {
template cudaError_t launch_reg_impl<3>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
template cudaError_t launch_reg_impl<4>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
template cudaError_t launch_reg_impl<5>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
template cudaError_t launch_reg_impl<6>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
template cudaError_t launch_reg_impl<7>(const RegBatch&, int, cudaStream_t, cudaEvent_t*, bool);
}  // namespace regk
}  // namespace sadi
