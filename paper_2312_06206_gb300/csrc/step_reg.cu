// step_reg.cu -- dispatch of the register-FFT step path by FFT length.
#include "../../include/sadi.h"
#include "sadi_internal.h"

namespace sadi {
namespace regk {
template <int LOGL>
cudaError_t launch_reg_impl(const RegBatch& b, int max_n, cudaStream_t st, cudaEvent_t* ev, bool dense);
}  // namespace regk

// both FP32 forms up to N' = 1024; the dense-inverse form's FFT part (its
// sweeps are GEMMs) up to N' = 2048
bool reg_path_supported(int logNp, int prec) {
  if (prec == SADI_PREC_FP32) return logNp >= 3 && logNp <= 10;
  if (prec == SADI_PREC_FP32_DENSE) return logNp >= 3 && logNp <= 11;
  return false;
}

cudaError_t launch_step_reg(const RegBatch& b, int logNp, int max_n, cudaStream_t st, cudaEvent_t* ev, bool dense) {
  if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
  switch (logNp) {
    case 3: return regk::launch_reg_impl<3>(b, max_n, st, ev, dense);
    case 4: return regk::launch_reg_impl<4>(b, max_n, st, ev, dense);
    case 5: return regk::launch_reg_impl<5>(b, max_n, st, ev, dense);
    case 6: return regk::launch_reg_impl<6>(b, max_n, st, ev, dense);
    case 7: return regk::launch_reg_impl<7>(b, max_n, st, ev, dense);
    case 8: return regk::launch_reg_impl<8>(b, max_n, st, ev, dense);
    case 9: return regk::launch_reg_impl<9>(b, max_n, st, ev, dense);
    case 10: return regk::launch_reg_impl<10>(b, max_n, st, ev, dense);
    case 11: return regk::launch_reg_impl<11>(b, max_n, st, ev, dense);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sadi
