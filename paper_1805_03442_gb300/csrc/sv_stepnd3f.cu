// sv_stepnd3f.cu -- the float 3D field-pair step (sv_stepnd3f.cuh) for float
// and compensated-float pressure, and the host entry points.
#include "sv_stepnd3f.cuh"

namespace sv {

int stepnd3f_default_seg() { return Tile3f::SEG; }

// Float (PREC_FP32), compensated-float (PREC_FP32_PC) and perturbation-layout
// (PREC_FP32_PS) 3D steps; n == nullptr: set the kernel's shared-memory limit
// (host side, at set-up).
cudaError_t stepnd3f_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                            const int64_t* n, int seg, cudaStream_t st) {
  if (precision == PREC_FP32_PS) return stepnd3f_launch_ps(kp, a, b, ctl, n, seg, st);
  if (precision == PREC_FP32_PC) return by_lim3f<2>(kp, a, b, ctl, n, seg, st);
  if (precision == PREC_FP32) return by_lim3f<0>(kp, a, b, ctl, n, seg, st);
  return cudaErrorInvalidValue;
}

}  // namespace sv
