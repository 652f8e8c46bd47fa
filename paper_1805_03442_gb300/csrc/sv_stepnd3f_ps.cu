// sv_stepnd3f_ps.cu -- the float 3D field-pair step (sv_stepnd3f.cuh) in the
// perturbation layout, compiled apart from the other pressure policies.
#include "sv_stepnd3f.cuh"

namespace sv {

cudaError_t stepnd3f_launch_ps(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n,
                               int seg, cudaStream_t st) {
  return by_lim3f<3>(kp, a, b, ctl, n, seg, st);
}

}  // namespace sv
