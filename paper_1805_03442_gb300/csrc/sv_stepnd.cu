// sv_stepnd.cu -- fused 2D/3D unsplit MUSCL-Hancock steps (placeholder until
// the multi-dimensional kernels land).
#include "sv_internal.h"
#include "sv_model.cuh"

namespace sv {

int stepnd_grid(int, int) { return 1; }

cudaError_t stepnd_launch(int, int, const KParams&, void*, void*, Ctl*, const int64_t*, int,
                          cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace sv
