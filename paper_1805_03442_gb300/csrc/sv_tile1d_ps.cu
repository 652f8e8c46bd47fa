// sv_tile1d_ps.cu -- the block-tile 1D step (sv_tile1d.cuh) in the
// perturbation layout.
#include "sv_tile1d.cuh"

namespace sv {

void* tile1d_pick_ps(const KParams& kp, int var) { return pick_lim<3>(kp, var); }

}  // namespace sv
