// sv_tile1d_pc.cu -- the block-tile 1D step (sv_tile1d.cuh) with the
// compensated-float pressure.
#include "sv_tile1d.cuh"

namespace sv {

void* tile1d_pick_pc(const KParams& kp, int var) { return pick_lim<2>(kp, var); }

}  // namespace sv
