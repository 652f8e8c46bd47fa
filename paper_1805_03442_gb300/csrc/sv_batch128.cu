// sv_batch128.cu -- the 128-thread instantiation of the batched sweep kernel
// (sv_batch_kernel.cuh), compiled apart from the 256-thread one.
#include "sv_batch_kernel.cuh"

namespace sv {

void* batch_pick128(int limiter, int precision) { return bpick<128>(limiter, precision); }

}  // namespace sv
