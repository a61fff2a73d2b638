// tct_stack_inc_r12.cu -- the incremental slice stack for an inflation window of
// radius 12 cells and a p_s patch of radius 2 (its own unit, compiled in parallel).
#include "tct_stack_inc.cuh"

namespace tct {
namespace inc {

cudaError_t run_r12(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s) {
    return run_radius<12, 2>(b, tile, ctas_per_sm, s);
}

}  // namespace inc
}  // namespace tct
