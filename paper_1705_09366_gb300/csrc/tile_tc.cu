// K5: tcgen05 tensor-core tile kernel (placeholder until the kernel lands).
#include "internal.cuh"

namespace stkde {

bool launch_tile_tc(const Plan&, const Bins&, float*, int*, int, cudaStream_t) { return false; }

}  // namespace stkde
