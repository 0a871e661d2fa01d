// Dual MM kernels on groups of 2 lane(s) (up to 32 labels), int16_t dual deltas.
#include "dmg_impl.cuh"

namespace dm {
template cudaError_t launch_g<2, int16_t>(const Dmm16Args&, int, cudaStream_t);
template cudaError_t launch_g_batch<2, int16_t>(const Batch16Args&, int, cudaStream_t);
}  // namespace dm
