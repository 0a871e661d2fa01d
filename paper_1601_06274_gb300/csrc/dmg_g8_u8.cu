// Dual MM kernels on groups of 8 lane(s) (up to 128 labels), uint8_t dual deltas.
#include "dmg_impl.cuh"

namespace dm {
template cudaError_t launch_g<8, uint8_t>(const Dmm16Args&, int, cudaStream_t);
template cudaError_t launch_g_batch<8, uint8_t>(const Batch16Args&, int, cudaStream_t);
}  // namespace dm
