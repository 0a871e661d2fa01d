// Dual MM kernels on groups of 16 lane(s) (up to 256 labels), uint8_t dual deltas.
#include "dmg_impl.cuh"

namespace dm {
template cudaError_t launch_g<16, uint8_t>(const Dmm16Args&, int, cudaStream_t);
template cudaError_t launch_g_batch<16, uint8_t>(const Batch16Args&, int, cudaStream_t);
}  // namespace dm
