// Packed 16-bit Dual MM kernels for 256 labels per warp row and uint8 dual deltas.
#include "dmm16_impl.cuh"

namespace dm {
template cudaError_t launch16<4, uint8_t>(const Dmm16Args&, int, cudaStream_t);
template cudaError_t launch16_batch<4, uint8_t>(const Batch16Args&, int, bool, cudaStream_t);
}  // namespace dm
