// Packed 16-bit Dual MM kernels for 64 labels per warp row and int16 dual deltas.
#include "dmm16_impl.cuh"

namespace dm {
template cudaError_t launch16<1, int16_t>(const Dmm16Args&, int, cudaStream_t);
template cudaError_t launch16_batch<1, int16_t>(const Batch16Args&, int, bool, cudaStream_t);
}  // namespace dm
