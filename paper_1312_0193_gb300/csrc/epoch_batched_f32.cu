// epoch_batched_f32.cu -- the batched worker kernel's instances for binary32 storage
// (one translation unit per storage format, compiled in parallel).
#include "epoch_batched.cuh"

namespace nomad {

const void* batched_kernel_f32(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp) {
  return batched_ptr_k4<kF32>(k4, debug, many, blk, smem_per_warp);
}

}  // namespace nomad
