// epoch_batched_fp8.cu -- the batched worker kernel's instances for E4M3 W storage
// (one translation unit per storage format, compiled in parallel).
#include "epoch_batched.cuh"

namespace nomad {

const void* batched_kernel_fp8(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp) {
  return batched_ptr_k4<kFP8>(k4, debug, many, blk, smem_per_warp);
}

}  // namespace nomad
