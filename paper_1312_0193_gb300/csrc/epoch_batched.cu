// epoch_batched.cu -- selection of the batched worker kernel (the kernel
// itself is in epoch_batched.cuh, its instances in epoch_batched_{f32,bf16,
// fp8}.cu, one translation unit per storage format).
#include "epoch_batched.cuh"

namespace nomad {

const void* batched_kernel_f32(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);
const void* batched_kernel_bf16(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);
const void* batched_kernel_fp8(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);

size_t batched_inbox_bytes() { return size_t(kInboxBytes); }
size_t batched_params_bytes() { return size_t(kParamsBytes); }

// Kernel pointer and per-warp shared memory (bytes) of the batched kernel,
// or of its several-problem form (`many`, which also takes
// batched_params_bytes() bytes per block).  The hybrid circulation (`blk`)
// adds batched_inbox_bytes() per warp.
const void* batched_kernel(int k4, bool debug, int precision, bool many, bool blk,
                           size_t* smem_per_warp) {
  if (precision == NOMAD_BF16) return batched_kernel_bf16(k4, debug, many, blk, smem_per_warp);
  if (precision == NOMAD_FP8) return batched_kernel_fp8(k4, debug, many, blk, smem_per_warp);
  return batched_kernel_f32(k4, debug, many, blk, smem_per_warp);
}

}  // namespace nomad
