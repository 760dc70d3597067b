// epoch_batched.cu -- selection of the batched worker kernel (the kernel
// itself is in epoch_batched.cuh, its instances in epoch_batched_{f32,bf16,
// fp8}.cu, one translation unit per storage format).
#include "epoch_batched.cuh"

namespace nomad {

const void* batched_kernel_f32(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);
const void* batched_kernel_bf16(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);
const void* batched_kernel_fp8(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp);

namespace {

// One warp per urgent segment: lane w of the segment's (record, pair of
// chunks) items draws the pair's bits with the kernel's own rule
// (w_bits_pair) and stores them where the record's visit reads them.
__global__ void draw_urgent_bits_kernel(const int32_t* __restrict__ useg_list, int64_t n_useg,
                                        const int64_t* __restrict__ seg_ptr,
                                        const int64_t* __restrict__ useg_off, int k4, int epoch,
                                        uint2 seed, uint2* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  const int npairs = (k4 + 1) >> 1;
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_useg;
       i += warps) {
    const int s = useg_list[i];
    const int64_t beg = seg_ptr[s];
    const int64_t items = (seg_ptr[s + 1] - beg) * npairs;
    uint2* dst = out + useg_off[s] * k4;
    for (int64_t w = lane; w < items; w += 32) {
      const int64_t u = w / npairs;
      const int q = int(w - u * npairs);
      const uint4 d = w_bits_pair(beg + u, epoch, q, seed);
      dst[u * k4 + 2 * q] = make_uint2(d.x, d.y);
      if (2 * q + 1 < k4) dst[u * k4 + 2 * q + 1] = make_uint2(d.z, d.w);
    }
  }
}

}  // namespace

cudaError_t draw_urgent_bits(const int32_t* useg_list, int64_t n_useg, const int64_t* seg_ptr,
                             const int64_t* useg_off, int k4, int epoch, uint2 seed, uint2* out,
                             cudaStream_t st) {
  if (n_useg <= 0) return cudaSuccess;
  int64_t blocks = (n_useg + 7) / 8;
  if (blocks > 152 * 32) blocks = 152 * 32;
  draw_urgent_bits_kernel<<<unsigned(blocks), 256, 0, st>>>(useg_list, n_useg, seg_ptr, useg_off,
                                                             k4, epoch, seed, out);
  return cudaGetLastError();
}

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
