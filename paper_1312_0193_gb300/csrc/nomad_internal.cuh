// nomad_internal.cuh -- internal declarations of libnomad (GB300 / sm_103a).
//
// Device-side building blocks shared by the translation units of the CUDA
// path: the counter-based generator, memory-order primitives written as
// inline PTX, the parameter blocks of the kernels and the handle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "nomad.h"

namespace nomad {

// ---------------------------------------------------------------- generator
// Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11): ten
// rounds of two 32x32->64 multiplies, the key advanced by the Weyl constants
// between rounds.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    // one widening 32x32->64 multiply gives both halves of each product
    const uint64_t p0 = 0xD2511F53ull * c.x, p1 = 0xCD9E8D57ull * c.z;
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Stream tags: the fourth counter word separates the uses of the generator.
constexpr uint32_t kTagInitW = 0u;       // W entries (factor 0)
constexpr uint32_t kTagInitH = 1u;       // H entries (factor 1)
constexpr uint32_t kTagItinerary = 0x49544e52u;  // epoch-mode visit orders
constexpr uint32_t kTagUniform = 0x554e4946u;    // uniform-mode routing
constexpr uint32_t kTagRounding = 0x53524e44u;   // stochastic rounding

// A worker of the batched kernel takes ready tokens from the first
// kRingWindow positions at the head of its ring, not only a contiguous
// prefix; rings have kRingWindow slots of headroom for the positions taken
// ahead of the head.
constexpr int kRingWindow = 16;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned long long ld_acquire_u64(
    const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p,
                                               unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(
    const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// With a preceding relaxed load of a flag, an acquire pattern: everything the
// releasing writer did before its release store is visible afterwards.
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- E4M3
// FP8-E4M3 storage of W (sign, 4 exponent bits with bias 7, 3 mantissa
// bits; exponent field 0 holds the subnormals m 2^-9; 448 is the largest
// finite value; 0x7f / 0xff is NaN; no infinity), one binary32 scale per row:
// the stored value of entry l of row i is scale_i * decode(code_il).

// Exact value of a code.
__device__ __forceinline__ float e4m3_value(uint32_t c) {
  const uint32_t e = (c >> 3) & 15u, m = c & 7u;
  float v = e == 0u ? float(m) * 0x1p-9f : __uint_as_float(((e + 120u) << 23) | (m << 20));
  if (e == 15u && m == 7u) v = __uint_as_float(0x7fc00000u);
  return (c & 0x80u) ? -v : v;
}

// Rounding of a binary32 x to E4M3.  Stochastic (r16 = 16 random bits) or
// to nearest with ties to even (stochastic = false):
//  - |x| >= 2^-6: on the bits of |x|, keeping 3 mantissa bits; stochastic
//    adds r16 << 4 to the 20 dropped bits, nearest adds 0x7ffff plus the
//    lowest kept bit; magnitudes above 448 saturate to 448;
//  - |x| < 2^-6: on the grid m 2^-9 (t = |x| 2^9 and its fraction f are
//    exact in binary32); stochastic rounds up when r16 < f 2^16, nearest when
//    f > 1/2 or f = 1/2 with floor(t) odd;
//  - infinities saturate, NaN gives the NaN code.
// The grid m 2^-9 below 2^-6 (rare after scaling by the row's inverse scale:
// kept out of line).
static __device__ __noinline__ uint32_t e4m3_round_small(uint32_t u, bool stochastic, uint32_t r16) {
  const float t = __fmul_rn(__uint_as_float(u), 512.0f);
  const float lo = floorf(t);
  const float f = __fsub_rn(t, lo);
  const uint32_t m = uint32_t(lo);
  const bool up = stochastic ? float(r16 & 0xffffu) < __fmul_rn(f, 65536.0f)
                             : (f > 0.5f || (f == 0.5f && (m & 1u)));
  return m + (up ? 1u : 0u);
}
__device__ __forceinline__ uint32_t e4m3_round(float x, bool stochastic, uint32_t r16) {
  const uint32_t bits = __float_as_uint(x);
  const uint32_t sign = (bits >> 24) & 0x80u;
  uint32_t u = bits & 0x7fffffffu;
  if (u < 0x3c800000u) return sign | e4m3_round_small(u, stochastic, r16);
  if (u > 0x7f800000u) return sign | 0x7fu;
  // |x| >= 2^-6 (infinity included): an integer add and truncation; the
  // exponent field of the result is at least 121 (2^-6)
  u += stochastic ? (r16 & 0xffffu) << 4 : 0x7ffffu + ((u >> 20) & 1u);
  const uint32_t q = (u >> 20) - (120u << 3);  // (E4M3 exponent << 3) | mantissa
  return sign | (q > 0x7eu ? 0x7eu : q);
}

// Scale and inverse scale of a row whose largest magnitude is a:
// s = a / 448, g = 448 / a (binary32 divisions), or 1, 1 for a < 2^-100.
__device__ __forceinline__ void e4m3_row_scale(float a, float* s, float* g) {
  if (a >= 0x1p-100f) {
    *s = __fdiv_rn(a, 448.0f);
    *g = __fdiv_rn(448.0f, a);
  } else {
    *s = 1.0f;
    *g = 1.0f;
  }
}

// Four codes (entry 4c+i in byte i) of the chunk v of a row with inverse
// scale g; stochastic with ra (entries 0, 1: low and high half) and rb
// (entries 2, 3), or to nearest.
__device__ __forceinline__ uint32_t e4m3_pack(float4 v, float g, bool stochastic, uint32_t ra,
                                              uint32_t rb) {
  return e4m3_round(__fmul_rn(v.x, g), stochastic, ra) |
         (e4m3_round(__fmul_rn(v.y, g), stochastic, ra >> 16) << 8) |
         (e4m3_round(__fmul_rn(v.z, g), stochastic, rb) << 16) |
         (e4m3_round(__fmul_rn(v.w, g), stochastic, rb >> 16) << 24);
}

// The chunk's four stored values: s * decode(code), binary32 products.  The
// codes are decoded by the hardware conversion to half precision, which
// holds every E4M3 value exactly.
__device__ __forceinline__ float4 e4m3_unpack(uint32_t c, float s) {
  uint32_t lo, hi;
  asm("{\n\t.reg .b16 a, b;\n\tmov.b32 {a, b}, %2;\n\t"
      "cvt.rn.f16x2.e4m3x2 %0, a;\n\tcvt.rn.f16x2.e4m3x2 %1, b;\n\t}"
      : "=r"(lo), "=r"(hi) : "r"(c));
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  return make_float4(__fmul_rn(s, a.x), __fmul_rn(s, a.y), __fmul_rn(s, b.x), __fmul_rn(s, b.y));
}

__device__ __forceinline__ float abs_max4(float4 v, float a) {
  return fmaxf(a, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
}

// int4 words of a token's next-visit record (the batched kernel; three used,
// padded to 64 bytes so that a record never straddles a cache line)
constexpr int kTokRecInts = 4;

// ---------------------------------------------------------------- kernels
// Status words written by device code: [0] error code (0 = ok), [1] worker,
// [2] detail, [3] count of ownership violations (debug).
constexpr int kStatusWords = 4;

struct SgdParams {
  void* W;                  // m x pitch (fp32, bf16 or E4M3 codes)
  void* H;                  // n x pitch (fp32 or bf16)
  float* Wscale;            // m: the scale of each row of W (E4M3 storage only)
  int32_t pitch;            // elements per row
  int32_t k4;               // 4-element chunks holding the k entries
  const int2* rec;          // {row, value bits} in segment order
  const int64_t* seg_ptr;   // S+1
  const int32_t* seg_col;   // S
  const int32_t* seg_worker;// S
  const int32_t* worker_seg_ptr;  // p+1
  const int32_t* col_seg_ptr;     // n+1
  const int32_t* col_segs;        // S: segments of each item, by worker
  // hybrid circulation (NOMAD_CIRCULATION_BLOCK): item j's segments
  // col_segs[col_seg_ptr[j] ..] fall into G_j runs of one thread block each;
  // grp_off[col_grp_ptr[j] + g] is the offset of run g, and
  // grp_off[col_grp_ptr[j] + G_j] = the item's number of segments
  const int32_t* col_grp_ptr;     // n+1 (null: flat circulation)
  const int32_t* grp_off;
  int32_t wpb;                    // warps (workers) per thread block
  int32_t batch_cap;              // batched kernel: tokens taken at once (0: the kernel's)
  unsigned long long* ring; // lap-tagged slots {lap:32 | segment:32}
  const int64_t* ring_base; // p
  const int32_t* ring_log2; // p: log2 of the ring capacity
  uint32_t* ring_tail;      // p: producer reservation counters
  uint32_t* ring_head;      // p: tokens taken so far (uniform mode), written by the owner
  int32_t routing;          // uniform mode: NOMAD_ROUTING_*
  unsigned long long* uring;  // p x 2^uring_log2 slots: tokens of urgent items
  uint32_t* uring_tail;       // p
  int32_t uring_log2;
  int32_t use_urgent;         // urgent items travel through the urgent rings
  int32_t* tok_hop;         // n: hop within the current epoch
  int32_t* tok_epoch;       // n: absolute epoch of the token
  const uint8_t* item_urgent;  // n: 1 for the items with the most ratings
  // batched kernel: per item, the token's next visit {segment, length, first
  // record, epoch} and {hop, first of its segments, number of segments, 0};
  // ring payloads are then item ids (null: payloads are segment ids)
  int4* tok_rec;
  const float* step;        // n_epochs step sizes (epoch mode)
  int32_t epoch0;
  int32_t n_epochs;
  int32_t p;
  float lambda;
  float alpha, beta;        // uniform mode computes s_t on the fly
  uint32_t seed_lo, seed_hi;
  int64_t timeout_ns;
  int32_t* status;
  unsigned long long* span;  // 2 words: first worker start, last worker end (globaltimer ns)
  // uniform mode
  unsigned long long* upd_done;
  unsigned long long upd_budget;
  int32_t* stop;
  // debug mode
  uint32_t* log_ticket;
  int32_t* log_seg;
  int32_t* log_epoch;
  int64_t log_cap;
  int32_t* owner;
  int32_t* rec_count;
  int32_t drop_item;
  // narrow formats, one epoch per launch: the W rounding bits of the urgent
  // items' ratings for this epoch, drawn before the launch (a record's bits
  // at ubits_pre[(useg_off[s] + r - seg_ptr[s]) * k4 + chunk] for record r
  // of urgent segment s), or null (the kernel draws them)
  const int64_t* useg_off;
  const uint2* ubits_pre;
};


// ---------------------------------------------------------------- handle
struct DeviceBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace nomad

struct nomad_handle {
  int64_t m = 0, n = 0;
  int32_t k = 0, k4 = 0, pitch = 0;
  int32_t elem = 4;                // bytes per stored entry of H
  int32_t w_elem = 4;              // bytes per stored entry of W (1: E4M3 codes)
  float lambda = 0.f;
  nomad_schedule sched{};
  int device = 0;
  int sm_count = 0;
  int32_t p = 0;
  int32_t warps_per_block = 0;
  int32_t blocks = 0;
  int64_t nnz = 0;
  int64_t n_seg = 0;
  int64_t epochs_done = 0;
  int64_t ring_slots = 0;
  bool loaded = false;
  std::string last_error;
  // factors
  void* W = nullptr;
  void* H = nullptr;
  float* Wscale = nullptr;         // m: row scales of W (E4M3 storage only)
  // layout
  int32_t* row_worker = nullptr;   // m
  int2* rec = nullptr;             // nnz
  int64_t* seg_ptr = nullptr;      // S+1
  int32_t* seg_col = nullptr;      // S
  int32_t* seg_worker = nullptr;   // S
  int32_t* worker_seg_ptr = nullptr;  // p+1
  int32_t* col_seg_ptr = nullptr;  // n+1
  int32_t* col_segs = nullptr;     // S
  int32_t* col_grp_ptr = nullptr;  // n+1: hybrid circulation's runs per item
  int32_t* grp_off = nullptr;      // runs + n
  // queues and tokens
  unsigned long long* ring = nullptr;
  int64_t* ring_base = nullptr;
  int32_t* ring_log2 = nullptr;
  uint32_t* ring_tail = nullptr;
  uint32_t* ring_head = nullptr;  // p: tokens taken (uniform mode, load-balanced routing)
  unsigned long long* uring = nullptr;  // per worker: tokens of urgent items
  uint32_t* uring_tail = nullptr;
  int32_t uring_log2 = 0;
  int32_t* tok_hop = nullptr;
  int32_t* tok_epoch = nullptr;
  uint8_t* item_urgent = nullptr;  // n: item degree >= half the largest
  // narrow formats: W rounding bits of the urgent items' ratings, drawn
  // before each launch (section 10b of the layout build); null if not used
  int64_t* useg_off = nullptr;     // S: offset (records) of an urgent segment's bits
  int32_t* useg_list = nullptr;    // the urgent segments
  int64_t n_useg = 0;
  int64_t upre_records = 0;        // records of the urgent segments
  uint2* ubits_pre = nullptr;      // urgent records x k4
  int4* tok_rec = nullptr;         // 4n: next-visit record of each token
  float* step = nullptr;
  int32_t step_cap = 0;
  int32_t* status = nullptr;       // kStatusWords
  unsigned long long* span = nullptr;  // device time span of the last batched launch
  unsigned long long* upd_done = nullptr;
  int32_t* stop = nullptr;
  // scratch for reductions
  double* partials = nullptr;
  int32_t partials_cap = 0;
  double* result = nullptr;
  // debug
  uint32_t* log_ticket = nullptr;
  int32_t* log_seg = nullptr;
  int32_t* log_epoch = nullptr;
  int64_t log_cap = 0;
  int32_t* owner = nullptr;
  int32_t* rec_count = nullptr;
  int64_t device_bytes = 0;
  int64_t launches = 0;            // kernels launched by this handle
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
  bool ev_recorded = false;
  std::unordered_map<void*, size_t> allocs;
};

namespace nomad {

// Allocation bookkeeping (nomad_api.cu).
cudaError_t dev_alloc(nomad_handle* h, void** p, size_t bytes);
void dev_free(nomad_handle* h, void** p);

// Layout construction (layout.cu).  Builds everything nomad_load_ratings
// needs from device COO arrays.  Returns a NOMAD_* code.
int build_layout(nomad_handle* h, int64_t nnz, const int32_t* d_rows,
                 const int32_t* d_cols, const float* d_vals,
                 cudaStream_t stream);

// Persistent SGD kernel launch (sgd.cu).
int launch_epochs(nomad_handle* h, int32_t n_epochs, cudaStream_t stream);
int launch_epochs_many(nomad_handle* const* hs, int count, int32_t n_epochs, cudaStream_t stream);
int max_resident_workers(int device, int warps_per_block, int k4, int precision,
                         int mode, int variant, int* blocks_per_sm, bool blk = false);
int default_warps_per_block();
// Batched epoch-mode worker kernel (epoch_batched.cu): pointer and dynamic
// shared memory per warp in bytes; nullptr for an unsupported k4.
const void* batched_kernel(int k4, bool debug, int precision, bool many, bool blk,
                           size_t* smem_per_warp);
size_t batched_inbox_bytes();   // per warp, hybrid circulation only
size_t batched_params_bytes();  // per block, several-problem form
// Draws the W rounding bits of epoch `epoch` for every record of the urgent
// segments useg_list[0 .. n_useg) into out (layout of SgdParams::ubits_pre).
cudaError_t draw_urgent_bits(const int32_t* useg_list, int64_t n_useg, const int64_t* seg_ptr,
                             const int64_t* useg_off, int k4, int epoch, uint2 seed, uint2* out,
                             cudaStream_t st);

// Initialisation, evaluation and factor copies (eval.cu).
int init_factors(nomad_handle* h, cudaStream_t stream);
int rmse_sum(nomad_handle* h, int64_t nnz, const int32_t* d_rows,
             const int32_t* d_cols, const float* d_vals, double* out,
             cudaStream_t stream);
int objective_sum(nomad_handle* h, double* out, cudaStream_t stream);
int factors_to_f32(nomad_handle* h, int which, float* d_dense,
                   cudaStream_t stream);
int factors_from_f32(nomad_handle* h, int which, const float* d_dense,
                     cudaStream_t stream);

}  // namespace nomad
