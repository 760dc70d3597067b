// eval.cu -- factor initialisation, test RMSE, objective and factor copies.
//
// Initialisation (Alg. 1; Sec. 5.1): every entry of W and H is an
// independent UniformReal(0, 1/sqrt(k)) (in E4M3 storage of W: those values
// rounded to nearest with each row's scale).  Entry (r, l) of factor f (0 = W,
// 1 = H) takes word (l mod 4) of Philox4x32-10(key = seed, counter =
// (l/4, r_lo, r_hi, f)); u = (word >> 8) 2^-24 and the entry is the binary32
// product u * c, c = binary32(1/sqrt k) computed on the host.
//
// Test RMSE (Sec. 5.1) and the objective J (Eq. obj_fcn, per-rating form):
// residuals and norms in binary32 per rating, sums in binary64: per-block
// partial sums are written to scratch memory and added in a fixed order by a
// second one-block kernel, so the result does not depend on scheduling.
#include <cmath>

#include "nomad_internal.cuh"

namespace nomad {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kEvalThreads = 256;

// bfloat16 (upper half of a binary32): widening is exact; narrowing rounds to
// nearest, ties to even (initial values and factors set by the caller).
__device__ __forceinline__ uint32_t bf16_rn(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return (u >> 16) | ((u & 0x007fffffu) ? 0x40u : 0u);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float4 widen4(uint2 c) {
  return make_float4(__uint_as_float(c.x << 16), __uint_as_float(c.x & 0xffff0000u),
                     __uint_as_float(c.y << 16), __uint_as_float(c.y & 0xffff0000u));
}
__device__ __forceinline__ float4 widen4(float4 c) { return c; }
// a chunk of W as binary32: binary32 / bfloat16 chunks, or four E4M3 codes
// times the row's scale
__device__ __forceinline__ float4 widen_w4(float4 c, const float*, int64_t) { return c; }
__device__ __forceinline__ float4 widen_w4(uint2 c, const float*, int64_t) { return widen4(c); }
__device__ __forceinline__ float4 widen_w4(uint32_t c, const float* scale, int64_t row) {
  return e4m3_unpack(c, scale[row]);
}
__device__ __forceinline__ uint2 narrow4(float4 v) {
  return make_uint2(bf16_rn(v.x) | (bf16_rn(v.y) << 16), bf16_rn(v.z) | (bf16_rn(v.w) << 16));
}
constexpr int kEvalBlocksPerSm = 8;

template <typename C>
__global__ void init_factor_kernel(C* __restrict__ F, int64_t rows, int32_t k,
                                   int32_t k4, int64_t pitch4, float c,
                                   uint32_t which, uint2 seed) {
  const int64_t total = rows * k4;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / k4;
    const int32_t ch = int32_t(t - r * k4);
    const uint4 w = philox4x32_10(
        make_uint4(uint32_t(ch), uint32_t(r), uint32_t(uint64_t(r) >> 32), which), seed);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float u = float(words[i] >> 8) * (1.0f / 16777216.0f);  // exact
      v[i] = (4 * ch + i < k) ? __fmul_rn(u, c) : 0.0f;
    }
    const float4 c4 = make_float4(v[0], v[1], v[2], v[3]);
    if constexpr (sizeof(C) == 16) F[r * pitch4 + ch] = c4;
    else F[r * pitch4 + ch] = narrow4(c4);
  }
}

// Initial W in E4M3 storage: the binary32 values of init_factor_kernel,
// then per row the scale (largest magnitude / 448) and codes rounded to
// nearest.  One warp per row, lane l holds chunks l, l + 32, ...
__global__ void init_w_e4m3_kernel(uint32_t* __restrict__ codes, float* __restrict__ scales,
                                   int64_t rows, int32_t k, int32_t k4, int64_t pitch4, float c,
                                   uint2 seed) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows; r += nwarps) {
    float4 v[4];
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ch = lane + 32 * i;
      v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ch < k4) {
        const uint4 w = philox4x32_10(
            make_uint4(uint32_t(ch), uint32_t(r), uint32_t(uint64_t(r) >> 32), kTagInitW), seed);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float u = float(words[j] >> 8) * (1.0f / 16777216.0f);  // exact
          x[j] = (4 * ch + j < k) ? __fmul_rn(u, c) : 0.0f;
        }
        v[i] = make_float4(x[0], x[1], x[2], x[3]);
      }
      a = abs_max4(v[i], a);
    }
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(kFull, a, o));
    float sc, g;
    e4m3_row_scale(a, &sc, &g);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ch = lane + 32 * i;
      if (ch < k4) codes[r * pitch4 + ch] = e4m3_pack(v[i], g, false, 0u, 0u);
    }
    if (lane == 0) scales[r] = sc;
  }
}

// Dense binary32 rows (k entries each) into E4M3 codes and scales, rounded
// to nearest; one warp per row.
__global__ void f32_rows_to_e4m3(const float* __restrict__ src, int64_t rows, int32_t k,
                                 int32_t k4, int64_t pitch4, uint32_t* __restrict__ codes,
                                 float* __restrict__ scales) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows; r += nwarps) {
    float4 v[4];
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ch = lane + 32 * i;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      if (ch < k4) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * ch + j < k) x[j] = src[r * k + 4 * ch + j];
      }
      v[i] = make_float4(x[0], x[1], x[2], x[3]);
      a = abs_max4(v[i], a);
    }
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(kFull, a, o));
    float sc, g;
    e4m3_row_scale(a, &sc, &g);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ch = lane + 32 * i;
      if (ch < k4) codes[r * pitch4 + ch] = e4m3_pack(v[i], g, false, 0u, 0u);
    }
    if (lane == 0) scales[r] = sc;
  }
}

__global__ void e4m3_rows_to_f32(const uint8_t* __restrict__ codes, const float* __restrict__ scales,
                                 int64_t rows, int32_t k, int32_t pitch, float* __restrict__ dst) {
  const int64_t total = rows * k;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / k, l = t - r * k;
    dst[t] = __fmul_rn(scales[r], e4m3_value(codes[r * pitch + l]));
  }
}

// Group of G lanes per rating (G = power of two >= number of 4-entry chunks,
// at most 32); each warp handles 32/G ratings at a time.
__device__ __forceinline__ float group_sum(float v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ void block_store_sum(double acc, double* __restrict__ partials) {
  __shared__ double red[kEvalThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kEvalThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

template <typename CW, typename CH>
__global__ void __launch_bounds__(kEvalThreads)
sq_error_kernel(const CW* __restrict__ W4, const float* __restrict__ Wscale,
                const CH* __restrict__ H4,
                int64_t pitch4, int32_t k4, int32_t G, const int32_t* __restrict__ rows,
                const int32_t* __restrict__ cols, const float* __restrict__ vals,
                int64_t nnz, int64_t m, int64_t n, int32_t* __restrict__ status,
                double* __restrict__ partials) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int per_warp = 32 / G;
  const int64_t gwarp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t base = gwarp * per_warp; base < nnz; base += nwarps * per_warp) {
    const int64_t r = base + lane / G;
    bool ok = r < nnz;
    int64_t i = ok ? rows[r] : 0, j = ok ? cols[r] : 0;
    if (ok && (i < 0 || i >= m || j < 0 || j >= n)) {  // caller's index out of range
      if (sub == 0) atomicCAS(status, 0, NOMAD_ERR_RANGE);
      ok = false;
      i = 0;
      j = 0;
    }
    float part = 0.f;
    for (int ch = sub; ch < k4; ch += G) {
      const float4 w = widen_w4(W4[i * pitch4 + ch], Wscale, i), h = widen4(H4[j * pitch4 + ch]);
      part = fmaf(w.x, h.x, part);
      part = fmaf(w.y, h.y, part);
      part = fmaf(w.z, h.z, part);
      part = fmaf(w.w, h.w, part);
    }
    const float dot = group_sum(part, G);
    if (ok && sub == 0) {
      const float e = vals[r] - dot;
      acc += double(e) * double(e);
    }
  }
  block_store_sum(acc, partials);
}

// J over the loaded training ratings, visiting segment by segment so that
// h_j of the segment's item is known.
template <typename CW, typename CH>
__global__ void __launch_bounds__(kEvalThreads)
objective_kernel(const CW* __restrict__ W4, const float* __restrict__ Wscale,
                 const CH* __restrict__ H4,
                 int64_t pitch4, int32_t k4, const int2* __restrict__ rec,
                 const int64_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_col,
                 int64_t n_seg, float lambda, double* __restrict__ partials) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t s = gwarp; s < n_seg; s += nwarps) {
    const int64_t j = seg_col[s];
    float hh = 0.f;
    for (int ch = lane; ch < k4; ch += 32) {
      const float4 h = widen4(H4[j * pitch4 + ch]);
      hh = fmaf(h.x, h.x, fmaf(h.y, h.y, fmaf(h.z, h.z, fmaf(h.w, h.w, hh))));
    }
    hh = group_sum(hh, 32);
    for (int64_t r = seg_ptr[s]; r < seg_ptr[s + 1]; ++r) {
      const int2 rc = rec[r];
      const int64_t i = rc.x;
      float dot = 0.f, ww = 0.f;
      for (int ch = lane; ch < k4; ch += 32) {
        const float4 w = widen_w4(W4[i * pitch4 + ch], Wscale, i),
                     h = widen4(H4[j * pitch4 + ch]);
        dot = fmaf(w.x, h.x, fmaf(w.y, h.y, fmaf(w.z, h.z, fmaf(w.w, h.w, dot))));
        ww = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, fmaf(w.w, w.w, ww))));
      }
      dot = group_sum(dot, 32);
      ww = group_sum(ww, 32);
      if (lane == 0) {
        const float e = __int_as_float(rc.y) - dot;
        acc += double(e) * double(e) + double(lambda) * (double(ww) + double(hh));
      }
    }
  }
  block_store_sum(acc, partials);
}

__global__ void sum_partials(const double* __restrict__ partials, int n,
                             double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x); ++w) t += red[w];
    *out = t;
  }
}

__global__ void bf16_rows_to_f32(const uint16_t* __restrict__ src, int64_t rows, int32_t k,
                                 int32_t pitch, float* __restrict__ dst) {
  const int64_t total = rows * k;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / k, l = t - r * k;
    dst[t] = __uint_as_float(uint32_t(src[r * pitch + l]) << 16);
  }
}

__global__ void f32_rows_to_bf16(const float* __restrict__ src, int64_t rows, int32_t k,
                                 int32_t pitch, uint16_t* __restrict__ dst) {
  const int64_t total = rows * int64_t(pitch);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / pitch, l = t - r * pitch;
    dst[t] = l < k ? uint16_t(bf16_rn(src[r * k + l])) : uint16_t(0);
  }
}

int eval_grid(nomad_handle* h) {
  int g = h->sm_count * kEvalBlocksPerSm;
  return g > 0 ? g : 1;
}

int ensure_partials(nomad_handle* h, int n) {
  if (h->partials_cap >= n) return NOMAD_OK;
  void* p = h->partials;
  dev_free(h, &p);
  h->partials = nullptr;
  if (dev_alloc(h, &p, sizeof(double) * n) != cudaSuccess) return NOMAD_ERR_OOM;
  h->partials = static_cast<double*>(p);
  h->partials_cap = n;
  return NOMAD_OK;
}

}  // namespace

int init_factors(nomad_handle* h, cudaStream_t st) {
  const float c = float(1.0 / std::sqrt(double(h->k)));
  const uint2 seed = make_uint2(uint32_t(h->sched.seed), uint32_t(h->sched.seed >> 32));
  const int64_t pitch4 = h->pitch / 4;
  const int grid = eval_grid(h);
  if (h->w_elem == 1) {
    init_w_e4m3_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<uint32_t*>(h->W), h->Wscale,
                                                     h->m, h->k, h->k4, pitch4, c, seed);
    init_factor_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<float4*>(h->H), h->n, h->k,
                                                     h->k4, pitch4, c, kTagInitH, seed);
  } else if (h->elem == 2) {
    init_factor_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<uint2*>(h->W), h->m, h->k,
                                                     h->k4, pitch4, c, kTagInitW, seed);
    init_factor_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<uint2*>(h->H), h->n, h->k,
                                                     h->k4, pitch4, c, kTagInitH, seed);
  } else {
    init_factor_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<float4*>(h->W), h->m, h->k,
                                                     h->k4, pitch4, c, kTagInitW, seed);
    init_factor_kernel<<<grid, kEvalThreads, 0, st>>>(static_cast<float4*>(h->H), h->n, h->k,
                                                     h->k4, pitch4, c, kTagInitH, seed);
  }
  h->launches += 2;
  return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
}

int rmse_sum(nomad_handle* h, int64_t nnz, const int32_t* d_rows, const int32_t* d_cols,
             const float* d_vals, double* out, cudaStream_t st) {
  const int grid = eval_grid(h);
  if (int rc = ensure_partials(h, grid)) return rc;
  int G = 1;
  while (G < h->k4 && G < 32) G <<= 1;
  if (h->w_elem == 1)
    sq_error_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const uint32_t*>(h->W), h->Wscale, static_cast<const float4*>(h->H),
        h->pitch / 4, h->k4, G, d_rows, d_cols, d_vals, nnz, h->m, h->n, h->status, h->partials);
  else if (h->elem == 2)
    sq_error_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const uint2*>(h->W), nullptr, static_cast<const uint2*>(h->H), h->pitch / 4,
        h->k4, G, d_rows, d_cols, d_vals, nnz, h->m, h->n, h->status, h->partials);
  else
    sq_error_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const float4*>(h->W), nullptr, static_cast<const float4*>(h->H), h->pitch / 4,
        h->k4, G, d_rows, d_cols, d_vals, nnz, h->m, h->n, h->status, h->partials);
  sum_partials<<<1, 256, 0, st>>>(h->partials, grid, h->result);
  h->launches += 2;
  if (cudaMemcpyAsync(out, h->result, sizeof(double), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return NOMAD_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
}

int objective_sum(nomad_handle* h, double* out, cudaStream_t st) {
  const int grid = eval_grid(h);
  if (int rc = ensure_partials(h, grid)) return rc;
  if (h->w_elem == 1)
    objective_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const uint32_t*>(h->W), h->Wscale, static_cast<const float4*>(h->H),
        h->pitch / 4, h->k4, h->rec, h->seg_ptr, h->seg_col, h->n_seg, h->lambda, h->partials);
  else if (h->elem == 2)
    objective_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const uint2*>(h->W), nullptr, static_cast<const uint2*>(h->H), h->pitch / 4,
        h->k4, h->rec, h->seg_ptr, h->seg_col, h->n_seg, h->lambda, h->partials);
  else
    objective_kernel<<<grid, kEvalThreads, 0, st>>>(
        static_cast<const float4*>(h->W), nullptr, static_cast<const float4*>(h->H), h->pitch / 4,
        h->k4, h->rec, h->seg_ptr, h->seg_col, h->n_seg, h->lambda, h->partials);
  sum_partials<<<1, 256, 0, st>>>(h->partials, grid, h->result);
  h->launches += 2;
  if (cudaMemcpyAsync(out, h->result, sizeof(double), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return NOMAD_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
}

int factors_to_f32(nomad_handle* h, int which, float* d_dense, cudaStream_t st) {
  const int64_t rows = which == 0 ? h->m : h->n;
  const void* src = which == 0 ? h->W : h->H;
  if (which == 0 && h->w_elem == 1) {
    e4m3_rows_to_f32<<<eval_grid(h), kEvalThreads, 0, st>>>(static_cast<const uint8_t*>(src),
                                                           h->Wscale, rows, h->k, h->pitch,
                                                           d_dense);
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
  }
  if (h->elem == 2) {
    bf16_rows_to_f32<<<eval_grid(h), kEvalThreads, 0, st>>>(static_cast<const uint16_t*>(src),
                                                           rows, h->k, h->pitch, d_dense);
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
  }
  const cudaError_t e =
      cudaMemcpy2DAsync(d_dense, sizeof(float) * h->k, src, sizeof(float) * h->pitch,
                        sizeof(float) * h->k, rows, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
}

int factors_from_f32(nomad_handle* h, int which, const float* d_dense, cudaStream_t st) {
  const int64_t rows = which == 0 ? h->m : h->n;
  void* dst = which == 0 ? h->W : h->H;
  if (which == 0 && h->w_elem == 1) {
    f32_rows_to_e4m3<<<eval_grid(h), kEvalThreads, 0, st>>>(d_dense, rows, h->k, h->k4,
                                                           h->pitch / 4, static_cast<uint32_t*>(dst),
                                                           h->Wscale);
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
  }
  if (h->elem == 2) {
    f32_rows_to_bf16<<<eval_grid(h), kEvalThreads, 0, st>>>(d_dense, rows, h->k, h->pitch,
                                                           static_cast<uint16_t*>(dst));
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
  }
  const cudaError_t e =
      cudaMemcpy2DAsync(dst, sizeof(float) * h->pitch, d_dense, sizeof(float) * h->k,
                        sizeof(float) * h->k, rows, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? NOMAD_OK : NOMAD_ERR_CUDA;
}

}  // namespace nomad
