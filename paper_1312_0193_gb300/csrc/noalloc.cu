// noalloc.cu -- test RMSE without any allocation by the library.
//
// nomad_rmse keeps its per-block partial sums in device memory that the
// handle allocates with cudaMalloc.  Some callers cannot let a library
// allocate: a service that reserves all device memory up front and hands out
// fixed buffers, a host thread that must not take the implicit device
// synchronisation of cudaMalloc/cudaFree in the middle of a latency-bound
// loop, or code that has no handle at all and only holds the factors.
// nomad_rmse_noalloc serves them: the caller passes W, H, the test ratings
// and the output in device memory, and the partial sums live in a file-scope
// __device__ array of fixed size that is part of the loaded library.
//
// The array is shared by every call on a device and keeps what the last call
// wrote; each call clears the flag it needs before it starts.  Two calls
// whose work overlaps on the GPU (different streams, no ordering between
// them) race on the array and give wrong results.
#include <cmath>
#include <mutex>

#include "nomad_internal.cuh"

namespace nomad {
namespace {

constexpr int kTileRatings = 8192;   // ratings per block
constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// One partial sum per tile, and a flag raised by an out-of-range index.
static __device__ __align__(256) double g_partials[NOMAD_NOALLOC_MAX_TILES];
static __device__ __align__(256) int g_range_flag[4];

struct SymbolAddresses {
  double* partials = nullptr;
  int* flag = nullptr;
  void* context = nullptr;  // the context the addresses belong to
  bool ready = false;
};

constexpr int kMaxDevices = 64;
SymbolAddresses g_addr[kMaxDevices];
std::mutex g_addr_mutex;

// The current driver context (cuCtxGetCurrent, reached through the runtime so
// that the library does not link the driver library); null if unavailable.
void* current_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<GetCurrent>(f);
  }();
  void* ctx = nullptr;
  if (fn == nullptr || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device addresses of the two arrays on the current device.  In host code
// the symbol names only stand in for the device objects, so the kernels get
// the addresses returned by cudaGetSymbolAddress, looked up with the device
// current: once per device, and again when the device's context is no longer
// the one the addresses were taken in (after cudaDeviceReset the module is
// loaded anew and the arrays can move).
cudaError_t symbol_addresses(int device, SymbolAddresses* out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  SymbolAddresses& a = g_addr[device];
  // null before the runtime has made the device's context current: then the
  // lookup below runs and makes it current
  void* ctx = current_context();
  if (!a.ready || ctx != a.context) {
    a.ready = false;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&a.partials), g_partials);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&a.flag), g_range_flag);
    if (e != cudaSuccess) return e;
    a.context = current_context();
    a.ready = true;
  }
  *out = a;
  return cudaSuccess;
}

__global__ void __launch_bounds__(kThreads)
tile_sq_error(const float* __restrict__ W, const float* __restrict__ H, int64_t pitch,
              int32_t k, int32_t G, const int32_t* __restrict__ rows,
              const int32_t* __restrict__ cols, const float* __restrict__ vals, int64_t nnz,
              int64_t m, int64_t n, double* __restrict__ partials, int* __restrict__ flag) {
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & (G - 1);
  const int per_warp = 32 / G;
  const int64_t tile_beg = int64_t(blockIdx.x) * kTileRatings;
  const int64_t tile_end = tile_beg + kTileRatings < nnz ? tile_beg + kTileRatings : nnz;
  double acc = 0.0;
  for (int64_t base = tile_beg + int64_t(warp) * per_warp; base < tile_end;
       base += int64_t(kThreads / 32) * per_warp) {
    const int64_t r = base + lane / G;
    bool ok = r < tile_end;
    int64_t i = ok ? rows[r] : 0, j = ok ? cols[r] : 0;
    if (ok && (i < 0 || i >= m || j < 0 || j >= n)) {
      if (sub == 0) atomicExch(flag, 1);
      ok = false;
      i = 0;
      j = 0;
    }
    float part = 0.f;
    for (int l = sub; l < k; l += G) part = fmaf(W[i * pitch + l], H[j * pitch + l], part);
    for (int o = G >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (ok && sub == 0) {
      const float e = vals[r] - part;
      acc += double(e) * double(e);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// Adds the tile sums in a fixed order and writes the RMSE (NaN when an index
// was out of range or nnz is 0).
__global__ void finish_rmse(const double* __restrict__ partials, int tiles, int64_t nnz,
                            const int* __restrict__ flag, double* __restrict__ out) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) s += partials[t];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int t = 0; t < int(blockDim.x); ++t) tot += red[t];
    *out = (nnz == 0 || *flag != 0) ? nan("") : sqrt(tot / double(nnz));
  }
}

}  // namespace
}  // namespace nomad

extern "C" int nomad_rmse_noalloc(const float* W, const float* H, int64_t m, int64_t n,
                                  int32_t k, int64_t pitch, int64_t nnz, const int32_t* rows,
                                  const int32_t* cols, const float* vals, double* out,
                                  void* stream) {
  using namespace nomad;
  if (!W || !H || !out || m < 1 || n < 1 || k < 1 || k > 512 || pitch < k || nnz < 0 ||
      (nnz > 0 && (!rows || !cols || !vals)))
    return NOMAD_ERR_INVALID_ARG;
  const int64_t tiles = (nnz + kTileRatings - 1) / kTileRatings;
  if (tiles > NOMAD_NOALLOC_MAX_TILES) return NOMAD_ERR_INVALID_ARG;  // over the fixed scratch
  // An error left pending by the caller's earlier work is reported as
  // NOMAD_ERR_CUDA and left in place (not consumed) for the caller to read.
  if (cudaPeekAtLastError() != cudaSuccess) return NOMAD_ERR_CUDA;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();  // this call's own failure
    return NOMAD_ERR_CUDA;
  }
  SymbolAddresses a;
  if (symbol_addresses(device, &a) != cudaSuccess) {
    cudaGetLastError();
    return NOMAD_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(a.flag, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return NOMAD_ERR_CUDA;
  }
  int G = 1;
  while (G < k && G < 32) G <<= 1;
  if (tiles > 0)
    tile_sq_error<<<unsigned(tiles), kThreads, 0, st>>>(W, H, pitch, k, G, rows, cols, vals, nnz,
                                                       m, n, a.partials, a.flag);
  finish_rmse<<<1, kThreads, 0, st>>>(a.partials, int(tiles), nnz, a.flag, out);
  // nothing was pending before the launches, so this is their own result
  if (cudaGetLastError() != cudaSuccess) return NOMAD_ERR_CUDA;
  return NOMAD_OK;
}
