// layout.cu -- builds the data layout of NOMAD's Sec. 3.1 on the device.
//
// Users are split into p contiguous row blocks I_q (equal numbers of ratings,
// the footnote's alternative, or equal numbers of users).  Worker q owns the
// sets Omega-bar_j^(q) = {(i,j) in Omega : i in I_q}; every non-empty one is a
// "segment".  Segments are stored worker-major, item-minor (a compressed CSC
// per worker: only items with ratings), rows ascending inside a segment, each
// rating as an 8-byte record {row, value}.  The data never move after this.
//
// Everything is built with device kernels: a stable LSD radix sort of 64-bit
// keys (worker | item | row), scans, and histograms.
#include <utility>

#include "nomad_internal.cuh"

namespace nomad {
namespace {

// Kernels launched by the layout build of the current call (added to the
// handle's launch counter at the end).
thread_local int64_t t_launches = 0;

// ------------------------------------------------------------------ scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile per block; the tile total goes to block_sums.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads)
scan_tiles(const TIn* __restrict__ in, TOut* __restrict__ out, int64_t n,
           TOut* __restrict__ block_sums) {
  __shared__ TOut warp_tot[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(tid) * kScanItems;
  TOut v[kScanItems];
  TOut run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    const TOut x = idx < n ? TOut(in[idx]) : TOut(0);
    v[i] = run;
    run += x;
  }
  // inclusive scan of the per-thread totals across the warp
  TOut incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const TOut y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  TOut warp_off = 0, tile_tot = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const TOut t = warp_tot[w];
    if (w < warp) warp_off += t;
    tile_tot += t;
  }
  const TOut thread_off = warp_off + incl - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n) out[idx] = v[i] + thread_off;
  }
  if (tid == 0 && block_sums) block_sums[blockIdx.x] = tile_tot;
}

template <typename T>
__global__ void add_block_offsets(T* __restrict__ out, int64_t n,
                                  const T* __restrict__ offs) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kScanTile];
}

// out[i] = sum_{i' < i} in[i'] for i in [0, n); returns the total in *total
// (device, may be null).  Temporaries come from the stream-ordered pool.
template <typename TIn, typename TOut>
cudaError_t exclusive_scan(const TIn* in, TOut* out, int64_t n, TOut* total,
                           cudaStream_t st) {
  if (n <= 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(TOut), st);
    return cudaSuccess;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  TOut* sums = nullptr;
  cudaError_t e = cudaMallocAsync(&sums, sizeof(TOut) * (nb + 1), st);
  if (e != cudaSuccess) return e;
  scan_tiles<TIn, TOut><<<unsigned(nb), kScanThreads, 0, st>>>(in, out, n, sums);
  ++t_launches;
  if (nb > 1) {
    TOut* sums_scanned = nullptr;
    e = cudaMallocAsync(&sums_scanned, sizeof(TOut) * (nb + 1), st);
    if (e != cudaSuccess) return e;
    e = exclusive_scan<TOut, TOut>(sums, sums_scanned, nb, total, st);
    if (e != cudaSuccess) return e;
    add_block_offsets<TOut><<<unsigned((n + 255) / 256), 256, 0, st>>>(out, n, sums_scanned);
    ++t_launches;
    cudaFreeAsync(sums_scanned, st);
  } else if (total) {
    e = cudaMemcpyAsync(total, sums, sizeof(TOut), cudaMemcpyDeviceToDevice, st);
  }
  cudaFreeAsync(sums, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kBins = 256;

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
radix_histogram(const K* __restrict__ keys, int64_t n, int shift,
                uint32_t* __restrict__ hist, int64_t ntiles) {
  __shared__ uint32_t h[kBins];
  for (int i = threadIdx.x; i < kBins; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t idx = base + int64_t(it) * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[uint32_t(keys[idx] >> shift) & (kBins - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBins; d += kSortThreads)
    hist[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: element order inside a tile is (round, warp, lane); the
// rank of an element among equal digits is the count of earlier rounds, of
// earlier warps in its round and of earlier lanes in its warp.
template <typename K, typename V>
__global__ void __launch_bounds__(kSortThreads)
radix_scatter(const K* __restrict__ kin, const V* __restrict__ vin,
              K* __restrict__ kout, V* __restrict__ vout, int64_t n, int shift,
              const uint32_t* __restrict__ offs, int64_t ntiles) {
  __shared__ uint32_t tile_off[kBins];
  __shared__ uint32_t run[kBins];
  __shared__ uint32_t wcnt[kSortWarps][kBins];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int d = tid; d < kBins; d += kSortThreads) {
    tile_off[d] = offs[int64_t(d) * ntiles + blockIdx.x];
    run[d] = 0;
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int it = 0; it < kSortItems; ++it) {
    for (int d = lane; d < kBins; d += 32) wcnt[warp][d] = 0;
    const int64_t idx = base + int64_t(it) * kSortThreads + tid;
    const bool valid = idx < n;
    K key{};
    V val{};
    uint32_t digit = kBins;  // invalid lanes share a digit no valid one has
    if (valid) {
      key = kin[idx];
      val = vin[idx];
      digit = uint32_t(key >> shift) & (kBins - 1);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const uint32_t rank = __popc(peers & lt_mask);
    __syncthreads();  // wcnt zeroed by every warp before any warp writes
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    for (int d = tid; d < kBins; d += kSortThreads) {
      uint32_t acc = run[d];
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = wcnt[w][d];
        wcnt[w][d] = acc;
        acc += c;
      }
      run[d] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = tile_off[digit] + wcnt[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

// Sorts (keys, vals) by the low `bits` bits of the key, stably.  The sorted
// data end in (*keys, *vals): the pointers are swapped with the temporaries
// when the number of passes is odd.
template <typename K, typename V>
cudaError_t radix_sort(K** keys, V** vals, K** tmp_keys, V** tmp_vals,
                       int64_t n, int bits, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* hist = nullptr;
  cudaError_t e = cudaMallocAsync(&hist, sizeof(uint32_t) * kBins * ntiles, st);
  if (e != cudaSuccess) return e;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_histogram<K><<<unsigned(ntiles), kSortThreads, 0, st>>>(*keys, n, shift, hist, ntiles);
    ++t_launches;
    e = exclusive_scan<uint32_t, uint32_t>(hist, hist, kBins * ntiles, nullptr, st);
    if (e != cudaSuccess) return e;
    radix_scatter<K, V><<<unsigned(ntiles), kSortThreads, 0, st>>>(
        *keys, *vals, *tmp_keys, *tmp_vals, n, shift, hist, ntiles);
    ++t_launches;
    std::swap(*keys, *tmp_keys);
    std::swap(*vals, *tmp_vals);
  }
  cudaFreeAsync(hist, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ layout kernels
__global__ void check_and_count_rows(const int32_t* __restrict__ rows,
                                     const int32_t* __restrict__ cols,
                                     int64_t nnz, int64_t m, int64_t n,
                                     unsigned long long* __restrict__ deg,
                                     int32_t* __restrict__ status) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nnz; r += stride) {
    const int32_t i = rows[r], j = cols[r];
    if (i < 0 || i >= m || j < 0 || j >= n) {
      atomicCAS(status, 0, NOMAD_ERR_RANGE);
      continue;
    }
    atomicAdd(&deg[i], 1ull);
  }
}

// Row block of every user (Sec. 3.1).  Ratings mode: the block in which the
// row's middle rating falls, min(p-1, floor(p (2 c_i + d_i) / (2 nnz))).
__global__ void assign_row_workers(const unsigned long long* __restrict__ deg,
                                   const unsigned long long* __restrict__ cum,
                                   int64_t m, int64_t nnz, int32_t p, int mode,
                                   int32_t* __restrict__ row_worker) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) {
    int64_t q;
    if (mode == NOMAD_PARTITION_USERS || nnz == 0) {
      q = mode == NOMAD_PARTITION_USERS ? (i * p) / m : 0;
    } else {
      const uint64_t mid2 = 2ull * cum[i] + deg[i];
      q = int64_t((uint64_t(p) * mid2) / (2ull * uint64_t(nnz)));
      if (q > p - 1) q = p - 1;
    }
    row_worker[i] = int32_t(q);
  }
}

__global__ void make_sort_keys(const int32_t* __restrict__ rows,
                               const int32_t* __restrict__ cols,
                               const float* __restrict__ vals, int64_t nnz,
                               const int32_t* __restrict__ row_worker,
                               int row_bits, int col_bits,
                               unsigned long long* __restrict__ keys,
                               uint32_t* __restrict__ payload) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nnz; r += stride) {
    const uint64_t i = uint32_t(rows[r]), j = uint32_t(cols[r]);
    const uint64_t q = uint32_t(row_worker[i]);
    keys[r] = (q << (row_bits + col_bits)) | (j << row_bits) | i;
    payload[r] = __float_as_uint(vals[r]);
  }
}

// flag[r] = 1 where a new (worker, item) pair starts; duplicates of a full
// key are an input error (Omega is a set).
__global__ void segment_flags(const unsigned long long* __restrict__ keys,
                              int64_t nnz, int row_bits,
                              uint32_t* __restrict__ flag,
                              int32_t* __restrict__ status) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nnz; r += stride) {
    const uint64_t k = keys[r];
    uint32_t f = 1;
    if (r > 0) {
      const uint64_t prev = keys[r - 1];
      if (prev == k) atomicCAS(status, 0, NOMAD_ERR_DUP_ENTRY);
      f = (prev >> row_bits) != (k >> row_bits);
    }
    flag[r] = f;
  }
}

__global__ void write_segments(const unsigned long long* __restrict__ keys,
                               const uint32_t* __restrict__ payload,
                               const uint32_t* __restrict__ flag,
                               const uint32_t* __restrict__ seg_id, int64_t nnz,
                               int row_bits, int col_bits,
                               int64_t* __restrict__ seg_ptr,
                               int32_t* __restrict__ seg_col,
                               int32_t* __restrict__ seg_worker,
                               int2* __restrict__ rec) {
  const uint64_t row_mask = (1ull << row_bits) - 1, col_mask = (1ull << col_bits) - 1;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nnz; r += stride) {
    const uint64_t k = keys[r];
    rec[r] = make_int2(int32_t(k & row_mask), int32_t(payload[r]));
    if (flag[r]) {
      const uint32_t s = seg_id[r];
      seg_ptr[s] = r;
      seg_col[s] = int32_t((k >> row_bits) & col_mask);
      seg_worker[s] = int32_t(k >> (row_bits + col_bits));
    }
  }
}

__global__ void count_by(const int32_t* __restrict__ ids, int64_t n,
                         uint32_t* __restrict__ counts) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += stride)
    atomicAdd(&counts[ids[s]], 1u);
}

// Ratings of each item, summed over its segments.
__global__ void item_degrees(const int64_t* __restrict__ seg_ptr,
                             const int32_t* __restrict__ seg_col, int64_t S,
                             uint32_t* __restrict__ deg) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < S; s += stride)
    atomicAdd(&deg[seg_col[s]], uint32_t(seg_ptr[s + 1] - seg_ptr[s]));
}

__global__ void max_u32(const uint32_t* __restrict__ x, int64_t n, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    m = x[i] > m ? x[i] : m;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Items whose tokens take the longest chains of visits: at least half the
// ratings of the most-rated item.
__global__ void urgent_flags(const uint32_t* __restrict__ deg, int64_t n,
                             const uint32_t* __restrict__ max_deg, uint8_t* __restrict__ flag) {
  const uint64_t top = *max_deg;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride)
    flag[j] = deg[j] > 0 && 2ull * deg[j] >= top ? 1 : 0;
}

// Segment s of an urgent item: its number of ratings in len[s] and 1 in
// flag[s] (0, 0 for the other segments).
__global__ void urgent_seg_lengths(const int64_t* __restrict__ seg_ptr,
                                   const int32_t* __restrict__ seg_col,
                                   const uint8_t* __restrict__ item_urgent, int64_t S,
                                   int64_t* __restrict__ len, uint32_t* __restrict__ flag) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < S; s += stride) {
    const bool u = item_urgent[seg_col[s]] != 0;
    len[s] = u ? seg_ptr[s + 1] - seg_ptr[s] : 0;
    flag[s] = u ? 1u : 0u;
  }
}

// The urgent segments in order: list[pos[s]] = s where flag[s].
__global__ void urgent_seg_scatter(const uint32_t* __restrict__ flag,
                                   const uint32_t* __restrict__ pos, int64_t S,
                                   int32_t* __restrict__ list) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < S; s += stride)
    if (flag[s]) list[pos[s]] = int32_t(s);
}

__global__ void count_flags(const uint8_t* __restrict__ flag, int64_t n,
                            uint32_t* __restrict__ count) {
  uint32_t c = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride)
    c += flag[j];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Hybrid circulation: the segments of an item (col_segs, ordered by worker)
// split into runs of one thread block each (blocks of wpb workers).  flag[i]
// is 1 where position i of col_segs starts a run.
__global__ void block_run_flags(const int32_t* __restrict__ col_segs,
                                const int32_t* __restrict__ seg_worker,
                                const int32_t* __restrict__ seg_col,
                                const int32_t* __restrict__ col_seg_ptr, int64_t S, int32_t wpb,
                                uint32_t* __restrict__ flag) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < S; i += stride) {
    const int32_t sg = col_segs[i];
    const bool first = i == col_seg_ptr[seg_col[sg]];
    flag[i] = first || seg_worker[sg] / wpb != seg_worker[col_segs[i - 1]] / wpb ? 1u : 0u;
  }
}

// Runs per item plus one (the terminal offset): run[S] = total runs.
__global__ void block_run_counts(const int32_t* __restrict__ col_seg_ptr,
                                 const uint32_t* __restrict__ run, int64_t n,
                                 uint32_t* __restrict__ cnt) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride)
    cnt[j] = run[col_seg_ptr[j + 1]] - run[col_seg_ptr[j]] + 1u;
}

// grp_off[col_grp_ptr[j] + g] = offset of run g of item j within its
// segments; grp_off[col_grp_ptr[j + 1] - 1] = the item's number of segments.
__global__ void block_run_offsets(const uint32_t* __restrict__ flag,
                                  const uint32_t* __restrict__ run,
                                  const int32_t* __restrict__ col_segs,
                                  const int32_t* __restrict__ seg_col,
                                  const int32_t* __restrict__ col_seg_ptr,
                                  const int32_t* __restrict__ col_grp_ptr, int64_t S, int64_t n,
                                  int32_t* __restrict__ grp_off) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < S + n; i += stride) {
    if (i < S) {
      if (flag[i]) {
        const int32_t j = seg_col[col_segs[i]];
        const int32_t a = col_seg_ptr[j];
        grp_off[col_grp_ptr[j] + int32_t(run[i] - run[a])] = int32_t(i - a);
      }
    } else {
      const int64_t j = i - S;
      grp_off[col_grp_ptr[j + 1] - 1] = col_seg_ptr[j + 1] - col_seg_ptr[j];
    }
  }
}

__global__ void iota_u32(uint32_t* __restrict__ out, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += stride)
    out[s] = uint32_t(s);
}

__global__ void copy_i32(const int32_t* __restrict__ in, uint32_t* __restrict__ out,
                         int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += stride)
    out[s] = uint32_t(in[s]);
}

// Ring capacity per worker: a power of two no smaller than the number of
// item tokens that can ever wait in that worker's queue at once.
__global__ void ring_sizes(const uint32_t* __restrict__ nseg, int32_t p,
                           int64_t uniform_items, int32_t* __restrict__ log2cap,
                           int64_t* __restrict__ cap) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p) return;
  const int64_t need =
      (uniform_items > 0 ? uniform_items : int64_t(nseg[q])) + kRingWindow + 1;
  int lg = 5;  // at least 32 slots
  while ((int64_t(1) << lg) < need) ++lg;
  log2cap[q] = lg;
  cap[q] = int64_t(1) << lg;
}

int bit_width(int64_t x) {  // bits needed for values 0..x (at least 1)
  int b = 1;
  while (b < 63 && (int64_t(1) << b) <= x) ++b;
  return b;
}

unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return unsigned(g);
}

#define TRY(expr)                                                   \
  do {                                                              \
    cudaError_t err_ = (expr);                                      \
    if (err_ != cudaSuccess) {                                      \
      h->last_error = std::string("layout: ") + #expr + ": " +      \
                      cudaGetErrorString(err_);                     \
      return err_ == cudaErrorMemoryAllocation ? NOMAD_ERR_OOM      \
                                               : NOMAD_ERR_CUDA;    \
    }                                                               \
  } while (0)

}  // namespace

int build_layout(nomad_handle* h, int64_t nnz, const int32_t* d_rows,
                 const int32_t* d_cols, const float* d_vals, cudaStream_t st) {
  const int64_t m = h->m, n = h->n;
  const int32_t p = h->p;
  const int row_bits = bit_width(m - 1), col_bits = bit_width(n - 1);
  const int wk_bits = bit_width(p - 1);
  if (row_bits + col_bits + wk_bits > 64) {
    h->last_error = "layout: worker|item|row key exceeds 64 bits";
    return NOMAD_ERR_UNSUPPORTED;
  }
  t_launches = 0;
  TRY(cudaMemsetAsync(h->status, 0, sizeof(int32_t) * kStatusWords, st));

  // 1. range check + row degrees, 2. prefix sums, 3. row blocks
  unsigned long long *deg = nullptr, *cum = nullptr;
  TRY(cudaMallocAsync(&deg, sizeof(unsigned long long) * (m + 1), st));
  TRY(cudaMallocAsync(&cum, sizeof(unsigned long long) * (m + 1), st));
  TRY(cudaMemsetAsync(deg, 0, sizeof(unsigned long long) * (m + 1), st));
  if (nnz > 0)
    check_and_count_rows<<<grid_for(nnz), 256, 0, st>>>(d_rows, d_cols, nnz, m, n, deg, h->status);
  if (nnz > 0) ++t_launches;
  int32_t status = 0;
  TRY(cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (status != 0) {
    cudaFreeAsync(deg, st);
    cudaFreeAsync(cum, st);
    h->last_error = "layout: rating index out of range";
    return status;
  }
  TRY((exclusive_scan<unsigned long long, unsigned long long>(deg, cum, m, nullptr, st)));
  assign_row_workers<<<grid_for(m), 256, 0, st>>>(deg, cum, m, nnz, p, h->sched.partition,
                                                 h->row_worker);
  ++t_launches;
  cudaFreeAsync(deg, st);
  cudaFreeAsync(cum, st);

  // 4. sort the ratings by (worker, item, row)
  unsigned long long *keys = nullptr, *keys_tmp = nullptr;
  uint32_t *pay = nullptr, *pay_tmp = nullptr;
  const int64_t nalloc = nnz > 0 ? nnz : 1;
  TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * nalloc, st));
  TRY(cudaMallocAsync(&keys_tmp, sizeof(unsigned long long) * nalloc, st));
  TRY(cudaMallocAsync(&pay, sizeof(uint32_t) * nalloc, st));
  TRY(cudaMallocAsync(&pay_tmp, sizeof(uint32_t) * nalloc, st));
  if (nnz > 0)
    make_sort_keys<<<grid_for(nnz), 256, 0, st>>>(d_rows, d_cols, d_vals, nnz, h->row_worker,
                                                 row_bits, col_bits, keys, pay);
  if (nnz > 0) ++t_launches;
  TRY((radix_sort<unsigned long long, uint32_t>(&keys, &pay, &keys_tmp, &pay_tmp, nnz,
                                                row_bits + col_bits + wk_bits, st)));

  // 5. segment boundaries, duplicate check, segment ids
  uint32_t* flag = pay_tmp;  // free now
  uint32_t* seg_id = nullptr;
  uint32_t* d_S = nullptr;
  TRY(cudaMallocAsync(&seg_id, sizeof(uint32_t) * nalloc, st));
  TRY(cudaMallocAsync(&d_S, sizeof(uint32_t), st));
  if (nnz > 0)
    segment_flags<<<grid_for(nnz), 256, 0, st>>>(keys, nnz, row_bits, flag, h->status);
  if (nnz > 0) ++t_launches;
  TRY((exclusive_scan<uint32_t, uint32_t>(flag, seg_id, nnz, d_S, st)));
  uint32_t S32 = 0;
  TRY(cudaMemcpyAsync(&S32, d_S, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (status != 0) {
    cudaFreeAsync(keys, st); cudaFreeAsync(keys_tmp, st); cudaFreeAsync(pay, st);
    cudaFreeAsync(pay_tmp, st); cudaFreeAsync(seg_id, st); cudaFreeAsync(d_S, st);
    h->last_error = "layout: duplicate rating (i,j)";
    return status;
  }
  const int64_t S = nnz > 0 ? int64_t(S32) : 0;
  if (S >= (int64_t(1) << 31)) {
    h->last_error = "layout: more than 2^31 segments";
    return NOMAD_ERR_UNSUPPORTED;
  }

  // 6. the layout proper
  void* vp = nullptr;
  TRY(dev_alloc(h, &vp, sizeof(int2) * nalloc)); h->rec = (int2*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int64_t) * (S + 1))); h->seg_ptr = (int64_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (S + 1))); h->seg_col = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (S + 1))); h->seg_worker = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (S + 1))); h->col_segs = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (p + 1))); h->worker_seg_ptr = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (n + 1))); h->col_seg_ptr = (int32_t*)vp;
  if (nnz > 0)
    write_segments<<<grid_for(nnz), 256, 0, st>>>(keys, pay, flag, seg_id, nnz, row_bits,
                                                 col_bits, h->seg_ptr, h->seg_col,
                                                 h->seg_worker, h->rec);
  if (nnz > 0) ++t_launches;
  const int64_t nnz64 = nnz;
  TRY(cudaMemcpyAsync(h->seg_ptr + S, &nnz64, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  cudaFreeAsync(keys, st);
  cudaFreeAsync(keys_tmp, st);
  cudaFreeAsync(pay, st);
  cudaFreeAsync(pay_tmp, st);
  cudaFreeAsync(seg_id, st);

  // 7. segments per worker and per item
  uint32_t* cnt = nullptr;
  const int64_t cnt_n = (p > n ? p : n) + 1;
  TRY(cudaMallocAsync(&cnt, sizeof(uint32_t) * cnt_n, st));
  TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * cnt_n, st));
  if (S > 0) count_by<<<grid_for(S), 256, 0, st>>>(h->seg_worker, S, cnt);
  if (S > 0) ++t_launches;
  uint32_t* nseg_per_worker = nullptr;
  TRY(cudaMallocAsync(&nseg_per_worker, sizeof(uint32_t) * (p + 1), st));
  TRY(cudaMemcpyAsync(nseg_per_worker, cnt, sizeof(uint32_t) * p, cudaMemcpyDeviceToDevice, st));
  TRY((exclusive_scan<uint32_t, uint32_t>(cnt, (uint32_t*)h->worker_seg_ptr, p,
                                          (uint32_t*)h->worker_seg_ptr + p, st)));
  TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * cnt_n, st));
  if (S > 0) count_by<<<grid_for(S), 256, 0, st>>>(h->seg_col, S, cnt);
  if (S > 0) ++t_launches;
  TRY((exclusive_scan<uint32_t, uint32_t>(cnt, (uint32_t*)h->col_seg_ptr, n,
                                          (uint32_t*)h->col_seg_ptr + n, st)));
  cudaFreeAsync(cnt, st);

  // 8. segments of each item ordered by worker: stable sort of the segment
  //    ids (already worker-major) by item
  uint32_t *ck = nullptr, *ck_tmp = nullptr, *cv = nullptr, *cv_tmp = nullptr;
  const int64_t salloc = S > 0 ? S : 1;
  TRY(cudaMallocAsync(&ck, sizeof(uint32_t) * salloc, st));
  TRY(cudaMallocAsync(&ck_tmp, sizeof(uint32_t) * salloc, st));
  TRY(cudaMallocAsync(&cv, sizeof(uint32_t) * salloc, st));
  TRY(cudaMallocAsync(&cv_tmp, sizeof(uint32_t) * salloc, st));
  if (S > 0) {
    copy_i32<<<grid_for(S), 256, 0, st>>>(h->seg_col, ck, S);
    ++t_launches;
    iota_u32<<<grid_for(S), 256, 0, st>>>(cv, S);
    ++t_launches;
  }
  TRY((radix_sort<uint32_t, uint32_t>(&ck, &cv, &ck_tmp, &cv_tmp, S, col_bits, st)));
  if (S > 0)
    TRY(cudaMemcpyAsync(h->col_segs, cv, sizeof(uint32_t) * S, cudaMemcpyDeviceToDevice, st));
  cudaFreeAsync(ck, st); cudaFreeAsync(ck_tmp, st);
  cudaFreeAsync(cv, st); cudaFreeAsync(cv_tmp, st);

  // 8b. hybrid circulation: runs of one thread block in each item's segments
  if (h->sched.circulation == NOMAD_CIRCULATION_BLOCK) {
    uint32_t *flag2 = nullptr, *run = nullptr, *rc = nullptr;
    TRY(cudaMallocAsync(&flag2, sizeof(uint32_t) * salloc, st));
    TRY(cudaMallocAsync(&run, sizeof(uint32_t) * (S + 1), st));
    TRY(cudaMallocAsync(&rc, sizeof(uint32_t) * (n + 1), st));
    if (S > 0) {
      block_run_flags<<<grid_for(S), 256, 0, st>>>(h->col_segs, h->seg_worker, h->seg_col,
                                                   h->col_seg_ptr, S, h->warps_per_block, flag2);
      ++t_launches;
    }
    TRY((exclusive_scan<uint32_t, uint32_t>(flag2, run, S, run + S, st)));
    block_run_counts<<<grid_for(n > 0 ? n : 1), 256, 0, st>>>(h->col_seg_ptr, run, n, rc);
    ++t_launches;
    TRY(dev_alloc(h, &vp, sizeof(int32_t) * (n + 1))); h->col_grp_ptr = (int32_t*)vp;
    TRY((exclusive_scan<uint32_t, uint32_t>(rc, (uint32_t*)h->col_grp_ptr, n,
                                            (uint32_t*)h->col_grp_ptr + n, st)));
    uint32_t runs_total = 0;
    TRY(cudaMemcpyAsync(&runs_total, h->col_grp_ptr + n, sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    TRY(dev_alloc(h, &vp, sizeof(int32_t) * (int64_t(runs_total) + 1))); h->grp_off = (int32_t*)vp;
    block_run_offsets<<<grid_for(S + n > 0 ? S + n : 1), 256, 0, st>>>(
        flag2, run, h->col_segs, h->seg_col, h->col_seg_ptr, h->col_grp_ptr, S, n, h->grp_off);
    ++t_launches;
    cudaFreeAsync(flag2, st);
    cudaFreeAsync(run, st);
    cudaFreeAsync(rc, st);
  }

  // 9. queues: one ring per worker
  int64_t* caps = nullptr;
  TRY(cudaMallocAsync(&caps, sizeof(int64_t) * (p + 1), st));
  TRY(dev_alloc(h, &vp, sizeof(int64_t) * (p + 1))); h->ring_base = (int64_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (p + 1))); h->ring_log2 = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(uint32_t) * (p + 1))); h->ring_tail = (uint32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(uint32_t) * (p + 1))); h->ring_head = (uint32_t*)vp;
  const int64_t uniform_items = h->sched.mode == NOMAD_MODE_UNIFORM ? n : 0;
  ring_sizes<<<(p + 255) / 256, 256, 0, st>>>(nseg_per_worker, p, uniform_items,
                                              h->ring_log2, caps);
  ++t_launches;
  TRY((exclusive_scan<int64_t, int64_t>(caps, h->ring_base, p, h->ring_base + p, st)));
  int64_t slots = 0;
  TRY(cudaMemcpyAsync(&slots, h->ring_base + p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(caps, st);
  cudaFreeAsync(nseg_per_worker, st);
  TRY(dev_alloc(h, &vp, sizeof(unsigned long long) * (slots > 0 ? slots : 1)));
  h->ring = (unsigned long long*)vp;
  h->ring_slots = slots;

  // 10. token state and debug arrays
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (n + 1))); h->tok_hop = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int32_t) * (n + 1))); h->tok_epoch = (int32_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(uint8_t) * (n + 1))); h->item_urgent = (uint8_t*)vp;
  TRY(dev_alloc(h, &vp, sizeof(int4) * kTokRecInts * (n + 1))); h->tok_rec = (int4*)vp;
  {
    uint32_t* deg = nullptr;
    TRY(cudaMallocAsync(&deg, sizeof(uint32_t) * (n + 2), st));
    TRY(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * (n + 2), st));
    if (S > 0) {
      item_degrees<<<grid_for(S), 256, 0, st>>>(h->seg_ptr, h->seg_col, S, deg);
      ++t_launches;
    }
    if (n > 0) {
      max_u32<<<grid_for(n), 256, 0, st>>>(deg, n, deg + n);
      urgent_flags<<<grid_for(n), 256, 0, st>>>(deg, n, deg + n, h->item_urgent);
      count_flags<<<grid_for(n), 256, 0, st>>>(h->item_urgent, n, deg + n + 1);
      t_launches += 3;
    }
    uint32_t n_urgent = 0;
    TRY(cudaMemcpyAsync(&n_urgent, deg + n + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(deg, st);
    // one urgent ring per worker, room for every urgent token at once
    int lgu = 5;
    while ((int64_t(1) << lgu) < int64_t(n_urgent) + 1) ++lgu;
    h->uring_log2 = lgu;
    TRY(dev_alloc(h, &vp, sizeof(unsigned long long) * (int64_t(p) << lgu)));
    h->uring = (unsigned long long*)vp;
    TRY(dev_alloc(h, &vp, sizeof(uint32_t) * (p + 1))); h->uring_tail = (uint32_t*)vp;

    // 10b. narrow formats: room for the W rounding bits of the urgent items'
    // ratings, drawn before each launch so that the chains of visits of
    // these items do not wait for them (the batched kernel at one chunk
    // per lane, epoch mode).  It pays where a few items with very long
    // chains bind the epoch: only when their ratings are at most a quarter
    // of all (with more, as for degrees close to uniform, the pass costs
    // more than the chains gain), and at most a quarter of the free device
    // memory or 32 GiB
    if (h->sched.precision != NOMAD_FP32 && h->sched.variant == NOMAD_VARIANT_BATCHED &&
        h->sched.mode == NOMAD_MODE_EPOCH && h->k4 <= 32 && S > 0 && n_urgent > 0) {
      int64_t* len = nullptr;
      uint32_t *flag3 = nullptr, *pos = nullptr;
      TRY(cudaMallocAsync(&len, sizeof(int64_t) * salloc, st));
      TRY(cudaMallocAsync(&flag3, sizeof(uint32_t) * salloc, st));
      TRY(cudaMallocAsync(&pos, sizeof(uint32_t) * (S + 1), st));
      TRY(dev_alloc(h, &vp, sizeof(int64_t) * (S + 1))); h->useg_off = (int64_t*)vp;
      urgent_seg_lengths<<<grid_for(S), 256, 0, st>>>(h->seg_ptr, h->seg_col, h->item_urgent, S,
                                                      len, flag3);
      ++t_launches;
      TRY((exclusive_scan<int64_t, int64_t>(len, h->useg_off, S, h->useg_off + S, st)));
      TRY((exclusive_scan<uint32_t, uint32_t>(flag3, pos, S, pos + S, st)));
      int64_t urecs = 0;
      uint32_t nus = 0;
      TRY(cudaMemcpyAsync(&urecs, h->useg_off + S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      TRY(cudaMemcpyAsync(&nus, pos + S, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      const double bytes = double(urecs) * double(h->k4) * sizeof(uint2);
      if (nus > 0 && urecs * 4 <= nnz && bytes <= double(free_b) / 4 &&
          bytes <= double(int64_t(32) << 30)) {
        TRY(dev_alloc(h, &vp, sizeof(int32_t) * nus)); h->useg_list = (int32_t*)vp;
        urgent_seg_scatter<<<grid_for(S), 256, 0, st>>>(flag3, pos, S, h->useg_list);
        ++t_launches;
        TRY(dev_alloc(h, &vp, size_t(bytes))); h->ubits_pre = (uint2*)vp;
        h->n_useg = int64_t(nus);
        h->upre_records = urecs;
      } else {
        vp = h->useg_off;
        dev_free(h, &vp);
        h->useg_off = nullptr;
      }
      cudaFreeAsync(len, st);
      cudaFreeAsync(flag3, st);
      cudaFreeAsync(pos, st);
    }
  }
  if (h->sched.debug || h->sched.mode == NOMAD_MODE_UNIFORM) {
    TRY(dev_alloc(h, &vp, sizeof(int32_t) * nalloc)); h->rec_count = (int32_t*)vp;
    TRY(cudaMemsetAsync(h->rec_count, 0, sizeof(int32_t) * nalloc, st));
  }
  if (h->sched.debug) {
    TRY(dev_alloc(h, &vp, sizeof(int32_t) * (n + 1))); h->owner = (int32_t*)vp;
    TRY(cudaMemsetAsync(h->owner, 0xff, sizeof(int32_t) * (n + 1), st));
  }
  TRY(cudaStreamSynchronize(st));
  h->nnz = nnz;
  h->n_seg = S;
  h->launches += t_launches;
  return NOMAD_OK;
}

#undef TRY

}  // namespace nomad
