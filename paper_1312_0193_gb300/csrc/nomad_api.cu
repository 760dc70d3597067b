// nomad_api.cu -- the extern "C" entry points declared in include/nomad.h.
//
// Host code only: argument checks, device memory of the handle, staging of
// host inputs, and the launches of the kernels in layout.cu, sgd.cu and
// eval.cu.  Every step of the computation runs in those kernels; there is
// no CPU fallback.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "nomad_internal.cuh"

namespace nomad {

namespace {

// Makes the handle's device current for the duration of a call and puts the
// caller's device back afterwards.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int fail(nomad_handle* h, int code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

int cuda_fail(nomad_handle* h, cudaError_t e, const char* what) {
  const int code = e == cudaErrorMemoryAllocation ? NOMAD_ERR_OOM : NOMAD_ERR_CUDA;
  cudaGetLastError();  // clear a sticky-free error so later calls can proceed
  return fail(h, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, expr, what)                               \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

void free_layout(nomad_handle* h) {
  void** ptrs[] = {(void**)&h->rec,        (void**)&h->seg_ptr,   (void**)&h->seg_col,
                   (void**)&h->seg_worker, (void**)&h->worker_seg_ptr,
                   (void**)&h->col_seg_ptr, (void**)&h->col_segs, (void**)&h->ring,
                   (void**)&h->ring_base,  (void**)&h->ring_log2, (void**)&h->ring_tail,
                   (void**)&h->tok_hop,    (void**)&h->tok_epoch, (void**)&h->owner,
                   (void**)&h->rec_count,  (void**)&h->log_seg,   (void**)&h->log_epoch,
                   (void**)&h->item_urgent, (void**)&h->uring,    (void**)&h->uring_tail,
                   (void**)&h->tok_rec,    (void**)&h->ring_head,  (void**)&h->col_grp_ptr,
                   (void**)&h->grp_off,    (void**)&h->useg_off,  (void**)&h->useg_list,
                   (void**)&h->ubits_pre};
  for (void** p : ptrs) dev_free(h, p);
  h->n_useg = 0;
  h->upre_records = 0;
  h->log_cap = 0;
  h->loaded = false;
  h->nnz = 0;
  h->n_seg = 0;
  h->ring_slots = 0;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Device copy of a caller array: the array itself when it already is device
// memory, else a stream-ordered temporary filled from the host.
template <typename T>
cudaError_t stage(const T* src, int64_t count, int32_t device_ptrs, cudaStream_t st,
                  const T** out, T** owned) {
  *owned = nullptr;
  if (count <= 0) {
    *out = nullptr;
    return cudaSuccess;
  }
  if (device_ptrs) {
    *out = src;
    return cudaSuccess;
  }
  T* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(T) * count, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, st);
  *out = d;
  *owned = d;
  return e;
}

__global__ void csc_expand_cols(const int64_t* __restrict__ colptr, int64_t n,
                                int32_t* __restrict__ cols, int32_t* __restrict__ status,
                                int64_t nnz) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
    const int64_t b = colptr[j], e = colptr[j + 1];
    if (b < 0 || e < b || e > nnz) {
      atomicCAS(status, 0, NOMAD_ERR_INVALID_ARG);
      continue;
    }
    for (int64_t r = b; r < e; ++r) cols[r] = int32_t(j);
  }
}

}  // namespace

cudaError_t dev_alloc(nomad_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    h->allocs[*p] = bytes;
    h->device_bytes += int64_t(bytes);
  }
  return e;
}

void dev_free(nomad_handle* h, void** p) {
  if (*p) {
    auto it = h->allocs.find(*p);
    if (it != h->allocs.end()) {
      h->device_bytes -= int64_t(it->second);
      h->allocs.erase(it);
    }
    cudaFree(*p);
  }
  *p = nullptr;
}


}  // namespace nomad

using namespace nomad;

extern "C" {

void nomad_schedule_default(nomad_schedule* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->alpha = 0.012f;
  s->beta = 0.05f;
  s->mode = NOMAD_MODE_EPOCH;
  s->precision = NOMAD_FP32;
  s->partition = NOMAD_PARTITION_RATINGS;
  s->n_workers = 0;
  s->warps_per_block = 0;
  s->debug = 0;
  s->seed = 1;
  s->spin_timeout_ns = 0;
  s->device = 0;
  s->debug_drop_item = -1;
  s->variant = NOMAD_VARIANT_BATCHED;
  s->routing = NOMAD_ROUTING_UNIFORM;
  s->circulation = NOMAD_CIRCULATION_FLAT;
}

const char* nomad_error_string(int32_t code) {
  switch (code) {
    case NOMAD_OK: return "ok";
    case NOMAD_ERR_INVALID_ARG: return "invalid argument";
    case NOMAD_ERR_OOM: return "out of memory";
    case NOMAD_ERR_DUP_ENTRY: return "duplicate rating (i,j)";
    case NOMAD_ERR_TIMEOUT: return "a worker timed out waiting for an item token";
    case NOMAD_ERR_OWNERSHIP: return "an item token was held by two workers";
    case NOMAD_ERR_CUDA: return "CUDA error";
    case NOMAD_ERR_RANGE: return "rating index out of range";
    case NOMAD_ERR_UNSUPPORTED: return "unsupported shape or option";
    case NOMAD_ERR_STATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* nomad_last_error_message(const nomad_t* h) {
  return h ? h->last_error.c_str() : "";
}

int nomad_create(int64_t m, int64_t n, int32_t k, float lambda, const nomad_schedule* s,
                 nomad_t** out) {
  if (!out) return NOMAD_ERR_INVALID_ARG;
  *out = nullptr;
  nomad_schedule sched;
  if (s) sched = *s; else nomad_schedule_default(&sched);
  if (m < 1 || n < 1 || m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31) || k < 1 ||
      k > 512 || !(lambda >= 0.f) || !std::isfinite(lambda) || !std::isfinite(sched.alpha) ||
      !std::isfinite(sched.beta) || sched.alpha < 0.f || sched.beta < 0.f ||
      (sched.mode != NOMAD_MODE_EPOCH && sched.mode != NOMAD_MODE_UNIFORM) ||
      (sched.partition != NOMAD_PARTITION_RATINGS && sched.partition != NOMAD_PARTITION_USERS) ||
      sched.n_workers < 0 || sched.warps_per_block < 0 || sched.spin_timeout_ns < 0 ||
      (sched.variant != NOMAD_VARIANT_BATCHED && sched.variant != NOMAD_VARIANT_SIMPLE) ||
      (sched.routing != NOMAD_ROUTING_UNIFORM && sched.routing != NOMAD_ROUTING_SHORTER) ||
      (sched.circulation != NOMAD_CIRCULATION_FLAT && sched.circulation != NOMAD_CIRCULATION_BLOCK) ||
      sched.batch_tokens < 0 || sched.batch_tokens > 16 || sched.epochs_per_launch < 0)
    return NOMAD_ERR_INVALID_ARG;
  if (sched.circulation == NOMAD_CIRCULATION_BLOCK &&
      (sched.mode != NOMAD_MODE_EPOCH || sched.variant != NOMAD_VARIANT_BATCHED))
    return NOMAD_ERR_UNSUPPORTED;  // the hybrid circulation: batched epoch-mode kernel only
  if (sched.precision != NOMAD_FP32 && sched.precision != NOMAD_BF16 &&
      sched.precision != NOMAD_FP8)
    return NOMAD_ERR_INVALID_ARG;
  if (sched.precision != NOMAD_FP32 &&
      (sched.mode != NOMAD_MODE_EPOCH || sched.variant != NOMAD_VARIANT_BATCHED))
    return NOMAD_ERR_UNSUPPORTED;  // narrow storage: batched epoch-mode kernel only
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || sched.device < 0 || sched.device >= ndev) {
    cudaGetLastError();
    return NOMAD_ERR_CUDA;
  }
  DeviceGuard guard(sched.device);
  nomad_handle* h = new nomad_handle();
  h->m = m;
  h->n = n;
  h->k = k;
  h->k4 = (k + 3) / 4;
  h->pitch = h->k4 * 4;
  h->lambda = lambda;
  h->elem = sched.precision == NOMAD_BF16 ? 2 : 4;
  h->w_elem = sched.precision == NOMAD_BF16 ? 2 : sched.precision == NOMAD_FP8 ? 1 : 4;
  h->sched = sched;
  h->device = sched.device;
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  h->warps_per_block = sched.warps_per_block > 0 ? sched.warps_per_block
                                                 : default_warps_per_block();
  int bps = 0;
  const int pmax = max_resident_workers(
      h->device, h->warps_per_block, h->k4, sched.precision, sched.mode, sched.variant, &bps,
      sched.circulation == NOMAD_CIRCULATION_BLOCK);
  if (pmax <= 0) {
    delete h;
    return NOMAD_ERR_UNSUPPORTED;
  }
  h->p = sched.n_workers > 0 ? sched.n_workers : pmax;
  if (h->p > pmax) {
    delete h;
    return NOMAD_ERR_INVALID_ARG;  // every worker must be resident at once
  }
  h->blocks = (h->p + h->warps_per_block - 1) / h->warps_per_block;

  const size_t esz = size_t(h->elem);
  const size_t wsz = size_t(h->w_elem);
  void* vp = nullptr;
  if (dev_alloc(h, &vp, wsz * size_t(m) * h->pitch) != cudaSuccess) goto oom;
  h->W = vp;
  if (dev_alloc(h, &vp, esz * size_t(n) * h->pitch) != cudaSuccess) goto oom;
  h->H = vp;
  if (sched.precision == NOMAD_FP8) {
    if (dev_alloc(h, &vp, sizeof(float) * size_t(m)) != cudaSuccess) goto oom;
    h->Wscale = static_cast<float*>(vp);
  }
  if (dev_alloc(h, &vp, sizeof(int32_t) * kStatusWords) != cudaSuccess) goto oom;
  h->status = static_cast<int32_t*>(vp);
  if (dev_alloc(h, &vp, sizeof(int32_t) * size_t(m)) != cudaSuccess) goto oom;
  h->row_worker = static_cast<int32_t*>(vp);
  if (dev_alloc(h, &vp, sizeof(double) * 2) != cudaSuccess) goto oom;
  h->result = static_cast<double*>(vp);
  if (dev_alloc(h, &vp, sizeof(unsigned long long) * 2) != cudaSuccess) goto oom;
  h->upd_done = static_cast<unsigned long long*>(vp);
  if (dev_alloc(h, &vp, sizeof(unsigned long long) * 2) != cudaSuccess) goto oom;
  h->span = static_cast<unsigned long long*>(vp);
  if (cudaMemset(h->span, 0, sizeof(unsigned long long) * 2) != cudaSuccess) goto cuda_err;
  if (dev_alloc(h, &vp, sizeof(int32_t) * 2) != cudaSuccess) goto oom;
  h->stop = static_cast<int32_t*>(vp);
  if (dev_alloc(h, &vp, sizeof(uint32_t) * 2) != cudaSuccess) goto oom;
  h->log_ticket = static_cast<uint32_t*>(vp);
  if (cudaMemset(h->status, 0, sizeof(int32_t) * kStatusWords) != cudaSuccess) goto cuda_err;
  if (cudaMemset(h->W, 0, wsz * size_t(m) * h->pitch) != cudaSuccess) goto cuda_err;
  if (cudaMemset(h->H, 0, esz * size_t(n) * h->pitch) != cudaSuccess) goto cuda_err;
  if (init_factors(h, nullptr) != NOMAD_OK) goto cuda_err;
  if (cudaDeviceSynchronize() != cudaSuccess) goto cuda_err;
  *out = h;
  return NOMAD_OK;
oom:
  nomad_destroy(h);
  cudaGetLastError();
  return NOMAD_ERR_OOM;
cuda_err:
  nomad_destroy(h);
  cudaGetLastError();
  return NOMAD_ERR_CUDA;
}

int nomad_load_ratings(nomad_t* h, int32_t fmt, int64_t nnz, const void* major,
                       const int32_t* minor, const float* vals, int32_t device_ptrs,
                       void* stream) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  if ((fmt != NOMAD_COO && fmt != NOMAD_CSC) || nnz < 0 || nnz >= (int64_t(1) << 32) ||
      (nnz > 0 && (!minor || !vals)) || (!major && (fmt == NOMAD_CSC || nnz > 0)))
    return fail(h, NOMAD_ERR_INVALID_ARG, "load_ratings: bad arguments");
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  free_layout(h);
  const int32_t *d_rows = nullptr, *d_cols = nullptr;
  const float* d_vals = nullptr;
  int32_t *own_rows = nullptr, *own_cols = nullptr;
  float* own_vals = nullptr;
  int64_t* own_colptr = nullptr;
  int32_t* exp_cols = nullptr;
  int rc = NOMAD_OK;
  if (fmt == NOMAD_COO) {
    CK(h, stage<int32_t>(static_cast<const int32_t*>(major), nnz, device_ptrs, st, &d_rows,
                         &own_rows),
       "load_ratings: rows");
    CK(h, stage<int32_t>(minor, nnz, device_ptrs, st, &d_cols, &own_cols), "load_ratings: cols");
  } else {
    const int64_t* d_colptr = nullptr;
    CK(h, stage<int64_t>(static_cast<const int64_t*>(major), h->n + 1, device_ptrs, st,
                         &d_colptr, &own_colptr),
       "load_ratings: colptr");
    CK(h, stage<int32_t>(minor, nnz, device_ptrs, st, &d_rows, &own_rows), "load_ratings: rows");
    CK(h, cudaMallocAsync(&exp_cols, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st),
       "load_ratings: cols");
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int32_t) * kStatusWords, st), "load_ratings");
    csc_expand_cols<<<unsigned((h->n + 255) / 256), 256, 0, st>>>(d_colptr, h->n, exp_cols,
                                                                h->status, nnz);
    ++h->launches;
    int32_t status = 0;
    CK(h, cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
       "load_ratings");
    CK(h, cudaStreamSynchronize(st), "load_ratings");
    if (status != 0) rc = fail(h, NOMAD_ERR_INVALID_ARG, "load_ratings: bad column pointers");
    d_cols = exp_cols;
  }
  if (rc == NOMAD_OK)
    CK(h, stage<float>(vals, nnz, device_ptrs, st, &d_vals, &own_vals), "load_ratings: vals");
  if (rc == NOMAD_OK) rc = build_layout(h, nnz, d_rows, d_cols, d_vals, st);
  if (own_rows) cudaFreeAsync(own_rows, st);
  if (own_cols) cudaFreeAsync(own_cols, st);
  if (own_vals) cudaFreeAsync(own_vals, st);
  if (own_colptr) cudaFreeAsync(own_colptr, st);
  if (exp_cols) cudaFreeAsync(exp_cols, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (rc != NOMAD_OK) {
    free_layout(h);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "load_ratings");
  h->loaded = true;
  h->epochs_done = 0;
  return NOMAD_OK;
}

namespace {

// Checks of one handle before n_epochs epochs, and its per-call buffers (the
// step-size table, the replay log) grown to the call's size.  The caller
// has made the handle's device current.
int prepare_call(nomad_t* h, int32_t n_epochs) {
  if (!h->loaded) return fail(h, NOMAD_ERR_STATE, "epoch: no ratings loaded");
  if (n_epochs < 1) return fail(h, NOMAD_ERR_INVALID_ARG, "epoch: n_epochs < 1");
  if (h->epochs_done + n_epochs >= (int64_t(1) << 31))
    return fail(h, NOMAD_ERR_INVALID_ARG, "epoch: epoch counter overflow");
  void* vp = nullptr;
  if (h->sched.mode == NOMAD_MODE_EPOCH && h->step_cap < n_epochs) {
    vp = h->step;
    dev_free(h, &vp);
    h->step = nullptr;
    CK(h, dev_alloc(h, &vp, sizeof(float) * n_epochs), "epoch: step table");
    h->step = static_cast<float*>(vp);
    h->step_cap = n_epochs;
  }
  if (h->sched.debug) {
    // one log entry per visit: S per epoch in epoch mode; uniform mode keeps
    // the first 8 |Omega| + 2^20 visits
    const int64_t need = h->sched.mode == NOMAD_MODE_EPOCH
                             ? h->n_seg * int64_t(n_epochs)
                             : 8 * h->nnz * int64_t(n_epochs) + (int64_t(1) << 20);
    if (need >= (int64_t(1) << 32))
      return fail(h, NOMAD_ERR_UNSUPPORTED, "epoch: replay log larger than 2^32 visits");
    if (h->log_cap < need) {
      dev_free(h, (void**)&h->log_seg);
      dev_free(h, (void**)&h->log_epoch);
      h->log_cap = 0;
      CK(h, dev_alloc(h, &vp, sizeof(int32_t) * need), "epoch: replay log");
      h->log_seg = static_cast<int32_t*>(vp);
      CK(h, dev_alloc(h, &vp, sizeof(int32_t) * need), "epoch: replay log");
      h->log_epoch = static_cast<int32_t*>(vp);
      h->log_cap = need;
    }
  }
  return NOMAD_OK;
}

// An error of handle h in a call over several handles, reported on h and on
// the first handle of the call.
int fail_many(nomad_t* h0, nomad_t* h, int code, const std::string& msg) {
  if (h != h0) fail(h0, code, msg);
  return fail(h, code, msg);
}

// Row width class of the batched kernel: one, two or four 16-byte chunks
// per lane.
int width_class(const nomad_t* h) { return h->k4 <= 32 ? 1 : h->k4 <= 64 ? 2 : 4; }

}  // namespace

int nomad_epoch(nomad_t* h, int32_t n_epochs, void* stream) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  int rc = prepare_call(h, n_epochs);
  if (rc != NOMAD_OK) return rc;
  rc = launch_epochs(h, n_epochs, st);
  if (rc != NOMAD_OK) return rc;
  h->epochs_done += n_epochs;
  return NOMAD_OK;
}

int nomad_epoch_many(nomad_t* const* hs, int32_t count, int32_t n_epochs, void* stream) {
  if (!hs || count < 1) return NOMAD_ERR_INVALID_ARG;
  for (int g = 0; g < count; ++g) {
    if (!hs[g]) return NOMAD_ERR_INVALID_ARG;
    for (int f = 0; f < g; ++f)
      if (hs[f] == hs[g]) return fail_many(hs[0], hs[g], NOMAD_ERR_INVALID_ARG, "epoch_many: a handle occurs twice");
  }
  nomad_t* h0 = hs[0];
  for (int g = 0; g < count; ++g) {
    nomad_t* h = hs[g];
    if (!h->loaded) return fail_many(h0, h, NOMAD_ERR_STATE, "epoch_many: no ratings loaded");
    if (h->sched.mode != NOMAD_MODE_EPOCH || h->sched.variant != NOMAD_VARIANT_BATCHED)
      return fail_many(h0, h, NOMAD_ERR_UNSUPPORTED,
                       "epoch_many: epoch mode with the batched variant only");
    if (h->device != h0->device || h->sched.precision != h0->sched.precision ||
        (h->sched.debug != 0) != (h0->sched.debug != 0) ||
        h->warps_per_block != h0->warps_per_block || width_class(h) != width_class(h0))
      return fail_many(h0, h, NOMAD_ERR_UNSUPPORTED,
                       "epoch_many: handles differ in device, precision, debug, warps per block or "
                  "row width");
  }
  DeviceGuard guard(h0->device);
  cudaStream_t st = as_stream(stream);
  for (int g = 0; g < count; ++g) {
    const int rc = prepare_call(hs[g], n_epochs);
    if (rc != NOMAD_OK) {
      if (hs[g] != h0) h0->last_error = hs[g]->last_error;
      return rc;
    }
  }
  const int rc = launch_epochs_many(hs, count, n_epochs, st);
  if (rc != NOMAD_OK) return rc;
  for (int g = 0; g < count; ++g) hs[g]->epochs_done += n_epochs;
  return NOMAD_OK;
}

int nomad_last_epoch_span_ns(nomad_t* h, int64_t* ns, void* stream) {
  if (!h || !ns) return NOMAD_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  unsigned long long span[2] = {0, 0};
  CK(h, cudaMemcpyAsync(span, h->span, sizeof(span), cudaMemcpyDeviceToHost, st),
     "last_epoch_span_ns");
  CK(h, cudaStreamSynchronize(st), "last_epoch_span_ns");
  *ns = span[1] > span[0] ? int64_t(span[1] - span[0]) : 0;
  return NOMAD_OK;
}

int nomad_check(nomad_t* h, void* stream) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  int32_t status[kStatusWords] = {0, 0, 0, 0};
  CK(h, cudaMemcpyAsync(status, h->status, sizeof(status), cudaMemcpyDeviceToHost, st),
     "check");
  CK(h, cudaStreamSynchronize(st), "check");
  if (status[0] != 0) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "device: %s (worker %d, detail %d, violations %d)",
                  nomad_error_string(status[0]), status[1], status[2], status[3]);
    h->last_error = buf;
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int32_t) * kStatusWords, st), "check");
    CK(h, cudaStreamSynchronize(st), "check");
    return status[0];
  }
  return NOMAD_OK;
}

int nomad_rmse(nomad_t* h, int64_t nnz, const int32_t* rows, const int32_t* cols,
               const float* vals, int32_t device_ptrs, double* out, void* stream) {
  if (!h || !out || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals)))
    return fail(h, NOMAD_ERR_INVALID_ARG, "rmse: bad arguments");
  if (int rc = nomad_check(h, stream)) return rc;
  if (nnz == 0) {
    *out = std::nan("");
    return NOMAD_OK;
  }
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  const int32_t *d_rows, *d_cols;
  const float* d_vals;
  int32_t *o_rows, *o_cols;
  float* o_vals;
  CK(h, stage<int32_t>(rows, nnz, device_ptrs, st, &d_rows, &o_rows), "rmse: rows");
  CK(h, stage<int32_t>(cols, nnz, device_ptrs, st, &d_cols, &o_cols), "rmse: cols");
  CK(h, stage<float>(vals, nnz, device_ptrs, st, &d_vals, &o_vals), "rmse: vals");
  CK(h, cudaMemsetAsync(h->status, 0, sizeof(int32_t), st), "rmse");
  double sum = 0.0;
  int rc = rmse_sum(h, nnz, d_rows, d_cols, d_vals, &sum, st);
  if (o_rows) cudaFreeAsync(o_rows, st);
  if (o_cols) cudaFreeAsync(o_cols, st);
  if (o_vals) cudaFreeAsync(o_vals, st);
  int32_t status = 0;
  CK(h, cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
     "rmse");
  CK(h, cudaStreamSynchronize(st), "rmse");
  if (rc != NOMAD_OK) return fail(h, rc, "rmse: kernel launch failed");
  if (status != 0) {
    cudaMemsetAsync(h->status, 0, sizeof(int32_t), st);
    cudaStreamSynchronize(st);
    return fail(h, status, "rmse: test index out of range");
  }
  *out = std::sqrt(sum / double(nnz));
  return NOMAD_OK;
}

int nomad_objective(nomad_t* h, double* out, void* stream) {
  if (!h || !out) return NOMAD_ERR_INVALID_ARG;
  if (!h->loaded) return fail(h, NOMAD_ERR_STATE, "objective: no ratings loaded");
  if (int rc = nomad_check(h, stream)) return rc;
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  double sum = 0.0;
  const int rc = objective_sum(h, &sum, st);
  CK(h, cudaStreamSynchronize(st), "objective");
  if (rc != NOMAD_OK) return fail(h, rc, "objective: kernel launch failed");
  *out = 0.5 * sum;
  return NOMAD_OK;
}

int nomad_get_factors(nomad_t* h, float* W, float* H, int32_t device_ptrs, void* stream) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  if (int rc = nomad_check(h, stream)) return rc;
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  float* outs[2] = {W, H};
  const int64_t rows[2] = {h->m, h->n};
  for (int f = 0; f < 2; ++f) {
    if (!outs[f]) continue;
    if (device_ptrs) {
      if (int rc = factors_to_f32(h, f, outs[f], st)) return fail(h, rc, "get_factors");
    } else {
      float* tmp = nullptr;
      CK(h, cudaMallocAsync(&tmp, sizeof(float) * rows[f] * h->k, st), "get_factors");
      const int rc = factors_to_f32(h, f, tmp, st);
      const cudaError_t e = cudaMemcpyAsync(outs[f], tmp, sizeof(float) * rows[f] * h->k,
                                            cudaMemcpyDeviceToHost, st);
      cudaFreeAsync(tmp, st);
      if (rc != NOMAD_OK) return fail(h, rc, "get_factors");
      CK(h, e, "get_factors: copy");
    }
  }
  CK(h, cudaStreamSynchronize(st), "get_factors");
  return NOMAD_OK;
}

int nomad_set_factors(nomad_t* h, const float* W, const float* H, int32_t device_ptrs,
                      int64_t epochs_done, void* stream) {
  if (!h || epochs_done < 0 || epochs_done >= (int64_t(1) << 31))
    return fail(h, NOMAD_ERR_INVALID_ARG, "set_factors: bad arguments");
  DeviceGuard guard(h->device);
  cudaStream_t st = as_stream(stream);
  const float* ins[2] = {W, H};
  const int64_t rows[2] = {h->m, h->n};
  for (int f = 0; f < 2; ++f) {
    if (!ins[f]) continue;
    const float* d = nullptr;
    float* owned = nullptr;
    CK(h, stage<float>(ins[f], rows[f] * h->k, device_ptrs, st, &d, &owned), "set_factors");
    const int rc = factors_from_f32(h, f, d, st);
    if (owned) cudaFreeAsync(owned, st);
    if (rc != NOMAD_OK) return fail(h, rc, "set_factors");
  }
  CK(h, cudaStreamSynchronize(st), "set_factors");
  h->epochs_done = epochs_done;
  return NOMAD_OK;
}

int nomad_get_info(const nomad_t* h, nomad_info* out) {
  if (!h || !out) return NOMAD_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->m = h->m;
  out->n = h->n;
  out->k = h->k;
  out->p = h->p;
  out->nnz = h->nnz;
  out->n_segments = h->n_seg;
  out->epochs_done = h->epochs_done;
  out->pitch = h->pitch;
  out->precision = h->sched.precision;
  out->mode = h->sched.mode;
  out->warps_per_block = h->warps_per_block;
  out->blocks = h->blocks;
  out->sm_count = h->sm_count;
  out->device_bytes = h->device_bytes;
  out->kernel_launches = h->launches;
  out->predrawn_ratings = h->ubits_pre ? h->upre_records : 0;
  return NOMAD_OK;
}

int nomad_last_epoch_kernel_ms(nomad_t* h, float* ms) {
  if (!h || !ms) return NOMAD_ERR_INVALID_ARG;
  if (!h->ev_recorded) return fail(h, NOMAD_ERR_STATE, "no epoch kernel has run yet");
  DeviceGuard guard(h->device);
  CK(h, cudaEventSynchronize(h->ev_stop), "epoch timing");
  CK(h, cudaEventElapsedTime(ms, h->ev_start, h->ev_stop), "epoch timing");
  return NOMAD_OK;
}

int nomad_get_layout(nomad_t* h, int32_t* row_worker, int32_t* seg_worker, int32_t* seg_col,
                     int64_t* seg_ptr, int32_t* rec_row, float* rec_val) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  if (!h->loaded) return fail(h, NOMAD_ERR_STATE, "get_layout: no ratings loaded");
  DeviceGuard guard(h->device);
  const int64_t S = h->n_seg;
  if (row_worker)
    CK(h, cudaMemcpy(row_worker, h->row_worker, sizeof(int32_t) * h->m, cudaMemcpyDeviceToHost),
       "get_layout");
  if (seg_worker && S)
    CK(h, cudaMemcpy(seg_worker, h->seg_worker, sizeof(int32_t) * S, cudaMemcpyDeviceToHost),
       "get_layout");
  if (seg_col && S)
    CK(h, cudaMemcpy(seg_col, h->seg_col, sizeof(int32_t) * S, cudaMemcpyDeviceToHost),
       "get_layout");
  if (seg_ptr)
    CK(h, cudaMemcpy(seg_ptr, h->seg_ptr, sizeof(int64_t) * (S + 1), cudaMemcpyDeviceToHost),
       "get_layout");
  if ((rec_row || rec_val) && h->nnz > 0) {
    int2* tmp = new int2[size_t(h->nnz)];
    const cudaError_t e =
        cudaMemcpy(tmp, h->rec, sizeof(int2) * h->nnz, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      for (int64_t r = 0; r < h->nnz; ++r) {
        if (rec_row) rec_row[r] = tmp[r].x;
        if (rec_val) std::memcpy(rec_val + r, &tmp[r].y, sizeof(float));
      }
    }
    delete[] tmp;
    CK(h, e, "get_layout");
  }
  return NOMAD_OK;
}

int nomad_get_replay_log(nomad_t* h, int64_t cap, int32_t* seg, int32_t* epoch,
                         int64_t* count) {
  if (!h || !count || cap < 0) return NOMAD_ERR_INVALID_ARG;
  if (!h->sched.debug) return fail(h, NOMAD_ERR_STATE, "replay log: debug mode is off");
  DeviceGuard guard(h->device);
  CK(h, cudaDeviceSynchronize(), "replay log");
  uint32_t ticket = 0;
  CK(h, cudaMemcpy(&ticket, h->log_ticket, sizeof(uint32_t), cudaMemcpyDeviceToHost),
     "replay log");
  *count = int64_t(ticket);
  int64_t nw = int64_t(ticket) < cap ? int64_t(ticket) : cap;
  if (nw > h->log_cap) nw = h->log_cap;
  if (nw > 0 && seg)
    CK(h, cudaMemcpy(seg, h->log_seg, sizeof(int32_t) * nw, cudaMemcpyDeviceToHost),
       "replay log");
  if (nw > 0 && epoch)
    CK(h, cudaMemcpy(epoch, h->log_epoch, sizeof(int32_t) * nw, cudaMemcpyDeviceToHost),
       "replay log");
  return NOMAD_OK;
}

int nomad_get_debug_counts(nomad_t* h, int32_t* rec_count, int64_t* ownership_violations) {
  if (!h) return NOMAD_ERR_INVALID_ARG;
  if (!h->rec_count) return fail(h, NOMAD_ERR_STATE, "debug counts: debug mode is off");
  DeviceGuard guard(h->device);
  CK(h, cudaDeviceSynchronize(), "debug counts");
  if (rec_count && h->nnz > 0)
    CK(h, cudaMemcpy(rec_count, h->rec_count, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost),
       "debug counts");
  if (ownership_violations) {
    int32_t st[kStatusWords];
    CK(h, cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost), "debug counts");
    *ownership_violations = st[3];
  }
  return NOMAD_OK;
}

void nomad_destroy(nomad_t* h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  cudaDeviceSynchronize();
  free_layout(h);
  void** ptrs[] = {&h->W, &h->H, (void**)&h->Wscale, (void**)&h->status, (void**)&h->row_worker,
                   (void**)&h->result, (void**)&h->upd_done, (void**)&h->stop,
                   (void**)&h->log_ticket, (void**)&h->step, (void**)&h->partials};
  for (void** p : ptrs) dev_free(h, p);
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->ev_stop) cudaEventDestroy(h->ev_stop);
  delete h;
}

}  // extern "C"
