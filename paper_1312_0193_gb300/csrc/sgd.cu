// sgd.cu -- the persistent NOMAD kernel (Sec. 3.1, Alg. 1) for GB300.
//
// One warp is one NOMAD worker q.  It owns the users of its row block I_q
// (their rows w_i stay in HBM/L2 and are only ever touched by this warp) and
// a ring queue of item tokens.  A visit is:
//   pop a token from the own ring (lane 0 polls with acquire loads, bounded
//   by a timeout) -> load h_j into registers -> for every rating (i,j) of the
//   set Omega-bar_j^(q): e = A_ij - <w_i,h_j> (warp-shuffle dot over k),
//   w_i += s (e h_j - lambda w_i), h_j += s (e w_i - lambda h_j) with the old
//   w_i (Eq. w_update / h_update, descent sign) -> store h_j -> route the
//   token -> push it into the next worker's ring with a release store.
// h_j is owned by exactly one warp at a time, so no update takes a lock and
// the visits are serialisable (the owner-computes rule of Sec. 3.1).
//
// Routing.  Epoch mode (Sec. 3.4's permutation circulation): item j visits
// the d_j workers that hold ratings of j once per epoch, in the order of a
// keyed pseudo-random permutation of [0, d_j) (a bijection on [0, 2^b)
// restricted to [0, d_j) by cycle walking), keyed by (seed, j, epoch).
// Uniform mode (Alg. 1 literally): the next worker is uniform over p.
//
// Rings.  Slot = {lap:32 | payload:32}.  A producer reserves a position with
// one atomicAdd on the ring's tail and publishes the payload with a release
// store tagged with the lap; the consumer, which alone advances its head,
// waits until the slot shows the lap it expects.  A ring never holds more
// tokens than its capacity (epoch mode: the number of items the worker
// holds; uniform mode: n), so a position is reused only after its previous
// payload was consumed.
#include "sgd_common.cuh"

namespace nomad {
namespace {

constexpr int kPrefetch = 4;   // W rows in flight per worker (simple kernel)

template <int CPL>
__device__ __forceinline__ void load_row(float4 (&w)[CPL], const float4* row,
                                         int lane, int k4) {
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int idx = lane + 32 * c;
    w[c] = idx < k4 ? row[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// The SGD updates of one visit: every rating of the segment [beg, end), in
// storage order (rows ascending).  h stays in registers; each lane holds
// CPL chunks of 4 entries of w_i and h_j.  Up to kPrefetch rows of W are in
// flight ahead of the serial chain through h_j (rows inside a segment are
// distinct, so the prefetches never alias an update in progress).
template <int CPL, bool COUNT>
__device__ __forceinline__ void sgd_segment(float4 (&h)[CPL], float4* __restrict__ W4,
                                            int64_t pitch4, int k4,
                                            const int2* __restrict__ rec,
                                            int64_t beg, int64_t end, float s,
                                            float lam, int lane,
                                            int32_t* __restrict__ rec_count,
                                            const SgdParams* P) {
  for (int64_t base = beg; base < end; base += 32) {
    const int nr = int(end - base < 32 ? end - base : 32);
    const int2 my = lane < nr ? __ldcs(rec + base + lane) : make_int2(0, 0);
    float4 wb[kPrefetch][CPL];
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int row = __shfl_sync(kFull, my.x, u);
      if (u < nr) load_row<CPL>(wb[u], W4 + row * pitch4, lane, k4);
    }
    for (int u0 = 0; u0 < nr; u0 += kPrefetch) {
#pragma unroll
      for (int pf = 0; pf < kPrefetch; ++pf) {
        const int u = u0 + pf;
        if (u < nr) {
          const int row = __shfl_sync(kFull, my.x, u);
          const float a = __int_as_float(__shfl_sync(kFull, my.y, u));
          float4 w[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) w[c] = wb[pf][c];
          const int un = u + kPrefetch;
          const int row_n = __shfl_sync(kFull, my.x, un & 31);
          if (un < nr) load_row<CPL>(wb[pf], W4 + row_n * pitch4, lane, k4);
          float part = 0.f;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            part = fmaf(w[c].x, h[c].x, part);
            part = fmaf(w[c].y, h[c].y, part);
            part = fmaf(w[c].z, h[c].z, part);
            part = fmaf(w[c].w, h[c].w, part);
          }
          float e = a - warp_sum(part);
          float step = s;
          if (COUNT) {
            // uniform mode: s_t from the per-rating update counter t.  Lane 0
            // alone reads it (it also increments it below) and broadcasts:
            // lanes of a warp need not run in lockstep, so a read by another
            // lane could see the increment.
            int t = 0;
            if (lane == 0) t = rec_count[base + u];
            t = __shfl_sync(kFull, t, 0);
            const float tf = float(t);
            step = P->alpha / (1.f + P->beta * tf * sqrtf(tf));
          }
          float4* wrow = W4 + row * pitch4;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int idx = lane + 32 * c;
            float4 wn, hn;
            wn.x = fmaf(step, fmaf(e, h[c].x, -lam * w[c].x), w[c].x);
            wn.y = fmaf(step, fmaf(e, h[c].y, -lam * w[c].y), w[c].y);
            wn.z = fmaf(step, fmaf(e, h[c].z, -lam * w[c].z), w[c].z);
            wn.w = fmaf(step, fmaf(e, h[c].w, -lam * w[c].w), w[c].w);
            hn.x = fmaf(step, fmaf(e, w[c].x, -lam * h[c].x), h[c].x);
            hn.y = fmaf(step, fmaf(e, w[c].y, -lam * h[c].y), h[c].y);
            hn.z = fmaf(step, fmaf(e, w[c].z, -lam * h[c].z), h[c].z);
            hn.w = fmaf(step, fmaf(e, w[c].w, -lam * h[c].w), h[c].w);
            if (idx < k4) {
              wrow[idx] = wn;
              h[c] = hn;
            }
          }
          if (rec_count != nullptr && lane == 0) rec_count[base + u] += 1;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ kernels
// Put every item token into its first queue of the launch.
__global__ void seed_tokens(const SgdParams P, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
    const int base = P.col_seg_ptr[j];
    const int d = P.col_seg_ptr[j + 1] - base;
    if (d == 0) continue;  // an item without ratings never circulates
    P.tok_hop[j] = 0;
    P.tok_epoch[j] = P.epoch0;
    if (j == P.drop_item) continue;  // planted lost message (tests only)
    if (P.stop == nullptr) {
      const uint4 key = philox4x32_10(
          make_uint4(uint32_t(j), uint32_t(P.epoch0), 0u, kTagItinerary),
          make_uint2(P.seed_lo, P.seed_hi));
      int seg = P.col_segs[base + itinerary_slot(0u, uint32_t(d), key)];
      if (P.tok_rec) {  // the batched kernel: the next-visit record, item payloads
        int4 c4 = make_int4(0, 0, 0, 0);
        if (P.col_grp_ptr) {  // hybrid circulation: the first worker of the first run
          const int gb = P.col_grp_ptr[j];
          const int G = P.col_grp_ptr[j + 1] - gb - 1;
          const int g = int(itinerary_slot(0u, uint32_t(G), key));
          const int o = P.grp_off[gb + g];
          const int z = P.grp_off[gb + g + 1] - o;
          seg = P.col_segs[base + o + int(itinerary_slot(
                                         0u, uint32_t(z), make_uint4(key.w, key.z, key.y, key.x)))];
          c4 = make_int4(gb, G, o, z);
        }
        const int64_t b0 = P.seg_ptr[seg];
        P.tok_rec[kTokRec * j] = make_int4(seg, int(P.seg_ptr[seg + 1] - b0), int(uint32_t(b0)),
                                           P.epoch0);
        P.tok_rec[kTokRec * j + 1] = make_int4(0, base, d, 0);
        P.tok_rec[kTokRec * j + 2] = c4;
        if (P.use_urgent && P.item_urgent[j]) push_urgent(P, P.seg_worker[seg], uint32_t(j));
        else push_token(P, P.seg_worker[seg], uint32_t(j));
      } else {
        push_token(P, P.seg_worker[seg], uint32_t(seg));
      }
    } else {
      const uint4 r = philox4x32_10(make_uint4(uint32_t(j), 0u, 0u, kTagUniform),
                                    make_uint2(P.seed_lo, P.seed_hi));
      const int q = int((static_cast<unsigned long long>(r.x) * uint32_t(P.p)) >> 32);
      push_token(P, q, uint32_t(j));
    }
  }
}

// Epoch mode: worker q makes exactly (segments of q) x n_epochs visits.
template <int CPL, bool DEBUG>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32)
nomad_epoch_kernel(const SgdParams P) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= P.p) return;
  const int64_t quota =
      int64_t(P.worker_seg_ptr[q + 1] - P.worker_seg_ptr[q]) * P.n_epochs;
  const int lg = P.ring_log2[q];
  const unsigned long long* ring_q = P.ring + P.ring_base[q];
  float4* __restrict__ W4 = reinterpret_cast<float4*>(P.W);
  float4* __restrict__ H4 = reinterpret_cast<float4*>(P.H);
  const int64_t pitch4 = P.pitch >> 2;
  const int k4 = P.k4;
  const uint2 seed = make_uint2(P.seed_lo, P.seed_hi);
  const int epoch_end = P.epoch0 + P.n_epochs;

  uint32_t head = 0;
  for (int64_t v = 0; v < quota; ++v, ++head) {
    int seg = 0, e = 0, hop = 0;
    if (lane == 0) {
      seg = pop_token(P, q, head, lg, ring_q);
      if (seg >= 0) {
        const int j = __ldg(P.seg_col + seg);
        e = __ldcg(P.tok_epoch + j);
        hop = __ldcg(P.tok_hop + j);
        if (DEBUG) {
          const uint32_t t = atomicAdd(P.log_ticket, 1u);
          if (int64_t(t) < P.log_cap) {
            P.log_seg[t] = seg;
            P.log_epoch[t] = e;
          }
          if (atomicExch(P.owner + j, q) != -1) flag_ownership(P, q, j);
        }
      }
    }
    seg = __shfl_sync(kFull, seg, 0);
    if (seg < 0) return;
    e = __shfl_sync(kFull, e, 0);
    hop = __shfl_sync(kFull, hop, 0);
    const int j = __ldg(P.seg_col + seg);
    const float s = P.step[e - P.epoch0];

    float4 h[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int idx = lane + 32 * c;
      h[c] = idx < k4 ? __ldcg(H4 + j * pitch4 + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    sgd_segment<CPL, false>(h, W4, pitch4, k4, P.rec, __ldg(P.seg_ptr + seg),
                            __ldg(P.seg_ptr + seg + 1), s, P.lambda, lane,
                            DEBUG ? P.rec_count : nullptr, &P);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int idx = lane + 32 * c;
      if (idx < k4) __stcg(H4 + j * pitch4 + idx, h[c]);
    }
    __syncwarp();  // every lane's h_j stores precede lane 0's release
    if (lane == 0) {
      const int base = __ldg(P.col_seg_ptr + j);
      const int d = __ldg(P.col_seg_ptr + j + 1) - base;
      int nh = hop + 1, ne = e;
      if (nh == d) {
        nh = 0;
        ne = e + 1;
      }
      __stcg(P.tok_hop + j, nh);
      __stcg(P.tok_epoch + j, ne);
      if (DEBUG && atomicExch(P.owner + j, -1) != q) flag_ownership(P, q, j);
      if (ne < epoch_end) {
        const uint4 key = philox4x32_10(
            make_uint4(uint32_t(j), uint32_t(ne), 0u, kTagItinerary), seed);
        const int nseg = __ldg(P.col_segs + base + itinerary_slot(uint32_t(nh), uint32_t(d), key));
        __threadfence();
        push_token(P, __ldg(P.seg_worker + nseg), uint32_t(nseg));
      }
    }
  }
}

// Uniform mode (Alg. 1 literally): the token carries the item id; a visit to
// a worker without ratings of j applies no update; the launch ends when
// upd_budget updates have been applied (the stop flag).
template <int CPL, bool DEBUG>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32)
nomad_uniform_kernel(const SgdParams P) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= P.p) return;
  const int lg = P.ring_log2[q];
  const unsigned long long* ring_q = P.ring + P.ring_base[q];
  float4* __restrict__ W4 = reinterpret_cast<float4*>(P.W);
  float4* __restrict__ H4 = reinterpret_cast<float4*>(P.H);
  const int64_t pitch4 = P.pitch >> 2;
  const int k4 = P.k4;
  const uint2 seed = make_uint2(P.seed_lo, P.seed_hi);

  for (uint32_t head = 0;; ++head) {
    int j = 0, hop = 0;
    if (lane == 0) {
      j = pop_token(P, q, head, lg, ring_q);
      // tokens taken, for senders that route to the shorter queue
      if (j >= 0 && P.routing == NOMAD_ROUTING_SHORTER) st_relaxed_u32(P.ring_head + q, head + 1);
      if (j >= 0) {
        hop = __ldcg(P.tok_hop + j);
        if (DEBUG && atomicExch(P.owner + j, q) != -1) flag_ownership(P, q, j);
      }
    }
    j = __shfl_sync(kFull, j, 0);
    if (j < 0) return;
    hop = __shfl_sync(kFull, hop, 0);
    // find the segment (q, j): 32-way search over item j's segments, which
    // are ordered by worker
    const int base = __ldg(P.col_seg_ptr + j);
    int lo = base, hi = __ldg(P.col_seg_ptr + j + 1);
    int seg = -1;
    while (hi - lo > 32) {
      const int step = (hi - lo + 31) >> 5;
      const int pos = lo + lane * step;
      const int wk = pos < hi ? __ldg(P.seg_worker + __ldg(P.col_segs + pos)) : 0x7fffffff;
      const unsigned le = __ballot_sync(kFull, wk <= q);
      if (le == 0) { hi = lo; break; }
      const int last = 31 - __clz(le);
      lo = lo + last * step;
      hi = min(hi, lo + step);
    }
    {
      const int pos = lo + lane;
      const int sg = pos < hi ? __ldg(P.col_segs + pos) : -1;
      const unsigned hit = __ballot_sync(kFull, sg >= 0 && __ldg(P.seg_worker + sg) == q);
      if (hit) seg = __shfl_sync(kFull, sg, __ffs(hit) - 1);
    }
    __syncwarp();
    if (DEBUG && lane == 0) {
      const uint32_t t = atomicAdd(P.log_ticket, 1u);
      if (int64_t(t) < P.log_cap) {
        P.log_seg[t] = seg;
        P.log_epoch[t] = j;
      }
    }
    if (seg >= 0) {
      float4 h[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int idx = lane + 32 * c;
        h[c] = idx < k4 ? __ldcg(H4 + j * pitch4 + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int64_t beg = __ldg(P.seg_ptr + seg), end = __ldg(P.seg_ptr + seg + 1);
      sgd_segment<CPL, true>(h, W4, pitch4, k4, P.rec, beg, end, 0.f, P.lambda, lane,
                             P.rec_count, &P);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int idx = lane + 32 * c;
        if (idx < k4) __stcg(H4 + j * pitch4 + idx, h[c]);
      }
      if (lane == 0) {
        const unsigned long long before =
            atomicAdd(P.upd_done, static_cast<unsigned long long>(end - beg));
        if (before + static_cast<unsigned long long>(end - beg) >= P.upd_budget)
          atomicExch(P.stop, 1);
      }
    }
    __syncwarp();
    if (lane == 0) {
      const int nh = hop + 1;
      __stcg(P.tok_hop + j, nh);
      if (DEBUG && atomicExch(P.owner + j, -1) != q) flag_ownership(P, q, j);
      const uint4 r = philox4x32_10(make_uint4(uint32_t(j), uint32_t(nh), 0u, kTagUniform), seed);
      int q2 = int((static_cast<unsigned long long>(r.x) * uint32_t(P.p)) >> 32);
      if (P.routing == NOMAD_ROUTING_SHORTER) {
        // Sec. 3.3: of two workers drawn uniformly, the one with fewer tokens
        // waiting (pushed minus taken; a snapshot, as a message payload is)
        const int qb = int((static_cast<unsigned long long>(r.y) * uint32_t(P.p)) >> 32);
        const uint32_t la = ld_relaxed_u32(P.ring_tail + q2) - ld_relaxed_u32(P.ring_head + q2);
        const uint32_t lb = ld_relaxed_u32(P.ring_tail + qb) - ld_relaxed_u32(P.ring_head + qb);
        if (lb < la) q2 = qb;
      }
      __threadfence();
      push_token(P, q2, uint32_t(j));
    }
    int stop_now = 0;
    if (lane == 0) stop_now = ld_relaxed_i32(P.stop);
    if (__shfl_sync(kFull, stop_now, 0)) return;
  }
}

__global__ void fill_step_sizes(float* step, int32_t epoch0, int32_t n_epochs,
                                double alpha, double beta) {
  for (int e = threadIdx.x; e < n_epochs; e += blockDim.x) {
    const double t = double(epoch0 + e);
    step[e] = float(alpha / (1.0 + beta * pow(t, 1.5)));
  }
}

template <int CPL>
const void* epoch_kernel_ptr(bool debug, int mode) {
  if (mode == NOMAD_MODE_UNIFORM)
    return debug ? (const void*)nomad_uniform_kernel<CPL, true>
                 : (const void*)nomad_uniform_kernel<CPL, false>;
  return debug ? (const void*)nomad_epoch_kernel<CPL, true>
               : (const void*)nomad_epoch_kernel<CPL, false>;
}

}  // namespace

// The worker kernel for a handle's settings and its dynamic shared memory per
// warp (bytes).
const void* worker_kernel(int k4, bool debug, int mode, int variant, int precision, bool blk,
                          size_t* smem_per_warp) {
  *smem_per_warp = 0;
  if (mode == NOMAD_MODE_EPOCH && variant == NOMAD_VARIANT_BATCHED)
    return batched_kernel(k4, debug, precision, false, blk, smem_per_warp);
  if (precision != NOMAD_FP32) return nullptr;  // narrow storage: batched kernel only
  if (k4 <= 32) return epoch_kernel_ptr<1>(debug, mode);
  if (k4 <= 64) return epoch_kernel_ptr<2>(debug, mode);
  if (k4 <= 128) return epoch_kernel_ptr<4>(debug, mode);
  return nullptr;
}

int max_resident_workers(int device, int warps_per_block, int k4, int precision, int mode,
                         int variant, int* blocks_per_sm, bool blk) {
  // the hybrid circulation's inboxes follow the warps' areas
  const size_t extra_smem_per_warp = blk ? batched_inbox_bytes() : 0;
  if (warps_per_block <= 0) warps_per_block = kDefaultWarpsPerBlock;
  if (warps_per_block > kMaxWarpsPerBlock) return -1;
  int per_sm = 1 << 30;
  // the debug variant must fit the same grid
  for (int dbg = 0; dbg < 2; ++dbg) {
    size_t spw = 0;
    const void* fn = worker_kernel(k4, dbg, mode, variant, precision, blk, &spw);
    if (!fn) return -1;
    const size_t smem = (spw + extra_smem_per_warp) * warps_per_block;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
      return -1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, warps_per_block * 32, smem) !=
        cudaSuccess)
      return -1;
    if (b < per_sm) per_sm = b;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (blocks_per_sm) *blocks_per_sm = per_sm;
  return per_sm * sms * warps_per_block;
}

int default_warps_per_block() { return kDefaultWarpsPerBlock; }

namespace {

// The worker kernel's parameters for the next n_epochs of handle h (in *out),
// after the launch's preparation on `st`: ring, queue and status resets, the
// step-size table and the initial tokens.
int prepare_epochs(nomad_handle* h, int32_t n_epochs, cudaStream_t st, SgdParams* out,
                   int32_t epoch_off = 0, bool first = true) {
  const bool uniform = h->sched.mode == NOMAD_MODE_UNIFORM;
  const bool debug = h->sched.debug != 0;
  SgdParams& P = *out;
  P = SgdParams{};
  P.W = h->W;
  P.H = h->H;
  P.Wscale = h->Wscale;
  P.pitch = h->pitch;
  P.k4 = h->k4;
  P.rec = h->rec;
  P.seg_ptr = h->seg_ptr;
  P.seg_col = h->seg_col;
  P.seg_worker = h->seg_worker;
  P.worker_seg_ptr = h->worker_seg_ptr;
  P.col_seg_ptr = h->col_seg_ptr;
  P.col_segs = h->col_segs;
  P.col_grp_ptr = (!uniform && h->sched.variant == NOMAD_VARIANT_BATCHED &&
                   h->sched.circulation == NOMAD_CIRCULATION_BLOCK) ? h->col_grp_ptr : nullptr;
  P.grp_off = h->grp_off;
  P.wpb = h->warps_per_block;
  P.batch_cap = h->sched.batch_tokens;
  P.ring = h->ring;
  P.ring_base = h->ring_base;
  P.ring_log2 = h->ring_log2;
  P.ring_tail = h->ring_tail;
  P.ring_head = h->ring_head;
  P.routing = h->sched.routing;
  P.tok_hop = h->tok_hop;
  P.tok_epoch = h->tok_epoch;
  P.item_urgent = h->item_urgent;
  P.tok_rec = (!uniform && h->sched.variant == NOMAD_VARIANT_BATCHED) ? h->tok_rec : nullptr;
  P.uring = h->uring;
  P.uring_tail = h->uring_tail;
  P.uring_log2 = h->uring_log2;
  // the batched kernel takes urgent items' visits out of turn (one chunk per lane)
  P.use_urgent = (!uniform && h->sched.variant == NOMAD_VARIANT_BATCHED && h->k4 <= 32 &&
                  h->uring != nullptr) ? 1 : 0;
  P.step = h->step;
  P.epoch0 = int32_t(h->epochs_done) + epoch_off;
  P.n_epochs = n_epochs;
  // the urgent items' rounding bits are drawn before a launch of one epoch
  if (h->ubits_pre && n_epochs == 1 && P.use_urgent) {
    P.useg_off = h->useg_off;
    P.ubits_pre = h->ubits_pre;
  }
  P.p = h->p;
  P.lambda = h->lambda;
  P.alpha = h->sched.alpha;
  P.beta = h->sched.beta;
  P.seed_lo = uint32_t(h->sched.seed);
  P.seed_hi = uint32_t(h->sched.seed >> 32);
  P.timeout_ns = h->sched.spin_timeout_ns > 0 ? h->sched.spin_timeout_ns : 10000000000ll;
  P.status = h->status;
  P.span = h->span;
  P.upd_done = uniform ? h->upd_done : nullptr;
  P.upd_budget = static_cast<unsigned long long>(n_epochs) * static_cast<unsigned long long>(h->nnz);
  P.stop = uniform ? h->stop : nullptr;
  P.log_ticket = h->log_ticket;
  P.log_seg = h->log_seg;
  P.log_epoch = h->log_epoch;
  P.log_cap = h->log_cap;
  P.owner = h->owner;
  P.rec_count = h->rec_count;
  P.drop_item = h->sched.debug_drop_item;

  cudaError_t e;
  if ((e = cudaMemsetAsync(h->ring, 0xff, sizeof(unsigned long long) * h->ring_slots, st)) ||
      (e = cudaMemsetAsync(h->ring_tail, 0, sizeof(uint32_t) * h->p, st)) ||
      (e = cudaMemsetAsync(h->ring_head, 0, sizeof(uint32_t) * h->p, st)) ||
      (h->uring && (e = cudaMemsetAsync(h->uring, 0xff,
                                        sizeof(unsigned long long) * (int64_t(h->p) << h->uring_log2),
                                        st))) ||
      (h->uring_tail && (e = cudaMemsetAsync(h->uring_tail, 0, sizeof(uint32_t) * h->p, st))) ||
      // status and span cover the whole call: an error of one launch stays
      // for nomad_check (the call's later launches see it and stop at their
      // first wait), and the span runs from the first launch's start
      (first && (e = cudaMemsetAsync(h->status, 0, sizeof(int32_t) * kStatusWords, st))) ||
      (first && (e = cudaMemsetAsync(h->span, 0xff, sizeof(unsigned long long), st))) ||
      (first && (e = cudaMemsetAsync(h->span + 1, 0, sizeof(unsigned long long), st)))) {
    h->last_error = std::string("epoch: ") + cudaGetErrorString(e);
    return NOMAD_ERR_CUDA;
  }
  if (uniform) {
    cudaMemsetAsync(h->upd_done, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(h->stop, 0, sizeof(int32_t), st);
  } else {
    fill_step_sizes<<<1, 256, 0, st>>>(h->step, P.epoch0, n_epochs, h->sched.alpha,
                                       h->sched.beta);
    ++h->launches;
  }
  if (debug && first) cudaMemsetAsync(h->log_ticket, 0, sizeof(uint32_t), st);
  const int64_t n = h->n;
  unsigned seed_grid = unsigned((n + 255) / 256);
  if (seed_grid < 1) seed_grid = 1;
  seed_tokens<<<seed_grid, 256, 0, st>>>(P, n);
  ++h->launches;
  if (!h->ev_start) {
    if (cudaEventCreate(&h->ev_start) != cudaSuccess ||
        cudaEventCreate(&h->ev_stop) != cudaSuccess) {
      h->last_error = "epoch: cudaEventCreate failed";
      return NOMAD_ERR_CUDA;
    }
  }
  return NOMAD_OK;
}

}  // namespace

// Epochs per launch of a call: one (the epochs kept in step), or the
// schedule's epochs_per_launch; uniform mode runs a call in one launch.
int32_t epochs_per_launch(const nomad_handle* h, int32_t n_epochs) {
  if (h->sched.mode == NOMAD_MODE_UNIFORM) return n_epochs;
  const int32_t e = h->sched.epochs_per_launch > 1 ? h->sched.epochs_per_launch : 1;
  return e < n_epochs ? e : n_epochs;
}

int launch_epochs(nomad_handle* h, int32_t n_epochs, cudaStream_t st) {
  const int32_t per = epochs_per_launch(h, n_epochs);
  for (int32_t done = 0; done < n_epochs; done += per) {
    const int32_t ne = n_epochs - done < per ? n_epochs - done : per;
    SgdParams P{};
    const int rc = prepare_epochs(h, ne, st, &P, done, done == 0);
    if (rc != NOMAD_OK || h->nnz == 0) return rc;
    const bool debug = h->sched.debug != 0;
    size_t spw = 0;
    const void* fn = worker_kernel(h->k4, debug, h->sched.mode, h->sched.variant,
                                   h->sched.precision, P.col_grp_ptr != nullptr, &spw);
    // the hybrid circulation's inboxes follow the warps' areas
    const size_t smem = (spw + (P.col_grp_ptr ? batched_inbox_bytes() : 0)) *
                        size_t(h->warps_per_block);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess) {
      h->last_error = "epoch: shared memory per block exceeds the device limit";
      return NOMAD_ERR_UNSUPPORTED;
    }
    void* args[] = {&P};
    if (done == 0) cudaEventRecord(h->ev_start, st);
    cudaError_t e = cudaSuccess;
    if (P.ubits_pre) {
      e = draw_urgent_bits(h->useg_list, h->n_useg, h->seg_ptr, h->useg_off, h->k4, P.epoch0,
                           make_uint2(P.seed_lo, P.seed_hi), h->ubits_pre, st);
      ++h->launches;
    }
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(fn, dim3(h->blocks), dim3(h->warps_per_block * 32), args,
                                      smem, st);
    if (e != cudaSuccess) {
      h->last_error = std::string("epoch: cooperative launch: ") + cudaGetErrorString(e);
      return NOMAD_ERR_CUDA;
    }
    ++h->launches;
  }
  cudaEventRecord(h->ev_stop, st);
  h->ev_recorded = true;
  return NOMAD_OK;
}

// Several handles' epochs in one launch of the batched kernel's several-
// problem form: handle g's blocks run its workers with its own parameters
// (copied to the device for the launch).  The caller has checked that the
// handles agree in mode, variant, precision, debug flag, warps per block and
// row width class.
int launch_epochs_many(nomad_handle* const* hs, int count, int32_t n_epochs, cudaStream_t st) {
  nomad_handle* h0 = hs[0];
  const bool debug = h0->sched.debug != 0;
  const int wpb = h0->warps_per_block;
  size_t spw = 0;
  const void* fn = batched_kernel(h0->k4, debug, h0->sched.precision, true, false, &spw);
  if (!fn) return NOMAD_ERR_UNSUPPORTED;
  int use_inboxes = 0;  // a problem with the hybrid circulation: inboxes after the parameters
  for (int g = 0; g < count; ++g)
    if (hs[g]->sched.circulation == NOMAD_CIRCULATION_BLOCK) use_inboxes = 1;
  const size_t smem = spw * size_t(wpb) + batched_params_bytes() +
                      (use_inboxes ? batched_inbox_bytes() * size_t(wpb) : 0);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
          cudaSuccess) {
    h0->last_error = "epoch_many: shared memory per block exceeds the device limit";
    return NOMAD_ERR_UNSUPPORTED;
  }
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wpb * 32, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h0->device) != cudaSuccess) {
    h0->last_error = "epoch_many: occupancy query failed";
    return NOMAD_ERR_CUDA;
  }
  int64_t total = 0;
  for (int g = 0; g < count; ++g)
    if (hs[g]->nnz > 0) total += hs[g]->blocks;
  if (total > int64_t(per_sm) * sms) {
    h0->last_error = "epoch_many: " + std::to_string(total) + " blocks do not fit on the device at once (" +
                     std::to_string(int64_t(per_sm) * sms) + ")";
    return NOMAD_ERR_UNSUPPORTED;
  }
  // one launch per epoch (or the first handle's epochs_per_launch)
  const int32_t per = epochs_per_launch(h0, n_epochs);
  for (int32_t done = 0; done < n_epochs; done += per) {
    const int32_t ne = n_epochs - done < per ? n_epochs - done : per;
    std::vector<SgdParams> Ps;
    std::vector<int2> blocks;
    std::vector<int> pre;  // handles whose urgent rounding bits are drawn first
    Ps.reserve(size_t(count));
    for (int g = 0; g < count; ++g) {
      SgdParams P{};
      const int rc = prepare_epochs(hs[g], ne, st, &P, done, done == 0);
      if (rc != NOMAD_OK) {
        if (hs[g] != h0) h0->last_error = hs[g]->last_error;
        return rc;
      }
      if (hs[g]->nnz == 0) continue;
      if (P.ubits_pre) pre.push_back(g);
      for (int b = 0; b < hs[g]->blocks; ++b) blocks.push_back(make_int2(int(Ps.size()), b));
      Ps.push_back(P);
    }
    if (blocks.empty()) return NOMAD_OK;
    void* dP = nullptr;
    void* dB = nullptr;
    cudaError_t e = cudaMallocAsync(&dP, sizeof(SgdParams) * Ps.size(), st);
    if (!e) e = cudaMallocAsync(&dB, sizeof(int2) * blocks.size(), st);
    if (!e) e = cudaMemcpyAsync(dP, Ps.data(), sizeof(SgdParams) * Ps.size(), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dB, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice, st);
    if (!e) {
      if (done == 0)
        for (int g = 0; g < count; ++g) cudaEventRecord(hs[g]->ev_start, st);
      for (size_t i = 0; i < pre.size() && !e; ++i) {
        nomad_handle* hg = hs[pre[i]];
        e = draw_urgent_bits(hg->useg_list, hg->n_useg, hg->seg_ptr, hg->useg_off, hg->k4,
                             int32_t(hg->epochs_done) + done,
                             make_uint2(uint32_t(hg->sched.seed), uint32_t(hg->sched.seed >> 32)),
                             hg->ubits_pre, st);
        ++hg->launches;
      }
      const SgdParams* aP = static_cast<const SgdParams*>(dP);
      const int2* aB = static_cast<const int2*>(dB);
      void* args[] = {&aP, &aB, &use_inboxes};
      if (!e)
        e = cudaLaunchCooperativeKernel(fn, dim3(unsigned(blocks.size())), dim3(wpb * 32), args,
                                        smem, st);
      if (!e) ++h0->launches;
    }
    if (dP) cudaFreeAsync(dP, st);
    if (dB) cudaFreeAsync(dB, st);
    if (e != cudaSuccess) {
      h0->last_error = std::string("epoch_many: ") + cudaGetErrorString(e);
      return NOMAD_ERR_CUDA;
    }
  }
  for (int g = 0; g < count; ++g) {
    cudaEventRecord(hs[g]->ev_stop, st);
    hs[g]->ev_recorded = true;
  }
  return NOMAD_OK;
}

}  // namespace nomad
