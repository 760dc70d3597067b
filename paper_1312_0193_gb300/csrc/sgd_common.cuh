// sgd_common.cuh -- device helpers shared by the NOMAD worker kernels:
// the epoch-mode visit order, the ring-queue push and the bounded pop.
#pragma once

#include "nomad_internal.cuh"

namespace nomad {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDefaultWarpsPerBlock = 8;
constexpr int kMaxWarpsPerBlock = 16;
constexpr unsigned kMaxSleepNs = 512;  // longest back-off of a waiting worker

__device__ __forceinline__ float warp_sum(float v) {
  v += __shfl_xor_sync(kFull, v, 16);
  v += __shfl_xor_sync(kFull, v, 8);
  v += __shfl_xor_sync(kFull, v, 4);
  v += __shfl_xor_sync(kFull, v, 2);
  v += __shfl_xor_sync(kFull, v, 1);
  return v;
}

// Position `hop` of item j's visit order in one epoch: a bijection of
// [0, d) built from two rounds of (odd multiply + add) mod 2^b and xorshift,
// walked until it lands in [0, d).  The walk ends within 2^b < 2d steps.
__device__ __forceinline__ uint32_t itinerary_slot(uint32_t hop, uint32_t d,
                                                   uint4 key) {
  if (d <= 1) return 0;
  const int b = 32 - __clz(d - 1);
  const uint32_t mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
  const int sh = (b + 1) >> 1;
  uint32_t x = hop;
  for (uint32_t guard = 0; guard <= mask; ++guard) {
    x = (x * (key.x | 1u) + key.y) & mask;
    x ^= x >> sh;
    x = (x * (key.z | 1u) + key.w) & mask;
    x ^= x >> sh;
    if (x < d) return x;
  }
  return hop;  // not reached: the orbit of hop returns to [0, d)
}

// The batched kernel's record of a token's next visit, kTokRec int4 per item
// (three used):
// a = {segment, ratings, first record, epoch}, b = {hop, first of the
// item's segments in col_segs, number of its segments d, gs}, c = {first run
// of the item in grp_off, runs G, offset and size of the current run} (gs
// and c: hybrid circulation only; gs = run hop << 16 | hop within the run).
constexpr int kTokRec = kTokRecInts;

// The visit that follows the one at flat hop `hop` (of the d per epoch) in
// epoch e of item j: segment (-1 past the last epoch), hop, epoch and the
// hybrid circulation's state.
struct Route {
  int seg, hop, epoch, gs, ro, rz;
};
template <bool BLK>
__device__ __forceinline__ Route route_next(const SgdParams& P, int j, int e, int hop, int cb,
                                            int d, int gs, int gb, int G, int ro, int rz,
                                            int epoch_end, uint2 seed) {
  Route r{-1, hop + 1, e, 0, 0, 0};
  if (r.hop == d) {
    r.hop = 0;
    r.epoch = e + 1;
  }
  if (r.epoch >= epoch_end) return r;
  const uint4 key = philox4x32_10(make_uint4(uint32_t(j), uint32_t(r.epoch), 0u, kTagItinerary),
                                  seed);
  if constexpr (!BLK) {  // permutation over all of the item's workers
    r.seg = __ldg(P.col_segs + cb + itinerary_slot(uint32_t(r.hop), uint32_t(d), key));
    return r;
  }
  // hybrid (Sec. 3.4): the runs of one thread block in the keyed order
  // itinerary_slot(gh, G); within a run, its workers in a second keyed
  // permutation (the key's words reversed)
  int gh = 0, wh = 0, o = 0, z = 0;
  if (r.hop != 0 && (gs & 0xffff) + 1 < rz) {  // the next worker of the same run
    gh = gs >> 16;
    wh = (gs & 0xffff) + 1;
    o = ro;
    z = rz;
  } else {  // the first worker of the next run
    gh = r.hop == 0 ? 0 : (gs >> 16) + 1;
    const int g = int(itinerary_slot(uint32_t(gh), uint32_t(G), key));
    o = __ldg(P.grp_off + gb + g);
    z = __ldg(P.grp_off + gb + g + 1) - o;
  }
  const uint4 kin = make_uint4(key.w, key.z, key.y, key.x);
  r.seg = __ldg(P.col_segs + cb + o + int(itinerary_slot(uint32_t(wh), uint32_t(z), kin)));
  r.gs = (gh << 16) | wh;
  r.ro = o;
  r.rz = z;
  return r;
}

// Appends `payload` to worker q's ring.  The slot is written with a release
// store: every write this thread performed or observed before it (the other
// lanes' stores of h_j, ordered by a preceding __syncwarp) is visible to the
// worker whose acquire reads the slot.
__device__ __forceinline__ void push_token(const SgdParams& P, int q,
                                           uint32_t payload) {
  const uint32_t pos = atomicAdd(P.ring_tail + q, 1u);
  const int lg = P.ring_log2[q];
  unsigned long long* slot = P.ring + P.ring_base[q] + (pos & ((1u << lg) - 1u));
  st_release_u64(slot, (static_cast<unsigned long long>(pos >> lg) << 32) | payload);
}

// Appends `payload` to worker q's urgent ring (the tokens of the items with
// most ratings), with the same release store as push_token.
__device__ __forceinline__ void push_urgent(const SgdParams& P, int q, uint32_t payload) {
  const uint32_t pos = atomicAdd(P.uring_tail + q, 1u);
  const int lg = P.uring_log2;
  unsigned long long* slot = P.uring + (int64_t(q) << lg) + (pos & ((1u << lg) - 1u));
  st_release_u64(slot, (static_cast<unsigned long long>(pos >> lg) << 32) | payload);
}

// Lane 0 only.  Waits until worker q's ring has a token at `head` or, when
// `uring_q` is not null, its urgent ring one at `head_u`, or when `itag` is
// not null, the shared-memory inbox slot's tag shows `iwant`; 0 then, -1 when
// the wait gave up (as pop_token).  The caller reads the slots again.
__device__ int wait_rings(const SgdParams& P, int q, uint32_t head, int lg,
                          const unsigned long long* ring_q, uint32_t head_u,
                          const unsigned long long* uring_q, const volatile int* itag = nullptr,
                          int iwant = 0) {
  const unsigned long long* slot = ring_q + (head & ((1u << lg) - 1u));
  const uint32_t lap = head >> lg;
  const int lgu = P.uring_log2;
  const unsigned long long* uslot = uring_q ? uring_q + (head_u & ((1u << lgu) - 1u)) : nullptr;
  const uint32_t ulap = head_u >> lgu;
  const unsigned long long t0 = globaltimer_ns();
  const unsigned long long max_iters =
      static_cast<unsigned long long>(P.timeout_ns) / 16ull + (1ull << 20);
  unsigned ns = 32;
  for (unsigned long long it = 0; it < max_iters; ++it) {
    if (uint32_t(ld_relaxed_u64(slot) >> 32) == lap ||
        (uslot && uint32_t(ld_relaxed_u64(uslot) >> 32) == ulap) || (itag && *itag == iwant)) {
      fence_acq_rel_gpu();
      return 0;
    }
    if ((it & 15) == 15) {
      if (ld_relaxed_i32(P.status) != 0) return -1;
      if (globaltimer_ns() - t0 > static_cast<unsigned long long>(P.timeout_ns)) break;
    }
    __nanosleep(ns);
    if (ns < kMaxSleepNs) ns <<= 1;
  }
  if (atomicCAS(P.status, 0, NOMAD_ERR_TIMEOUT) == 0) {
    atomicExch(P.status + 1, q);
    atomicExch(P.status + 2, int(head));
  }
  return -1;
}

// Lane 0 only.  Returns the payload at position `head` of worker q's ring,
// or -1 when the wait gave up (another worker failed, the stop flag of
// uniform mode was raised, or this wait exceeded the timeout, in which case
// the status word records it).  The slot is polled with relaxed loads (an
// acquire load would also invalidate the SM's L1, which the working warps of
// the SM use) and a backoff of up to kMaxSleepNs; the acquire is one fence
// once the slot is seen ready.
__device__ int pop_token(const SgdParams& P, int q, uint32_t head, int lg,
                         const unsigned long long* ring_q) {
  const unsigned long long* slot = ring_q + (head & ((1u << lg) - 1u));
  const uint32_t lap = head >> lg;
  unsigned long long v = ld_relaxed_u64(slot);
  if (uint32_t(v >> 32) == lap) {
    fence_acq_rel_gpu();
    return int(uint32_t(v));
  }
  const unsigned long long t0 = globaltimer_ns();
  const unsigned long long max_iters =
      static_cast<unsigned long long>(P.timeout_ns) / 16ull + (1ull << 20);
  unsigned ns = 32;
  for (unsigned long long it = 0; it < max_iters; ++it) {
    v = ld_relaxed_u64(slot);
    if (uint32_t(v >> 32) == lap) {
      fence_acq_rel_gpu();
      return int(uint32_t(v));
    }
    if ((it & 15) == 15) {
      if (ld_relaxed_i32(P.status) != 0) return -1;
      if (P.stop != nullptr && ld_relaxed_i32(P.stop) != 0) return -1;
      if (globaltimer_ns() - t0 > static_cast<unsigned long long>(P.timeout_ns)) break;
    }
    __nanosleep(ns);
    if (ns < kMaxSleepNs) ns <<= 1;
  }
  if (atomicCAS(P.status, 0, NOMAD_ERR_TIMEOUT) == 0) {
    atomicExch(P.status + 1, q);
    atomicExch(P.status + 2, int(head));
  }
  return -1;
}

__device__ __forceinline__ void flag_ownership(const SgdParams& P, int q, int j) {
  atomicAdd(P.status + 3, 1);
  if (atomicCAS(P.status, 0, NOMAD_ERR_OWNERSHIP) == 0) {
    atomicExch(P.status + 1, q);
    atomicExch(P.status + 2, j);
  }
}


}  // namespace
}  // namespace nomad
