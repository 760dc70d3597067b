// epoch_batched.cuh -- the batched NOMAD worker kernel (epoch mode).
//
// Same worker semantics as the one-token kernel of sgd.cu (one warp = one
// worker q of Sec. 3.1, item tokens on lap-tagged rings, permutation
// circulation of Sec. 3.4), organised so that the latency of global memory is
// paid per batch of tokens instead of per visit:
//
//  1. take the ready tokens among the first kRingWindow positions of the own
//     ring (up to Batch<CPL>; a position reserved but not yet written does
//     not hold back the ones behind it), one acquire load per lane;
//  2. read every token's record of its next visit (written by the previous
//     holder before its push) lane-parallel, lane b = token b;
//  3. order the visits: long visits (>= kHeavy ratings) first, then the
//     rest in ring order;
//  4. copy every h_j of the batch into shared memory and the rating records
//     of the batch, as one stream of positions, into a shared circular
//     buffer (cp.async); compute each token's next hop meanwhile;
//  5. run the long visits in block form (long_visit), each token handed on
//     right after its visit;
//  6. walk the stream of short visits: W rows are copied into a ring of R
//     shared-memory slots R-1 positions ahead of the update (cp.async); the
//     update itself is the fused SGD step of Eq. w_update / h_update
//     (descent sign, old w_i in the h update);
//  7. hand on the remaining tokens together: one __syncwarp, then one
//     release store per token lane.
//
// The tokens of the items with most ratings travel through a second, urgent
// ring per worker and are visited out of turn between visits (urgent_visit);
// visits are never split, so the serial order stays a valid NOMAD order.
//
// A row can appear in two visits of one batch (a user who rated both items).
// Its copy for the later position must not be taken before the earlier
// position has updated it: when the row being prefetched is the row of a
// position still in flight, no copy is made, and the latest such position
// writes its updated row into the later position's slot as well.
//
// Storage formats (template parameter PR): binary32 W and H; bfloat16 W and
// H; FP8-E4M3 W with one binary32 scale per row and binary32 H.  Arithmetic
// is binary32 in every format.  The narrow formats round W stochastically at
// every update (and bfloat16 H once per visit) with 16 random bits per entry
// from Philox4x32-10: W of record r in epoch e at counter
// (r lo, r hi, e, 0x57000000 | chunk/2); H at
// (segment, e, 0, 0x48000000 | chunk), words z,w; entry 4c+i takes half i%2
// of word i/2 (word 2 + i/2 for H); one W draw serves two chunks (words x,y
// for chunk 2q, z,w for chunk 2q+1 at counter word 0x57000000 | q).  The
// draws do not depend on the updates, so they are made ahead of them in
// bulk (32 positions of the stream, or a block of a long visit, spread over
// the lanes as independent draws) and kept in shared memory.
//
// The worker body is shared by the one-problem kernel and a form that runs
// several independent problems in one launch (nomad_batched_many_kernel).
#pragma once

#include "sgd_common.cuh"

namespace nomad {
namespace {

// Tokens taken from the ring at once: 16 when a row is one chunk per lane,
// 8 otherwise (shared memory holds their h).
template <int CPL>
constexpr int Batch = CPL == 1 ? 16 : 8;
constexpr int kRecBuf = 128;   // circular buffer of record positions
constexpr int kRecInit = 64;   // positions loaded before the first row copy
constexpr int kHeavy = 32;     // visits this long go first and are pushed at once

constexpr int kStreamChunks = 16;  // row-ring chunks per lane of the generic stream
constexpr int kBatchedWarps = 8;   // warps per thread block at most (register budget)

constexpr int kVisitChunks = 21;   // ring chunks of a long visit at one chunk per lane
constexpr int kUrgentChunks = 14;  // ring chunks of a visit taken out of turn

constexpr int kF32 = 0, kBF16 = 1, kFP8 = 2;  // storage formats

// Hybrid circulation (Sec. 3.4): a token whose next worker is a warp of the
// same thread block is handed over through that warp's inbox in shared
// memory: kInboxSlots slots, filled by the warps of the block (a slot is
// reserved with a compare-and-swap on the tail, then written, then tagged
// with its position + 1 after a block-scope fence) and emptied in order by
// the owner (which publishes its head after a fence).  A full inbox sends
// the token through the global ring instead.  Slot positions 16..30 of the
// intake window are read by lanes 16..30.
constexpr int kInboxSlots = 16;

// Row ring per lane: CHUNKS chunks.  The generic stream uses the first
// kStreamChunks and a long visit of the batch the first VISIT (each runs
// alone); at one chunk per lane a visit of an urgent item that interrupts
// either of them uses the kUrgentChunks after those.  A row slot is CPL
// chunks per lane; FP8 rows also keep their scale, one float per slot.
template <int CPL>
struct RowRing {
  static constexpr int VISIT = CPL == 1 ? kVisitChunks : kStreamChunks;
  static constexpr int CHUNKS = CPL == 1 ? kVisitChunks + kUrgentChunks : kStreamChunks;
  static constexpr int R = kStreamChunks / CPL;  // slots; R-1 rows in flight
  static_assert(kStreamChunks <= VISIT, "the stream's slots lie in the batch's region");
};

// A chunk is 4 consecutive entries of a row: float4 (binary32), uint2
// (bfloat16) or uint32_t (four E4M3 codes, entry 4c+i in byte i).
template <int PR>
struct Fmt;
template <>
struct Fmt<kF32> {
  using w_t = float4;
  using h_t = float4;
};
template <>
struct Fmt<kBF16> {
  using w_t = uint2;
  using h_t = uint2;
};
template <>
struct Fmt<kFP8> {
  using w_t = uint32_t;
  using h_t = float4;
};

__device__ __forceinline__ float4 bf16_widen(uint2 c) {
  return make_float4(__uint_as_float(c.x << 16), __uint_as_float(c.x & 0xffff0000u),
                     __uint_as_float(c.y << 16), __uint_as_float(c.y & 0xffff0000u));
}
__device__ __forceinline__ float4 widen_h(float4 c) { return c; }
__device__ __forceinline__ float4 widen_h(uint2 c) { return bf16_widen(c); }
// a W chunk as binary32 (s: the row's scale, FP8 only)
__device__ __forceinline__ float4 widen_w(float4 c, float) { return c; }
__device__ __forceinline__ float4 widen_w(uint2 c, float) { return bf16_widen(c); }
__device__ __forceinline__ float4 widen_w(uint32_t c, float s) { return e4m3_unpack(c, s); }

// binary32 -> bfloat16 with 16 random bits added to the dropped bits of the
// magnitude (stochastic rounding); infinities and NaN are truncated.
__device__ __forceinline__ uint32_t bf16_sr(float x, uint32_t r16) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return (u >> 16) | ((u & 0x007fffffu) ? 0x40u : 0u);
  return (u + (r16 & 0xffffu)) >> 16;
}
__device__ __forceinline__ uint2 pack_sr(float4 v, uint32_t ra, uint32_t rb) {
  return make_uint2(bf16_sr(v.x, ra) | (bf16_sr(v.y, ra >> 16) << 16),
                    bf16_sr(v.z, rb) | (bf16_sr(v.w, rb >> 16) << 16));
}

// The rounding bits of chunks 2q and 2q+1 of the W row written by the update
// of record `rix` in epoch `e`: words x,y and z,w of one draw.
__device__ __forceinline__ uint4 w_bits_pair(int64_t rix, int e, int q, uint2 seed) {
  return philox4x32_10(make_uint4(uint32_t(rix), uint32_t(uint64_t(rix) >> 32), uint32_t(e),
                                  0x57000000u | uint32_t(q)),
                       seed);
}

// The draws of `nu` updates, one per (update u, pair of chunks q), spread
// over the lanes; the bits of chunk c of update u go to buf[u * CPL * 32 + c].
// rix(u) and e(u) name the record and epoch of update u: lane u holds them
// (u < nu <= 32).  w / npairs is taken as umulhi(w, m) with
// m = floor((2^32 - 1) / npairs) + 1, exact for w < 2^16 and npairs <= 64.
template <int CPL>
__device__ __forceinline__ void draw_w_bits(uint2* buf, int nu, int64_t rix, int e, int k4,
                                            uint2 seed, int lane) {
  const int npairs = (k4 + 1) >> 1;
  const uint32_t m = 0xffffffffu / uint32_t(npairs) + 1u;
  const int items = nu * npairs;
  for (int base = 0; base < items; base += 32) {
    const int w = base + lane;
    const int u = int(__umulhi(uint32_t(w), m));
    const int q = w - u * npairs;
    const int us = w < items ? u : 0;
    const int64_t rx = __shfl_sync(kFull, rix, us);
    const int ex = __shfl_sync(kFull, e, us);
    if (w < items) {
      const uint4 d = w_bits_pair(rx, ex, q, seed);
      uint2* dst = buf + u * CPL * 32 + 2 * q;
      dst[0] = make_uint2(d.x, d.y);
      if (2 * q + 1 < k4) dst[1] = make_uint2(d.z, d.w);
    }
  }
}

// h of a visit written back to H (bfloat16: rounded with the bits of
// segment `seg` in epoch `e`).
__device__ __forceinline__ void store_h(float4* dst, float4 h, int, int, int, uint2) {
  __stcg(dst, h);
}
__device__ __forceinline__ void store_h(uint2* dst, float4 h, int seg, int e, int idx, uint2 seed) {
  const uint4 r = philox4x32_10(
      make_uint4(uint32_t(seg), uint32_t(e), 0u, 0x48000000u | uint32_t(idx)), seed);
  __stcg(dst, pack_sr(h, r.z, r.w));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// The stored form of an updated W row (warp-collective: every lane calls,
// lanes past the row hold zeros).  wn: this lane's chunks; rb: their
// rounding bits.  FP8: the new scale (the row's largest magnitude / 448) is
// returned in *scale.
template <int PR, int CPL>
__device__ __forceinline__ void narrow_w(const float4 (&wn)[CPL], const uint2 (&rb)[CPL],
                                         typename Fmt<PR>::w_t (&out)[CPL], float* scale) {
#pragma unroll
  for (int cc = 0; cc < CPL; ++cc) {
    if constexpr (PR == kF32) out[cc] = wn[cc];
    if constexpr (PR == kBF16) out[cc] = pack_sr(wn[cc], rb[cc].x, rb[cc].y);
  }
  if constexpr (PR == kFP8) {
    float a = 0.f;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) a = abs_max4(wn[cc], a);
    a = warp_max(a);
    float s, g;
    e4m3_row_scale(a, &s, &g);
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) out[cc] = e4m3_pack(wn[cc], g, true, rb[cc].x, rb[cc].y);
    *scale = s;
  }
}

// Packed binary32 pairs (Blackwell's two-wide FMA): a chunk of 4 entries is
// handled as two float2 halves.
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// acc + a.b over the 4 entries, kept as two partial sums
__device__ __forceinline__ float2 dot4_acc(float4 a, float4 b, float2 acc) {
  acc = __ffma2_rn(lo2(a), lo2(b), acc);
  return __ffma2_rn(hi2(a), hi2(b), acc);
}
// per entry: fma(b, y, a * x)
__device__ __forceinline__ float4 axpby(float2 a2, float4 x, float2 b2, float4 y) {
  return cat4(__ffma2_rn(b2, lo2(y), __fmul2_rn(a2, lo2(x))),
              __ffma2_rn(b2, hi2(y), __fmul2_rn(a2, hi2(x))));
}

// Shared memory of one warp.  Offsets in bytes, each a multiple of 16: row
// slots, their scales (FP8), h of the batch, the rounding bits of the stream
// and of the batch's long visits (narrow formats: SRB positions of CPL*32
// chunks), those of an urgent visit, records (int2) and two int4 tables of
// batch metadata.  The inboxes of the hybrid circulation lie after the
// warps' areas (and the parameters of the several-problem form), one per
// warp, in shared memory the launch adds only for that circulation.
template <int CPL, int PR>
struct WarpSmem {
  using F = Fmt<PR>;
  static constexpr int SRB = 32 / CPL;  // stream positions per bulk draw
  static constexpr int kRows = 0;
  static constexpr int kScales = kRows + RowRing<CPL>::CHUNKS * 32 * int(sizeof(typename F::w_t));
  static constexpr int kH = kScales + (PR == kFP8 ? (RowRing<CPL>::CHUNKS * 4 + 15) / 16 * 16 : 0);
  static constexpr int kSr = kH + Batch<CPL> * CPL * 32 * int(sizeof(typename F::h_t));
  static constexpr int kUbits = kSr + (PR == kF32 ? 0 : SRB * CPL * 32 * 8);
  // an urgent visit's block of rounding bits (one chunk per lane, 7 rows)
  static constexpr int kRecs = kUbits + (PR == kF32 || CPL != 1 ? 0 : 7 * 32 * 8);
  static constexpr int kMeta = kRecs + kRecBuf * 8;
  static constexpr int bytes = kMeta + 2 * Batch<CPL> * 16;
};
template <int CPL, int PR>
__host__ __device__ constexpr int warp_smem_bytes() {
  return WarpSmem<CPL, PR>::bytes;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_chunk(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 16) cp_async16(smem, gmem);
  else if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}
// cp_chunk under a predicate, without a branch (so that it can be scheduled
// among independent instructions); nothing is read when `pred` is false
template <typename T>
__device__ __forceinline__ void cp_chunk_if(bool pred, T* smem, const T* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(T) == 16)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
                 "@p cp.async.cg.shared.global [%0], [%1], 16;\n\t}\n" ::"r"(sa), "l"(gmem),
                 "r"(int(pred)) : "memory");
  else if constexpr (sizeof(T) == 8)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
                 "@p cp.async.ca.shared.global [%0], [%1], 8;\n\t}\n" ::"r"(sa), "l"(gmem),
                 "r"(int(pred)) : "memory");
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
                 "@p cp.async.ca.shared.global [%0], [%1], 4;\n\t}\n" ::"r"(sa), "l"(gmem),
                 "r"(int(pred)) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The visit rank of stream position p (p0 <= p < p0 + 32): the last rank
// r < nb whose offset is <= p.  Lane r < nb holds the stream offset `soff`
// of the rank-r visit (offsets increase strictly with the rank): the visits
// that start before p0 are counted with one ballot, those that start in
// [p0, p] with one OR-reduction of their start bits.
template <int KB>
__device__ __forceinline__ int rank_of(int soff, int nb, int p0, int p, int lane) {
  const int d = soff - p0;
  const bool in = lane < nb && d >= 0 && d < 32;
  const unsigned starts = __reduce_or_sync(kFull, in ? 1u << d : 0u);
  const int before = __popc(__ballot_sync(kFull, lane < nb && soff < p0));
  const int q = p - p0;
  const unsigned upto = q >= 31 ? 0xffffffffu : (2u << q) - 1u;
  return before + __popc(starts & upto) - 1;
}

// Copies the records of stream positions [p0, p0 + count) (count <= 32) into
// the circular buffer.  Lane r < nb holds the stream offset `soff` and first
// record `beg` of the rank-r visit.
template <int KB>
__device__ __forceinline__ void load_records(int2* recs, const int2* __restrict__ rec, int soff,
                                             int64_t beg, int nb, int p0, int count, int lane) {
  const int p = p0 + lane;
  const int r = rank_of<KB>(soff, nb, p0, p, lane);
  const int o = __shfl_sync(kFull, soff, r);
  const int64_t b = __shfl_sync(kFull, beg, r);
  if (lane < count) cp_async8(recs + (p % kRecBuf), rec + b + (p - o));
}

// The rounding bits of stream positions [p0, min(p0 + SRB, T)), all chunks,
// into srb[(p - p0) * CPL * 32 + chunk].  Lane r < nb holds the offset,
// first record and epoch of the rank-r visit.
template <int KB, int CPL>
__device__ __forceinline__ void draw_stream_bits(uint2* srb, int soff, int64_t beg, int ep, int nb,
                                                 int p0, int T, int k4, uint2 seed, int lane) {
  constexpr int SRB = 32 / CPL;
  const int p = p0 + (lane < SRB ? lane : 0);  // lane u < SRB: position p0 + u
  const int r = rank_of<KB>(soff, nb, p0, p, lane);
  const int o = __shfl_sync(kFull, soff, r);
  const int64_t b = __shfl_sync(kFull, beg, r);
  const int e = __shfl_sync(kFull, ep, r);
  const int nu = T - p0 < SRB ? T - p0 : SRB;
  draw_w_bits<CPL>(srb, nu, b + (p - o), e, k4, seed, lane);
}

// Transposed warp reduction: v[0..31] are this lane's partial sums of 32
// quantities; on return lane l holds the warp-wide sum of quantity l.  Each
// level halves the values a lane keeps and exchanges the other half with the
// partner lane, so the 32 sums take 31 shuffles that are mostly independent.
__device__ __forceinline__ float warp_sum_transposed(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// The updates of one long visit (>= kHeavy ratings) of token j, the serial
// chain through h_j that bounds an epoch for the items with most ratings.
//
// The visit applies the per-rating step of Eq. w_update / h_update to its
// ratings u = 0, 1, ... in order.  The rows of one visit are distinct users,
// so within a block of B consecutive ratings every w_u is read before it is
// written and only h changes from one update to the next.  With
// a = 1 - s*lambda the recurrence h_{u+1} = a h_u + s e_u w_u unrolls to
//
//   e_u = A_u - a^u <w_u, h_0> - s * sum_{v<u} a^(u-1-v) <w_u, w_v> e_v,
//
// so the block needs the B dot products <w_u, h_0> and the B(B-1)/2 dot
// products <w_u, w_v> (one transposed reduction), a B-step scalar forward
// substitution for e_0..e_{B-1}, and then the vector updates
// w_u' = a w_u + s e_u h_u, h_{u+1} = a h_u + s e_u w_u.  In exact arithmetic
// this is the sequential update; the dependent chain per rating shrinks from
// a full warp reduction to one shuffle and one multiply-add.
//
// W rows come through NCH chunk slots per lane of the warp's shared-memory
// ring (`rows`, with the scale of each row slot in `rsc` for FP8), LB blocks
// ahead with cp.async; each lane copies and reads only its own chunk of a
// row.  Records are held in lane registers, three 32-record chunks (lane i
// holds record i of a chunk).  Earlier stores of this warp precede these
// loads in program order.
//
// Narrow formats: the rounding bits of a block are drawn into `rbuf` while
// the block's products are reduced, or, with PRE, read from `pre` (drawn
// before the launch, record u of the visit at pre + u * k4): copied with the
// block's rows into `pbuf` (LB + 1 blocks of B records, each lane its own
// chunks), which takes the draws off the chain of the visit.
template <int CPL>
__host__ __device__ constexpr int long_visit_b() {
  return CPL == 4 ? 4 : 7;
}
// blocks of rows in flight; positions up to B*(b + LB) + B - 1 must lie in
// record chunks c0 and c0 + 1
template <int CPL, int NCH>
__host__ __device__ constexpr int long_visit_lb() {
  constexpr int B = long_visit_b<CPL>();
  return (NCH / CPL) / B < 33 / B - 1 ? (NCH / CPL) / B : 33 / B - 1;
}

template <int CPL, int PR, bool DEBUG, int NCH, bool PRE = false>
__device__ __forceinline__ void long_visit(float4 (&h)[CPL], typename Fmt<PR>::w_t* rows, float* rsc,
                                           uint2* rbuf, typename Fmt<PR>::w_t* W4, float* Wscale,
                                           int64_t pitch4, int k4, const int2* __restrict__ rec,
                                           int64_t beg, int c, float s, float lam, int epoch,
                                           uint2 seed, int lane, int32_t* rec_count,
                                           const uint2* pre, uint2* pbuf) {
  constexpr int B = long_visit_b<CPL>();
  constexpr int NS = B + B * (B - 1) / 2;
  static_assert(NS <= 32, "one transposed reduction per block");
  constexpr int LB = long_visit_lb<CPL, NCH>();
  static_assert(LB >= 1 && B * (LB + 1) - 1 <= 32, "row ring holds the blocks in flight");
  using w_t = typename Fmt<PR>::w_t;
  const float al = 1.f - s * lam;
  // lane u < B: a^u, and s a^(u-1-v) for v < u
  float aD = 1.f;
#pragma unroll
  for (int i = 0; i < B - 1; ++i)
    if (i < lane) aD *= al;
  float cg[B - 1];
#pragma unroll
  for (int v = 0; v < B - 1; ++v) {
    float x = s;
#pragma unroll
    for (int i = 0; i < B - 2; ++i)
      if (i < lane - 1 - v) x *= al;
    cg[v] = x;
  }
  const int2 z2 = make_int2(0, 0);
  int2 r0 = lane < c ? __ldcs(rec + beg + lane) : z2;
  int2 r1 = lane + 32 < c ? __ldcs(rec + beg + 32 + lane) : z2;
  int2 r2 = lane + 64 < c ? __ldcs(rec + beg + 64 + lane) : z2;
  int c0 = 0;  // record chunk held in r0; r1, r2 hold the next two
  // row of position u (warp-uniform, in chunk c0 or c0 + 1)
  auto row_at = [&](int u) {
    const int src = (u >> 5) == c0 ? r0.x : r1.x;
    return __shfl_sync(kFull, src, u & 31);
  };
  auto fetch = [&](int bb) {  // the rows of block bb, one commit group
    const int set = int(unsigned(bb) % unsigned(LB));
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int u = bb * B + i;
      const int row = row_at(u);
      if (u < c) {
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          const int idx = lane + 32 * cc;
          if (idx < k4)
            cp_chunk(rows + ((set * B + i) * CPL + cc) * 32 + lane, W4 + int64_t(row) * pitch4 + idx);
        }
        if constexpr (PR == kFP8)
          if (lane == 0) cp_async4(rsc + set * B + i, Wscale + row);
        if constexpr (PR != kF32) {
          if constexpr (PRE) {
            const int pset = int(unsigned(bb) % unsigned(LB + 1));
#pragma unroll
            for (int cc = 0; cc < CPL; ++cc) {
              const int idx = lane + 32 * cc;
              if (idx < k4)
                cp_async8(pbuf + ((pset * B + i) * CPL + cc) * 32 + lane, pre + int64_t(u) * k4 + idx);
            }
          }
        }
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int l = 0; l < LB; ++l) fetch(l);

  const float2 al2 = make_float2(al, al);
  const int nblk = (c + B - 1) / B;
  for (int b = 0; b < nblk; ++b) {
    if (((b * B) >> 5) != c0) {  // next record chunk
      r0 = r1;
      r1 = r2;
      ++c0;
      const int p2 = (c0 + 2) * 32 + lane;
      r2 = p2 < c ? __ldcs(rec + beg + p2) : z2;
    }
    cp_wait<LB - 1>();
    if constexpr (PR == kFP8) __syncwarp();  // lane 0's copies of the scales have landed
    const int set = int(unsigned(b) % unsigned(LB));
    float4 w[B][CPL];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const float sc = PR == kFP8 ? rsc[set * B + i] : 1.f;
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc)
        w[i][cc] = lane + 32 * cc < k4 && b * B + i < c
                       ? widen_w(rows[((set * B + i) * CPL + cc) * 32 + lane], sc)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (PR == kFP8) __syncwarp();  // every lane has read the scales before they are refilled
    // lane partials: slots 0..B-1 <w_u, h_0>, then <w_u, w_v> for v < u
    // (two-wide FMAs, the halves summed at the end)
    float v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = 0.f;
#pragma unroll
    for (int u = 0; u < B; ++u) {
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) a = dot4_acc(w[u][cc], h[cc], a);
      v[u] = a.x + a.y;
    }
#pragma unroll
    for (int u = 1; u < B; ++u)
#pragma unroll
      for (int q = 0; q < u; ++q) {
        const int t = B + u * (u - 1) / 2 + q;
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) a = dot4_acc(w[u][cc], w[q][cc], a);
        v[t] = a.x + a.y;
      }
    // the slots just read take the rows of block b + LB (the partials above
    // consumed every value read from them)
    fetch(b + LB);
    // the block's rounding bits (narrow formats): independent of the
    // updates, drawn here so that the draws overlap the reduction below
    if constexpr (PR != kF32) {
      if constexpr (!PRE) {
        __syncwarp();  // every lane has read the previous block's bits
        draw_w_bits<CPL>(rbuf, B, beg + b * B + (lane < B ? lane : 0), epoch, k4, seed, lane);
      }
    }
    // the block's rounding bits
    const uint2* bits = PRE ? pbuf + int(unsigned(b) % unsigned(LB + 1)) * B * CPL * 32 : rbuf;
    const float red = warp_sum_transposed(v, lane);
    // lane u < B: A_u - a^u <w_u, h_0>, then the forward substitution
    float acc;
    {
      const int u = b * B + (lane < B ? lane : 0);
      const int y0 = __shfl_sync(kFull, r0.y, u & 31);
      const int y1 = __shfl_sync(kFull, r1.y, u & 31);
      acc = __int_as_float((u >> 5) == c0 ? y0 : y1) - aD * red;
    }
    float gs[B - 1];
#pragma unroll
    for (int q = 0; q < B - 1; ++q) {
      const int src = lane > q && lane < B ? B + lane * (lane - 1) / 2 + q : 0;
      gs[q] = cg[q] * __shfl_sync(kFull, red, src);
    }
    float e[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      e[q] = __shfl_sync(kFull, acc, q);
      if (q < B - 1 && lane > q) acc = fmaf(-gs[q], e[q], acc);
    }
    if constexpr (PR != kF32) __syncwarp();  // the bits drawn above are visible
    // vector updates in rating order
    const int nu = c - b * B < B ? c - b * B : B;
    if constexpr (PR == kFP8) {
      // E4M3: the block's updated rows first (the chain through h), then
      // their scales from one interleaved max-reduction of the B rows, so
      // that the B reductions and divisions overlap instead of each
      // waiting for the one before
      float4 wn[B][CPL];
      float am[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const float se = s * e[i];
        const float2 se2 = make_float2(se, se);
        am[i] = 0.f;
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          if (i < nu) {
            wn[i][cc] = axpby(al2, w[i][cc], se2, h[cc]);  // a w_u + s e_u h_u
            h[cc] = axpby(se2, w[i][cc], al2, h[cc]);      // a h_u + s e_u w_u
          } else {
            wn[i][cc] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          am[i] = abs_max4(wn[i][cc], am[i]);
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int i = 0; i < B; ++i) am[i] = fmaxf(am[i], __shfl_xor_sync(kFull, am[i], o));
#pragma unroll
      for (int i = 0; i < B; ++i) {
        if (i >= nu) break;
        const int u = b * B + i;
        const int row = row_at(u);
        w_t* wrow = W4 + int64_t(row) * pitch4;
        float sc, g;
        e4m3_row_scale(am[i], &sc, &g);
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          const uint2 rb = bits[i * CPL * 32 + lane + 32 * cc];
          if (lane + 32 * cc < k4) wrow[lane + 32 * cc] = e4m3_pack(wn[i][cc], g, true, rb.x, rb.y);
        }
        if (lane == 0) Wscale[row] = sc;
        if (DEBUG && lane == 0) rec_count[beg + u] += 1;
      }
    } else {
#pragma unroll
      for (int i = 0; i < B; ++i) {
        if (i >= nu) break;
        const int u = b * B + i;
        const float se = s * e[i];
        const float2 se2 = make_float2(se, se);
        const int row = row_at(u);
        w_t* wrow = W4 + int64_t(row) * pitch4;
        float4 wn[CPL];
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          wn[cc] = axpby(al2, w[i][cc], se2, h[cc]);  // a w_u + s e_u h_u
          h[cc] = axpby(se2, w[i][cc], al2, h[cc]);   // a h_u + s e_u w_u
        }
        uint2 rb[CPL];
        if constexpr (PR != kF32) {
#pragma unroll
          for (int cc = 0; cc < CPL; ++cc) rb[cc] = bits[i * CPL * 32 + lane + 32 * cc];
        }
        w_t out[CPL];
        float scale = 1.f;
        narrow_w<PR, CPL>(wn, rb, out, &scale);
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc)
          if (lane + 32 * cc < k4) wrow[lane + 32 * cc] = out[cc];
        if (DEBUG && lane == 0) rec_count[beg + u] += 1;
      }
    }
  }
  cp_wait<0>();
  if constexpr (PR == kFP8) __syncwarp();
}

// An inbox: kInboxSlots slots of 4 int4 (the three record words and
// {item, tag}), then {head, tail}.
constexpr int kInboxBytes = kInboxSlots * 64 + 16;
__device__ __forceinline__ int4* inbox_slots(unsigned char* ib) {
  return reinterpret_cast<int4*>(ib);
}
__device__ __forceinline__ int* inbox_ctl(unsigned char* ib) {
  return reinterpret_cast<int*>(ib + kInboxSlots * 64);
}

// Hands the token of item j over through the inbox `ib` (one lane; the
// caller's H stores are ordered before this call by a __syncwarp).  False
// when the inbox is full: the caller uses the global ring.
__device__ __forceinline__ bool inbox_push(unsigned char* ib, int j, int4 a, int4 b, int4 c) {
  int4* slots = inbox_slots(ib);
  int* ctl = inbox_ctl(ib);
  volatile int* vctl = ctl;
  int t = vctl[1];
  for (int tries = 0; tries < 64; ++tries) {
    if (t - vctl[0] >= kInboxSlots) return false;
    const int old = atomicCAS(ctl + 1, t, t + 1);
    if (old == t) {
      int4* sl = slots + 4 * (t % kInboxSlots);
      sl[0] = a;
      sl[1] = b;
      sl[2] = c;
      sl[3].x = j;
      __threadfence_block();  // the record (and the warp's H stores) before the tag
      reinterpret_cast<volatile int*>(sl + 3)[1] = t + 1;
      return true;
    }
    t = old;
  }
  return false;
}

// A visit of an urgent item's token taken out of turn by worker q (one
// chunk of a row per lane): segment `useg`, just popped from q's ring.  The
// steps of a long visit of a batch: metadata, h_j into registers, the
// updates (in the ring slots `rows` / `rsc`, disjoint from those of the
// interrupted work), h_j back to H, the token handed on at once.  Visits are
// never split: the check runs between visits.  Not inlined: it is reached
// from two places and runs a few hundred times per worker and epoch.
// An urgent visit with pre-drawn bits keeps LB + 1 blocks of them in the
// stream's rounding-bits area (the stream draws its bits again afterwards).
static_assert((long_visit_lb<1, kUrgentChunks>() + 1) * long_visit_b<1>() <= 32,
              "the stream's bits area holds an urgent visit's blocks of bits");
template <int PR, bool DEBUG, bool BLK, bool PRE>
__device__ __noinline__ void urgent_visit(const SgdParams& P, int q, int lane, uint32_t item,
                                          typename Fmt<PR>::w_t* rows, float* rsc, uint2* rbuf,
                                          uint2* pbuf) {
  using w_t = typename Fmt<PR>::w_t;
  using h_t = typename Fmt<PR>::h_t;
  w_t* __restrict__ W4 = reinterpret_cast<w_t*>(P.W);
  h_t* __restrict__ H4 = reinterpret_cast<h_t*>(P.H);
  const int64_t pitch4 = P.pitch >> 2;
  const int k4 = P.k4;
  const uint2 seed = make_uint2(P.seed_lo, P.seed_hi);
  const int uj = int(item);
  const int4 ra = __ldcg(P.tok_rec + kTokRec * uj);
  const int4 rb4 = __ldcg(P.tok_rec + kTokRec * uj + 1);
  const int4 rc4 = BLK ? __ldcg(P.tok_rec + kTokRec * uj + 2) : make_int4(0, 0, 0, 0);
  const uint32_t useg = uint32_t(ra.x);
  const int uc = ra.y;
  const int64_t ubeg = int64_t(uint32_t(ra.z));
  const int ue = ra.w;
  float4 uh[1];
  uh[0] = lane < k4 ? widen_h(__ldcg(H4 + int64_t(uj) * pitch4 + lane))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
  const float us = __ldg(P.step + (ue - P.epoch0));
  const Route nx = route_next<BLK>(P, uj, ue, rb4.x, rb4.y, rb4.z, rb4.w, rc4.x, rc4.y, rc4.z,
                                   rc4.w, P.epoch0 + P.n_epochs, seed);
  const int unseg = nx.seg;
  int uq2 = -1, unc = 0;
  int64_t unbeg = 0;
  if (unseg >= 0) {
    uq2 = __ldg(P.seg_worker + unseg);
    unbeg = __ldg(P.seg_ptr + unseg);
    unc = int(__ldg(P.seg_ptr + unseg + 1) - unbeg);
  }
  if (DEBUG && lane == 0) {
    const uint32_t tk = atomicAdd(P.log_ticket, 1u);
    if (int64_t(tk) < P.log_cap) {
      P.log_seg[tk] = int(useg);
      P.log_epoch[tk] = ue;
    }
    if (atomicExch(P.owner + uj, q) != -1) flag_ownership(P, q, uj);
  }
  // PRE: the rounding bits were drawn before the launch (narrow formats)
  const uint2* pre = PRE ? P.ubits_pre + P.useg_off[useg] * k4 : nullptr;
  long_visit<1, PR, DEBUG, kUrgentChunks, PRE>(uh, rows, rsc, rbuf, W4, P.Wscale, pitch4, k4,
                                               P.rec, ubeg, uc, us, P.lambda, ue, seed, lane,
                                               P.rec_count, pre, pbuf);
  if (lane < k4) store_h(H4 + int64_t(uj) * pitch4 + lane, uh[0], int(useg), ue, lane, seed);
  if (lane == 0) {
    if (unseg >= 0) {
      __stcg(P.tok_rec + kTokRec * uj, make_int4(unseg, unc, int(uint32_t(unbeg)), nx.epoch));
      __stcg(P.tok_rec + kTokRec * uj + 1, make_int4(nx.hop, rb4.y, rb4.z, nx.gs));
      if (BLK) __stcg(P.tok_rec + kTokRec * uj + 2, make_int4(rc4.x, rc4.y, nx.ro, nx.rz));
    }
    if (DEBUG && atomicExch(P.owner + uj, -1) != q) flag_ownership(P, q, uj);
  }
  __syncwarp();  // orders every lane's H stores before the release below
  if (lane == 0 && unseg >= 0) push_urgent(P, uq2, uint32_t(uj));
}

// Worker q of the problem P (one warp), with its shared memory at `wsmem`
// (warp_smem_bytes<CPL, PR>() bytes).
template <int CPL, int PR, bool DEBUG, bool BLK>
__device__ __forceinline__ void batched_worker(const SgdParams& P, int q, unsigned char* wsmem,
                                               unsigned char* inboxes, int wib) {
  constexpr int R = RowRing<CPL>::R;
  using SM = WarpSmem<CPL, PR>;
  using w_t = typename Fmt<PR>::w_t;
  using h_t = typename Fmt<PR>::h_t;
  constexpr int SRB = SM::SRB;
  const int lane = threadIdx.x & 31;
  w_t* rows = reinterpret_cast<w_t*>(wsmem + SM::kRows);
  float* rsc = reinterpret_cast<float*>(wsmem + SM::kScales);  // FP8: scale of each row slot
  h_t* hbuf = reinterpret_cast<h_t*>(wsmem + SM::kH);
  uint2* srb = reinterpret_cast<uint2*>(wsmem + SM::kSr);      // narrow formats: stream draws
  uint2* ubits = reinterpret_cast<uint2*>(wsmem + SM::kUbits);  // and an urgent visit's
  constexpr int kBatch = Batch<CPL>;
  int2* recs = reinterpret_cast<int2*>(wsmem + SM::kRecs);
  int4* meta_a = reinterpret_cast<int4*>(wsmem + SM::kMeta);  // {j, c, e, seg}
  int4* meta_b = meta_a + kBatch;                             // {beg_lo, beg_hi, lane, soff}

  const int64_t quota = int64_t(P.worker_seg_ptr[q + 1] - P.worker_seg_ptr[q]) * P.n_epochs;
  if (lane == 0) atomicMin(P.span, globaltimer_ns());  // the launch's time span on the device
  const int lg = P.ring_log2[q];
  const uint32_t qmask = (1u << lg) - 1u;
  const unsigned long long* ring_q = P.ring + P.ring_base[q];
  w_t* __restrict__ W4 = reinterpret_cast<w_t*>(P.W);
  h_t* __restrict__ H4 = reinterpret_cast<h_t*>(P.H);
  float* __restrict__ Wscale = P.Wscale;
  const int64_t pitch4 = P.pitch >> 2;
  const int k4 = P.k4;
  const float lam = P.lambda;
  const uint2 seed = make_uint2(P.seed_lo, P.seed_hi);
  const int epoch_end = P.epoch0 + P.n_epochs;
  const unsigned below = (1u << lane) - 1u;

  uint32_t head = 0;      // first ring position not yet taken
  uint32_t taken = 0;     // bit i: position head + i already taken (out of order)
  int64_t done = 0;
  // hybrid circulation: this warp's inbox (read by lanes 16..30) and the
  // block of this worker (a next worker in it is handed the token there)
  constexpr bool use_in = BLK;
  int4* islots = inbox_slots(inboxes + size_t(wib) * kInboxBytes);
  int* ictl = inbox_ctl(inboxes + size_t(wib) * kInboxBytes);
  int head_in = 0;
  const int qblock = q - wib;  // first worker of this block
  // tokens taken at once: the schedule's batch_tokens, at most kBatch
  const int cap = P.batch_cap > 0 && P.batch_cap < kBatch ? P.batch_cap : kBatch;
  // urgent ring: tokens of the items with most ratings, taken out of turn
  const bool use_u = CPL == 1 && P.use_urgent != 0;
  const int lgu = P.uring_log2;
  const uint32_t umask = (1u << lgu) - 1u;
  const unsigned long long* uring_q = use_u ? P.uring + (int64_t(q) << lgu) : nullptr;
  uint32_t head_u = 0;
  // lane 0: urgent slot `pv_pos` as read at the previous check
  unsigned long long pv = 0;
  uint32_t pv_pos = ~0u;

  // Between visits: take a token waiting in the urgent ring.  Lane 0 looks
  // at the slot as read at the previous check (reading it again for the next
  // check while it is empty), so the check never waits for memory.  Returns
  // true after such a visit.
  auto try_urgent = [&]() -> bool {
    if constexpr (CPL != 1) {
      return false;
    } else {
      if (!use_u) return false;
      int go = 0;
      uint32_t useg = 0;
      if (lane == 0) {
        if (pv_pos == head_u && uint32_t(pv >> 32) == (head_u >> lgu)) {
          go = 1;
          useg = uint32_t(pv);
          fence_acq_rel_gpu();  // with the relaxed read of the slot: an acquire
        } else {
          pv = ld_relaxed_u64(uring_q + (head_u & umask));
          pv_pos = head_u;
        }
      }
      if (!__shfl_sync(kFull, go, 0)) return false;
      __syncwarp();
      useg = __shfl_sync(kFull, useg, 0);
      ++head_u;
      ++done;
      if (PR != kF32 && P.ubits_pre)
        urgent_visit<PR, DEBUG, BLK, PR != kF32>(P, q, lane, useg, rows + kVisitChunks * 32,
                                                 rsc + kVisitChunks, ubits, srb);
      else
        urgent_visit<PR, DEBUG, BLK, false>(P, q, lane, useg, rows + kVisitChunks * 32,
                                            rsc + kVisitChunks, ubits, srb);
      return true;
    }
  };

  while (done < quota) {
    // ---- 1. ready tokens among the first kRingWindow positions of the ring
    // (a position reserved by a pusher that has not written it yet does not
    // hold back the ones behind it), and the urgent ring
    unsigned long long sv = 0;
    bool ready = false;
    if (lane < kRingWindow) {
      const uint32_t pos = head + uint32_t(lane);
      if (!((taken >> lane) & 1u)) {
        sv = ld_acquire_u64(ring_q + (pos & qmask));
        ready = uint32_t(sv >> 32) == (pos >> lg);
      }
    } else if (lane < 31) {  // the inbox (hybrid circulation)
      if (use_in && lane - kRingWindow < kInboxSlots) {
        const int pos = head_in + (lane - kRingWindow);
        const volatile int* tag =
            reinterpret_cast<const volatile int*>(islots + 4 * (pos % kInboxSlots) + 3) + 1;
        ready = *tag == pos + 1;
        if (ready) __threadfence_block();  // with the tag seen: an acquire
      }
    } else if (use_u) {  // lane 31: the urgent ring, read alongside
      sv = ld_acquire_u64(uring_q + (head_u & umask));
      ready = uint32_t(sv >> 32) == (head_u >> lgu);
    }
    const unsigned rmask = __ballot_sync(kFull, ready);
    if (rmask >> 31) {  // an urgent item's token first
      __syncwarp();
      const uint32_t item = uint32_t(__shfl_sync(kFull, sv, 31));
      ++head_u;
      ++done;
      if (PR != kF32 && P.ubits_pre)
        urgent_visit<PR, DEBUG, BLK, PR != kF32>(P, q, lane, item, rows + kVisitChunks * 32,
                                                 rsc + kVisitChunks, ubits, srb);
      else
        urgent_visit<PR, DEBUG, BLK, false>(P, q, lane, item, rows + kVisitChunks * 32,
                                            rsc + kVisitChunks, ubits, srb);
      continue;
    }
    // inbox tokens: the ready positions from the head on, in order
    int n_in = __ffs(~((rmask >> kRingWindow) & 0x7fffu)) - 1;
    if (n_in > cap) n_in = cap;
    unsigned tmask = rmask & ((1u << kRingWindow) - 1u);
    if (tmask == 0u && n_in == 0) {
      int got = 0;
      if (lane == 0) {
        const volatile int* itag =
            use_in ? reinterpret_cast<const volatile int*>(islots + 4 * (head_in % kInboxSlots) + 3) + 1
                   : nullptr;
        got = wait_rings(P, q, head, lg, ring_q, head_u, uring_q, itag, head_in + 1);
      }
      if (__shfl_sync(kFull, got, 0) < 0) return;
      continue;  // a slot is ready now; read the rings again
    }
    // batch lanes 0 .. n_in-1 take the inbox tokens, the next ones the first
    // ready ring positions
    while (__popc(tmask) > cap - n_in) tmask &= ~(1u << (31 - __clz(tmask)));
    const int nb = n_in + __popc(tmask);
    {
      const int src = lane >= n_in && lane < nb ? int(__fns(tmask, 0, lane - n_in + 1)) : 0;
      sv = __shfl_sync(kFull, sv, src);
    }
    __syncwarp();  // each lane's acquire precedes every lane's reads below
    taken |= tmask;
    {
      const int adv = __ffs(~taken) - 1;  // taken positions at the head
      head += uint32_t(adv);
      taken >>= adv;
    }
    done += nb;
    const bool mine = lane < nb;

    // ---- 2. token `lane`: item and its visit, from the inbox slot or from
    // the ring and the token's record
    int j = 0, seg = 0, c = 0, e = 0, hop = 0, cb = 0, dseg = 0;
    int4 rb4 = make_int4(0, 0, 0, 0), rc4 = make_int4(0, 0, 0, 0);
    int64_t beg = 0;
    if (mine) {
      int4 ra;
      if (lane < n_in) {
        const int4* sl = islots + 4 * ((head_in + lane) % kInboxSlots);
        ra = sl[0];
        rb4 = sl[1];
        rc4 = sl[2];
        j = sl[3].x;
      } else {
        j = int(uint32_t(sv));
        ra = __ldcg(P.tok_rec + kTokRec * j);
        rb4 = __ldcg(P.tok_rec + kTokRec * j + 1);
        if (use_in) rc4 = __ldcg(P.tok_rec + kTokRec * j + 2);
      }
      seg = ra.x;
      c = ra.y;
      beg = int64_t(uint32_t(ra.z));
      e = ra.w;
      hop = rb4.x;
      cb = rb4.y;
      dseg = rb4.z;
    }
    if (n_in > 0) {  // the slots are read: hand them back to the producers
      head_in += n_in;
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        reinterpret_cast<volatile int*>(ictl)[0] = head_in;
      }
    }

    // ---- 3. processing order: long visits first, then ring order
    const unsigned hv = __ballot_sync(kFull, mine && c >= kHeavy);
    const unsigned lt = ((1u << nb) - 1u) & ~hv;
    int rank = 0;
    if (mine) rank = ((hv >> lane) & 1u) ? __popc(hv & below) : __popc(hv) + __popc(lt & below);
    if (mine) {
      meta_a[rank] = make_int4(j, c, e, seg);
      meta_b[rank] = make_int4(int(uint32_t(beg)), int(uint32_t(uint64_t(beg) >> 32)), lane, 0);
    }
    __syncwarp();
    int T;
    {  // stream offsets: exclusive prefix of the lengths in processing order
      const int cr = lane < nb ? meta_a[lane].y : 0;
      int incl = cr;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      T = __shfl_sync(kFull, incl, 31);
      if (lane < nb) meta_b[lane].w = incl - cr;
    }
    __syncwarp();

    // ---- 4. h of every token and the first records of the stream
    for (int r = 0; r < nb; ++r) {
      const int64_t jr = meta_a[r].x;
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int idx = lane + 32 * cc;
        if (idx < k4) cp_chunk(hbuf + (r * CPL + cc) * 32 + lane, H4 + jr * pitch4 + idx);
      }
    }
    // lane r < nb: stream offset, first record and epoch of the rank-r visit
    int v_soff = 0, v_ep = 0;
    int64_t v_beg = 0;
    if (lane < nb) {
      const int4 mb = meta_b[lane];
      v_soff = mb.w;
      v_beg = (int64_t(mb.y) << 32) | uint32_t(mb.x);
      v_ep = meta_a[lane].z;
    }
    // long visits (ranks 0 .. nhv-1) take stream positions [0, T0) and run
    // first on their own path; the generic stream starts at T0
    const int nhv = __popc(hv);
    int T0 = 0;
    for (int r = 0; r < nhv; ++r) T0 += meta_a[r].y;
    int loaded = T - T0 < kRecInit ? T : T0 + kRecInit;
    for (int p0 = T0; p0 < loaded; p0 += 32)
      load_records<kBatch>(recs, P.rec, v_soff, v_beg, nb, p0, loaded - p0 < 32 ? loaded - p0 : 32,
                   lane);
    cp_commit();

    // step size and routing of token `lane` (loads overlap the copies)
    int nseg = -1;
    Route nx{-1, 0, 0, 0, 0, 0};
    float s_tok = 0.f;
    if (mine) {
      s_tok = __ldg(P.step + (e - P.epoch0));
      nx = route_next<BLK>(P, j, e, hop, cb, dseg, rb4.w, rc4.x, rc4.y, rc4.z, rc4.w, epoch_end,
                           seed);
      nseg = nx.seg;
    }
    cp_wait_all();
    __syncwarp();
    int q2 = -1, nc = 0;  // the next visit: worker, length, first record
    int64_t nbeg = 0;
    if (mine && nseg >= 0) {
      q2 = __ldg(P.seg_worker + nseg);
      nbeg = __ldg(P.seg_ptr + nseg);
      nc = int(__ldg(P.seg_ptr + nseg + 1) - nbeg);
    }
    // Hand-over of token `lane` in two steps around the __syncwarp that
    // orders the warp's H stores: a next worker in this block gets the token
    // in its inbox, with the record of its next visit; otherwise the record
    // goes to the token's global record (before the __syncwarp) and the item
    // to the worker's ring (release store, after it).  A full inbox falls
    // back to the global path after the __syncwarp.
    const bool intra = use_in && nseg >= 0 && q2 - qblock >= 0 && q2 - qblock < P.wpb;
    auto write_record = [&]() {
      __stcg(P.tok_rec + kTokRec * j, make_int4(nseg, nc, int(uint32_t(nbeg)), nx.epoch));
      __stcg(P.tok_rec + kTokRec * j + 1, make_int4(nx.hop, cb, dseg, nx.gs));
      if (use_in) __stcg(P.tok_rec + kTokRec * j + 2, make_int4(rc4.x, rc4.y, nx.ro, nx.rz));
    };
    auto hand_on = [&]() {
      if (intra) {
        if (inbox_push(inboxes + size_t(q2 - qblock) * kInboxBytes, j,
                       make_int4(nseg, nc, int(uint32_t(nbeg)), nx.epoch),
                       make_int4(nx.hop, cb, dseg, nx.gs),
                       make_int4(rc4.x, rc4.y, nx.ro, nx.rz)))
          return;
        write_record();
      }
      push_token(P, q2, uint32_t(j));
    };

    // ---- 5h. the long visits
    for (int kh = 0; kh < nhv; ++kh) {
      while (try_urgent()) {
      }
      const int4 ma = meta_a[kh];
      const int4 mb = meta_b[kh];
      const int vl = mb.z;
      const int64_t vb = (int64_t(mb.y) << 32) | uint32_t(mb.x);
      const float sv = __shfl_sync(kFull, s_tok, vl);
      float4 hh[CPL];
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc)
        hh[cc] = lane + 32 * cc < k4 ? widen_h(hbuf[(kh * CPL + cc) * 32 + lane])
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
      if (DEBUG && lane == 0) {
        const uint32_t tk = atomicAdd(P.log_ticket, 1u);
        if (int64_t(tk) < P.log_cap) {
          P.log_seg[tk] = ma.w;
          P.log_epoch[tk] = ma.z;
        }
        if (atomicExch(P.owner + ma.x, q) != -1) flag_ownership(P, q, ma.x);
      }
      long_visit<CPL, PR, DEBUG, RowRing<CPL>::VISIT>(hh, rows, rsc, srb, W4, Wscale, pitch4, k4,
                                                      P.rec, vb, ma.y, sv, lam, ma.z, seed, lane,
                                                      P.rec_count, nullptr, nullptr);
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int idx = lane + 32 * cc;
        if (idx < k4) store_h(H4 + int64_t(ma.x) * pitch4 + idx, hh[cc], ma.w, ma.z, idx, seed);
      }
      if (lane == vl) {
        if (nseg >= 0 && !intra) write_record();
        if (DEBUG && atomicExch(P.owner + j, -1) != q) flag_ownership(P, q, j);
      }
      __syncwarp();  // orders every lane's H stores before the hand-over below
      if (lane == vl && nseg >= 0) hand_on();
    }

    // ---- 5a. cold start of the row ring: positions 0 .. R-2
    // A row that a position in flight also updates (a user who rated two
    // items of the batch) is not copied: the latest such position writes its
    // updated row into this position's slot as well (each lane its own chunk).
    int win = -1;    // lane L < R: row of the position in flight in slot L
    int fwd = -1;    // lane L < R: the slot that takes that position's updated row
    auto copy_row = [&](int slot, int row) {
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int idx = lane + 32 * cc;
        if (idx < k4)
          cp_chunk(rows + (slot * CPL + cc) * 32 + lane, W4 + int64_t(row) * pitch4 + idx);
      }
      if constexpr (PR == kFP8)
        if (lane == 0) cp_async4(rsc + slot, Wscale + row);
    };
    // one commit group per position: at tick t exactly R-1 groups are
    // younger than position t's group, so cp.async.wait_group R-1 suffices.
    // The R-1 positions are decided together: lane L < R takes the position
    // o = (L - T0) mod R of the cold start (slot L); lanes with the same row
    // are found at once, a position with an earlier one of its row is not
    // copied, and each position forwards to the next one of its row.
    {
      const int sh = int(unsigned(T0) % unsigned(R));
      const int o = int(unsigned(lane - sh + R) % unsigned(R));
      const bool live = lane < R && o < R - 1 && T0 + o < T;
      const int row = live ? recs[unsigned(T0 + o) % kRecBuf].x : -(lane + 1);
      const unsigned m = __match_any_sync(kFull, row);
      const unsigned full = (1u << R) - 1u;
      const unsigned mr = m & full;
      const unsigned rot = ((mr >> sh) | (mr << (R - sh))) & full;  // bit o: order o
      const bool has_src = live && (rot & ((1u << o) - 1u)) != 0u;
      const unsigned later = live ? rot & ~((2u << o) - 1u) & full : 0u;
      fwd = later ? int(unsigned(__ffs(later) - 1 + sh) % unsigned(R)) : -1;
      win = live ? row : -1;
      const unsigned copy = __ballot_sync(kFull, live && !has_src);
      for (int q = 0; q < R - 1; ++q) {
        const int slot = int(unsigned(q + sh) % unsigned(R));
        const int rq = __shfl_sync(kFull, row, slot);
        if ((copy >> slot) & 1u) copy_row(slot, rq);
        cp_commit();
      }
    }

    // ---- 5b. the stream
    int k = nhv - 1, vend = T0, vsoff = 0, vlane = 0, vseg = 0, vep = 0;
    int64_t vbeg = 0;
    float s = 0.f;
    float2 al2 = make_float2(1.f, 1.f);
    int sr_lo = T0, sr_hi = T0;  // stream positions whose rounding bits are in srb
    float4 h[CPL];
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) h[cc] = make_float4(0.f, 0.f, 0.f, 0.f);
    // the row the next tick prefetches, read a tick ahead (its record landed
    // with a group at least R ticks old)
    int nrow = T0 + R - 1 < T ? recs[(T0 + R - 1) % kRecBuf].x : 0;
    for (int t = T0; t < T; ++t) {
      if (t == vend) {  // a visit starts
        // an urgent item's token waiting in the ring goes first: the tokens
        // of the items with most ratings make the longest chains of visits
        if (try_urgent()) {
          // rows copied or forwarded for the positions in flight may be stale:
          // copy them all again (a forward still to come overwrites the copy)
          for (int pos = t; pos < t + R - 1 && pos < T; ++pos)
            copy_row(pos % R, recs[pos % kRecBuf].x);
          cp_commit();
          cp_wait<0>();
          // a visit with pre-drawn bits used the stream's bits area: draw
          // from t again
          if constexpr (PR != kF32)
            if (P.ubits_pre) sr_hi = t;
        }
        ++k;
        const int4 ma = meta_a[k];
        const int4 mb = meta_b[k];
        vsoff = t;
        vend = t + ma.y;
        vseg = ma.w;
        vep = ma.z;
        vlane = mb.z;
        vbeg = (int64_t(mb.y) << 32) | uint32_t(mb.x);
        s = __shfl_sync(kFull, s_tok, vlane);
        al2 = make_float2(1.f - s * lam, 1.f - s * lam);
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc)  // lanes past k/4 hold zeros, never smem
          h[cc] = lane + 32 * cc < k4 ? widen_h(hbuf[(k * CPL + cc) * 32 + lane])
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        if (DEBUG && lane == 0) {
          const uint32_t tk = atomicAdd(P.log_ticket, 1u);
          if (int64_t(tk) < P.log_cap) {
            P.log_seg[tk] = vseg;
            P.log_epoch[tk] = ma.z;
          }
          if (atomicExch(P.owner + ma.x, q) != -1) flag_ownership(P, q, ma.x);
        }
      }
      if constexpr (PR != kF32) {
        if (t == sr_hi) {  // the next SRB positions' rounding bits, drawn in bulk
          __syncwarp();    // every lane has read the previous draws
          draw_stream_bits<kBatch, CPL>(srb, v_soff, v_beg, v_ep, nb, t, T, k4, seed, lane);
          sr_lo = t;
          sr_hi = t + SRB;
        }
      }
      // keep the records one chunk ahead of the row prefetch
      if (loaded < T && loaded < t + R + 32) {
        const int cnt = T - loaded < 32 ? T - loaded : 32;
        load_records<kBatch>(recs, P.rec, v_soff, v_beg, nb, loaded, cnt, lane);
        loaded += cnt;
      }
      // position t's row was copied R-1 ticks ago; the copy of position
      // t + R - 1 (issued below, after t's slot is read) is not committed
      // yet, so R-2 younger groups may still be in flight
      cp_wait<R - 2>();
      __syncwarp();

      const int2 rc = recs[unsigned(t) % kRecBuf];
      const int slot = int(unsigned(t) % R);
      w_t* wrow = W4 + int64_t(rc.x) * pitch4;
      const float sc = PR == kFP8 ? rsc[slot] : 1.f;
      float4 w[CPL];
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int idx = lane + 32 * cc;
        w[cc] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < k4) w[cc] = widen_w(rows[(slot * CPL + cc) * 32 + lane], sc);
      }
      uint2 rb[CPL];
      if constexpr (PR != kF32) {
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) rb[cc] = srb[(t - sr_lo) * CPL * 32 + lane + 32 * cc];
      }
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) acc = dot4_acc(w[cc], h[cc], acc);
      float dsum = acc.x + acc.y;
      dsum += __shfl_xor_sync(kFull, dsum, 16);
      {  // the copy of position pp = t + R - 1 into the slot t - 1 left, decided
         // and issued without branches while the reduction's shuffles are in
         // flight; its row (nrow) was read from the records a tick ahead
        const int pp = t + R - 1;
        const bool live = pp < T;
        const int pslot = int(unsigned(pp) % R);
        const unsigned m = __ballot_sync(kFull, live && lane < R && lane != pslot && win == nrow);
        // the latest position in flight with that row: going back from pp - 1
        // the slots are pslot - 1, ..., 0, R - 1, ..., pslot + 1; it writes
        // its updated row into pslot as well
        const unsigned mm = (m | (m << R)) & ((1u << (pslot + R)) - 1u);
        const int tgt = m ? int(unsigned(31 - __clz(mm)) % R) : -1;
        const bool copy = live && m == 0u;
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          const int idx = lane + 32 * cc;
          cp_chunk_if(copy && idx < k4, rows + (pslot * CPL + cc) * 32 + lane,
                      W4 + int64_t(nrow) * pitch4 + idx);
        }
        if constexpr (PR == kFP8) cp_chunk_if(copy && lane == 0, rsc + pslot, Wscale + nrow);
        fwd = lane == tgt ? pslot : fwd;
        win = lane == pslot ? (live ? nrow : -1) : win;
        fwd = lane == pslot ? -1 : fwd;
        cp_commit();
      }
      dsum += __shfl_xor_sync(kFull, dsum, 8);
      dsum += __shfl_xor_sync(kFull, dsum, 4);
      dsum += __shfl_xor_sync(kFull, dsum, 2);
      dsum += __shfl_xor_sync(kFull, dsum, 1);
      const int fslot = __shfl_sync(kFull, fwd, slot);  // a later position's slot, or -1
      const float err = __int_as_float(rc.y) - dsum;
      const float se = s * err;
      const float2 se2 = make_float2(se, se);
      float4 wn[CPL];
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        wn[cc] = axpby(al2, w[cc], se2, h[cc]);  // (1 - s lam) w + s e h
        h[cc] = axpby(se2, w[cc], al2, h[cc]);   // (1 - s lam) h + s e w
      }
      w_t out[CPL];
      float nscale = 1.f;
      narrow_w<PR, CPL>(wn, rb, out, &nscale);
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int idx = lane + 32 * cc;
        if (idx < k4) {
          wrow[idx] = out[cc];
          if (fslot >= 0) rows[(fslot * CPL + cc) * 32 + lane] = out[cc];
        }
      }
      if constexpr (PR == kFP8) {
        if (lane == 0) {
          Wscale[rc.x] = nscale;
          if (fslot >= 0) rsc[fslot] = nscale;
        }
      }
      if (DEBUG && lane == 0) P.rec_count[vbeg + (t - vsoff)] += 1;
      if (t + R < T) nrow = recs[(t + R) % kRecBuf].x;

      if (t == vend - 1) {  // the visit ends: publish h_j
        const int jv = meta_a[k].x;
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          const int idx = lane + 32 * cc;
          if (idx < k4) store_h(H4 + int64_t(jv) * pitch4 + idx, h[cc], vseg, vep, idx, seed);
        }
      }
    }

    // ---- 6. hand on the remaining tokens together
    const bool late = mine && c < kHeavy;
    if (late) {
      if (nseg >= 0 && !intra) write_record();
      if (DEBUG && atomicExch(P.owner + j, -1) != q) flag_ownership(P, q, j);
    }
    __syncwarp();  // orders every lane's H stores before the hand-overs below
    if (late && nseg >= 0) hand_on();
  }
  if (lane == 0) atomicMax(P.span + 1, globaltimer_ns());
}

// Empties warp wib's inbox.
__device__ __forceinline__ void clear_inbox(unsigned char* inboxes, int wib, int lane) {
  int* w = reinterpret_cast<int*>(inboxes + size_t(wib) * kInboxBytes);
  for (int i = lane; i < kInboxBytes / 4; i += 32) w[i] = 0;
}

template <int CPL, int PR, bool DEBUG, bool BLK>
__global__ void __launch_bounds__(kBatchedWarps * 32, 1)
nomad_batched_kernel(const __grid_constant__ SgdParams P) {
  extern __shared__ float4 smem_f4[];
  unsigned char* base = reinterpret_cast<unsigned char*>(smem_f4);
  const int nw = blockDim.x >> 5;
  const int wib = threadIdx.x >> 5;
  unsigned char* inboxes = base + size_t(nw) * warp_smem_bytes<CPL, PR>();
  if constexpr (BLK) {  // hybrid circulation: inboxes empty before any hand-over
    clear_inbox(inboxes, wib, threadIdx.x & 31);
    __syncthreads();
  }
  const int q = blockIdx.x * nw + wib;
  if (q >= P.p) return;
  batched_worker<CPL, PR, DEBUG, BLK>(P, q, base + size_t(wib) * warp_smem_bytes<CPL, PR>(),
                                      inboxes, wib);
}

// Several independent problems in one launch: block b runs block
// `blocks[b].y` of problem `blocks[b].x`, whose parameters (Ps[blocks[b].x])
// are copied into shared memory after the warps' areas (and the inboxes
// after them, when some problem uses the hybrid circulation: use_inboxes).  Every block of a
// problem is resident with the others (cooperative launch), as in the
// one-problem kernel; problems share nothing.
constexpr int kParamsBytes = int((sizeof(SgdParams) + 15) / 16 * 16);

template <int CPL, int PR, bool DEBUG>
__global__ void __launch_bounds__(kBatchedWarps * 32, 1)
nomad_batched_many_kernel(const SgdParams* __restrict__ Ps, const int2* __restrict__ blocks,
                          int use_inboxes) {
  extern __shared__ float4 smem_f4[];
  const int nw = blockDim.x >> 5;
  unsigned char* base = reinterpret_cast<unsigned char*>(smem_f4);
  SgdParams* Pb = reinterpret_cast<SgdParams*>(base + size_t(nw) * warp_smem_bytes<CPL, PR>());
  const int2 bp = blocks[blockIdx.x];
  const int* src = reinterpret_cast<const int*>(Ps + bp.x);
  int* dst = reinterpret_cast<int*>(Pb);
  for (int i = threadIdx.x; i < int(sizeof(SgdParams) / sizeof(int)); i += blockDim.x)
    dst[i] = src[i];
  const int wib = threadIdx.x >> 5;
  unsigned char* inboxes = reinterpret_cast<unsigned char*>(Pb) + kParamsBytes;
  if (use_inboxes) clear_inbox(inboxes, wib, threadIdx.x & 31);
  __syncthreads();
  const int q = bp.y * nw + wib;
  if (q >= Pb->p) return;
  // problems of either circulation share the launch: the worker body of each
  if (Pb->col_grp_ptr != nullptr)
    batched_worker<CPL, PR, DEBUG, true>(*Pb, q, base + size_t(wib) * warp_smem_bytes<CPL, PR>(),
                                         inboxes, wib);
  else
    batched_worker<CPL, PR, DEBUG, false>(*Pb, q, base + size_t(wib) * warp_smem_bytes<CPL, PR>(),
                                          inboxes, wib);
}

template <int CPL, int PR>
const void* batched_ptr(bool debug, bool many, bool blk, size_t* smem_per_warp) {
  *smem_per_warp = size_t(warp_smem_bytes<CPL, PR>());
  if (many)
    return debug ? (const void*)nomad_batched_many_kernel<CPL, PR, true>
                 : (const void*)nomad_batched_many_kernel<CPL, PR, false>;
  if (blk)
    return debug ? (const void*)nomad_batched_kernel<CPL, PR, true, true>
                 : (const void*)nomad_batched_kernel<CPL, PR, false, true>;
  return debug ? (const void*)nomad_batched_kernel<CPL, PR, true, false>
               : (const void*)nomad_batched_kernel<CPL, PR, false, false>;
}

// The kernels of storage format PR for the row width class of k4.
template <int PR>
const void* batched_ptr_k4(int k4, bool debug, bool many, bool blk, size_t* smem_per_warp) {
  if (k4 <= 32) return batched_ptr<1, PR>(debug, many, blk, smem_per_warp);
  if (k4 <= 64) return batched_ptr<2, PR>(debug, many, blk, smem_per_warp);
  if (k4 <= 128) return batched_ptr<4, PR>(debug, many, blk, smem_per_warp);
  return nullptr;
}

}  // namespace
}  // namespace nomad
