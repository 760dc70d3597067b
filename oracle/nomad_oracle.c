/*
 * nomad_oracle.c -- serial CPU oracle for NOMAD matrix completion
 * (Yun, Yu, Hsieh, Vishwanathan, Dhillon, "NOMAD: Non-locking, stOchastic
 * Multi-machine algorithm for Asynchronous and Decentralized matrix
 * completion", arXiv 1312.0193).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this library.
 * It shares no source, header, table or helper with the CUDA path.
 *
 * Everything here is deliberately plain: one rating at a time, in the order
 * the paper states, in IEEE binary64 unless a function says otherwise.
 * Build with -ffp-contract=off so that no multiply-add is fused behind the
 * reader's back.
 *
 * Readings of the paper that this file commits to (each also listed in the
 * design notes of the repository):
 *  R1  Sign of the SGD step (Sec. 2.3, Eq. w_update / h_update).  The
 *      derivative of 1/2 (A_ij - <w_i,h_j>)^2 w.r.t. w_i is -(A_ij-<w,h>) h_j,
 *      so a descent step is  w_i += s (e h_j - lambda w_i),
 *      h_j += s (e w_i - lambda h_j)  with  e = A_ij - <w_i,h_j>.
 *  R2  The "w_j" inside the printed h-update is a typo for w_i.
 *  R3  Both updates use the OLD w_i (one gradient evaluation per rating).
 *      The alternative (h-update sees the new w_i) is available through the
 *      flag h_uses_new_w so that the choice is explicit and testable.
 *  R4  t in the step size (Sec. 5.1, Eq. stepsize_method) counts the updates
 *      already applied to the rating (i,j); the first visit uses s_0 = alpha.
 *  R5  The regulariser is applied per rating with plain lambda (the
 *      simplified form of Eq. obj_fcn): no division by |Omega_i|.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Used for the     */
/* factor initialisation of Alg. 1 and for every random draw of the oracle. */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_KEY_STEP_A = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_KEY_STEP_B = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* the key is bumped before every round but the first */
      k0 += PHILOX_KEY_STEP_A;
      k1 += PHILOX_KEY_STEP_B;
    }
    uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
    uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
    uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
    uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
    uint32_t y0 = hi_b ^ x1 ^ k0;
    uint32_t y1 = lo_b;
    uint32_t y2 = hi_a ^ x3 ^ k1;
    uint32_t y3 = lo_a;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 32-bit word of the stream (seed; c0,c1,c2,c3), word index w in 0..3. */
static uint32_t rand_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, int w) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[w];
}

/* Uniform integer in [0, bound) from one 32-bit word (multiply-shift). */
static uint32_t bounded(uint32_t word, uint32_t bound) {
  return (uint32_t)(((uint64_t)word * (uint64_t)bound) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Initialisation (Alg. 1 "initialize parameters"; Sec. 5.1 set-up):        */
/* every entry of W and H independent UniformReal(0, 1/sqrt(k)).            */
/*                                                                          */
/* Entry (r, l) of the factor `which` (0 = W, 1 = H) takes word (l mod 4)   */
/* of Philox4x32-10 with key = seed and counter = (l/4, r_lo, r_hi, which). */
/* u = (word >> 8) * 2^-24 is exact in binary32; the entry is the binary32  */
/* product u * c with c = binary32(1/sqrt(k)), stored here widened to       */
/* double (the widening is exact).                                          */
/* ------------------------------------------------------------------------ */
void orc_init_factor(int64_t rows, int32_t k, uint64_t seed, uint32_t which,
                     double *F) {
  const float c = (float)(1.0 / sqrt((double)k));
  for (int64_t r = 0; r < rows; ++r) {
    for (int32_t l = 0; l < k; ++l) {
      uint32_t word = rand_word(seed, (uint32_t)(l / 4), (uint32_t)r,
                                (uint32_t)((uint64_t)r >> 32), which, l % 4);
      float u = (float)(word >> 8) * (1.0f / 16777216.0f);
      float v = u * c; /* one binary32 rounding */
      F[r * (int64_t)k + l] = (double)v;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Step size, Sec. 5.1 Eq. stepsize_method: s_t = alpha / (1 + beta t^1.5). */
/* ------------------------------------------------------------------------ */
double orc_step_size(double alpha, double beta, int64_t t) {
  return alpha / (1.0 + beta * pow((double)t, 1.5));
}

/* ------------------------------------------------------------------------ */
/* One SGD update on rating (i,j) with value a (Sec. 2.3, Eq. w_update and  */
/* h_update under readings R1-R3).                                          */
/* ------------------------------------------------------------------------ */
void orc_sgd_update(int32_t k, double *w, double *h, double a, double lambda,
                    double s, int32_t h_uses_new_w) {
  double dot = 0.0;
  for (int32_t l = 0; l < k; ++l) dot += w[l] * h[l];
  const double e = a - dot;
  for (int32_t l = 0; l < k; ++l) {
    const double w_old = w[l];
    const double h_old = h[l];
    const double w_new = w_old + s * (e * h_old - lambda * w_old);
    const double w_for_h = h_uses_new_w ? w_new : w_old;
    w[l] = w_new;
    h[l] = h_old + s * (e * w_for_h - lambda * h_old);
  }
}

/* The same update carried out entirely in binary32 (for the FP32 replay). */
void orc_sgd_update_f32(int32_t k, float *w, float *h, float a, float lambda,
                        float s) {
  float dot = 0.0f;
  for (int32_t l = 0; l < k; ++l) dot += w[l] * h[l];
  const float e = a - dot;
  for (int32_t l = 0; l < k; ++l) {
    const float w_old = w[l];
    const float h_old = h[l];
    w[l] = w_old + s * (e * h_old - lambda * w_old);
    h[l] = h_old + s * (e * w_old - lambda * h_old);
  }
}

/* ------------------------------------------------------------------------ */
/* Objective J(W,H), simplified form of Eq. obj_fcn (Sec. 2):               */
/*   J = 1/2 sum_{(i,j) in Omega} [ (A_ij - <w_i,h_j>)^2                    */
/*                                  + lambda (|w_i|^2 + |h_j|^2) ]          */
/* ------------------------------------------------------------------------ */
double orc_objective(int64_t nnz, const int32_t *rows, const int32_t *cols,
                     const double *vals, int32_t k, double lambda,
                     const double *W, const double *H) {
  double total = 0.0;
  for (int64_t r = 0; r < nnz; ++r) {
    const double *w = W + (int64_t)rows[r] * k;
    const double *h = H + (int64_t)cols[r] * k;
    double dot = 0.0, ww = 0.0, hh = 0.0;
    for (int32_t l = 0; l < k; ++l) {
      dot += w[l] * h[l];
      ww += w[l] * w[l];
      hh += h[l] * h[l];
    }
    const double e = vals[r] - dot;
    total += e * e + lambda * (ww + hh);
  }
  return 0.5 * total;
}

/* Test RMSE (Sec. 5.1): sqrt( sum_test (A_ij - <w_i,h_j>)^2 / |Omega_test| ).
 * Returns the sum of squares; the caller divides and takes the root so that
 * an empty test set is handled where the count is known. */
double orc_sq_error_sum(int64_t nnz, const int32_t *rows, const int32_t *cols,
                        const double *vals, int32_t k, const double *W,
                        const double *H) {
  double total = 0.0;
  for (int64_t r = 0; r < nnz; ++r) {
    const double *w = W + (int64_t)rows[r] * k;
    const double *h = H + (int64_t)cols[r] * k;
    double dot = 0.0;
    for (int32_t l = 0; l < k; ++l) dot += w[l] * h[l];
    const double e = vals[r] - dot;
    total += e * e;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Replay of a given serial order of token visits (Sec. 3.1: processing     */
/* item j at worker q runs the SGD updates on Omega-bar_j^(q); Alg. 1, the  */
/* loop over Omega-bar_j^(q)).                                              */
/*                                                                          */
/* visit_seg[v] names the segment Omega-bar_j^(q) processed by visit v.     */
/* Segment s holds records seg_ptr[s] .. seg_ptr[s+1]-1, whose rows are     */
/* rec_row and values rec_val; its item is seg_col[s].  Within a visit the  */
/* records are applied in storage order.  rec_count[r] is the number of     */
/* updates already applied to record r (reading R4); it is advanced here.   */
/* W is m x k and H is n x k, row-major with pitch k.                       */
/* Returns 0, or -1 if a segment index is out of range.                     */
/* ------------------------------------------------------------------------ */
int32_t orc_replay_f64(int32_t k, double lambda, double alpha, double beta,
                       int64_t n_visits, const int64_t *visit_seg,
                       int64_t n_seg, const int64_t *seg_ptr,
                       const int32_t *seg_col, const int32_t *rec_row,
                       const double *rec_val, double *W, double *H,
                       int32_t *rec_count, int32_t h_uses_new_w) {
  for (int64_t v = 0; v < n_visits; ++v) {
    const int64_t s = visit_seg[v];
    if (s < 0 || s >= n_seg) return -1;
    double *h = H + (int64_t)seg_col[s] * k;
    for (int64_t r = seg_ptr[s]; r < seg_ptr[s + 1]; ++r) {
      double *w = W + (int64_t)rec_row[r] * k;
      const double step = orc_step_size(alpha, beta, rec_count[r]);
      orc_sgd_update(k, w, h, rec_val[r], lambda, step, h_uses_new_w);
      rec_count[r] += 1;
    }
  }
  return 0;
}

/* The same replay with W, H and all arithmetic in binary32; the step size is
 * evaluated in binary64 and rounded once. */
int32_t orc_replay_f32(int32_t k, float lambda, double alpha, double beta,
                       int64_t n_visits, const int64_t *visit_seg,
                       int64_t n_seg, const int64_t *seg_ptr,
                       const int32_t *seg_col, const int32_t *rec_row,
                       const float *rec_val, float *W, float *H,
                       int32_t *rec_count) {
  for (int64_t v = 0; v < n_visits; ++v) {
    const int64_t s = visit_seg[v];
    if (s < 0 || s >= n_seg) return -1;
    float *h = H + (int64_t)seg_col[s] * k;
    for (int64_t r = seg_ptr[s]; r < seg_ptr[s + 1]; ++r) {
      float *w = W + (int64_t)rec_row[r] * k;
      const float step = (float)orc_step_size(alpha, beta, rec_count[r]);
      orc_sgd_update_f32(k, w, h, rec_val[r], lambda, step);
      rec_count[r] += 1;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Serial simulation of NOMAD (Alg. 1) with p simulated worker queues.      */
/*                                                                          */
/* mode 0 ("epoch", permutation circulation of Sec. 3.4): in every epoch    */
/*   item j visits each worker that holds ratings of j exactly once, in a   */
/*   fresh uniformly random order (Fisher-Yates on the list of its          */
/*   segments, stream (seed; j, epoch, 0, 0x4f524331)).  Its first queue is */
/*   the first worker of epoch 0's order (Alg. 1 places every item in a     */
/*   random queue).  The run ends when every item has finished n_epochs.    */
/* mode 1 ("uniform", Alg. 1 literally): the first queue and every next     */
/*   queue are uniform over all p workers (streams (seed; j, hop, 1, tag)), */
/*   a visit to a worker without ratings of j does nothing, and the run     */
/*   stops once n_epochs * nnz updates have been applied.                   */
/* mode 2 (uniform with the dynamic load balancing of Sec. 3.3): as mode 1, */
/*   but every next queue is the shorter of two uniform draws (streams      */
/*   (seed; j, hop, 1, tag) and (seed; j, hop, 2, tag)), the first one on a */
/*   tie.                                                                   */
/* queue_stats (may be NULL): [0] the longest queue met by a push, [1] the  */
/* sum over pushes of the length of the queue pushed to.                    */
/*                                                                          */
/* Workers are served round-robin q = 0,1,...,p-1, each popping at most one */
/* item per round from the front of its FIFO queue; an empty queue is       */
/* skipped.  The order of segments of item j is col_segs[col_seg_ptr[j] ..],*/
/* and seg_worker[s] is the worker of segment s.  Visits are appended to    */
/* visit_log (segment index, or -1 for an empty uniform-mode visit) when    */
/* visit_log is not NULL and there is room (log_cap).                       */
/* Returns the number of visits, or -1 on a bad argument.                   */
/* ------------------------------------------------------------------------ */
int64_t orc_serial_nomad(int32_t k, double lambda, double alpha, double beta,
                         int32_t p, int64_t n, int64_t n_seg,
                         const int64_t *seg_ptr, const int32_t *seg_col,
                         const int32_t *seg_worker, const int32_t *rec_row,
                         const double *rec_val, const int64_t *col_seg_ptr,
                         const int64_t *col_segs, int32_t n_epochs,
                         uint64_t seed, int32_t mode, double *W, double *H,
                         int32_t *rec_count, int64_t *visit_log,
                         int64_t log_cap, int64_t *queue_stats) {
  if (p <= 0 || n < 0 || mode < 0 || mode > 2) return -1;
  const int uniform = mode != 0;
  const uint32_t TAG = 0x4f524331u;
  /* FIFO queue per worker, each able to hold all n items. */
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p * (n + 1)));
  int64_t *qhead = (int64_t *)calloc((size_t)p, sizeof(int64_t));
  int64_t *qlen = (int64_t *)calloc((size_t)p, sizeof(int64_t));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_seg + 1));
  int64_t *hop = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  int32_t *epoch = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
  if (!queue || !qhead || !qlen || !order || !hop || !epoch) {
    free(queue); free(qhead); free(qlen); free(order); free(hop); free(epoch);
    return -1;
  }
  int64_t total_nnz = seg_ptr[n_seg];
  int64_t n_visits = 0, n_updates = 0;

  if (queue_stats) queue_stats[0] = queue_stats[1] = 0;
#define PUSH(q, j)                                                    \
  do {                                                                \
    int64_t pos_ = (qhead[(q)] + qlen[(q)]) % (n + 1);                \
    queue[(int64_t)(q) * (n + 1) + pos_] = (j);                       \
    if (queue_stats) {                                                \
      if (qlen[(q)] > queue_stats[0]) queue_stats[0] = qlen[(q)];     \
      queue_stats[1] += qlen[(q)];                                    \
    }                                                                 \
    qlen[(q)] += 1;                                                   \
  } while (0)

  /* A fresh uniformly random order of item j's segments for epoch e. */
#define SHUFFLE(j, e)                                                       \
  do {                                                                      \
    int64_t b_ = col_seg_ptr[(j)], d_ = col_seg_ptr[(j) + 1] - b_;          \
    for (int64_t t_ = 0; t_ < d_; ++t_) order[b_ + t_] = col_segs[b_ + t_]; \
    for (int64_t t_ = d_ - 1; t_ > 0; --t_) {                               \
      uint32_t wd_ = rand_word(seed, (uint32_t)(j), (uint32_t)(e),          \
                               (uint32_t)t_, TAG, 0);                       \
      int64_t u_ = (int64_t)bounded(wd_, (uint32_t)(t_ + 1));               \
      int64_t tmp_ = order[b_ + t_];                                        \
      order[b_ + t_] = order[b_ + u_];                                      \
      order[b_ + u_] = tmp_;                                                \
    }                                                                       \
  } while (0)

  /* Initial queues (Alg. 1 "initialize queues"). */
  for (int64_t j = 0; j < n; ++j) {
    if (mode == 0) {
      if (col_seg_ptr[j + 1] == col_seg_ptr[j] || n_epochs <= 0) continue;
      SHUFFLE(j, 0);
      PUSH(seg_worker[order[col_seg_ptr[j]]], j);
    } else {
      uint32_t wd = rand_word(seed, (uint32_t)j, 0u, 1u, TAG, 1);
      PUSH((int32_t)bounded(wd, (uint32_t)p), j);
    }
  }

  const int64_t budget = (int64_t)n_epochs * total_nnz;
  int busy = 1;
  while (busy) {
    busy = 0;
    for (int32_t q = 0; q < p; ++q) {
      if (qlen[q] == 0) continue;
      if (uniform && n_updates >= budget) break;
      busy = 1;
      int64_t j = queue[(int64_t)q * (n + 1) + qhead[q]];
      qhead[q] = (qhead[q] + 1) % (n + 1);
      qlen[q] -= 1;
      /* Find segment (q, j): linear search over item j's segments. */
      int64_t seg = -1;
      for (int64_t t = col_seg_ptr[j]; t < col_seg_ptr[j + 1]; ++t)
        if (seg_worker[col_segs[t]] == q) { seg = col_segs[t]; break; }
      if (visit_log && n_visits < log_cap) visit_log[n_visits] = seg;
      n_visits += 1;
      if (seg >= 0 && seg_col[seg] != j) seg = -2; /* corrupt layout */
      if (seg == -2) break;
      if (seg >= 0) {
        double *h = H + j * (int64_t)k;
        for (int64_t r = seg_ptr[seg]; r < seg_ptr[seg + 1]; ++r) {
          double *w = W + (int64_t)rec_row[r] * k;
          double step = orc_step_size(alpha, beta, rec_count[r]);
          orc_sgd_update(k, w, h, rec_val[r], lambda, step, 0);
          rec_count[r] += 1;
          n_updates += 1;
        }
      }
      if (mode == 0) {
        int64_t d = col_seg_ptr[j + 1] - col_seg_ptr[j];
        hop[j] += 1;
        if (hop[j] == d) {
          hop[j] = 0;
          epoch[j] += 1;
          if (epoch[j] >= n_epochs) continue; /* item j is finished */
          SHUFFLE(j, epoch[j]);
        }
        PUSH(seg_worker[order[col_seg_ptr[j] + hop[j]]], j);
      } else {
        hop[j] += 1;
        uint32_t wd = rand_word(seed, (uint32_t)j, (uint32_t)hop[j], 1u, TAG, 1);
        int32_t qn = (int32_t)bounded(wd, (uint32_t)p);
        if (mode == 2) { /* Sec. 3.3: the shorter of two queues */
          uint32_t wb = rand_word(seed, (uint32_t)j, (uint32_t)hop[j], 2u, TAG, 1);
          int32_t qb = (int32_t)bounded(wb, (uint32_t)p);
          if (qlen[qb] < qlen[qn]) qn = qb;
        }
        PUSH(qn, j);
      }
    }
    if (uniform && n_updates >= budget) break;
  }
#undef PUSH
#undef SHUFFLE
  free(queue); free(qhead); free(qlen); free(order); free(hop); free(epoch);
  return n_visits;
}

/* ------------------------------------------------------------------------ */
/* Textbook SGD (Sec. 2.3): each epoch visits every rating once in a fresh  */
/* uniformly random order (Fisher-Yates, stream (seed; t, epoch, 2, tag)).  */
/* Step size from the per-rating update count (reading R4).                 */
/* ------------------------------------------------------------------------ */
int32_t orc_shuffled_sgd(int32_t k, double lambda, double alpha, double beta,
                         int64_t nnz, const int32_t *rows, const int32_t *cols,
                         const double *vals, int32_t n_epochs, uint64_t seed,
                         double *W, double *H, int32_t *rec_count) {
  const uint32_t TAG = 0x4f524332u;
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz + 1));
  if (!perm) return -1;
  for (int32_t e = 0; e < n_epochs; ++e) {
    for (int64_t r = 0; r < nnz; ++r) perm[r] = r;
    for (int64_t t = nnz - 1; t > 0; --t) {
      uint32_t wd = rand_word(seed, (uint32_t)t, (uint32_t)e,
                              (uint32_t)((uint64_t)t >> 32), TAG, 2);
      int64_t u = (int64_t)bounded(wd, (uint32_t)(t + 1));
      int64_t tmp = perm[t];
      perm[t] = perm[u];
      perm[u] = tmp;
    }
    for (int64_t v = 0; v < nnz; ++v) {
      int64_t r = perm[v];
      double *w = W + (int64_t)rows[r] * k;
      double *h = H + (int64_t)cols[r] * k;
      double step = orc_step_size(alpha, beta, rec_count[r]);
      orc_sgd_update(k, w, h, vals[r], lambda, step, 0);
      rec_count[r] += 1;
    }
  }
  free(perm);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* bfloat16 storage (the precision variant of the GPU path: W and H stored  */
/* as bfloat16, every update computed in binary32, stochastic rounding on   */
/* write-back).  A bfloat16 is the upper 16 bits of a binary32.             */
/*                                                                          */
/* Round to nearest, ties to even (used for the initial values):            */
/*   add 0x7fff plus the lowest kept bit, then truncate.                    */
/* Stochastic rounding with 16 random bits r: add r to the 16 dropped bits  */
/* of the magnitude and truncate, so the magnitude rounds up with           */
/* probability (dropped bits) / 2^16 and the expected value is exact.       */
/* Infinities and NaN are truncated (NaN kept quiet).                       */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float bits_f32(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

uint16_t orc_bf16_rn(float x) {
  uint32_t u = f32_bits(x);
  if ((u & 0x7f800000u) == 0x7f800000u)
    return (uint16_t)((u >> 16) | ((u & 0x007fffffu) ? 0x0040u : 0u));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

uint16_t orc_bf16_sr(float x, uint32_t r16) {
  uint32_t u = f32_bits(x);
  if ((u & 0x7f800000u) == 0x7f800000u)
    return (uint16_t)((u >> 16) | ((u & 0x007fffffu) ? 0x0040u : 0u));
  u += (r16 & 0xffffu);
  return (uint16_t)(u >> 16);
}

float orc_bf16_to_f32(uint16_t b) { return bits_f32((uint32_t)b << 16); }

/* The 16 random bits for entry l of a row written back by the end of the
 * visit of segment s in epoch e (factor H): Philox4x32-10 with key = seed
 * and counter (s, e, 0, 0x48000000 | l/4); entry l takes word
 * 2 + (l mod 4)/2, its low half for even l and high half for odd l. */
static uint32_t sr_bits(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                        uint32_t tag, int32_t l, int word_base) {
  uint32_t w = rand_word(seed, c0, c1, c2, tag | (uint32_t)(l / 4),
                         word_base + (l % 4) / 2);
  return (l % 2) ? (w >> 16) : (w & 0xffffu);
}

/* The 16 random bits for entry l of the W row written back by the update of
 * record r in epoch e.  Entries come in chunks of four (chunk c = l/4), and
 * one Philox4x32-10 draw with key = seed and counter
 * (r_lo, r_hi, e, 0x57000000 | c/2) serves the pair of chunks (2q, 2q+1):
 * chunk c takes words 2(c mod 2) and 2(c mod 2) + 1, entry l word
 * 2(c mod 2) + (l mod 4)/2, its low half for even l and high half for odd
 * l. */
static uint32_t sr_bits_w(uint64_t seed, int64_t r, uint32_t e, int32_t l) {
  const int32_t c = l / 4;
  uint32_t w = rand_word(seed, (uint32_t)r, (uint32_t)((uint64_t)r >> 32), e,
                         0x57000000u | (uint32_t)(c / 2), 2 * (c % 2) + (l % 4) / 2);
  return (l % 2) ? (w >> 16) : (w & 0xffffu);
}

/* Replay in bfloat16 storage: W and H are arrays of bfloat16 bit patterns,
 * rows of k entries.  Per visit: h_j is widened to binary32, every rating of
 * the segment is applied in binary32 (same update as orc_sgd_update_f32) and
 * w_i is written back with stochastic rounding; at the end of the visit h_j
 * is written back with stochastic rounding.  visit_epoch[v] is the epoch of
 * visit v (it enters the rounding counters); the step size comes from the
 * per-record update count as in the other replays. */
int32_t orc_replay_bf16(int32_t k, float lambda, double alpha, double beta,
                        int64_t n_visits, const int64_t *visit_seg,
                        const int32_t *visit_epoch, int64_t n_seg,
                        const int64_t *seg_ptr, const int32_t *seg_col,
                        const int32_t *rec_row, const float *rec_val,
                        uint16_t *W, uint16_t *H, int32_t *rec_count,
                        uint64_t seed) {
  float *h = (float *)malloc(sizeof(float) * (size_t)k);
  float *w = (float *)malloc(sizeof(float) * (size_t)k);
  if (!h || !w) { free(h); free(w); return -2; }
  for (int64_t v = 0; v < n_visits; ++v) {
    const int64_t s = visit_seg[v];
    if (s < 0 || s >= n_seg) { free(h); free(w); return -1; }
    const uint32_t e = (uint32_t)visit_epoch[v];
    uint16_t *hb = H + (int64_t)seg_col[s] * k;
    for (int32_t l = 0; l < k; ++l) h[l] = orc_bf16_to_f32(hb[l]);
    for (int64_t r = seg_ptr[s]; r < seg_ptr[s + 1]; ++r) {
      uint16_t *wb = W + (int64_t)rec_row[r] * k;
      for (int32_t l = 0; l < k; ++l) w[l] = orc_bf16_to_f32(wb[l]);
      const float step = (float)orc_step_size(alpha, beta, rec_count[r]);
      orc_sgd_update_f32(k, w, h, rec_val[r], lambda, step);
      for (int32_t l = 0; l < k; ++l)
        wb[l] = orc_bf16_sr(w[l], sr_bits_w(seed, r, e, l));
      rec_count[r] += 1;
    }
    for (int32_t l = 0; l < k; ++l)
      hb[l] = orc_bf16_sr(h[l], sr_bits(seed, (uint32_t)s, e, 0u, 0x48000000u,
                                        l, 2));
  }
  free(h);
  free(w);
  return 0;
}

/* Array forms of the conversions above (for the Python side). */
void orc_bf16_rn_n(int64_t n, const float *x, uint16_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_rn(x[i]);
}
void orc_bf16_sr_n(int64_t n, const float *x, const uint32_t *r16, uint16_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_sr(x[i], r16[i]);
}
void orc_bf16_to_f32_n(int64_t n, const uint16_t *b, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_to_f32(b[i]);
}

/* ------------------------------------------------------------------------ */
/* FP8-E4M3 storage of W with one binary32 scale per row (a storage variant */
/* like the bfloat16 one; H stays binary32).                                */
/*                                                                          */
/* E4M3: sign, 4 exponent bits (bias 7), 3 mantissa bits.  Exponent field 0 */
/* holds the subnormals m * 2^-9 (m = 0..7); otherwise the value is         */
/* (1 + m/8) * 2^(E-7).  The largest finite magnitude is 448 (E=15, m=6);   */
/* E=15, m=7 is NaN; there is no infinity.                                  */
/*                                                                          */
/* Rounding of a binary32 x to E4M3 (sign kept, magnitude |x| rounded):    */
/*  - |x| >= 2^-6 (normal range): keep 3 of the 23 mantissa bits.  Nearest */
/*    (ties to even): add 0x7ffff plus the lowest kept bit, truncate.       */
/*    Stochastic with 16 random bits r: add r << 4 to the 20 dropped bits,   */
/*    truncate; the magnitude rounds up with probability (dropped bits      */
/*    >> 4) / 2^16.                                                          */
/*  - |x| < 2^-6: the grid is m * 2^-9.  With t = |x| * 2^9 and             */
/*    f = t - floor(t) (both exact in binary32): nearest rounds up when      */
/*    f > 1/2, or f = 1/2 with floor(t) odd; stochastic rounds up when        */
/*    r < f * 2^16.  m = 8 is the smallest normal, code 0x08.               */
/*  - Magnitudes above 448 after rounding, and infinities, become 448; NaN  */
/*    becomes the NaN code.                                                  */
/*                                                                          */
/* A row w (k binary32 entries) is stored as codes c_l and a scale s:      */
/*   a = max_l |w_l|; if a >= 2^-100: s = a / 448, g = 448 / a (binary32    */
/*   divisions), else s = 1, g = 1; c_l = round(w_l * g) (binary32 product). */
/* Its stored value is s * decode(c_l) (binary32 product).                  */
/* ------------------------------------------------------------------------ */
static uint8_t e4m3_from_rounded(uint32_t sign, uint32_t u) {
  /* u: a binary32 magnitude with at most 3 mantissa bits, >= 2^-6 */
  const int32_t e = (int32_t)((u >> 23) & 0xffu) - 127;
  if (e > 8 || (e == 8 && ((u >> 20) & 7u) == 7u)) return (uint8_t)(sign | 0x7eu);
  return (uint8_t)(sign | ((uint32_t)(e + 7) << 3) | ((u >> 20) & 7u));
}

static uint8_t e4m3_round(float x, int stochastic, uint32_t r16) {
  const uint32_t bits = f32_bits(x);
  const uint32_t sign = (bits >> 24) & 0x80u;
  uint32_t u = bits & 0x7fffffffu;
  if (u > 0x7f800000u) return (uint8_t)(sign | 0x7fu);  /* NaN */
  if (u == 0x7f800000u) return (uint8_t)(sign | 0x7eu); /* infinity saturates */
  if (u >= 0x3c800000u) {                                /* |x| >= 2^-6 */
    if (stochastic) u += (r16 & 0xffffu) << 4;
    else u += 0x7ffffu + ((u >> 20) & 1u);
    u &= ~0xfffffu;
    return e4m3_from_rounded(sign, u);
  }
  const float t = bits_f32(u) * 512.0f;
  const float lo = floorf(t);
  const float f = t - lo;
  uint32_t m = (uint32_t)lo;
  int up;
  if (stochastic) up = (float)(r16 & 0xffffu) < f * 65536.0f;
  else up = f > 0.5f || (f == 0.5f && (m & 1u));
  if (up) m += 1u;
  return (uint8_t)(sign | m); /* m <= 8: code m (8 is the smallest normal) */
}

uint8_t orc_e4m3_rn(float x) { return e4m3_round(x, 0, 0u); }
uint8_t orc_e4m3_sr(float x, uint32_t r16) { return e4m3_round(x, 1, r16); }

float orc_e4m3_to_f32(uint8_t c) {
  const uint32_t e = (c >> 3) & 15u, m = c & 7u;
  float v;
  if (e == 15u && m == 7u) v = NAN;
  else if (e == 0u) v = ldexpf((float)m, -9);
  else v = ldexpf(1.0f + (float)m / 8.0f, (int)e - 7);
  return (c & 0x80u) ? -v : v;
}

/* Codes and scale of a row (r16 = NULL: round to nearest). */
void orc_e4m3_row(int32_t k, const float *w, const uint32_t *r16, uint8_t *codes,
                  float *scale) {
  float a = 0.0f;
  for (int32_t l = 0; l < k; ++l) a = fmaxf(a, fabsf(w[l]));
  float s = 1.0f, g = 1.0f;
  if (a >= 0x1p-100f) {
    s = a / 448.0f;
    g = 448.0f / a;
  }
  for (int32_t l = 0; l < k; ++l)
    codes[l] = r16 ? orc_e4m3_sr(w[l] * g, r16[l]) : orc_e4m3_rn(w[l] * g);
  *scale = s;
}

/* Replay with W in E4M3 codes plus a binary32 scale per row and H in
 * binary32: per rating, w_i is decoded (scale * value), the update of
 * orc_sgd_update_f32 is applied, and w_i is re-encoded with stochastic
 * rounding (the 16 random bits of entry l as for the bfloat16 W); h_j is
 * updated in place in binary32. */
int32_t orc_replay_e4m3(int32_t k, float lambda, double alpha, double beta,
                        int64_t n_visits, const int64_t *visit_seg,
                        const int32_t *visit_epoch, int64_t n_seg,
                        const int64_t *seg_ptr, const int32_t *seg_col,
                        const int32_t *rec_row, const float *rec_val,
                        uint8_t *Wc, float *Ws, float *H, int32_t *rec_count,
                        uint64_t seed) {
  float *w = (float *)malloc(sizeof(float) * (size_t)k);
  uint32_t *r16 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
  if (!w || !r16) { free(w); free(r16); return -2; }
  for (int64_t v = 0; v < n_visits; ++v) {
    const int64_t s = visit_seg[v];
    if (s < 0 || s >= n_seg) { free(w); free(r16); return -1; }
    const uint32_t e = (uint32_t)visit_epoch[v];
    float *h = H + (int64_t)seg_col[s] * k;
    for (int64_t r = seg_ptr[s]; r < seg_ptr[s + 1]; ++r) {
      const int64_t i = rec_row[r];
      uint8_t *c = Wc + i * k;
      for (int32_t l = 0; l < k; ++l) w[l] = Ws[i] * orc_e4m3_to_f32(c[l]);
      const float step = (float)orc_step_size(alpha, beta, rec_count[r]);
      orc_sgd_update_f32(k, w, h, rec_val[r], lambda, step);
      for (int32_t l = 0; l < k; ++l)
        r16[l] = sr_bits_w(seed, r, e, l);
      orc_e4m3_row(k, w, r16, c, &Ws[i]);
      rec_count[r] += 1;
    }
  }
  free(w);
  free(r16);
  return 0;
}

/* Array forms for the Python side. */
void orc_e4m3_rn_n(int64_t n, const float *x, uint8_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3_rn(x[i]);
}
void orc_e4m3_sr_n(int64_t n, const float *x, const uint32_t *r16, uint8_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3_sr(x[i], r16[i]);
}
void orc_e4m3_to_f32_n(int64_t n, const uint8_t *c, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3_to_f32(c[i]);
}
void orc_e4m3_rows(int64_t rows, int32_t k, const float *w, const uint32_t *r16,
                   uint8_t *codes, float *scale) {
  for (int64_t i = 0; i < rows; ++i)
    orc_e4m3_row(k, w + i * k, r16 ? r16 + i * k : NULL, codes + i * k, scale + i);
}
