/*
 * nomad.h -- C ABI of libnomad, a GB300 (sm_103a) implementation of the SGD
 * hot path of NOMAD (Yun, Yu, Hsieh, Vishwanathan, Dhillon, "NOMAD:
 * Non-locking, stOchastic Multi-machine algorithm for Asynchronous and
 * Decentralized matrix completion", arXiv 1312.0193).
 *
 * The library learns W (m x k) and H (n x k) with A ~ W H^T over the observed
 * ratings Omega (Sec. 2) by per-rating SGD (Sec. 2.3) under NOMAD's ownership
 * passing schedule (Sec. 3.1, Alg. 1): users are split into p row blocks,
 * each owned by one worker (one warp of a persistent kernel); each item
 * vector h_j is a token owned by exactly one worker at a time and handed
 * between workers through device-resident queues.
 *
 * Conventions for every entry point:
 *  - Indices are 0-based int32; m, n < 2^31; nnz < 2^32.
 *  - Pointers are plain host or device addresses, as the `device_ptrs`
 *    argument says (1 = device memory of the handle's device, 0 = host
 *    memory, pinned or pageable).  The library copies what it needs; the
 *    caller keeps ownership of its buffers and may reuse them on return
 *    (for device inputs: once the work queued on `stream` has passed).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - The handle owns all device memory it allocates (cudaMalloc) and frees it
 *    in nomad_destroy.  A handle is not thread-safe: one host thread at a
 *    time.
 *  - Return value: NOMAD_OK (0) or a negative NOMAD_ERR_* code; the text of
 *    the last error of a handle is available from nomad_last_error_message.
 */
#ifndef NOMAD_H_
#define NOMAD_H_

#include <stdint.h>

#if defined(__GNUC__)
#define NOMAD_API __attribute__((visibility("default")))
#else
#define NOMAD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define NOMAD_OK 0
#define NOMAD_ERR_INVALID_ARG (-1) /* bad size, pointer, mode or order of calls */
#define NOMAD_ERR_OOM (-2)         /* device or host allocation failed */
#define NOMAD_ERR_DUP_ENTRY (-3)   /* a pair (i,j) occurs twice: Omega is a set (Sec. 2) */
#define NOMAD_ERR_TIMEOUT (-4)     /* a worker waited longer than spin_timeout_ns for a token */
#define NOMAD_ERR_OWNERSHIP (-5)   /* debug check: an item token held by two workers */
#define NOMAD_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define NOMAD_ERR_RANGE (-7)       /* an index is outside [0,m) or [0,n) */
#define NOMAD_ERR_UNSUPPORTED (-8) /* shape or option the library does not handle */
#define NOMAD_ERR_STATE (-9)       /* e.g. nomad_epoch before nomad_load_ratings */

/* ---------------------------------------------------------------- options */
/* Routing of an item token after a visit (Sec. 3.1 / Alg. 1 / Sec. 3.4). */
#define NOMAD_MODE_EPOCH 0   /* permutation circulation: in every epoch item j
                                visits each worker that holds ratings of j
                                exactly once, in a fresh pseudo-random order
                                (Sec. 3.4); t of Eq. stepsize_method is the
                                epoch index */
#define NOMAD_MODE_UNIFORM 1 /* Alg. 1 literally: the next worker is uniform
                                over all p workers; a per-rating counter gives
                                t; one "epoch" is |Omega| updates */

#define NOMAD_FP32 0 /* W, H stored in binary32 */
#define NOMAD_BF16 1 /* W, H stored in bfloat16, FP32 arithmetic, stochastic
                        rounding on write-back */
#define NOMAD_FP8 2  /* W stored as FP8-E4M3 codes with one binary32 scale
                        per row (scale = the row's largest magnitude / 448),
                        H in binary32; FP32 arithmetic; W rounded
                        stochastically at every update.  The paper has no
                        such format: this is the capacity variant for the
                        largest shapes (Hugewiki-sized W: 5 GB instead of
                        20 GB).  Batched epoch-mode kernel only. */

#define NOMAD_PARTITION_RATINGS 0 /* blocks with equal numbers of ratings
                                     (footnote of Sec. 3.1) */
#define NOMAD_PARTITION_USERS 1   /* blocks with equal numbers of users
                                     (Sec. 3.1) */

#define NOMAD_VARIANT_BATCHED 0 /* a worker takes up to 16 ready tokens at once,
                                   streams W rows through shared memory
                                   (default) */
#define NOMAD_VARIANT_SIMPLE 1  /* a worker handles one token at a time */

/* Epoch mode, batched kernel: how a token circulates (Sec. 3.4). */
#define NOMAD_CIRCULATION_FLAT 0  /* every worker holding ratings of the item
                                     once per epoch, in one keyed
                                     pseudo-random order over all of them */
#define NOMAD_CIRCULATION_BLOCK 1 /* the hybrid of Sec. 3.4: the token visits
                                     all of its workers inside one thread
                                     block (the workers of one SM) before it
                                     moves to another block, blocks in a keyed
                                     order and the workers of a block in a
                                     second keyed order; a hand-over inside a
                                     block goes through a shared-memory inbox
                                     of the receiving warp instead of the
                                     global ring (the global ring when the
                                     inbox is full) */

/* Uniform mode: choice of the next worker (Alg. 1 / Sec. 3.3). */
#define NOMAD_ROUTING_UNIFORM 0  /* uniform over all p workers (Alg. 1) */
#define NOMAD_ROUTING_SHORTER 1  /* of two workers drawn uniformly, the one with
                                    fewer tokens waiting in its queue (dynamic
                                    load balancing, Sec. 3.3) */

#define NOMAD_COO 0 /* rating input as (row, col, value) triples */
#define NOMAD_CSC 1 /* rating input as column pointers + row indices */

/* Schedule and hyper-parameters.  Fill with nomad_schedule_default first. */
typedef struct nomad_schedule {
  float alpha;      /* step size s_t = alpha / (1 + beta t^1.5), Sec. 5.1 */
  float beta;       /* Eq. stepsize_method; Table 1 gives (alpha, beta) */
  int32_t mode;     /* NOMAD_MODE_* */
  int32_t precision;/* NOMAD_FP32, NOMAD_BF16 or NOMAD_FP8 */
  int32_t partition;/* NOMAD_PARTITION_* */
  int32_t n_workers;/* p; 0 = every warp the persistent kernel can keep
                       resident on the device */
  int32_t warps_per_block; /* 0 = library default */
  int32_t debug;    /* 1 = record the serial visit order (replay log),
                       per-rating update counts and item-ownership checks */
  uint64_t seed;    /* factor initialisation, routing and rounding draws */
  int64_t spin_timeout_ns; /* a worker that waits longer than this for a
                       token stops and nomad_epoch reports NOMAD_ERR_TIMEOUT;
                       0 = 10 s */
  int32_t device;   /* CUDA device ordinal */
  int32_t debug_drop_item; /* testing only: item id whose token is never
                       handed to a worker in nomad_epoch (a planted lost
                       message); -1 = none */
  int32_t variant;  /* epoch-mode worker kernel: NOMAD_VARIANT_* */
  int32_t routing;  /* uniform mode: NOMAD_ROUTING_* */
  int32_t circulation; /* epoch mode, batched kernel: NOMAD_CIRCULATION_* */
  int32_t batch_tokens; /* batched kernel: most tokens a worker takes from
                       its queues at once, 1..16; 0 = 16 for k <= 128, 8
                       above (larger values are capped there) */
  int32_t epochs_per_launch; /* epoch mode: 0 or 1 = one kernel launch per
                       epoch, so every token finishes epoch e before any
                       token starts e+1 (the epochs of the permutation
                       circulation, Sec. 3.4, stay in step; the default);
                       n > 1 = up to n epochs in one launch, tokens free to
                       run epochs ahead of each other (no end-of-epoch wait,
                       but the descent per epoch is slower on skewed data) */
  int32_t reserved32;
  int64_t reserved[3];
} nomad_schedule;

typedef struct nomad_handle nomad_t;

/* Facts about a handle (sizes of the layout built by nomad_load_ratings). */
typedef struct nomad_info {
  int64_t m, n;
  int32_t k;
  int32_t p;               /* number of workers (row blocks) */
  int64_t nnz;             /* training ratings loaded */
  int64_t n_segments;      /* non-empty sets Omega-bar_j^(q) (Sec. 3.1) */
  int64_t epochs_done;     /* epochs completed since load / set_factors */
  int32_t pitch;           /* row pitch of W and H on the device, elements */
  int32_t precision;
  int32_t mode;
  int32_t warps_per_block;
  int32_t blocks;          /* persistent grid size */
  int32_t sm_count;
  int64_t device_bytes;    /* device memory held by the handle */
  int64_t kernel_launches; /* kernels launched by the handle so far */
  int64_t predrawn_ratings; /* ratings whose W rounding bits are drawn before
                               each launch (see nomad_load_ratings); 0 = none */
  int64_t reserved[2];
} nomad_info;

/* Library defaults: alpha 0.012, beta 0.05 (Table 1, Netflix), epoch mode,
 * FP32, ratings-balanced partition, automatic p, seed 1, 10 s timeout. */
NOMAD_API void nomad_schedule_default(nomad_schedule *s);

/* Create a problem with m users, n items, rank k and regularisation lambda
 * (Eq. obj_fcn).  Allocates and initialises W and H with independent
 * UniformReal(0, 1/sqrt(k)) entries (Alg. 1, Sec. 5.1).  1 <= k <= 512.
 * On success *out is a new handle; on failure *out is NULL. */
NOMAD_API int nomad_create(int64_t m, int64_t n, int32_t k, float lambda,
                 const nomad_schedule *s, nomad_t **out);

/* Load the training ratings and build the layout of Sec. 3.1: rows split
 * into p blocks I_q, and for every worker q the sets Omega-bar_j^(q) of its
 * ratings of item j, stored as a compressed per-worker CSC (only non-empty
 * columns), rows ascending inside a set.  The data are never moved again.
 *  fmt NOMAD_COO: major = const int32_t rows[nnz], minor = cols[nnz].
 *  fmt NOMAD_CSC: major = const int64_t colptr[n+1], minor = rows[nnz].
 *  vals = const float[nnz].
 * Errors: NOMAD_ERR_RANGE (index out of range), NOMAD_ERR_DUP_ENTRY.
 * Synchronises with the device before returning.  May be called again to
 * replace the ratings (the factors are kept).
 * With NOMAD_BF16 or NOMAD_FP8 storage (batched kernel, epoch mode, k <=
 * 128) it may also reserve 8 ceil(k/4) bytes per rating of the items with
 * the most ratings (at least half the largest item degree): their W
 * rounding bits are then drawn there before each one-epoch launch, off the
 * chains of visits of those items.  Only when those ratings are at most a
 * quarter of all and the reservation fits in a quarter of the free device
 * memory and 32 GiB; otherwise the kernel draws the bits itself.
 * nomad_get_info's device_bytes includes the reservation. */
NOMAD_API int nomad_load_ratings(nomad_t *h, int32_t fmt, int64_t nnz, const void *major,
                       const int32_t *minor, const float *vals,
                       int32_t device_ptrs, void *stream);

/* Run n_epochs epochs of NOMAD (Alg. 1) in persistent launches (one per
 * epoch, or schedule.epochs_per_launch epochs each): every worker pops item
 * tokens from its queue, applies the SGD updates of Eq. w_update / h_update
 * to its ratings of that item, and hands the token on.  In NOMAD_MODE_EPOCH
 * every rating is updated exactly once per epoch.
 * Asynchronous on `stream`; errors raised on the device (timeout, ownership)
 * are reported by the next nomad_check / nomad_rmse / nomad_objective /
 * nomad_get_factors call. */
NOMAD_API int nomad_epoch(nomad_t *h, int32_t n_epochs, void *stream);

/* nomad_epoch for `count` independent problems at once: per epoch one
 * persistent launch (or per the first handle's epochs_per_launch) in which
 * each problem runs on its own blocks (h[g]->n_workers
 * workers, i.e. its schedule's n_workers / warps_per_block blocks), as in a
 * sweep over lambda, k or data (App. A/B).  The problems share no data; each
 * one's updates, visit order, replay log and errors are those nomad_epoch
 * would give with the same workers.
 *  - h: `count` distinct loaded handles on the same device, all in
 *    NOMAD_MODE_EPOCH with NOMAD_VARIANT_BATCHED, the same precision, the
 *    same debug flag, the same warps_per_block and the same row width class
 *    (k <= 128, k <= 256 or k <= 512); the caller keeps the array.
 *  - Their blocks together must fit on the device at once (one block of
 *    warps_per_block warps per SM with the default shared memory use):
 *    otherwise NOMAD_ERR_UNSUPPORTED and nothing runs.
 *  - Asynchronous on `stream`; per-handle errors as for nomad_epoch, and
 *    nomad_last_epoch_kernel_ms of every handle reports the call's
 *    launches (first start to last end).
 * Errors: NOMAD_ERR_INVALID_ARG (count < 1, a NULL or repeated handle,
 * n_epochs < 1), NOMAD_ERR_STATE (a handle without ratings),
 * NOMAD_ERR_UNSUPPORTED (handles that differ in the above, or too many
 * blocks). */
NOMAD_API int nomad_epoch_many(nomad_t *const *h, int32_t count, int32_t n_epochs,
                               void *stream);

/* Device time span, in nanoseconds, of the handle's workers in its last
 * nomad_epoch / nomad_epoch_many call with the batched variant: from the
 * first worker's start to the last worker's end (the device's global
 * timer).  In a nomad_epoch_many launch this is the handle's own problem,
 * which is how a caller sees which problem the launch waited for.  Waits for
 * the handle's work on `stream`.  *ns = 0 when no such call has run (or the
 * simple variant or uniform mode ran). */
NOMAD_API int nomad_last_epoch_span_ns(nomad_t *h, int64_t *ns, void *stream);

/* Wait for the handle's work on `stream` and report any device-side error
 * of earlier nomad_epoch calls (then clears it). */
NOMAD_API int nomad_check(nomad_t *h, void *stream);

/* Test RMSE (Sec. 5.1) over nnz ratings: sqrt(sum (A_ij - <w_i,h_j>)^2 /
 * nnz).  Products and residuals in binary32, sums in binary64.  Writes the
 * result to *out (host).  Synchronous.  nnz = 0 gives NaN. */
NOMAD_API int nomad_rmse(nomad_t *h, int64_t nnz, const int32_t *rows,
               const int32_t *cols, const float *vals, int32_t device_ptrs,
               double *out, void *stream);

/* Objective J(W,H) of Eq. obj_fcn over the loaded training ratings:
 * 1/2 sum_Omega [ (A_ij - <w_i,h_j>)^2 + lambda (|w_i|^2 + |h_j|^2) ],
 * per-rating terms in binary32, sums in binary64.  Synchronous. */
NOMAD_API int nomad_objective(nomad_t *h, double *out, void *stream);

/* Copy the factors out as dense row-major binary32 arrays W[m*k], H[n*k]
 * (BF16 storage is widened exactly; an E4M3 row is scale * code value, one
 * binary32 product per entry).  Either pointer may be NULL.  Synchronous. */
NOMAD_API int nomad_get_factors(nomad_t *h, float *W, float *H, int32_t device_ptrs,
                      void *stream);

/* Replace the factors (checkpoint resume); epochs_done is set to
 * `epochs_done` so that the step-size schedule continues from there.
 * BF16 storage rounds to nearest; E4M3 storage takes each row's scale from
 * its largest magnitude and rounds the codes to nearest.  Either pointer may
 * be NULL. Synchronous. */
NOMAD_API int nomad_set_factors(nomad_t *h, const float *W, const float *H,
                      int32_t device_ptrs, int64_t epochs_done, void *stream);

/* Device time in milliseconds of the persistent NOMAD kernel of the last
 * nomad_epoch call, from CUDA events recorded on that call's stream right
 * before and after the launch.  Waits for the second event. */
NOMAD_API int nomad_last_epoch_kernel_ms(nomad_t *h, float *ms);

/* Sizes and settings of the handle. */
NOMAD_API int nomad_get_info(const nomad_t *h, nomad_info *out);

/* Host copies of the layout built by nomad_load_ratings, each pointer may be
 * NULL: row_worker[m] (the block of every user), seg_worker[S], seg_col[S],
 * seg_ptr[S+1] (record offsets), rec_row[nnz], rec_val[nnz] (records in
 * segment order).  S = nomad_info.n_segments.  Synchronous. */
NOMAD_API int nomad_get_layout(nomad_t *h, int32_t *row_worker, int32_t *seg_worker,
                     int32_t *seg_col, int64_t *seg_ptr, int32_t *rec_row,
                     float *rec_val);

/* Debug mode only (schedule.debug = 1): the serial visit order of the last
 * nomad_epoch call.  Visits are ordered by a ticket each worker takes right
 * after it pops a token; that order is a valid serialisation (two visits that
 * share an item or a worker are ordered as they happened).  seg[v] is the
 * segment (index into the layout) and epoch[v] the epoch of visit v.  Writes
 * min(cap, count) entries and the total count to *count.  Synchronous. */
NOMAD_API int nomad_get_replay_log(nomad_t *h, int64_t cap, int32_t *seg, int32_t *epoch,
                         int64_t *count);

/* Debug mode only: per-record update counts since load (records in segment
 * order) and the number of ownership violations seen.  Synchronous. */
NOMAD_API int nomad_get_debug_counts(nomad_t *h, int32_t *rec_count,
                           int64_t *ownership_violations);

/* Largest number of 8192-rating tiles nomad_rmse_noalloc can reduce: its
 * partial sums live in a fixed __device__ array of this many doubles
 * (512 KiB, held by every GPU that loads the library until exit). */
#define NOMAD_NOALLOC_MAX_TILES 65536

/* Test RMSE for callers that cannot let the library allocate memory (the
 * paper has no counterpart: this serves deployment, not the method).  For
 * example a service that reserves all device memory up front, or a loop that
 * must not take the implicit device synchronisation of cudaMalloc/cudaFree.
 * It needs no handle and calls no allocator: everything is caller memory
 * except a fixed scratch array inside the library.
 *  W (m x pitch), H (n x pitch): binary32 factors in device memory, row
 *    major, entries 0..k-1 of each row used; 1 <= k <= 512, pitch >= k.
 *  rows, cols, vals: nnz test ratings in device memory.
 *  out: one double in device memory; receives sqrt(sum (A_ij -
 *    <w_i,h_j>)^2 / nnz) (binary32 residuals, binary64 sums), or NaN when
 *    nnz is 0 or an index lies outside [0,m) x [0,n).
 * The result equals nomad_rmse's on the same factors up to the order of the
 * binary64 additions (within about 1e-6 relative), and is the same from call
 * to call for the same inputs.
 * Asynchronous on `stream` (a cudaStream_t as void*), on the current device.
 * Rejects nnz > NOMAD_NOALLOC_MAX_TILES * 8192 (536,870,912) with
 * NOMAD_ERR_INVALID_ARG.  The first call on a device looks up the scratch
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is looked up again after the
 * device's context changes (e.g. after cudaDeviceReset).  All calls share
 * the scratch array: calls whose work may overlap on the GPU (unordered
 * streams) race and must not be issued.  A CUDA error already pending when
 * the call starts (from the caller's earlier work) makes it return
 * NOMAD_ERR_CUDA without launching anything; the pending error is left for
 * the caller to read. */
NOMAD_API int nomad_rmse_noalloc(const float *W, const float *H, int64_t m,
                                 int64_t n, int32_t k, int64_t pitch,
                                 int64_t nnz, const int32_t *rows,
                                 const int32_t *cols, const float *vals,
                                 double *out, void *stream);

/* Free every resource of the handle (NULL is ignored). */
NOMAD_API void nomad_destroy(nomad_t *h);

/* Static text for an error code. */
NOMAD_API const char *nomad_error_string(int32_t code);

/* Text of the last error of the handle ("" if none). */
NOMAD_API const char *nomad_last_error_message(const nomad_t *h);

#ifdef __cplusplus
}
#endif

#endif /* NOMAD_H_ */
