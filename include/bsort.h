/*
 * bsort.h -- C ABI of a GB300 (sm_103a) implementation of GPU Bucket Sort,
 * the deterministic sample sort of Dehne & Zaboli ("Deterministic Sample Sort
 * for GPUs", Section 4, Algorithm 1).
 *
 * The problem (Algorithm 1, "Input"/"Output"): an array A of n items in
 * global memory is to be sorted.  Every call below computes exactly the
 * sorted permutation: keys in nondecreasing order, and for key/value pairs
 * the stable order (equal keys keep their input order).  Steps 1-9 of
 * Algorithm 1 each run as hand-written CUDA kernels on one GPU; nothing here
 * falls back to the CPU.
 *
 * Conventions common to all entry points
 *   - Pointers named d_* are device pointers on the handle's device; h_* are
 *     host pointers.  The caller owns every key/value buffer and the stream.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Sort calls are asynchronous on that stream: they return
 *     after enqueueing work.  bsort_sync() waits and reports device-side
 *     errors.
 *   - Input and output may be the same buffer (in-place sort, as in the
 *     paper); otherwise they must not overlap.  The input is never modified
 *     when it differs from the output.
 *   - n = 0 and n = 1 are valid.  Key-value pairs, 64-bit keys, batches and
 *     served jobs take n < 2^32 - 2^16 (their positions are 32-bit on the
 *     device).  Keys-only sorts of 32-bit keys (bsort_sort_keys,
 *     bsort_sort_keys_host) take n up to 2^34, with a two-level plan above
 *     2^30 keys (see bsort_plan_info.levels; planner-chosen t, s and b
 *     only); such a call waits for its stream once, after Step 8, to read the
 *     b bucket sizes and plan the bucket sorts.  Larger n returns
 *     BSORT_EUNSUPPORTED.
 *   - A handle is not thread-safe; use one handle per host thread.  Calls on
 *     one handle must be ordered on one stream (they share its workspace).
 *   - Errors: argument and launch errors are returned directly.  A device
 *     consistency check or a bounded device wait that ran out sets a device
 *     error word; bsort_sync() returns it (BSORT_EINTERNAL / BSORT_ETIMEOUT)
 *     and clears it.  No kernel aborts, traps or spins without a limit.
 */
#ifndef BSORT_H
#define BSORT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsort_ctx *bsort_t;

typedef enum {
    BSORT_OK = 0,
    BSORT_EINVAL = 1,        /* bad argument (null pointer, bad size, bad flag) */
    BSORT_ENOMEM = 2,        /* workspace too small / device allocation failed */
    BSORT_ECUDA = 3,         /* a CUDA runtime call failed; see bsort_last_error */
    BSORT_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
    BSORT_EBUSY = 5,         /* the handle serves a request stream
                                (bsort_submit) and refuses other sort calls */
    BSORT_ENOTREADY = 6,     /* no completed call to report on */
    BSORT_EUNSUPPORTED = 7,  /* valid request that this library does not serve */
    BSORT_EINTERNAL = 8      /* a device-side consistency check failed */
} bsort_status;

typedef enum {
    BSORT_U32 = 0,  /* unsigned 32-bit keys */
    BSORT_F32 = 1,  /* IEEE binary32 keys, total order
                       -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN;
                       bit patterns are preserved */
    BSORT_U64 = 2   /* unsigned 64-bit keys: keys-only sorts (bsort_sort_keys,
                       bsort_sort_keys_host, batches, served jobs) and pairs
                       (bsort_sort_pairs: two stable passes of the 32-bit
                       pair sort, low key half first); not the
                       no-allocation entry (BSORT_EUNSUPPORTED) */
} bsort_key_type;

/* bsort_config.buckets: let the planner choose b for the given t and s. */
#define BSORT_BUCKETS_AUTO 0xFFFFFFFFu

/* Flags for bsort_config.flags. */
#define BSORT_FLAG_TIMING 0x1u   /* record CUDA events between the kernels of
                                    every call; see bsort_kernel_times() */
#define BSORT_FLAG_LOW_MEMORY 0x2u /* do not materialise the relocated array
                                      of Step 8: Step 9 gathers its items from
                                      the runs A_ij of the sorted sublists
                                      directly.  Same result; the workspace
                                      shrinks by n'*(key+value) bytes, at some
                                      cost in speed; BSORT_IM_RELOCATED is then
                                      not available */
#define BSORT_FLAG_GRAPHS 0x4u     /* bsort_sort_keys / bsort_sort_pairs
                                      capture their launch sequence as a CUDA
                                      graph the first time they see a call
                                      (key type, value bytes, n, the four
                                      buffer pointers, the stream, the
                                      workspace) and replay it with one graph
                                      launch when the same call repeats (new
                                      contents in the same buffers are fine);
                                      the handle keeps the 16 most recent
                                      graphs and drops them all when its
                                      workspace moves.  Not combined with
                                      BSORT_FLAG_TIMING (no kernel times are
                                      recorded for captured calls); calls on
                                      the legacy default stream (NULL), or on
                                      a stream that is already capturing,
                                      are issued as usual */
#define BSORT_FLAG_TEST_STALL_SCAN 0x10u /* test of the bounded device
                                      waits, for 32-bit keys that need
                                      sampling: Step 7 runs as the
                                      decoupled look-back scan (the form
                                      batches use; sorts otherwise scan
                                      each bucket row on its own, with no
                                      waits) and its first chunk never
                                      publishes its prefix, so the waits of
                                      later chunks
                                      give up after a few thousand polls; the
                                      call then stops after Step 7 (the
                                      offsets are wrong, so Steps 8-9 are not
                                      run and the output is not written) and
                                      bsort_sync returns BSORT_ETIMEOUT.
                                      Device-buffer calls only (EINVAL for
                                      bsort_sort_keys_host).  Never set it
                                      otherwise */
#define BSORT_FLAG_PLAN_MODEL 0x20u /* plan every sort with the analytic
                                      cost model, also where a measured
                                      (t, s) is tabled for n's size class
                                      (keys-only 32-bit sorts); kept to
                                      compare the two */
#define BSORT_FLAG_TEST_TWO_LEVEL 0x40u /* test of the two-level plan:
                                      keys-only 32-bit sorts of more than
                                      65536 keys take it at any size, with
                                      top-level buckets of about 2^16 keys
                                      (so that small inputs exercise it);
                                      never set it otherwise */
#define BSORT_FLAG_MERGE_SORT 0x8u /* keys-only 32-bit sorts: a unit of
                                      32768 keys sorted by one CTA (a Step-9
                                      bucket unit, a Step-2 sublist of
                                      t = 32768) is sorted by comparisons
                                      (register networks and merges) instead
                                      of by 7-bit digits over the bits that
                                      vary in the unit (the default).  Same
                                      result; kept to measure one against the
                                      other */

typedef struct {
    int device;                /* CUDA device ordinal the handle works on */
    uint64_t mem_budget_bytes; /* library-owned workspace: if > 0 and
                                  workspace == NULL, allocated once at create;
                                  a job that needs more returns BSORT_ENOMEM.
                                  0 with workspace == NULL: the library grows
                                  its workspace on demand (cudaMalloc). */
    void *workspace;           /* caller-owned device workspace (may be NULL);
                                  when set, the library never allocates device
                                  memory and must not outlive it */
    uint64_t workspace_bytes;  /* size of workspace */
    uint32_t tile;             /* t = n/m of Step 1 (0 = planner's choice) */
    uint32_t samples;          /* s of Step 3 (0 = planner's choice) */
    uint32_t flags;            /* BSORT_FLAG_* */
    uint32_t buckets;          /* b, the number of buckets of Steps 5-9
                                  (0 = b = s when samples is given, else the
                                  planner's choice; BSORT_BUCKETS_AUTO = the
                                  planner's choice also when samples is
                                  given); the splitters are the
                                  sorted samples of rank floor((j+1)ms/b) - 1,
                                  which for b = s is the paper's S[(j+1)m - 1]
                                  (Section 4, Step 5).  1 <= b <= m*s and
                                  b <= 12288, else EINVAL / EUNSUPPORTED. */
    uint32_t batch_direct_max; /* bsort_sort_batch: largest segment sorted
                                  whole by one CTA or cluster (0 = 131072;
                                  at most 262144) */
    uint32_t pad_;
    uint64_t serve_budget_bytes; /* bsort_submit: device memory of the request
                                  loop (0 = 4 GiB): half (at most 15 GiB)
                                  holds admitted requests' keys, the rest is
                                  split between the workspaces of its two
                                  lanes */
} bsort_config;

/* The plan of one job (Step 1 parameters and the Step-9 unit). */
typedef struct {
    uint64_t n;              /* items */
    uint64_t n_padded;       /* n' = m * t (the last sublist padded) */
    uint32_t t;              /* sublist size n/m (Step 1) */
    uint32_t s;              /* samples per sublist (Step 3) */
    uint32_t m;              /* number of sublists */
    uint32_t w;              /* t / s, distance between samples (Step 3) */
    uint64_t bucket_bound;   /* max |B_j| = ceil(ms/b) w + (m-1)(w-1); for
                                b = s this is n'/s + (m-1)(w-1) <= 2n'/s */
    uint32_t tile_ctas;      /* CTAs that sort one sublist (Step 2) */
    uint32_t unit_ctas;      /* CTAs that sort one bucket (Step 9) */
    uint64_t unit_capacity;  /* items one Step-9 unit holds (>= bucket_bound) */
    uint32_t single_tile;    /* 1: n fits one unit, sorted directly */
    uint32_t num_kernels;    /* kernel launches per call */
    uint64_t workspace_bytes;/* device workspace this job needs */
    uint32_t b;              /* buckets (Steps 5-9); b = s is the paper's rule */
    uint32_t unit_small;     /* when unit_ctas > 1: buckets of at most this
                                many items are sorted by one CTA each, the
                                others by a unit of unit_ctas CTAs (0: one
                                tier) */
    uint32_t levels;         /* 1; 2 above 2^30 keys (keys-only 32-bit keys,
                                planner's t/s/b): Step 9 sorts each of the b
                                buckets, at most bucket_bound keys, by a
                                plan of its own */
    uint32_t pad_;
} bsort_plan_info;

/* The plan of one batch (bsort_plan_batch). */
typedef struct {
    uint64_t n;               /* keys in all segments */
    uint32_t num_segs;
    uint32_t direct_segs;     /* sorted whole by one CTA or cluster */
    uint32_t sampled_segs;    /* sorted by segment-aware Algorithm 1 */
    uint32_t large_segs;      /* above 524288 32-bit or 1048576 64-bit keys:
                                 one plain sort each */
    uint32_t sublists;        /* sublists of the sampled segments */
    uint32_t buckets;         /* buckets of the sampled segments */
    uint32_t num_kernels;     /* kernel launches per call */
    uint32_t pad_;
    uint64_t workspace_bytes; /* device workspace the batch needs */
} bsort_batch_info;

/* Intermediates of the last call (for parity checks), see bsort_get_intermediate. */
typedef enum {
    BSORT_IM_TILES = 0,      /* Step 2: sorted sublists, n' keys (transformed
                                key domain for F32), sublist-major */
    BSORT_IM_SAMPLES = 1,    /* Step 3: m*s records (key << 32 | p), p = i*t + r,
                                sublist-major; for BSORT_U64 two uint64 words
                                per record (key, p) */
    BSORT_IM_SPLITTERS = 2,  /* Step 5: b records g_0..g_{b-1} (same format) */
    BSORT_IM_COUNTS = 3,     /* Step 6: a_ij, uint32, bucket-major a[j*m + i], m*b */
    BSORT_IM_OFFSETS = 4,    /* Step 7: l_ij, uint32, bucket-major, m*b */
    BSORT_IM_RELOCATED = 5   /* Step 8: n' keys B_1 ... B_b (not with
                                BSORT_FLAG_LOW_MEMORY) */
} bsort_intermediate;

/* Create a handle on cfg->device.  cfg may be NULL (device 0, on-demand
 * workspace, planner's t and s).  Returns BSORT_ENOMEM if mem_budget_bytes
 * cannot be allocated. */
bsort_status bsort_create(const bsort_config *cfg, bsort_t *out);

/* Release the handle and any workspace the library allocated.  Waits for
 * no stream; the caller must make sure no call is in flight. */
bsort_status bsort_destroy(bsort_t h);

/* Compute the plan for sorting n items of key type kt (val_bytes = 0 for
 * keys only, 4 or 8 for pairs).  Host-only; touches no device memory. */
bsort_status bsort_plan(bsort_t h, bsort_key_type kt, uint32_t val_bytes,
                        uint64_t n, bsort_plan_info *out);

/* Algorithm 1 on n keys: d_keys_out receives the keys in nondecreasing
 * order.  Returns BSORT_ENOMEM if the workspace cannot hold the job. */
bsort_status bsort_sort_keys(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                             void *d_keys_out, uint64_t n, void *cuda_stream);

/* Algorithm 1 on n (key, value) pairs, stable: equal keys keep their input
 * order.  val_bytes is 4 or 8; values are moved, never interpreted. */
bsort_status bsort_sort_pairs(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              const void *d_vals_in, void *d_keys_out,
                              void *d_vals_out, uint32_t val_bytes, uint64_t n,
                              void *cuda_stream);

/* Batched sort (no counterpart in the paper, which sorts one array):
 * num_segs independent arrays, segment q = keys [seg_offsets[q],
 * seg_offsets[q+1]) of d_keys_in, each sorted on its own into the same
 * range of d_keys_out (d_keys_out == d_keys_in allowed).  seg_offsets is
 * HOST memory, num_segs + 1 nondecreasing values, the last below 2^32 -
 * 2^16; keys outside every segment are left untouched.  Segments up to
 * batch_direct_max keys are sorted whole by one CTA or thread-block cluster
 * (as Step 9 sorts a bucket); larger ones up to 524288 keys by Algorithm 1
 * (Section 4) with segment-aware sublists (32768 keys), s = 1024 samples
 * per sublist and per-segment splitters, all segments together in one
 * sequence of launches; larger ones by one plain sort each.  The segment
 * table is copied to the device from pinned staging owned by the handle.
 * kt: BSORT_U32, BSORT_F32 or BSORT_U64 (64-bit keys: segments up to
 * 262144 keys, or batch_direct_max when given, sorted whole — above 131072
 * by a 16-CTA cluster, where the device schedules one, else the limit is
 * 131072 —, larger ones up to 1048576 keys by the segment-aware Algorithm 1
 * with sublists of 16384 keys and s = 256 samples per sublist (128 above
 * 32 sublists), larger ones one plain sort each).  Errors: EINVAL (null
 * pointers, decreasing offsets, partial overlap), EUNSUPPORTED (too many
 * keys), ENOMEM. */
bsort_status bsort_sort_batch(bsort_t h, bsort_key_type kt, const void *d_keys_in,
                              void *d_keys_out, const uint64_t *seg_offsets,
                              uint32_t num_segs, void *cuda_stream);

/* ---- Served stream (no counterpart in the paper) ------------------------
 * bsort_submit queues one independent sort job; a request loop owned by the
 * handle (one worker thread, started by the first submit) admits queued
 * jobs while its device arena has room (the serving budget,
 * bsort_config.serve_budget_bytes) and copies their keys in.  Small jobs
 * (up to 524288 32-bit or 1048576 64-bit keys: those bsort_sort_batch sorts
 * whole or by its segment-aware sample sort) are admitted in arrival order
 * and sorted together as a batch (bsort_sort_batch's path) as soon as the
 * previous small batch has finished sorting, on a high-priority stream;
 * jobs that arrive meanwhile are copied in and form the next batch
 * (continuous batching).  Larger jobs are admitted in arrival order, at most
 * four at a time, and sorted one at a time on a low-priority stream with a
 * workspace of their own, so small jobs are not held behind them.  Every job's result is
 * exactly the sort of its keys.  Once a handle has served a request its
 * plain sort calls return BSORT_EBUSY. */
typedef struct {
    bsort_key_type key_type;  /* BSORT_U32, BSORT_F32 or BSORT_U64 */
    uint32_t pad_;
    uint64_t n;               /* keys */
    const void *h_keys_in;    /* host memory (pinned for asynchronous copies);
                                 must stay valid until the job is polled */
    void *h_keys_out;         /* host memory for the sorted keys (may equal
                                 h_keys_in) */
} bsort_request;

typedef struct {
    bsort_status status;      /* BSORT_OK, or the failure of the job */
    uint32_t batch_size;      /* jobs sorted in the same batch */
    uint64_t submit_ns;       /* bsort_clock_ns() at bsort_submit */
    uint64_t start_ns;        /* when its batch was launched */
    uint64_t done_ns;         /* when its sorted keys were in h_keys_out */
} bsort_result;

typedef struct {
    uint64_t arena_bytes;      /* device bytes for admitted jobs' keys */
    uint64_t workspace_bytes;  /* workspace of the batches */
    uint64_t arena_used_bytes; /* in use now */
    uint64_t arena_peak_bytes; /* most ever in use (<= arena_bytes) */
    uint64_t queued;           /* submitted, waiting for arena room */
    uint64_t completed;        /* jobs finished */
    uint64_t batches;          /* batches launched */
    uint64_t max_batch;        /* most jobs in one batch */
    uint64_t large_jobs;       /* jobs sorted one at a time (large lane) */
    uint64_t worker_busy_ns;   /* time the request loop spent working */
} bsort_serve_info;

/* Queue one job; *ticket identifies it for bsort_poll.  Errors: EINVAL,
 * ENOMEM (the job alone exceeds the arena or the workspace), and the
 * errors of starting the loop (ENOMEM, ECUDA). */
bsort_status bsort_submit(bsort_t h, const bsort_request *req, uint64_t *ticket);

/* Non-blocking: BSORT_ENOTREADY while the job runs; BSORT_OK once its keys
 * are in h_keys_out, with *out filled (the ticket is then released);
 * BSORT_EINVAL for an unknown ticket. */
bsort_status bsort_poll(bsort_t h, uint64_t ticket, bsort_result *out);

/* Non-blocking: up to cap finished jobs, in completion order, each with its
 * ticket and result, released as by bsort_poll; *count receives how many
 * (0 when none has finished). */
bsort_status bsort_poll_any(bsort_t h, uint64_t *tickets, bsort_result *results, uint32_t cap,
                            uint32_t *count);

/* Counters of the request loop (all zero before the first submit). */
bsort_status bsort_serve_stats(bsort_t h, bsort_serve_info *out);

/* The clock of bsort_result (a monotonic clock, nanoseconds). */
uint64_t bsort_clock_ns(void);

/* The plan bsort_sort_batch would use for these segments.  Host-only. */
bsort_status bsort_plan_batch(bsort_t h, bsort_key_type kt, const uint64_t *seg_offsets,
                              uint32_t num_segs, bsort_batch_info *out);

/* bsort_sort_keys on HOST buffers: copies h_keys_in to the device, sorts,
 * and copies the result back into h_keys_out, all ordered on cuda_stream
 * (the copies are part of the call; h_keys_out is complete once the work
 * issued on cuda_stream so far has finished).  Pinned host memory gives
 * asynchronous copies.  For 32-bit keys over several sublists the copies
 * overlap the sort from 2^23 keys on: the keys go in as chunks of whole
 * sublists (one per 8 MiB, at most 16), Steps 1-3 starting on each chunk
 * once it has arrived, and Step 9 runs in as many groups of units by output
 * position, each group's slice of h_keys_out copied out while the next
 * group sorts (on a copy stream of the handle, ordered against cuda_stream
 * by events).  Uses extra workspace: the device copy of
 * the keys (n * key bytes, rounded up to 256) plus 256 bytes. */
bsort_status bsort_sort_keys_host(bsort_t h, bsort_key_type kt, const void *h_keys_in,
                                  void *h_keys_out, uint64_t n, void *cuda_stream);

/* Wait for cuda_stream, then return and clear the device error word:
 * BSORT_OK, BSORT_ETIMEOUT or BSORT_EINTERNAL. */
bsort_status bsort_sync(bsort_t h, void *cuda_stream);

/* Copy one intermediate of the last sort call into host memory (waits for
 * the device).  bytes must equal the intermediate's size for that call's
 * plan; intermediates that the plan skipped (single_tile) give
 * BSORT_ENOTREADY. */
bsort_status bsort_get_intermediate(bsort_t h, bsort_intermediate which,
                                    void *h_dst, uint64_t bytes);

/* With BSORT_FLAG_TIMING: milliseconds spent in each kernel launch, in
 * launch order, summed over the calls made since the previous
 * bsort_kernel_times (at most the last 64 calls, and only those with the same
 * launch sequence as the last call; *calls receives how many were summed).
 * Waits for the last call.  *written receives the number of entries
 * (<= count).  bsort_kernel_name(h, i) names entry i of the last call. */
bsort_status bsort_kernel_times(bsort_t h, float *ms, uint32_t count,
                                uint32_t *written, uint32_t *calls);
const char *bsort_kernel_name(bsort_t h, uint32_t index);

/* Largest n that bsort_sort_keys_noalloc accepts. */
#define BSORT_NOALLOC_MAX_KEYS (1ull << 20)

/* Keys-only sort that allocates nothing, for callers that cannot allocate
 * device memory: code running where cudaMalloc is not allowed or not wanted
 * (inside a memory pool that must not grow, under a strict memory budget, in
 * a plugin whose host owns every allocation).  It needs no handle.  The paper
 * has no counterpart: this is a packaging of the same sort.
 *
 * It sorts n <= BSORT_NOALLOC_MAX_KEYS (2^20) uint32 or float32 keys on the
 * current CUDA device (kt = BSORT_U32 or BSORT_F32), from d_keys_in into
 * d_keys_out (the same buffer or disjoint), with the same result as
 * bsort_sort_keys.  Its scratch memory is one fixed array of 12 MiB inside
 * the library, which every GPU that loads the library keeps until the
 * process exits.  The first call in a CUDA context (per device, and again
 * after a device reset) looks up that array's device address
 * (cudaGetSymbolAddress) and sets the kernels' attributes; make that first
 * call before any stream capture.  The call makes no cudaMalloc, cudaFree or
 * other allocating call.  Every call uses the same array, so calls whose
 * work overlaps on the GPU (on different streams, or from different threads)
 * race and corrupt each other; order them on one stream.
 *
 * Returns BSORT_EINVAL for n > BSORT_NOALLOC_MAX_KEYS, a null or partially
 * overlapping pointer, or a key type other than U32/F32 (BSORT_EUNSUPPORTED
 * for U64).  The call is asynchronous on cuda_stream; with wait != 0 it
 * waits for the stream and also returns the device error status
 * (BSORT_ETIMEOUT / BSORT_EINTERNAL) recorded since the last call that
 * reported one: this call's, or that of an earlier call made with wait = 0
 * (whose status is kept, not lost, until such a call reads and clears it). */
bsort_status bsort_sort_keys_noalloc(bsort_key_type kt, const void *d_keys_in,
                                     void *d_keys_out, uint64_t n, void *cuda_stream,
                                     int wait);

/* Last error message on this handle (never NULL). */
const char *bsort_last_error(bsort_t h);

/* Name of a status code (never NULL). */
const char *bsort_status_string(bsort_status st);

#ifdef __cplusplus
}
#endif

#endif /* BSORT_H */
