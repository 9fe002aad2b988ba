/*
 * ldpc.h - C ABI of the GB300 (sm_103a) LDPC belief-propagation decoding library.
 *
 * The library decodes many codewords of a quasi-cyclic LDPC code at once on one GPU:
 * check-node update, variable-node update, a-posteriori LLR sum, hard decision and
 * syndrome early exit (Amiri & Mehrpouyan, arXiv 1812.06545: Sec. II decoding
 * algorithms, Algorithm 1 loop order; Sec. III-A frame-level parallelism over F frames;
 * Sec. III-B interleaving of frames; Sec. III-C concurrent streams).
 *
 * Conventions shared by every entry point
 *   - LLR sign: L = ln P(c = 0) / P(c = 1); BPSK maps bit 0 to +1.  Hard decision
 *     c = [APP < 0] (an APP of exactly zero decodes to 0).
 *   - User layouts are row-major per codeword: llr[n_cw][N], bits[n_cw][N] (one byte per
 *     bit, values 0/1), iters[n_cw], app[n_cw][N].
 *   - Device pointers are CUDA device (or managed) memory owned by the caller; host
 *     pointers are host memory owned by the caller (pinned memory lets copies overlap).
 *   - Decoding is asynchronous on the caller's CUDA stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream).  Argument errors are reported synchronously
 *     before anything is launched; CUDA launch errors return LDPC_ECUDA.
 *   - The library owns ldpc_code objects and its own internal buffers; nothing the
 *     caller passes in is retained after a call returns (except inside the stream's
 *     queued work, which the caller must keep alive until the stream reaches it).
 *   - No C++ exception crosses this interface.  ldpc_last_error() returns a message for
 *     the calling thread's most recent failure.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDPC_OK = 0,
    LDPC_EINVAL = -1,    /* bad argument: null pointer, bad size, bad code, bad params  */
    LDPC_ENOMEM = -2,    /* host or device allocation failed, or workspace too small    */
    LDPC_ECUDA = -3,     /* a CUDA call or launch failed                                */
    LDPC_EBUSY = -4,     /* resource in use                                             */
    LDPC_ETIMEDOUT = -5, /* a bounded wait ran out                                      */
    LDPC_ENOTSUP = -6    /* combination not supported (e.g. code too large for a form)  */
} ldpc_status;

typedef enum { LDPC_SCHED_FLOODING = 0, LDPC_SCHED_LAYERED = 1 } ldpc_schedule;
typedef enum { LDPC_ALGO_SPA = 0, LDPC_ALGO_NMS = 1 } ldpc_algo;
typedef enum { LDPC_MSG_F32 = 0, LDPC_MSG_F16 = 1, LDPC_MSG_I8 = 2 } ldpc_msg_type;
typedef enum { LDPC_LLR_F32 = 0, LDPC_LLR_I8 = 1 } ldpc_llr_type;
typedef enum {
    LDPC_IMPL_AUTO = 0,     /* the fastest kernels for the requested form: for flooding, the */
                            /* on-chip slot decoder when one codeword's posterior and        */
                            /* messages fit in shared memory, else the cluster decoder when  */
                            /* they fit two SMs, else the streaming kernels                  */
    LDPC_IMPL_PLAIN = 1,    /* the plain FP32 flooding comparator (one codeword per thread,  */
                            /* library expm1f/log1pf phi, state streamed through HBM)        */
    LDPC_IMPL_STREAMING = 2, /* flooding with all state streamed through HBM in the         */
                             /* codeword-interleaved layout (check-node and variable-node   */
                             /* kernels per iteration); layered min-sum with a fixed group  */
                             /* of codewords per CTA instead of persistent refilled slots   */
    LDPC_IMPL_CLUSTER = 3    /* flooding SPA on the cluster decoder: one codeword per two-SM */
                             /* thread-block cluster, its rows and columns split between the */
                             /* two CTAs' shared memories (AUTO uses it when a codeword does */
                             /* not fit one CTA but fits a cluster)                          */
} ldpc_impl;

/* Opaque code object (library-owned, immutable after creation, usable from any thread). */
typedef struct ldpc_code ldpc_code;

/* Decoder parameters.  Supported forms:
 *   sched FLOODING + algo SPA + msg F32 or F16  (sum-product; Algorithm 1 order)
 *   sched LAYERED  + algo SPA + msg F32 or F16  (sum-product on the layered schedule of
 *                                                "Algorithm 2": block rows in order, each
 *                                                computed from the current posteriors and
 *                                                updating them at once; impl AUTO only, for
 *                                                codes whose slot fits in shared memory)
 *   sched LAYERED  + algo NMS + msg I8          (bit-exact integer normalised min-sum)
 * Every field must be set; ldpc_default_params() fills the defaults below. */
typedef struct {
    int32_t sched;           /* ldpc_schedule; default FLOODING                               */
    int32_t algo;            /* ldpc_algo; default SPA                                        */
    int32_t msg;             /* ldpc_msg_type; default F32                                    */
    int32_t max_iter;        /* >= 1; default 20                                              */
    int32_t early_exit;      /* 0/1: stop a codeword once H.c = 0 after an iteration (1)      */
    float phi_clamp;         /* X > 1: |Q| is clamped to [phi(X), X] before phi (80.0)        */
    int32_t nms_alpha_num;   /* min-sum scaling (alpha_num * mag) >> alpha_shift (3)          */
    int32_t nms_alpha_shift; /* (2): alpha = 0.75                                             */
    int32_t msg_sat;         /* min-sum message saturation, 1..127 (31)                       */
    int32_t app_sat;         /* min-sum posterior saturation, msg_sat..127 (127)              */
    float llr_scale;         /* fp32 LLR quantiser q = sat(rint(llr_scale * L)) (2.0)         */
    int32_t impl;            /* ldpc_impl (AUTO)                                              */
    int32_t reserved[4];     /* must be zero                                                  */
} ldpc_decode_params;

/* Fill *p with the defaults listed above.  Returns LDPC_EINVAL if p is NULL. */
ldpc_status ldpc_default_params(ldpc_decode_params *p);

/* Create a code from a QC base matrix (Sec. II, Eq. 1 gives H as an edge set between
 * check and variable nodes; the quasi-cyclic lifting defines H block by block).
 *   base  host pointer, row-major int32 [mb][nb], copied; entry -1 = zero block, entry
 *         s in [0, Z) = Z x Z identity shifted so that row r has its one in column
 *         (r + s) mod Z.  Check l*Z + r therefore joins variable j*Z + (r + s_lj) mod Z.
 *   Limits: 1 <= mb < nb, mb <= 64, nb <= 128, 1 <= Z <= 1024, nonzero blocks <= 1024,
 *   every block row holds >= 2 nonzero blocks, every block column >= 1.
 * Returns LDPC_EINVAL on a bad matrix (shift out of range, empty row, mb >= nb), LDPC_ENOMEM
 * or LDPC_ECUDA if the device tables cannot be created.  *out is set only on success. */
ldpc_status ldpc_code_create(const int32_t *base, int32_t mb, int32_t nb, int32_t Z, ldpc_code **out);

/* Destroy a code (NULL is ignored).  Work already queued with it must have completed. */
void ldpc_code_destroy(ldpc_code *code);

/* Query sizes: N = nb*Z variables, K = N - M, M = mb*Z checks, E = edges.  Any output
 * pointer may be NULL. */
ldpc_status ldpc_code_info(const ldpc_code *code, int32_t *N, int32_t *K, int32_t *M, int64_t *E);

/* Device workspace needed by ldpc_decode_batch for n_cw codewords with these params. */
ldpc_status ldpc_workspace_size(const ldpc_code *code, const ldpc_decode_params *p, int64_t n_cw,
                                size_t *bytes);

/* Decode n_cw codewords (Sec. II: Algorithm 1 loop order for the flooding schedule,
 * "Algorithm 2" for the layered schedule; Sec. III-A: all codewords in parallel).
 *   llr_dev    device, [n_cw][N], fp32 (LDPC_LLR_F32) or int8 already quantised to
 *              [-msg_sat, msg_sat] (LDPC_LLR_I8, layered NMS only).  fp32 input to the
 *              layered NMS form is quantised with p->llr_scale inside the library.
 *   bits_dev   device, [n_cw][N] uint8 0/1 hard decisions after the last iteration run.
 *   iters_dev  device, [n_cw] int32: iterations run (1..max_iter).
 *   app_dev    device, [n_cw][N] fp32 posterior LLRs after the last iteration, or NULL
 *              (integer forms write their integer APP converted exactly to fp32).
 *   workspace  device scratch of >= ldpc_workspace_size() bytes, 256-byte aligned, or NULL
 *              to let the library allocate and free it stream-ordered on `stream`.
 * n_cw == 0 returns LDPC_OK with nothing launched. */
ldpc_status ldpc_decode_batch(const ldpc_code *code, const ldpc_decode_params *p,
                              const void *llr_dev, int32_t llr_type, int64_t n_cw,
                              uint8_t *bits_dev, int32_t *iters_dev, float *app_dev,
                              void *workspace, size_t workspace_bytes, void *stream);

/* Choose, by timing, the schedule ldpc_decode_batch / ldpc_decode_multi use for this code
 * and form with impl AUTO, and remember it in the code object.
 *   Flooding forms: the on-chip slot decoder with one or two codewords per thread (where
 *   the code fits), or the HBM-streaming kernels.  Layered min-sum: persistent slots with one
 *   codeword per thread (32-bit integer arithmetic) or two per thread (packed half-precision
 *   integer arithmetic, offered when it is exact for the params: every message magnitude
 *   (alpha_num * msg_sat) >> alpha_shift <= 127 and 2 * alpha_num * msg_sat +
 *   2^alpha_shift <= 2047), or the fixed group per CTA.  Untuned, AUTO takes two per thread
 *   where offered.  The layered sum-product has one schedule: LDPC_ENOTSUP.
 *   llr_dev / llr_type / n_cw  a representative device sample of the workload (>= 1 codeword).
 *   choice     receives the pick: 1 slots (1 codeword per thread), 2 slots (2 per thread),
 *              3 streaming / fixed group (may be NULL).
 *   ms         receives up to 3 candidate times in milliseconds, -1 for absent candidates,
 *              in the order slots-1, slots-2, streaming (may be NULL).
 * Synchronizes `stream` and allocates temporary device buffers; call it at set-up, before
 * decoding with the code from other threads. */
ldpc_status ldpc_autotune(ldpc_code *code, const ldpc_decode_params *p, const void *llr_dev, int32_t llr_type,
                          int64_t n_cw, void *stream, int32_t *choice, float *ms);

/* One decode request of a mixed-code launch (caller-owned device buffers, layouts as in
 * ldpc_decode_batch). */
typedef struct {
    const ldpc_code *code;
    const void *llr_dev;   /* [n_cw][N]: fp32, or int8 for the layered form with LDPC_LLR_I8 */
    int64_t n_cw;          /* >= 0 (0: skipped)                                            */
    uint8_t *bits_dev;     /* [n_cw][N]                                                    */
    int32_t *iters_dev;    /* [n_cw]                                                       */
    float *app_dev;        /* [n_cw][N] or NULL                                            */
} ldpc_request;

/* Decode several requests, possibly of different codes, in one persistent launch (Sec. III-A
 * frame-level parallelism extended across codes).  Every codeword of every request is an item
 * of a work queue: requests of one code form a group with its own counter, CTAs start on
 * groups in proportion to their work and move to the group with the most work left once
 * theirs runs dry, and a codeword's slot is refilled the moment it converges.  A codeword
 * decodes to exactly the same result as in ldpc_decode_batch (alone or in any mix).
 *   reqs       host array of n_req <= 128 requests over <= 16 distinct codes, all decoded
 *              with the same params (impl must be AUTO; every code must fit the form's
 *              on-chip decoders: a slot of one CTA, or for flooding a two-SM cluster -
 *              ldpc_decode_batch with LDPC_IMPL_STREAMING serves larger codes).
 *   llr_type   applies to every request.
 *   workspace  >= ldpc_multi_workspace_size() bytes of device memory (work counters),
 *              256-byte aligned, or NULL for a stream-ordered allocation on `stream`.
 * The flooding forms run all slot-sized requests in one launch and the requests of each
 * cluster-sized code in one launch per code; the layered min-sum runs the requests of each
 * code in one launch per code; the layered sum-product issues one persistent launch per
 * request.  All launches go on `stream`. */
ldpc_status ldpc_decode_multi(const ldpc_request *reqs, int32_t n_req, const ldpc_decode_params *p,
                              int32_t llr_type, void *workspace, size_t workspace_bytes, void *stream);

/* Device workspace bytes ldpc_decode_multi needs (independent of the requests). */
ldpc_status ldpc_multi_workspace_size(size_t *bytes);

/* Multi-stream host-to-host decoding (Sec. III-C: W streams, each decoding its own set
 * of frames so that copies and kernels of different sets overlap).
 *   llr_host   host, [n_cw][N] fp32 (pinned memory recommended).
 *   bits_host  host, [n_cw][N] uint8;  iters_host host [n_cw] int32 (may be NULL).
 *   n_streams  W >= 1; the batch is cut into chunks of at most chunk_cw codewords
 *              (chunk_cw <= 0: n_cw / W rounded up) issued round-robin over W internal
 *              streams, each chunk being H2D copy -> decode -> D2H copy on its stream.
 * Blocks until every chunk has finished.  Device buffers are owned by the library and
 * kept for reuse between calls on the same thread. */
ldpc_status ldpc_decode_host(const ldpc_code *code, const ldpc_decode_params *p, const float *llr_host,
                             int64_t n_cw, uint8_t *bits_host, int32_t *iters_host, int32_t n_streams,
                             int64_t chunk_cw);

/* ------------------------------------------------------------------ serving loop
 *
 * A session decodes requests submitted from any host thread, continuously batching them
 * onto the GPU (Sec. III-C: several sets of frames in flight on their own streams).  A
 * dispatcher thread keeps up to max_inflight launches going; whenever one finishes (or a
 * request arrives while a slot is free) it admits the head of the FIFO queue together with
 * the queued requests that share its parameter set (at most max_batch requests over at most
 * 16 codes, as the remaining device-memory budget allows; no request overtakes one waiting
 * for memory), and issues them on their own stream as: host-to-device
 * copies, one persistent multi-request decode (the codewords of every admitted request are
 * items of one work queue; codes the on-chip decoders cannot hold are decoded alone), and
 * device-to-host copies.  A request's result does not depend on what it was batched with. */
typedef struct ldpc_session ldpc_session;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory for request buffers, reserved at creation (>= 1 MiB) */
    int32_t max_inflight;     /* concurrent launches / streams, 1..16 (default 4)                    */
    int32_t max_batch;        /* requests per launch, 1..128 (default 128)                           */
    int32_t start_paused;     /* 1: admit nothing until ldpc_session_pause(s, 0)                     */
    int32_t fail_alloc_after; /* fault injection: the n-th buffer allocation fails (0: off); that     */
                              /* request finishes with LDPC_ENOMEM and the session carries on         */
    int32_t reserved[4];      /* zero                                                                */
} ldpc_session_config;

typedef struct {
    int64_t submitted, completed, failed, cancelled, queued, launches;
    size_t budget_bytes, bytes_in_use, peak_bytes; /* request-buffer memory of the arena */
} ldpc_session_stats;

/* Request states reported by ldpc_session_poll. */
enum { LDPC_REQ_QUEUED = 0, LDPC_REQ_RUNNING = 1, LDPC_REQ_DONE = 2, LDPC_REQ_FAILED = 3, LDPC_REQ_CANCELLED = 4 };

ldpc_status ldpc_session_default_config(ldpc_session_config *cfg);

/* Create a session on the current device: reserves hbm_budget_bytes of device memory and
 * starts the dispatcher thread. */
ldpc_status ldpc_session_create(const ldpc_session_config *cfg, ldpc_session **out);

/* Queue n_cw >= 1 codewords of `code` for decoding with params *p.
 *   llr_host   host [n_cw][N] fp32 LLRs; bits_host host [n_cw][N]; iters_host [n_cw] or NULL.
 *              Caller-owned; they must stay valid until the request is reported finished
 *              (pinned memory lets the copies overlap the decoding of other requests).
 *   req_id     receives the request's id.
 * Returns LDPC_ENOMEM if the request alone exceeds the memory budget, LDPC_EINVAL /
 * LDPC_ENOTSUP for bad arguments; nothing is queued then. */
ldpc_status ldpc_session_submit(ldpc_session *s, const ldpc_code *code, const ldpc_decode_params *p,
                                const float *llr_host, int64_t n_cw, uint8_t *bits_host, int32_t *iters_host,
                                uint64_t *req_id);

/* Non-blocking status: *state receives LDPC_REQ_*.  Once a finished state is reported the
 * request's record is released (its id becomes unknown) and the return value is the
 * request's own status (LDPC_OK, or e.g. LDPC_ENOMEM / LDPC_ECUDA for a failed request);
 * *latency_s then receives the time from submission to completion. */
ldpc_status ldpc_session_poll(ldpc_session *s, uint64_t req_id, int32_t *state, double *latency_s);

/* Block until the request finishes (then as ldpc_session_poll) or timeout_s elapses
 * (LDPC_ETIMEDOUT, record kept). */
ldpc_status ldpc_session_wait(ldpc_session *s, uint64_t req_id, double timeout_s, double *latency_s);

/* Cancel a queued request (LDPC_EBUSY once it is on the GPU; finished ones are left alone). */
ldpc_status ldpc_session_cancel(ldpc_session *s, uint64_t req_id);

/* Stop (paused = 1) or restart (0) admitting queued requests; launches in flight finish. */
ldpc_status ldpc_session_pause(ldpc_session *s, int32_t paused);

ldpc_status ldpc_session_stats_get(ldpc_session *s, ldpc_session_stats *out);

/* Stop the dispatcher, wait for launches in flight and free the session (queued requests
 * are dropped). */
void ldpc_session_destroy(ldpc_session *s);

/* Release the device buffers and streams ldpc_decode_host keeps for the calling thread. */
void ldpc_release_host_buffers(void);

/* Per-kernel timing: when enabled, every kernel the library launches is bracketed by CUDA
 * events on its launch stream; ldpc_profile_read returns, per kernel family, the number
 * of launches and the summed event time in milliseconds (it synchronizes the pending
 * events).  Families: 0 interleave, 1 check-node, 2 variable-node, 3 deinterleave,
 * 4 layered min-sum, 5 plain check-node, 6 plain variable-node, 7 on-chip flooding slot
 * decoder, 8 on-chip layered sum-product slot decoder. */
ldpc_status ldpc_profile_enable(int32_t on);
ldpc_status ldpc_profile_read(int32_t family, int64_t *launches, double *ms);
ldpc_status ldpc_profile_reset(void);

/* Measured special-function throughput of the current device in operations per second:
 * independent ex2.approx and lg2.approx chains on every SM (the units the exponentials and
 * logarithms of the sum-product check rule run on).  Synchronizes `stream`; allocates 4 bytes. */
ldpc_status ldpc_sfu_throughput(double *ex2_per_s, double *lg2_per_s, void *stream);

/* Device status word: the decoding kernels flag bad channel input without a host pass over
 * the data.  Bits: 1 = a non-finite fp32 LLR was decoded (NaN or infinity; the decode ran
 * on it as given), 2 = an int8 LLR outside [-msg_sat, msg_sat] was decoded (it was
 * saturated to the range).  The word is per device and shared by every stream and thread on
 * it.  ldpc_stream_check orders itself after the work queued on `stream`, takes the word
 * (swapping in zero, so no flag set concurrently is lost) and synchronizes the stream.
 *   flags  receives the bits taken (may be NULL).
 * Returns LDPC_OK when no bit was set, LDPC_EINVAL (with a message naming the bits) when
 * one was, LDPC_ECUDA if the stream or the copy failed.  Allocates nothing after the first
 * code was created on the device.  (An input check of the boundary; the paper's decoder has
 * no counterpart.) */
ldpc_status ldpc_stream_check(void *stream, uint32_t *flags);

/* Number of kernel launches the library has issued since the last reset (all families). */
int64_t ldpc_launch_count(void);
void ldpc_launch_count_reset(void);

/* Flooding decode that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory at decode time - for example a real-time receive pipeline that reserves all
 * of its memory at start-up (a cudaMalloc can synchronize the device and has no latency
 * bound), or a host process whose device memory is owned by another framework's pool.
 * It runs the same flooding sum-product kernels as ldpc_decode_batch, but their scratch
 * (interleaved LLRs, posteriors, messages and per-codeword flags) lives in one fixed
 * array of LDPC_STATIC_SCRATCH_BYTES bytes compiled into the library.  Every GPU that
 * loads the library holds that array until the process exits.
 *   - Same arguments and layouts as ldpc_decode_batch with llr_type LDPC_LLR_F32 and no
 *     workspace; only the flooding SPA forms (F32 / F16 messages) are accepted.
 *   - n_cw must satisfy ldpc_workspace_size(code, p, n_cw) <= LDPC_STATIC_SCRATCH_BYTES;
 *     larger batches are rejected with LDPC_ENOMEM before anything is launched (decode
 *     them in several calls).  With LDPC_IMPL_AUTO a code whose codeword state fits on
 *     chip needs only a few bytes of scratch, so any batch fits; with LDPC_IMPL_STREAMING
 *     or LDPC_IMPL_PLAIN the scratch grows in tiles of 128 codewords (up to 896 codewords
 *     of the N = 1944 rate-1/2 code with FP32 messages).
 *   - The first call on each device looks up the array's device address (with that device
 *     current) and keeps it; make that first call before any stream capture begins.  Under
 *     CUDA's lazy module loading (the default) that lookup is also what loads the part of
 *     the library holding the array, so the first call is the one that reserves the array's
 *     device memory (a failure there is reported as LDPC_ECUDA).  Make it at start-up, with
 *     a small batch; later calls reserve nothing.
 *   - All calls share the one array and it keeps whatever the last call left in it (the
 *     kernels initialise every part they read).  Calls whose work overlaps on the GPU -
 *     on different streams, or from different host threads without ordering - corrupt each
 *     other's scratch: issue them on one stream, or order them.
 * Returns LDPC_OK, LDPC_EINVAL / LDPC_ENOTSUP for bad arguments, LDPC_ENOMEM for a batch
 * beyond the array, LDPC_ECUDA for a failed address lookup or launch. */
#define LDPC_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
ldpc_status ldpc_decode_batch_static(const ldpc_code *code, const ldpc_decode_params *p, const float *llr_dev,
                                     int64_t n_cw, uint8_t *bits_dev, int32_t *iters_dev, float *app_dev,
                                     void *stream);

/* Message for the calling thread's most recent failure ("" if none).  Valid until the
 * thread's next call into the library. */
const char *ldpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */
