/*
 * gbfft.h -- C ABI of the GB300 batched complex FFT library.
 *
 * The library executes the DFT problem dft(N, V, I, O) of Johnson & Frigo,
 * "Implementing FFTs in Practice", sec. 4.1: a loop over the vector I/O
 * tensor V (the "howmany" dimensions) of rank-|N| complex DFTs whose
 * dimensions are the I/O dimensions of the size tensor N.  Each 1-D DFT is
 * eq. (1) of sec. 2, Y[k] = sum_{l<n} X[l] w^{l k}, with
 * w = exp(sign * 2 pi i / n); sign = -1 is the paper's forward transform
 * and sign = +1 the unnormalised backward transform (so a forward then a
 * backward transform multiplies the data by the product of the lengths).
 * A multi-dimensional DFT is the separable product over its dimensions.
 *
 * Data are complex64: interleaved FP32 (re, im) pairs, 8 bytes per element.
 * All strides are in complex elements (not bytes) and may be negative; a
 * pointer argument addresses element 0 of its array.
 *
 * The interface follows the paper's "lowest-common-denominator" rule for a
 * numerical library (sec. 7): plain C types, no language-specific objects.
 * Plans are created once (sec. 4: problems, algorithmic steps, planner) and
 * executed many times; they do not depend on the data pointers.
 *
 * Threading: plan creation and destruction may be called from any host
 * thread; fft_execute on one plan must not run concurrently from two host
 * threads.  The last error is per host thread.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- types */

/* An I/O dimension (n, is, os), sec. 4.1: length n >= 0, input stride is,
 * output stride os, both counted in complex elements. */
typedef struct {
    int64_t n;
    int64_t is;
    int64_t os;
} fft_iodim;

/* Opaque plan handle (sec. 4: a composition of algorithmic steps). */
typedef struct fft_plan_s *fft_plan;

/* ---------------------------------------------------------------- errors */

enum {
    FFT_OK = 0,
    FFT_ERR_INVALID_ARG = 1,      /* bad rank, length, sign, flag or NULL pointer */
    FFT_ERR_UNSUPPORTED = 2,      /* valid problem outside this library's limits */
    FFT_ERR_ALIAS = 3,            /* input and output overlap without FFT_INPLACE */
    FFT_ERR_INPLACE_MISMATCH = 4, /* FFT_INPLACE with is != os, or in != out */
    FFT_ERR_OOM = 5,              /* device allocation failed */
    FFT_ERR_BUDGET = 6,           /* a byte budget (serving, group) was exceeded */
    FFT_ERR_CUDA = 7,             /* a CUDA runtime call failed */
    FFT_ERR_DEVICE_TIMEOUT = 8,   /* a bounded device-side wait gave up */
    FFT_ERR_WISDOM = 9,           /* malformed wisdom, or FFT_WISDOM_ONLY without an entry */
    FFT_ERR_NO_DEVICE = 10,       /* no usable CUDA device */
    FFT_ERR_OUTPUT_OVERLAP = 11   /* the output map is not injective */
};

/* ---------------------------------------------------------------- flags */

#define FFT_MEASURE 0u             /* default: time candidate plans on the device (sec. 4.3) */
#define FFT_ESTIMATE (1u << 0)     /* heuristic plan, no timing (sec. 4.3, "estimate mode") */
#define FFT_WISDOM_ONLY (1u << 1)  /* use only imported wisdom; fail otherwise */
#define FFT_INPLACE (1u << 2)      /* executed with in == out; requires is == os everywhere */
#define FFT_EXTERNAL_SCRATCH (1u << 3) /* no plan-owned scratch: pass a work area to fft_execute_scratch */
#define FFT_PREC_TC_FP16 (1u << 4) /* radix-16 stages as FP16 tensor-core MMAs */
#define FFT_PREC_TC_BF16 (1u << 5) /* radix-16 stages as BF16 tensor-core MMAs */
#define FFT_PREC_SPLIT (1u << 6)   /* with a TC flag: split operands (FP16 hi+lo, BF16 hi+mid+lo) */
/* Testing only: the plan's first step is one device wait, bounded at 50 ms,
 * on an mbarrier nothing arrives on.  It runs out and records
 * FFT_ERR_DEVICE_TIMEOUT in the plan's status word exactly as a kernel whose
 * tile copy never landed would (see fft_sync_status); nothing faults and the
 * transform itself still runs. */
#define FFT_DEBUG_STALL (1u << 11)

/* ---------------------------------------------------------------- plans */

/*
 * fft_plan_dft -- plan dft(N, V, I, O) (sec. 4.1).
 *   rank, dims             : the size tensor N, rank in [0, 3]; rank 0 is a
 *                            copy (sec. 4.1.1, "a size-1 DFT is a copy")
 *   howmany_rank, howmany_dims : the vector tensor V, rank in [0, 3]
 *   sign                   : -1 forward, +1 backward (eq. (1)); else error
 *   flags                  : FFT_* bits above
 * The arrays are read, not kept.  Any length 0 gives an empty problem whose
 * plan executes as a no-op.  Length-1 dimensions are dropped and vector
 * dimensions that form one stride run are merged (canonical form).
 * Returns NULL on error and sets fft_last_error(): INVALID_ARG,
 * OUTPUT_OVERLAP (two index tuples write one output element),
 * INPLACE_MISMATCH, UNSUPPORTED, WISDOM, OOM, CUDA or NO_DEVICE.
 * Planning uses the current CUDA device and allocates the plan's twiddle
 * tables and scratch there; the plan owns them until fft_destroy.
 */
fft_plan fft_plan_dft(int rank, const fft_iodim *dims, int howmany_rank,
                      const fft_iodim *howmany_dims, int sign, unsigned flags);

/*
 * fft_plan_dft_r2c / fft_plan_dft_c2r -- DFTs of real data (sec. 5: the
 * real-input specialisation saves about a factor of two; sec. 7: real-data
 * transforms as part of the library's generality).  The problem is
 * dft(N, V, I, O) of a real array:
 *   r2c: real input x (FP32), complex64 output Y[k] = sum_l x[l] w^{l k}
 *        (sign -1, eq. (1) over every dimension) for the indices whose last
 *        component k_last <= n_last / 2 (integer division): the
 *        non-redundant half of the conjugate-symmetric spectrum, so the last
 *        output dimension has n_last / 2 + 1 entries;
 *   c2r: complex64 input holding such a half spectrum, real output
 *        y[l] = Re( sum_{k_last <= n_last/2} c(k_last) X[k] w^{-l k} ), c = 1
 *        for k_last = 0 and (n_last even) k_last = n_last / 2, else 2 -- the
 *        unnormalised backward transform of the conjugate-symmetric extension
 *        (c2r(r2c(x)) = prod(n) x); the imaginary parts of the
 *        self-conjugate planes k_last = 0, n_last / 2 drop out.
 * dims[i] = (n, is, os) with n the real (logical) length; strides count
 * elements of the array they step through: FP32 values on the real side,
 * complex64 values on the complex side (so the last complex dimension has
 * n_last / 2 + 1 entries along its stride).  howmany_dims likewise.
 *   rank in [1, 3], howmany_rank in [0, 3]; flags: FFT_ESTIMATE,
 *   FFT_WISDOM_ONLY, FFT_DEBUG_STALL (FFT_INPLACE, FFT_EXTERNAL_SCRATCH and
 *   the tensor-core flags return FFT_ERR_UNSUPPORTED).
 * Execute with fft_execute(plan, in, out, stream): in and out do not
 * overlap; element 0 of the real array must be 8-byte aligned (even
 * lengths with unit real stride read or write it as complex pairs).  The
 * input is not modified.  Errors as fft_plan_dft.
 */
fft_plan fft_plan_dft_r2c(int rank, const fft_iodim *dims, int howmany_rank,
                          const fft_iodim *howmany_dims, unsigned flags);
fft_plan fft_plan_dft_c2r(int rank, const fft_iodim *dims, int howmany_rank,
                          const fft_iodim *howmany_dims, unsigned flags);

/*
 * fft_execute -- run a plan (sec. 4.2: the plan's steps, in order).
 *   in, out : device pointers to element 0 of complex64 arrays that cover
 *             every addressed element; caller-owned.  For an out-of-place
 *             plan the input is not modified and the footprints of in and
 *             out must not overlap (else FFT_ERR_ALIAS).  A plan made with
 *             FFT_INPLACE must be given in == out.
 *   stream  : a cudaStream_t (NULL = legacy default stream); the call only
 *             enqueues work and returns.
 * Returns FFT_OK or an error code (INVALID_ARG, ALIAS, INPLACE_MISMATCH,
 * CUDA); also reported by fft_last_error().  If an earlier execution of the
 * plan has left a device-side error in its status word that nobody collected
 * (visible to the host without synchronising, once that kernel has run), the
 * call returns it (FFT_ERR_DEVICE_TIMEOUT), clears it and enqueues nothing.
 */
int fft_execute(fft_plan p, const void *in, void *out, void *stream);

/*
 * fft_sync_status -- wait for the plan's last execution (the last
 * fft_execute / fft_execute_scratch not made during a stream capture) and
 * return its device-side status: FFT_OK, or FFT_ERR_DEVICE_TIMEOUT when one
 * of its kernels' bounded waits gave up (a tile copy or an MMA that did not
 * complete within 2 s); the status is cleared.  Every wait in the library's
 * kernels is bounded, so a stuck copy turns into this error, not a hang.
 * The status word is page-locked host memory mapped into the device.  Returns
 * FFT_ERR_INVALID_ARG for NULL and FFT_ERR_CUDA if the wait itself failed.
 */
int fft_sync_status(fft_plan p);

/*
 * fft_execute_scratch -- run a plan made with FFT_EXTERNAL_SCRATCH, using the
 * caller's device work area `scratch` (256-byte aligned, at least
 * fft_plan_scratch_bytes(p) bytes; may be NULL when that is 0) instead of
 * plan-owned scratch, so that one plan can run concurrently on several
 * streams with separate work areas.  Otherwise as fft_execute; plans with
 * external scratch must be run with this call (fft_execute returns
 * FFT_ERR_INVALID_ARG for them when they need scratch).
 */
int fft_execute_scratch(fft_plan p, const void *in, void *out, void *scratch, void *stream);

/* fft_destroy -- free a plan and its device memory; NULL is ignored.  The
 * caller must make sure no enqueued execution of the plan is still running. */
void fft_destroy(fft_plan p);

/* Error reporting: last error code of this host thread, and its text. */
int fft_last_error(void);
const char *fft_error_string(int code);

/*
 * fft_plan_info -- the printed plan tree (its steps, radices, tilings), a
 * NUL-terminated string.  Writes at most len bytes; returns the full length
 * (excluding the NUL) or -1 on error.
 */
int fft_plan_info(fft_plan p, char *buf, size_t len);

/*
 * fft_plan_explain -- the plan tree fft_plan_dft would build in estimate
 * mode, computed on the host only (no device, no allocation); same
 * arguments as fft_plan_dft plus the output buffer as in fft_plan_info.
 * Returns the full length, or -1 with fft_last_error() set.
 */
int fft_plan_explain(int rank, const fft_iodim *dims, int howmany_rank,
                     const fft_iodim *howmany_dims, int sign, unsigned flags, char *buf,
                     size_t len);

/* Algorithmic bytes of one execution: 16 bytes per transformed point
 * (8 read + 8 written), the unit used for the HBM roofline; for real-data
 * plans 4 bytes per real value plus 8 per complex value of the half
 * spectrum. */
double fft_plan_bytes(fft_plan p);

/* Flops of one execution under the 5 N log2 N convention (sec. 1); real-data
 * plans count half of it, 2.5 N log2 N. */
double fft_plan_flops(fft_plan p);

/* Number of kernel launches one fft_execute enqueues. */
int fft_plan_launches(fft_plan p);

/* Device scratch bytes the plan holds, or (FFT_EXTERNAL_SCRATCH) needs in the
 * caller's work area; excludes twiddle tables. */
size_t fft_plan_scratch_bytes(fft_plan p);

/* ---------------------------------------------------------------- tables */

/*
 * Twiddle and chirp tables (sec. 6: the accuracy of the transform rests on
 * twiddle factors computed to about machine precision from an exactly
 * reduced exponent; sec. 4.2.5: Bluestein's chirp, Rader's permutation).
 * These two calls expose, for checking, what the planner computes for one
 * table: fft_twiddle_exponents evaluates on the host the same inline integer
 * code the device generators run (gb_index.h) and writes the exponent of
 * every entry; fft_twiddle_table runs the device generator itself.  An entry
 * with exponent m holds w_N^m = exp(-2 pi i m / N) rounded once from FP64 to
 * FP32 (the chirp: exp(-pi i m / N); exponent -1: the entry is 1).
 *   FFT_TABLE_ROOTS      entry i: (i a) mod N, any count (a >= 0)
 *   FFT_TABLE_STAGE      power-of-two stage table of (L, R) = (a, b): entry
 *                        4k + t: (2^t k N/(L R)) mod N, -1 where 2^t >= R;
 *                        count = 4 L
 *   FFT_TABLE_FULL_STAGE mixed-radix stage table, L = a, R = b, N = L R:
 *                        entry k W + r - 1 (W = R-1 rounded up to even):
 *                        (r k) mod N, -1 for r = R; count = L W
 *   FFT_TABLE_POSTTW     four-step twiddle w_N^{c k} of eq. (2), L = a,
 *                        columns c < b: entries c L + j: (c j) mod N, then
 *                        entries b L + 4c + t: (c L 2^t) mod N; count = b (L+4)
 *   FFT_TABLE_CHIRP      entry k: k^2 mod 2N, count = N
 *   FFT_TABLE_RADER      entry i: a^i mod N (exponents only; a a generator of
 *                        the prime N); any count
 * Arguments: N <= 2^31; out is a host int64_t array that receives the
 * exponents of the first `count` entries (count <= the table's size), or a
 * device complex64 array that receives the whole table (count = its size;
 * `stream` a cudaStream_t, the call only enqueues).
 * Returns FFT_OK, FFT_ERR_INVALID_ARG (kind, sizes or count inconsistent) or
 * FFT_ERR_CUDA.
 */
#define FFT_TABLE_ROOTS 0
#define FFT_TABLE_STAGE 1
#define FFT_TABLE_FULL_STAGE 2
#define FFT_TABLE_POSTTW 3
#define FFT_TABLE_CHIRP 4
#define FFT_TABLE_RADER 5
int fft_twiddle_exponents(int kind, int64_t N, int64_t a, int64_t b, int64_t count, int64_t *out);
int fft_twiddle_table(int kind, int64_t N, int64_t a, int64_t b, int64_t count, void *out, void *stream);

/* ---------------------------------------------------------------- wisdom */

/*
 * Wisdom (sec. 4: plans "precomputed and loaded at a later time").
 * fft_export_wisdom writes the planner's recorded decisions as text into
 * buf (at most len bytes, NUL-terminated) and returns the full length.
 * fft_import_wisdom merges such text; later plans of the same canonical
 * problems reuse the recorded decisions without timing, giving the
 * identical plan.  Returns FFT_OK or FFT_ERR_WISDOM (nothing merged).
 * fft_forget_wisdom clears everything recorded or imported.
 */
int fft_export_wisdom(char *buf, size_t len);
int fft_import_wisdom(const char *text);
void fft_forget_wisdom(void);

/* ---------------------------------------------------------------- groups */

/*
 * Uneven batches.  A group holds several plans of any kind and executes all
 * of them together, with one of two executors, chosen at creation by timing
 * both on buffers shaped like the plans' arrays (the measuring of sec. 4.3
 * applied to the whole batch) unless a flag fixes it:
 *   persistent queue (FFT_GROUP_PERSISTENT): one persistent kernel takes
 *     (step, tile) work items from a device queue ordered by step level, each
 *     item waiting (bounded, about 1 s) until the previous step of its own
 *     plan has completed; a plan's specialised pass kernels are replaced there
 *     by its generic pass over the same sub-problem, so each transform's
 *     result matches executing its plan alone to within the library's
 *     rounding (not bit for bit).  Plans with a step that has no generic
 *     form (a cluster pass beyond one CTA) cannot use it.
 *   graph of plan launches (FFT_GROUP_GRAPH): every plan's own kernels on one
 *     of up to eight forked streams, joined back into the caller's stream and
 *     captured into a CUDA graph (bit-identical to executing each plan alone).
 *   fft_group_create  : nplans >= 1 plans, kept by pointer (they must outlive
 *                       the group); flags 0, FFT_GROUP_PERSISTENT,
 *                       FFT_GROUP_GRAPH, FFT_GROUP_DEBUG_STALL (implies the
 *                       queue).  NULL on error (INVALID_ARG, UNSUPPORTED, OOM,
 *                       CUDA).  Timing both executors synchronises the device.
 *   fft_group_execute : ins[i], outs[i] are the device arrays of plan i, with
 *                       the same rules as fft_execute.  On a non-default
 *                       stream the work is captured into a CUDA graph once
 *                       and replayed (the queue's pointer table is rewritten,
 *                       the plan graph updated in place, when pointers
 *                       change).  Executions of one group must not overlap.
 *   fft_group_status  : waits for the device, returns FFT_OK or
 *                       FFT_ERR_DEVICE_TIMEOUT if a wait gave up (and clears it).
 *   fft_group_launches: kernel launches per execution (1 for the queue).
 *   fft_group_mode    : 1 persistent queue, 2 graph of plan launches.
 * FFT_GROUP_DEBUG_STALL adds one work item that waits on a segment no item
 * belongs to, with a 50 ms bound: for testing that a device wait that runs
 * out reports FFT_ERR_DEVICE_TIMEOUT and leaves the context usable.
 * Neither executor has a counterpart in the paper; they serve the vector
 * loops of sec. 4.1 when the transforms of a batch differ in size.
 */
#define FFT_GROUP_DEBUG_STALL (1u << 8)
#define FFT_GROUP_PERSISTENT (1u << 9)
#define FFT_GROUP_GRAPH (1u << 10)
typedef struct fft_group_s *fft_group;
fft_group fft_group_create(int nplans, const fft_plan *plans, unsigned flags);
int fft_group_execute(fft_group g, const void *const *ins, void *const *outs, void *stream);
int fft_group_status(fft_group g);
int fft_group_launches(fft_group g);
int fft_group_mode(fft_group g);
void fft_group_destroy(fft_group g);

/* ---------------------------------------------------------------- serving */

/*
 * A continuous-batching request loop (no counterpart in the paper; it serves
 * many independent problems of sec. 4.1 as they arrive).  Requests are dense
 * row-major transforms: rank in [1, 3], lengths n[0..rank-1] (last index
 * fastest), `batch` transforms back to back, sign -1/+1, with HOST input and
 * output buffers (pinned memory gives asynchronous copies).  A worker thread
 * admits waiting requests in arrival order whenever their device work buffers
 * (input, output and plan scratch, carved from one pool of `budget_bytes`) fit
 * in the unused budget and one of `nstreams` compute streams has a free slot;
 * waiting requests with the same shape and sign are merged into one launch.
 * Each launch is a pipeline over streams joined by events: its host->device
 * copies on one copy-in stream (admission order), the transform on a compute
 * stream, its device->host copies on one copy-out stream, so both directions
 * of the host link and the transforms of different launches overlap.  Plans
 * stay cached; making one does not synchronise the device.
 *   fft_server_create : budget_bytes >= 4096, nstreams in [1, 64], flags 0;
 *                       allocates the pool on the current device.
 *   fft_server_submit : enqueues; `arrival` is the request's arrival time in
 *                       seconds on the server clock (fft_server_now), or < 0
 *                       for "now"; *ticket identifies it.  The host buffers
 *                       must stay valid until the request completes.
 *   fft_server_poll   : FFT_OK when done, 1 while queued or running, else the
 *                       request's error (FFT_ERR_BUDGET if it can never fit).
 *   fft_server_wait   : like poll, blocking up to timeout_s seconds.
 *   fft_server_drain  : waits until nothing is queued or running (1 on timeout).
 *   fft_server_stats  : JSON text (completed, launches, merged requests, p50 /
 *                       p99 latency from arrival to completion, throughput,
 *                       budget high-water mark, cached plans, and the seconds
 *                       the queue head waited for a stream slot or for
 *                       memory); length as fft_plan_info.
 *   fft_server_destroy: finishes queued work, then frees everything.
 */
typedef struct fft_server_s *fft_server;
fft_server fft_server_create(size_t budget_bytes, int nstreams, unsigned flags);
double fft_server_now(fft_server s);
int fft_server_submit(fft_server s, int rank, const int64_t *n, int64_t batch, int sign,
                      const void *host_in, void *host_out, double arrival, uint64_t *ticket);
int fft_server_poll(fft_server s, uint64_t ticket);
int fft_server_wait(fft_server s, uint64_t ticket, double timeout_s);
int fft_server_drain(fft_server s, double timeout_s);
int fft_server_stats(fft_server s, char *buf, size_t len);
void fft_server_destroy(fft_server s);

/* ---------------------------------------------------------------- no allocation */

/* Largest batch * n that fft_execute_1d_noalloc accepts: 2^21 complex values,
 * i.e. 16 MiB of static device scratch (plus about 129 KiB of tables and
 * descriptors) that every GPU loading this library holds until exit. */
#define GBFFT_NOALLOC_MAX_POINTS (1LL << 21)

/*
 * fft_execute_1d_noalloc -- a batched 1-D complex DFT that allocates no
 * device memory, for callers that cannot allocate when they need the
 * transform: a host thread that must not block on the device-wide
 * synchronisation cudaMalloc/cudaFree may imply, a process whose device
 * memory is owned by another allocator (a framework's caching allocator or a
 * fixed pool), or a callback that is not allowed to allocate.  The paper has
 * no counterpart; the computation is the same two-pass Cooley-Tukey step
 * that fft_plan_dft plans for large n (n = n1 n2, both factors at most 4096
 * with prime factors in {2,3,5,7,11,13}), using scratch, twiddle tables and
 * pass descriptors held in one static device array.
 *   n, batch : batch contiguous transforms of length n; element l of
 *              transform b is at b*n + l in both in and out (complex64)
 *   sign     : -1 forward, +1 backward (unnormalised), as fft_plan_dft
 *   in, out  : caller-owned device arrays; in == out (in place) is allowed,
 *              any other overlap returns FFT_ERR_ALIAS
 *   stream   : cudaStream_t; the work is enqueued and the call returns
 * Returns FFT_OK; FFT_ERR_UNSUPPORTED when n * batch exceeds
 * GBFFT_NOALLOC_MAX_POINTS or n has no such split (n < 4, or a prime factor
 * above 13); FFT_ERR_INVALID_ARG, FFT_ERR_ALIAS, FFT_ERR_CUDA.
 * Set-up: the first call on each device looks up the static array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call rewrites the tables and the
 * scratch it uses, so nothing carries over from the previous call, but all
 * calls share the one array: calls that overlap on the GPU (other streams,
 * or another host thread) race and must be serialised by the caller.
 */
int fft_execute_1d_noalloc(int64_t n, int64_t batch, int sign, const void *in, void *out,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
