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
#define FFT_PREC_TC_FP16 (1u << 4) /* radix-16 stages as FP16 tensor-core MMAs */
#define FFT_PREC_TC_BF16 (1u << 5) /* radix-16 stages as BF16 tensor-core MMAs */
#define FFT_PREC_SPLIT (1u << 6)   /* with a TC flag: split hi+lo operands */

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
 * fft_execute -- run a plan (sec. 4.2: the plan's steps, in order).
 *   in, out : device pointers to element 0 of complex64 arrays that cover
 *             every addressed element; caller-owned.  For an out-of-place
 *             plan the input is not modified and the footprints of in and
 *             out must not overlap (else FFT_ERR_ALIAS).  A plan made with
 *             FFT_INPLACE must be given in == out.
 *   stream  : a cudaStream_t (NULL = legacy default stream); the call only
 *             enqueues work and returns.
 * Returns FFT_OK or an error code (INVALID_ARG, ALIAS, INPLACE_MISMATCH,
 * CUDA); also reported by fft_last_error().
 */
int fft_execute(fft_plan p, const void *in, void *out, void *stream);

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
 * (8 read + 8 written), the unit used for the HBM roofline. */
double fft_plan_bytes(fft_plan p);

/* Flops of one execution under the 5 N log2 N convention (sec. 1). */
double fft_plan_flops(fft_plan p);

/* Number of kernel launches one fft_execute enqueues. */
int fft_plan_launches(fft_plan p);

/* Device scratch bytes the plan holds (excludes twiddle tables). */
size_t fft_plan_scratch_bytes(fft_plan p);

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
