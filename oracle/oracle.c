/*
 * oracle.c -- plain FP64 CPU reference for the DFT problem dft(N, V, I, O).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes (Johnson & Frigo, "Implementing FFTs in Practice"):
 *   - eq. (1), sec. 2: Y[k] = sum_{l<n} X[l] w_n^{l k}, with w_n = exp(s 2 pi i/n).
 *     The paper defines the forward transform with s = -1; s = +1 is read as
 *     the unnormalised backward transform.
 *   - eq. (2), sec. 2: Cooley-Tukey with n = n1 n2, l = l1 n2 + l2,
 *     k = k1 + k2 n1, used recursively with n2 = p (the smallest prime
 *     factor of n) as a decimation-in-time radix; this generalises the
 *     depth-first radix-2 recursion of Algorithm 1 to mixed radix.
 *   - sec. 4.1: the problem dft(N, V, I, O) -- a loop over the vector
 *     tensor V of rank-|N| transforms with I/O dimensions (n, is, os);
 *     strides are counted in complex elements and may be negative or zero
 *     on the input side.  A multi-dimensional transform is evaluated
 *     separably, one dimension at a time, through an FP64 temporary.
 *
 * Precision: every operation is IEEE FP64.  Roots of unity come from one
 * table per transform length, R[m] = exp(s 2 pi i m/n) for 0 <= m < n,
 * looked up at (l*k) mod n computed exactly in 64-bit integers, so no angle
 * ever grows beyond 2 pi.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cplx;

static cplx cmul(cplx a, cplx b) {
    cplx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}

/* R[m] = exp(sign * 2 pi i m / n), 0 <= m < n (eq. (1): w_n^m). */
static cplx *root_table(int64_t n, int sign) {
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    if (!r) return NULL;
    for (int64_t m = 0; m < n; ++m) {
        double a = 2.0 * M_PI * (double)m / (double)n;
        r[m].re = cos(a);
        r[m].im = (double)sign * sin(a);
    }
    return r;
}

/*
 * Direct evaluation of eq. (1) (the "generic" Theta(n^2) plan of sec. 4.2).
 * x[l*xs] for l < n  ->  y[k*ys] for k < n.  roots[m] = w_n^m.
 */
static void dft_direct_t(int64_t n, const cplx *roots, const cplx *x, int64_t xs,
                         cplx *y, int64_t ys) {
    for (int64_t k = 0; k < n; ++k) {
        cplx acc = {0.0, 0.0};
        for (int64_t l = 0; l < n; ++l) {
            cplx t = cmul(x[l * xs], roots[(l * k) % n]);
            acc.re += t.re;
            acc.im += t.im;
        }
        y[k * ys] = acc;
    }
}

static int64_t smallest_prime_factor(int64_t n) {
    if (n % 2 == 0) return 2;
    for (int64_t p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

/*
 * Recursive mixed-radix decimation-in-time Cooley-Tukey, eq. (2).
 * Computes the length-n DFT of x[l*xs] into y[0..n-1] (unit stride).
 * rootN[m] = w_N^m for the top-level length N; w_n^e = w_N^{e N/n}.
 * With n = n1 n2, n2 = p the smallest prime factor of n and n1 = m:
 *   1. for each l2 < p: the length-m DFT of x[(l1 p + l2) xs] over l1
 *      (recursively), stored at y[l2 m + k1];
 *   2. for each k1 < m: multiply by the twiddle w_n^{l2 k1} and take the
 *      length-p DFT over l2, giving Y[k1 + k2 m].
 * Step 2 reads and writes the same p locations {l2 m + k1}, so it runs in
 * place, as the radix-2 butterfly loop of Algorithm 1 does.
 * A prime length is evaluated directly (eq. (1)).
 */
static void dft_ct_rec(int64_t n, int64_t N, const cplx *rootN, const cplx *x, int64_t xs,
                       cplx *y, cplx *tmp) {
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    int64_t p = smallest_prime_factor(n);
    int64_t scale = N / n; /* w_n^e = w_N^{e*scale} */
    if (p == n) {
        for (int64_t k = 0; k < n; ++k) {
            cplx acc = {0.0, 0.0};
            for (int64_t l = 0; l < n; ++l) {
                cplx t = cmul(x[l * xs], rootN[((l * k) % n) * scale]);
                acc.re += t.re;
                acc.im += t.im;
            }
            y[k] = acc;
        }
        return;
    }
    int64_t m = n / p;
    for (int64_t l2 = 0; l2 < p; ++l2)
        dft_ct_rec(m, N, rootN, x + l2 * xs, p * xs, y + l2 * m, tmp);
    for (int64_t k1 = 0; k1 < m; ++k1) {
        for (int64_t l2 = 0; l2 < p; ++l2)
            tmp[l2] = cmul(y[l2 * m + k1], rootN[((l2 * k1) % n) * scale]);
        for (int64_t k2 = 0; k2 < p; ++k2) {
            cplx acc = {0.0, 0.0};
            for (int64_t l2 = 0; l2 < p; ++l2) {
                /* w_p^{l2 k2} = w_n^{(l2 k2 mod p) m} */
                cplx t = cmul(tmp[l2], rootN[(((l2 * k2) % p) * m) * scale]);
                acc.re += t.re;
                acc.im += t.im;
            }
            y[k1 + k2 * m] = acc;
        }
    }
}

/* algo: 0 = auto (direct for n <= 4096, Cooley-Tukey above), 1 = direct, 2 = Cooley-Tukey */
#define ORACLE_DIRECT_MAX 4096

typedef struct {
    int64_t n;
    int sign;
    int algo;
    cplx *roots; /* w_n^m, m < n */
    cplx *work;  /* n values, Cooley-Tukey output */
    cplx *tmp;   /* n values, Cooley-Tukey radix scratch */
} dft1;

static int dft1_init(dft1 *d, int64_t n, int sign, int algo) {
    memset(d, 0, sizeof(*d));
    d->n = n;
    d->sign = sign;
    d->algo = (algo == 0) ? (n <= ORACLE_DIRECT_MAX ? 1 : 2) : algo;
    d->roots = root_table(n, sign);
    d->work = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    d->tmp = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    return (d->roots && d->work && d->tmp) ? 0 : -1;
}

static void dft1_free(dft1 *d) {
    free(d->roots);
    free(d->work);
    free(d->tmp);
}

/* One length-n 1-D DFT, x[l*xs] -> y[k*ys]; x and y must not overlap. */
static void dft1_run(dft1 *d, const cplx *x, int64_t xs, cplx *y, int64_t ys) {
    if (d->algo == 1) {
        dft_direct_t(d->n, d->roots, x, xs, y, ys);
    } else {
        dft_ct_rec(d->n, d->n, d->roots, x, xs, d->work, d->tmp);
        for (int64_t k = 0; k < d->n; ++k) y[k * ys] = d->work[k];
    }
}

/* ------------------------------------------------------------------------ */
/* The problem dft(N, V, I, O) of sec. 4.1.                                  */

#define ORACLE_MAX_RANK 8

typedef struct {
    int rank;
    int64_t n[ORACLE_MAX_RANK], is[ORACLE_MAX_RANK], os[ORACLE_MAX_RANK];
    int vrank;
    int64_t vn[ORACLE_MAX_RANK], vis[ORACLE_MAX_RANK], vos[ORACLE_MAX_RANK];
    int sign, algo;
    const cplx *in;
    cplx *out;
    int64_t total_vec;  /* product of vector lengths */
    int64_t total_pts;  /* product of transform lengths */
    int64_t next;       /* next vector index to process (guarded by lock) */
    pthread_mutex_t lock;
    int failed;
} job;

/* Vector index v (row-major over the vector loops) -> input/output offsets. */
static void vec_offsets(const job *jb, int64_t v, int64_t *io, int64_t *oo) {
    int64_t a = 0, b = 0;
    for (int d = jb->vrank - 1; d >= 0; --d) {
        int64_t i = v % jb->vn[d];
        v /= jb->vn[d];
        a += i * jb->vis[d];
        b += i * jb->vos[d];
    }
    *io = a;
    *oo = b;
}

static void *worker(void *arg) {
    job *jb = (job *)arg;
    int64_t P = jb->total_pts;
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)(P > 0 ? P : 1));
    cplx *line_in = NULL, *line_out = NULL;
    dft1 plans[ORACLE_MAX_RANK];
    memset(plans, 0, sizeof(plans));
    int ok = buf != NULL;
    int64_t maxn = 1;
    for (int d = 0; d < jb->rank; ++d) maxn = jb->n[d] > maxn ? jb->n[d] : maxn;
    line_in = (cplx *)malloc(sizeof(cplx) * (size_t)maxn);
    line_out = (cplx *)malloc(sizeof(cplx) * (size_t)maxn);
    ok = ok && line_in && line_out;
    for (int d = 0; d < jb->rank; ++d)
        if (ok && dft1_init(&plans[d], jb->n[d], jb->sign, jb->algo) != 0) ok = 0;
    if (!ok) {
        pthread_mutex_lock(&jb->lock);
        jb->failed = 1;
        pthread_mutex_unlock(&jb->lock);
    }
    /* row-major strides of the FP64 temporary over the transform dims */
    int64_t tstride[ORACLE_MAX_RANK];
    {
        int64_t s = 1;
        for (int d = jb->rank - 1; d >= 0; --d) {
            tstride[d] = s;
            s *= jb->n[d];
        }
    }
    while (ok) {
        int64_t v;
        pthread_mutex_lock(&jb->lock);
        v = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (v >= jb->total_vec) break;
        int64_t io, oo;
        vec_offsets(jb, v, &io, &oo);
        /* gather X[I + sum_j l_j is_j] into the temporary */
        for (int64_t e = 0; e < P; ++e) {
            int64_t r = e, off = 0;
            for (int d = jb->rank - 1; d >= 0; --d) {
                off += (r % jb->n[d]) * jb->is[d];
                r /= jb->n[d];
            }
            buf[e] = jb->in[io + off];
        }
        /* separable multi-dimensional DFT: 1-D transforms along each dim */
        for (int d = 0; d < jb->rank; ++d) {
            int64_t nd = jb->n[d], st = tstride[d];
            int64_t lines = P / nd;
            for (int64_t q = 0; q < lines; ++q) {
                /* q enumerates all index tuples with dim d removed */
                int64_t hi = q / st, lo = q % st;
                int64_t base = hi * st * nd + lo;
                for (int64_t l = 0; l < nd; ++l) line_in[l] = buf[base + l * st];
                dft1_run(&plans[d], line_in, 1, line_out, 1);
                for (int64_t k = 0; k < nd; ++k) buf[base + k * st] = line_out[k];
            }
        }
        /* scatter Y[O + sum_j k_j os_j] */
        for (int64_t e = 0; e < P; ++e) {
            int64_t r = e, off = 0;
            for (int d = jb->rank - 1; d >= 0; --d) {
                off += (r % jb->n[d]) * jb->os[d];
                r /= jb->n[d];
            }
            jb->out[oo + off] = buf[e];
        }
    }
    for (int d = 0; d < jb->rank; ++d) dft1_free(&plans[d]);
    free(buf);
    free(line_in);
    free(line_out);
    return NULL;
}

/*
 * oracle_dft: evaluate dft(N, V, I, O) (sec. 4.1) in FP64.
 *   rank, n[], is[], os[]      : the size tensor N (rank 0 = copy, sec. 4.1.1)
 *   vrank, vn[], vis[], vos[]  : the vector tensor V (loops, order irrelevant)
 *   in, out                    : complex FP64 arrays addressed at element 0;
 *                                strides in complex elements
 *   sign                       : -1 forward (eq. (1)), +1 backward (unnormalised)
 *   algo                       : 0 auto, 1 direct eq. (1), 2 Cooley-Tukey eq. (2)
 *   nthreads                   : worker threads over the vector loops
 * Returns 0 on success, -1 on invalid arguments or allocation failure.
 */
int oracle_dft(int rank, const int64_t *n, const int64_t *is, const int64_t *os, int vrank,
               const int64_t *vn, const int64_t *vis, const int64_t *vos, const double *in,
               double *out, int sign, int algo, int nthreads) {
    if (rank < 0 || rank > ORACLE_MAX_RANK || vrank < 0 || vrank > ORACLE_MAX_RANK) return -1;
    if (sign != -1 && sign != 1) return -1;
    if (algo < 0 || algo > 2) return -1;
    job jb;
    memset(&jb, 0, sizeof(jb));
    jb.rank = rank;
    jb.vrank = vrank;
    jb.sign = sign;
    jb.algo = algo;
    jb.in = (const cplx *)in;
    jb.out = (cplx *)out;
    jb.total_pts = 1;
    jb.total_vec = 1;
    for (int d = 0; d < rank; ++d) {
        if (n[d] < 0) return -1;
        jb.n[d] = n[d];
        jb.is[d] = is[d];
        jb.os[d] = os[d];
        jb.total_pts *= n[d];
    }
    for (int d = 0; d < vrank; ++d) {
        if (vn[d] < 0) return -1;
        jb.vn[d] = vn[d];
        jb.vis[d] = vis[d];
        jb.vos[d] = vos[d];
        jb.total_vec *= vn[d];
    }
    if (jb.total_pts == 0 || jb.total_vec == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > jb.total_vec) nthreads = (int)jb.total_vec;
    pthread_mutex_init(&jb.lock, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, worker, &jb) != 0) break;
        started = t;
    }
    worker(&jb);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&jb.lock);
    return jb.failed ? -1 : 0;
}
