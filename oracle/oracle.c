/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the verification
 * in C. Hercher, "On the Sum of Squarefree Integers and a Power of Two"
 * (arXiv 2411.01964).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference leg load this library. The GPU library shares no
 * code, header, table or constant with it, and neither calls the other.
 *
 * Definitions used throughout (Sec. 1 Conjecture; Sec. 4 Theorem):
 *   squarefree(s)  : s >= 1 and no prime p with p^2 | s.  1 is squarefree.
 *   mink(n), odd n >= 3 : the smallest k >= 1 with 2^k < n and n - 2^k
 *                    squarefree (s = n - 2^k must be a positive integer, as in
 *                    the Theorem); "failure" when no such k exists.
 * k = 0 is excluded (Sec. 3, "The sieve..."), n = 1 is excluded (Conjecture:
 * n > 1), so a range [lo, hi) covers the odd n with max(lo, 3) <= n < hi.
 *
 * Two independent ways to get mink are provided:
 *   - the definition written out: trial division of every n - 2^k
 *     (or_min_k, or_verify_range_brute);
 *   - the paper's method: Algorithm 1 (sieve of the odd squarefree integers of
 *     an interval) followed by Algorithm 2 (the k loop per odd n), with the
 *     paper's look-back into the preceding interval (Sec. 3, after
 *     Algorithm 2) generalised to a look-back margin W and with the k_max cap
 *     removed: any n - 2^k below the sieved window is decided by trial
 *     division (or_verify_range).
 * Pinned by the test suite against Table 3, Table 4, the squarefree counting
 * function Q(x), sympy, brute force and the CRT construction of the Remark
 * in Sec. 2. All arithmetic is exact unsigned 64-bit integer arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

#define OR_NO_N UINT64_MAX

/* floor(sqrt(x)), digit-by-digit binary method (integer only). */
uint64_t or_isqrt(uint64_t x)
{
    uint64_t r = 0, bit = (uint64_t)1 << 62;
    while (bit > x) bit >>= 2;
    while (bit) {
        if (x >= r + bit) {
            x -= r + bit;
            r = (r >> 1) + bit;
        } else {
            r >>= 1;
        }
        bit >>= 2;
    }
    return r;
}

/*
 * Sieve of Eratosthenes: writes the odd primes 3 <= p <= limit, ascending,
 * into out (if out != NULL and room remains) and returns how many there are.
 * Primes enter Algorithm 1 as "forall primes 3 <= p < sqrt(end)".
 */
int64_t or_odd_primes(uint64_t limit, uint32_t *out, int64_t cap)
{
    if (limit < 3) return 0;
    if (limit > 0xFFFFFFFFull) return OR_EINVAL;
    uint8_t *composite = (uint8_t *)calloc(limit + 1, 1);
    if (!composite) return OR_ENOMEM;
    for (uint64_t i = 2; i * i <= limit; i++)
        if (!composite[i])
            for (uint64_t j = i * i; j <= limit; j += i) composite[j] = 1;
    int64_t count = 0;
    for (uint64_t i = 3; i <= limit; i += 2)
        if (!composite[i]) {
            if (out && count < cap) out[count] = (uint32_t)i;
            count++;
        }
    free(composite);
    return count;
}

/* squarefree(s) by the definition: no d >= 2 with d*d | s. Slow; no primes needed. */
int or_is_squarefree_brute(uint64_t s)
{
    if (s == 0) return 0;
    for (uint64_t d = 2; d <= s / d; d++)
        if (s % (d * d) == 0) return 0;
    return 1;
}

/*
 * squarefree(s) for odd s by trial division with the odd primes p, p*p <= s.
 * primes[] holds every odd prime <= cover, ascending.  Returns -1 if
 * isqrt(s) > cover (the list is too short to decide).
 */
static int is_squarefree_odd_primes(uint64_t s, const uint32_t *primes, int64_t np,
                                    uint64_t cover)
{
    if (s == 0) return 0;
    for (int64_t i = 0; i < np; i++) {
        uint64_t p = primes[i];
        uint64_t q = p * p;
        if (q > s) return 1;
        if (s % q == 0) return 0;
    }
    return (or_isqrt(s) <= cover) ? 1 : -1;
}

/*
 * Algorithm 1: for every odd n in [start, end) set is_squarefree(n) <- true,
 * then for every prime 3 <= p with p^2 < end find the smallest odd multiple m
 * of p^2 with m >= start and clear m + 2*i*p^2 for all such numbers < end.
 * sqf[(n - first_odd) / 2] holds the flag of odd n, first_odd = start | 1.
 */
static void alg1_sieve(uint64_t start, uint64_t end, const uint32_t *primes,
                       int64_t np, uint8_t *sqf)
{
    uint64_t first = start | 1;
    if (end <= first) return;
    uint64_t count = (end - first + 1) / 2;
    memset(sqf, 1, count);
    for (int64_t i = 0; i < np; i++) {
        uint64_t p = primes[i];
        uint64_t q = p * p;
        if (q >= end) break;
        uint64_t m = ((start + q - 1) / q) * q; /* smallest multiple of q >= start */
        if ((m & 1) == 0) m += q;               /* q is odd: the next one is odd */
        for (; m < end; m += 2 * q) sqf[(m - first) / 2] = 0;
    }
}

/* Public form of Algorithm 1 over [lo, hi) with its own prime list. */
int or_sieve_odd(uint64_t lo, uint64_t hi, uint8_t *out)
{
    if (hi <= (lo | 1)) return OR_OK;
    uint64_t pmax = or_isqrt(hi - 1);
    int64_t np = or_odd_primes(pmax, NULL, 0);
    if (np < 0) return (int)np;
    uint32_t *pr = (uint32_t *)malloc((size_t)(np + 1) * sizeof(uint32_t));
    if (!pr) return OR_ENOMEM;
    or_odd_primes(pmax, pr, np);
    alg1_sieve(lo, hi, pr, np, out);
    free(pr);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Range verification                                                  */
/* ------------------------------------------------------------------ */

typedef struct {
    /* in */
    uint64_t lo, hi;
    uint32_t list_k_threshold; /* n with mink >= this go to the list */
    uint32_t pad;
    /* out: counts */
    uint64_t n_odd;
    uint64_t hist[64];    /* hist[k] = #odd n with mink(n) = k */
    uint64_t first_n[64]; /* smallest n with mink(n) = k, OR_NO_N if none */
    uint64_t ksum;
    uint64_t kmax;
    /* out: caller-owned buffers (may be NULL with cap 0) */
    uint64_t *list;  /* n with mink >= threshold, ascending */
    uint8_t *list_k; /* their mink */
    uint64_t list_cap, list_len;
    uint64_t list_overflow;
    uint64_t *failures; /* odd n with no k, ascending */
    uint64_t fail_cap, fail_len;
    uint8_t *per_n_k; /* optional: mink of odd n at (n - nlo)/2, 255 = failure */
} or_result;

typedef struct {
    uint64_t n;
    uint8_t k;
} list_item;

typedef struct {
    /* shared */
    const or_result *job;
    const uint32_t *primes;
    int64_t np;
    uint64_t cover; /* primes[] holds every odd prime <= cover */
    uint64_t nlo, margin, chunk;
    uint64_t nchunks;
    uint64_t next_chunk; /* guarded by mu */
    pthread_mutex_t mu;
    int use_sieve;
    /* per-thread accumulators live in worker_state */
} shared_state;

typedef struct {
    shared_state *sh;
    uint64_t hist[64];
    uint64_t first_n[64];
    list_item *items;
    uint64_t nitems, cap_items;
    uint64_t *fails;
    uint64_t nfails, cap_fails;
    int err;
} worker_state;

static int push_item(worker_state *w, uint64_t n, uint8_t k)
{
    if (w->nitems == w->cap_items) {
        uint64_t nc = w->cap_items ? 2 * w->cap_items : 1024;
        list_item *p = (list_item *)realloc(w->items, nc * sizeof(list_item));
        if (!p) return OR_ENOMEM;
        w->items = p;
        w->cap_items = nc;
    }
    w->items[w->nitems].n = n;
    w->items[w->nitems].k = k;
    w->nitems++;
    return OR_OK;
}

static int push_fail(worker_state *w, uint64_t n)
{
    if (w->nfails == w->cap_fails) {
        uint64_t nc = w->cap_fails ? 2 * w->cap_fails : 64;
        uint64_t *p = (uint64_t *)realloc(w->fails, nc * sizeof(uint64_t));
        if (!p) return OR_ENOMEM;
        w->fails = p;
        w->cap_fails = nc;
    }
    w->fails[w->nfails++] = n;
    return OR_OK;
}

/*
 * Algorithm 2 for the odd n of one chunk [a, b): k <- 1 and increase k while
 * n - 2^k is not squarefree.  The flag of n - 2^k is read from the chunk's
 * Algorithm 1 window [wbase, b) when it lies inside, and decided by trial
 * division otherwise (brute mode: always by trial division).
 */
static int scan_chunk(worker_state *w, uint64_t a, uint64_t b, uint8_t *sqf)
{
    shared_state *sh = w->sh;
    const or_result *job = sh->job;
    uint64_t wbase = 1;
    if (sh->use_sieve) {
        wbase = (a > sh->margin + 1) ? a - sh->margin : 1;
        alg1_sieve(wbase, b, sh->primes, sh->np, sqf);
    }
    uint64_t wfirst = wbase | 1;
    uint64_t n = a | 1;
    for (; n < b; n += 2) {
        uint32_t k = 1;
        uint32_t found = 0;
        for (;;) {
            if (k >= 63 || ((uint64_t)1 << k) >= n) break; /* s = n - 2^k < 1 */
            uint64_t s = n - ((uint64_t)1 << k);
            int sf;
            if (sh->use_sieve && s >= wbase)
                sf = sqf[(s - wfirst) / 2];
            else {
                sf = is_squarefree_odd_primes(s, sh->primes, sh->np, sh->cover);
                if (sf < 0) return OR_EINVAL;
            }
            if (sf) {
                found = k;
                break;
            }
            k++;
        }
        if (found) {
            w->hist[found]++;
            if (n < w->first_n[found]) w->first_n[found] = n;
            if (found >= job->list_k_threshold)
                if (push_item(w, n, (uint8_t)found)) return OR_ENOMEM;
        } else {
            if (push_fail(w, n)) return OR_ENOMEM;
        }
        if (job->per_n_k) job->per_n_k[(n - sh->nlo) / 2] = found ? (uint8_t)found : 255;
    }
    return OR_OK;
}

static void *worker_main(void *arg)
{
    worker_state *w = (worker_state *)arg;
    shared_state *sh = w->sh;
    uint8_t *sqf = NULL;
    if (sh->use_sieve) {
        sqf = (uint8_t *)malloc(sh->chunk / 2 + sh->margin / 2 + 2);
        if (!sqf) {
            w->err = OR_ENOMEM;
            return NULL;
        }
    }
    for (;;) {
        pthread_mutex_lock(&sh->mu);
        uint64_t c = sh->next_chunk++;
        pthread_mutex_unlock(&sh->mu);
        if (c >= sh->nchunks) break;
        uint64_t a = sh->nlo + c * sh->chunk;
        uint64_t b = a + sh->chunk;
        if (b > sh->job->hi || b < a) b = sh->job->hi;
        int e = scan_chunk(w, a, b, sqf);
        if (e) {
            w->err = e;
            break;
        }
    }
    free(sqf);
    return NULL;
}

static int cmp_item(const void *x, const void *y)
{
    uint64_t a = ((const list_item *)x)->n, b = ((const list_item *)y)->n;
    return (a > b) - (a < b);
}

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/*
 * One range, Algorithm 1 + Algorithm 2 per chunk (or the definition, when
 * use_sieve is 0).  table/table_np/table_cover: a prime list the caller built
 * already (every odd prime <= table_cover, ascending), used when it covers
 * isqrt(hi - 1); NULL builds the range's own list.  Primes beyond the range's
 * own sqrt change nothing: Algorithm 1 stops at p^2 >= end and the trial
 * division at p^2 > s.
 */
static int verify_range_impl(or_result *r, int nthreads, int use_sieve, uint64_t margin,
                             uint64_t chunk, const uint32_t *table, int64_t table_np,
                             uint64_t table_cover)
{
    if (!r || r->hi > ((uint64_t)1 << 62)) return OR_EINVAL;
    uint64_t lo = r->lo < 3 ? 3 : r->lo;
    uint64_t nlo = lo | 1;
    memset(r->hist, 0, sizeof(r->hist));
    for (int k = 0; k < 64; k++) r->first_n[k] = OR_NO_N;
    r->n_odd = 0;
    r->ksum = 0;
    r->kmax = 0;
    r->list_len = 0;
    r->list_overflow = 0;
    r->fail_len = 0;
    if (r->hi <= nlo) return OR_OK;
    r->n_odd = (r->hi - nlo + 1) / 2;

    if (nthreads < 1) nthreads = 1;
    if (chunk < 64) chunk = 64;
    chunk &= ~(uint64_t)1; /* even, so that every chunk starts on an odd n */
    if (margin & 1) margin++;

    uint64_t pmax = or_isqrt(r->hi - 1);
    int64_t np;
    uint32_t *primes = NULL;      /* owned here when the range builds its own list */
    const uint32_t *plist;
    if (table && table_cover >= pmax) {
        plist = table;
        np = table_np;
        pmax = table_cover;
    } else {
        np = or_odd_primes(pmax, NULL, 0);
        if (np < 0) return (int)np;
        primes = (uint32_t *)malloc((size_t)(np + 1) * sizeof(uint32_t));
        if (!primes) return OR_ENOMEM;
        or_odd_primes(pmax, primes, np);
        plist = primes;
    }

    shared_state sh;
    memset(&sh, 0, sizeof(sh));
    sh.job = r;
    sh.primes = plist;
    sh.np = np;
    sh.cover = pmax;
    sh.nlo = nlo;
    sh.margin = margin;
    sh.chunk = chunk;
    sh.nchunks = (r->hi - nlo + chunk - 1) / chunk;
    sh.use_sieve = use_sieve;
    pthread_mutex_init(&sh.mu, NULL);

    worker_state *ws = (worker_state *)calloc((size_t)nthreads, sizeof(worker_state));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int err = (!ws || !th) ? OR_ENOMEM : OR_OK;
    int started = 0;
    if (!err) {
        for (int t = 0; t < nthreads; t++) {
            ws[t].sh = &sh;
            for (int k = 0; k < 64; k++) ws[t].first_n[k] = OR_NO_N;
        }
        for (int t = 0; t < nthreads; t++) {
            if (pthread_create(&th[t], NULL, worker_main, &ws[t]) != 0) {
                err = OR_ENOMEM;
                break;
            }
            started++;
        }
        for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    }

    /* merge: sums of counts, minima of first occurrences, sorted lists */
    uint64_t total_items = 0, total_fails = 0;
    for (int t = 0; t < started && !err; t++) {
        if (ws[t].err) err = ws[t].err;
        for (int k = 0; k < 64; k++) {
            r->hist[k] += ws[t].hist[k];
            if (ws[t].first_n[k] < r->first_n[k]) r->first_n[k] = ws[t].first_n[k];
        }
        total_items += ws[t].nitems;
        total_fails += ws[t].nfails;
    }
    if (!err) {
        list_item *all = (list_item *)malloc((total_items + 1) * sizeof(list_item));
        uint64_t *fl = (uint64_t *)malloc((total_fails + 1) * sizeof(uint64_t));
        if (!all || !fl) err = OR_ENOMEM;
        if (!err) {
            uint64_t ni = 0, nf = 0;
            for (int t = 0; t < started; t++) {
                memcpy(all + ni, ws[t].items, ws[t].nitems * sizeof(list_item));
                ni += ws[t].nitems;
                memcpy(fl + nf, ws[t].fails, ws[t].nfails * sizeof(uint64_t));
                nf += ws[t].nfails;
            }
            qsort(all, ni, sizeof(list_item), cmp_item);
            qsort(fl, nf, sizeof(uint64_t), cmp_u64);
            for (uint64_t i = 0; i < ni; i++) {
                if (r->list_len < r->list_cap) {
                    if (r->list) r->list[r->list_len] = all[i].n;
                    if (r->list_k) r->list_k[r->list_len] = all[i].k;
                    r->list_len++;
                } else {
                    r->list_overflow = 1;
                }
            }
            for (uint64_t i = 0; i < nf; i++)
                if (r->fail_len < r->fail_cap) {
                    if (r->failures) r->failures[r->fail_len] = fl[i];
                    r->fail_len++;
                }
        }
        free(all);
        free(fl);
    }
    for (int t = 0; t < nthreads && ws; t++) {
        free(ws[t].items);
        free(ws[t].fails);
    }
    free(ws);
    free(th);
    free(primes); /* NULL when the caller's list was used */
    pthread_mutex_destroy(&sh.mu);
    if (err) return err;
    for (int k = 1; k < 64; k++) {
        r->ksum += (uint64_t)k * r->hist[k];
        if (r->hist[k]) r->kmax = (uint64_t)k;
    }
    return OR_OK;
}

/* The paper's method: Algorithm 1 + Algorithm 2 per chunk, look-back margin W. */
int or_verify_range(or_result *r, int nthreads, uint64_t margin, uint64_t chunk)
{
    return verify_range_impl(r, nthreads, 1, margin, chunk, NULL, 0, 0);
}

/* The definition written out: every n - 2^k decided by trial division. */
int or_verify_range_brute(or_result *r, int nthreads)
{
    return verify_range_impl(r, nthreads, 0, 0, (uint64_t)1 << 16, NULL, 0, 0);
}

/*
 * Many independent ranges: the same computation as or_verify_range for each
 * of rs[0 .. count), with one prime list (for the largest hi) shared by all,
 * and the ranges handed out to nthreads workers, one whole range each, in
 * the order given.
 */
typedef struct {
    or_result *rs;
    int64_t count;
    int64_t next; /* guarded by mu */
    pthread_mutex_t mu;
    const uint32_t *primes;
    int64_t np;
    uint64_t cover, margin, chunk;
    int err;
} batch_state;

static void *batch_worker(void *arg)
{
    batch_state *b = (batch_state *)arg;
    for (;;) {
        pthread_mutex_lock(&b->mu);
        int64_t i = b->next++;
        int stop = b->err != 0;
        pthread_mutex_unlock(&b->mu);
        if (stop || i >= b->count) break;
        int e = verify_range_impl(&b->rs[i], 1, 1, b->margin, b->chunk, b->primes, b->np, b->cover);
        if (e) {
            pthread_mutex_lock(&b->mu);
            if (!b->err) b->err = e;
            pthread_mutex_unlock(&b->mu);
        }
    }
    return NULL;
}

int or_verify_ranges(or_result *rs, int64_t count, int nthreads, uint64_t margin, uint64_t chunk)
{
    if (count < 0 || (count && !rs)) return OR_EINVAL;
    uint64_t max_hi = 2;
    for (int64_t i = 0; i < count; i++) {
        if (rs[i].hi > ((uint64_t)1 << 62)) return OR_EINVAL;
        if (rs[i].hi > max_hi) max_hi = rs[i].hi;
    }
    batch_state b;
    memset(&b, 0, sizeof(b));
    b.rs = rs;
    b.count = count;
    b.margin = margin;
    b.chunk = chunk;
    b.cover = or_isqrt(max_hi - 1);
    b.np = or_odd_primes(b.cover, NULL, 0);
    if (b.np < 0) return (int)b.np;
    uint32_t *primes = (uint32_t *)malloc((size_t)(b.np + 1) * sizeof(uint32_t));
    if (!primes) return OR_ENOMEM;
    or_odd_primes(b.cover, primes, b.np);
    b.primes = primes;
    pthread_mutex_init(&b.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int started = 0;
    if (!th) b.err = OR_ENOMEM;
    for (int t = 0; t < nthreads && th; t++) {
        if (pthread_create(&th[t], NULL, batch_worker, &b) != 0) {
            if (!started) b.err = OR_ENOMEM;
            break;
        }
        started++;
    }
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    free(primes);
    pthread_mutex_destroy(&b.mu);
    return b.err;
}

/*
 * mink of single points by the definition (trial division of each n - 2^k).
 * out[i] = mink(points[i]); 0 if points[i] is even or < 3; 255 on failure.
 */
int or_min_k(const uint64_t *points, uint64_t count, uint8_t *out)
{
    uint64_t maxp = 0;
    for (uint64_t i = 0; i < count; i++)
        if (points[i] > maxp) maxp = points[i];
    if (maxp > ((uint64_t)1 << 62)) return OR_EINVAL;
    uint64_t pmax = maxp > 1 ? or_isqrt(maxp - 1) : 1;
    int64_t np = or_odd_primes(pmax, NULL, 0);
    if (np < 0) return (int)np;
    uint32_t *primes = (uint32_t *)malloc((size_t)(np + 1) * sizeof(uint32_t));
    if (!primes) return OR_ENOMEM;
    or_odd_primes(pmax, primes, np);
    for (uint64_t i = 0; i < count; i++) {
        uint64_t n = points[i];
        if (n < 3 || (n & 1) == 0) {
            out[i] = 0;
            continue;
        }
        uint8_t res = 255;
        for (uint32_t k = 1; k < 63 && ((uint64_t)1 << k) < n; k++) {
            int sf = is_squarefree_odd_primes(n - ((uint64_t)1 << k), primes, np, pmax);
            if (sf < 0) {
                free(primes);
                return OR_EINVAL;
            }
            if (sf) {
                res = (uint8_t)k;
                break;
            }
        }
        out[i] = res;
    }
    free(primes);
    return OR_OK;
}

/* squarefree(s) for any s >= 1, by trial division with 2 and the odd primes. */
int or_is_squarefree(uint64_t s)
{
    if (s == 0) return 0;
    if (s % 4 == 0) return 0;
    if ((s & 1) == 0) s >>= 1;
    uint64_t pmax = or_isqrt(s);
    int64_t np = or_odd_primes(pmax, NULL, 0);
    if (np < 0) return (int)np;
    uint32_t *primes = (uint32_t *)malloc((size_t)(np + 1) * sizeof(uint32_t));
    if (!primes) return OR_ENOMEM;
    or_odd_primes(pmax, primes, np);
    int r = is_squarefree_odd_primes(s, primes, np, pmax);
    free(primes);
    return r;
}
