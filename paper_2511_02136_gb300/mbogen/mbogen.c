/*
 * mbogen.c -- seeded synthetic market-by-order (MBO) message streams.
 *
 * This is the input module shared by the CPU oracle and the CUDA engine: it
 * writes message bytes and nothing else.  It holds none of the matching,
 * agent, observation or reward arithmetic of the environment step; it only
 * plays the role of the historical message store of Sec. 4 (Design): all
 * messages of all episodes in one contiguous array, plus the per-step start
 * indices into it ("index the data at runtime").  The LOBSTER data the paper
 * replays is not available, so the stream is drawn from a small stochastic
 * message model instead:
 *
 *   - a latent mid price (int32 ticks) that, before every message, moves by
 *     +1 or -1 (equal odds) with probability p_move;
 *   - message type drawn from a four-way mix: add limit, partial cancel,
 *     full delete, market order;
 *   - side 50/50;
 *   - add prices: buy at mid - g, sell at mid + g, g ~ Geom0(p_price) on
 *     {0, 1, ...} (failures before the first success);
 *   - sizes 1 + Geom0(p_size), or min(size_cap, floor(X)) with
 *     X ~ Pareto(x_m = 1, alpha) for the heavy-tailed mix;
 *   - partial cancels and deletes target a uniformly chosen order from the
 *     generator's own pool of issued, not yet fully cancelled ids.  The
 *     generator does not see executions, so such a message may name an order
 *     that no longer rests; the engine treats that as a no-op;
 *   - optional cancel bursts: with probability p_burst per env-step the step
 *     starts with min(floor(pool/2), M) deletes of pool orders;
 *   - messages per step fixed (M) or Poisson(lambda_env) with lambda_env
 *     log-uniform in [lam_lo, lam_hi];
 *   - optionally the latent mid at every step boundary, from which the
 *     Python side draws synthetic book snapshots for episode starts.
 *
 * All random draws are integers: SplitMix64 outputs compared against uint64
 * CDF threshold tables.  The tables are built with IEEE double + - * / only
 * (no libm), so they are the same on every host that rounds to nearest.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define MBO_ADD 1
#define MBO_PARTIAL 2
#define MBO_DELETE 3
#define MBO_MARKET 4
#define MBO_BUY 1
#define MBO_SELL (-1)

/* 32-byte message record; the layout is the wire format both consumers read. */
typedef struct mbo_msg {
    int64_t ts;   /* generator clock: message index within the env's stream */
    int64_t oid;  /* order id (>= 0) */
    int32_t px;   /* price in ticks (0 for market orders) */
    int32_t qty;  /* size (add/market), cancelled amount (partial), known size (delete) */
    int16_t type; /* MBO_ADD .. MBO_MARKET */
    int16_t side; /* MBO_BUY / MBO_SELL */
    int32_t pad;
} mbo_msg;

typedef struct mbogen_params {
    int32_t start_mid;
    int32_t msgs_mode;      /* 0: fixed msgs_fixed per step, 1: Poisson(lambda_env) */
    int32_t msgs_fixed;
    int32_t size_model;     /* 0: 1 + Geom0(size_p); 1: min(size_cap, floor(Pareto(1, alpha))) */
    int32_t size_cap;
    int32_t pad0;
    double p_move;
    double mix_add, mix_partial, mix_delete, mix_market;
    double price_p;
    double size_p;
    double pareto_alpha;
    double p_burst;
    double lam_lo, lam_hi;
} mbogen_params;

/* ---- SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ---------------------- */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL
static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t sm_next(uint64_t *s) { *s += SM_GAMMA; return sm_mix(*s); }
/* Lemire's multiply-shift map of the high 32 bits onto [0, n). */
static inline uint32_t lemire32(uint64_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)(uint32_t)(u >> 32) * (uint64_t)n) >> 32);
}

#define TAG_MSGS   0x4D424F4D53475331ULL
#define TAG_COUNT  0x4D424F434E545331ULL
#define TAG_LAMBDA 0x4D424F4C414D4231ULL
#define TAG_CAPS   0x4D424F4341505331ULL

uint64_t mbogen_env_seed(uint64_t seed, int64_t env) {
    uint64_t s = seed ^ (uint64_t)env;
    return sm_next(&s);
}

/* ---- deterministic exp / log from + - * / only ---------------------------- */
static double det_exp(double x) {
    /* exp(x) = (exp(x / 2^k))^(2^k); Taylor series on the reduced argument */
    int k = 0;
    while (x > 0.5 || x < -0.5) { x *= 0.5; k++; }
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 30; i++) { term = term * x / (double)i; sum += term; }
    for (int i = 0; i < k; i++) sum = sum * sum;
    return sum;
}
static double det_log(double x) {
    /* x > 0: x = m * 2^e with m in [0.75, 1.5); ln m = 2 atanh((m-1)/(m+1)) */
    const double LN2 = 0.6931471805599453094;
    int e = 0;
    while (x >= 1.5) { x *= 0.5; e++; }
    while (x < 0.75) { x *= 2.0; e--; }
    double y = (x - 1.0) / (x + 1.0), y2 = y * y, term = y, sum = 0.0;
    for (int i = 1; i < 80; i += 2) { sum += term / (double)i; term *= y2; }
    return 2.0 * sum + (double)e * LN2;
}

static inline uint64_t prob_to_u64(double c) {
    if (!(c > 0.0)) return 0;
    if (c >= 1.0) return UINT64_MAX;
    return (uint64_t)(c * 18446744073709551616.0);
}

/* CDF threshold table: value k is returned when thr[k-1] <= u < thr[k]. */
typedef struct cdf_table { uint64_t *thr; int32_t n; int32_t base; } cdf_table;

static int32_t cdf_sample(const cdf_table *t, uint64_t u) {
    int32_t lo = 0, hi = t->n; /* first index with u < thr[i] */
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (u < t->thr[mid]) hi = mid; else lo = mid + 1;
    }
    return t->base + lo; /* lo == n means the (negligible) tail: clamp to last+1 */
}

static int build_geom(cdf_table *t, double p, int32_t base, int32_t max_n) {
    t->thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)max_n);
    if (!t->thr) return -1;
    t->base = base;
    double surv = 1.0;
    int32_t n = 0;
    while (n < max_n) {
        surv = surv * (1.0 - p);
        uint64_t th = prob_to_u64(1.0 - surv);
        t->thr[n++] = th;
        if (th == UINT64_MAX || surv < 1e-300) break;
    }
    t->n = n;
    return 0;
}

static int build_pareto(cdf_table *t, double alpha, int32_t cap) {
    /* P(floor X = k) for k = 1..cap-1, X ~ Pareto(1, alpha); the rest is cap */
    int32_t n = cap - 1;
    if (n < 1) n = 1;
    t->thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    if (!t->thr) return -1;
    t->base = 1;
    for (int32_t i = 0; i < n; i++) {
        double k1 = (double)(i + 2); /* P(floor X <= i+1) = 1 - (i+2)^(-alpha) */
        double surv = det_exp(-alpha * det_log(k1));
        t->thr[i] = prob_to_u64(1.0 - surv);
    }
    t->n = n;
    return 0;
}

static int build_poisson(cdf_table *t, double lam) {
    /* the tail beyond 2*lambda + 100 is below 1e-20 for lambda <= 1e4 */
    int32_t maxk = (int32_t)(2.0 * lam) + 100;
    t->thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)maxk);
    if (!t->thr) return -1;
    t->base = 0;
    double pk = det_exp(-lam), cdf = pk;
    int32_t n = 0;
    for (int32_t k = 0; k < maxk; k++) {
        uint64_t th = prob_to_u64(cdf);
        t->thr[n++] = th;
        if (th == UINT64_MAX) break;
        pk = pk * lam / (double)(k + 1);
        cdf += pk;
    }
    t->n = n;
    return 0;
}

typedef struct pool_entry { int64_t oid; int32_t px; int32_t q; int16_t side; } pool_entry;

typedef struct shared_ctx {
    const mbogen_params *p;
    const uint64_t *env_seeds;
    int64_t n_envs;
    int32_t n_steps;
    const int32_t *counts; /* [n_envs][n_steps] */
    const int64_t *offsets;/* [n_envs][n_steps+1] absolute */
    mbo_msg *out;
    int32_t *mids;         /* [n_envs][n_steps+1] latent mid at each step boundary, or NULL */
    cdf_table geom_price, size_tab;
    uint64_t thr_move, thr_add, thr_partial, thr_delete, thr_burst;
    int64_t next_env;
    pthread_mutex_t mu;
    int error;
} shared_ctx;

static int gen_env(shared_ctx *c, int64_t e) {
    const mbogen_params *p = c->p;
    uint64_t s = sm_mix(c->env_seeds[e] ^ TAG_MSGS);
    int32_t mid = p->start_mid;
    int64_t next_oid = 0, clock = 0;
    int64_t pool_n = 0, pool_cap = 1024;
    pool_entry *pool = (pool_entry *)malloc(sizeof(pool_entry) * (size_t)pool_cap);
    if (!pool) return -1;
    for (int32_t t = 0; t < c->n_steps; t++) {
        int32_t m = c->counts[e * (int64_t)c->n_steps + t];
        mbo_msg *o = c->out + c->offsets[e * (int64_t)(c->n_steps + 1) + t];
        if (c->mids) c->mids[e * (int64_t)(c->n_steps + 1) + t] = mid;
        int32_t n_burst = 0;
        if (c->thr_burst) {
            uint64_t u = sm_next(&s);
            if (u < c->thr_burst) {
                int64_t b = pool_n / 2;
                n_burst = (int32_t)(b < m ? b : m);
            }
        }
        for (int32_t i = 0; i < m; i++) {
            mbo_msg *r = o + i;
            uint64_t u = sm_next(&s);
            if (u < c->thr_move) mid += (sm_next(&s) >> 63) ? 1 : -1;
            int type;
            if (i < n_burst) {
                type = MBO_DELETE;
            } else {
                u = sm_next(&s);
                type = u < c->thr_add ? MBO_ADD : u < c->thr_partial ? MBO_PARTIAL
                     : u < c->thr_delete ? MBO_DELETE : MBO_MARKET;
            }
            if ((type == MBO_PARTIAL || type == MBO_DELETE) && pool_n == 0) type = MBO_ADD;
            memset(r, 0, sizeof(*r));
            r->ts = clock++;
            r->type = (int16_t)type;
            if (type == MBO_ADD || type == MBO_MARKET) {
                int16_t side = (sm_next(&s) >> 63) ? MBO_SELL : MBO_BUY;
                int32_t qty = cdf_sample(&c->size_tab, sm_next(&s));
                if (p->size_model == 0) qty += 1; /* 1 + Geom0 */
                r->side = side;
                r->qty = qty;
                r->oid = next_oid++;
                if (type == MBO_ADD) {
                    int32_t g = cdf_sample(&c->geom_price, sm_next(&s));
                    r->px = side == MBO_BUY ? mid - g : mid + g;
                    if (pool_n == pool_cap) {
                        pool_cap *= 2;
                        pool_entry *np = (pool_entry *)realloc(pool, sizeof(pool_entry) * (size_t)pool_cap);
                        if (!np) { free(pool); return -1; }
                        pool = np;
                    }
                    pool[pool_n].oid = r->oid; pool[pool_n].px = r->px;
                    pool[pool_n].q = qty; pool[pool_n].side = side;
                    pool_n++;
                }
            } else {
                uint32_t k = lemire32(sm_next(&s), (uint32_t)pool_n);
                pool_entry *pe = pool + k;
                r->oid = pe->oid; r->px = pe->px; r->side = pe->side;
                int remove = 0;
                if (type == MBO_PARTIAL) {
                    int32_t span = pe->q - 1 > 1 ? pe->q - 1 : 1;
                    int32_t amt = 1 + (int32_t)lemire32(sm_next(&s), (uint32_t)span);
                    r->qty = amt;
                    pe->q -= amt;
                    remove = pe->q <= 0;
                } else {
                    r->qty = pe->q;
                    remove = 1;
                }
                if (remove) pool[k] = pool[--pool_n];
            }
        }
    }
    if (c->mids) c->mids[e * (int64_t)(c->n_steps + 1) + c->n_steps] = mid;
    free(pool);
    return 0;
}

static void *worker(void *arg) {
    shared_ctx *c = (shared_ctx *)arg;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        int64_t e = c->next_env++;
        pthread_mutex_unlock(&c->mu);
        if (e >= c->n_envs) break;
        if (gen_env(c, e)) { pthread_mutex_lock(&c->mu); c->error = -1; pthread_mutex_unlock(&c->mu); }
    }
    return NULL;
}

/* Per-env, per-step message counts.  Fixed mode fills msgs_fixed; Poisson mode
 * draws lambda_env log-uniform in [lam_lo, lam_hi] and M_t ~ Poisson(lambda). */
int mbogen_counts(const mbogen_params *p, int64_t n_envs, const uint64_t *env_seeds,
                  int32_t n_steps, int32_t *counts_out, double *lambda_out) {
    for (int64_t e = 0; e < n_envs; e++) {
        int32_t *row = counts_out + e * (int64_t)n_steps;
        if (p->msgs_mode == 0) {
            for (int32_t t = 0; t < n_steps; t++) row[t] = p->msgs_fixed;
            if (lambda_out) lambda_out[e] = (double)p->msgs_fixed;
            continue;
        }
        uint64_t sl = sm_mix(env_seeds[e] ^ TAG_LAMBDA);
        double u = (double)(sm_next(&sl) >> 11) * (1.0 / 9007199254740992.0);
        double lam = p->lam_lo * det_exp(u * det_log(p->lam_hi / p->lam_lo));
        if (lambda_out) lambda_out[e] = lam;
        cdf_table tab;
        if (build_poisson(&tab, lam)) return -1;
        uint64_t sc = sm_mix(env_seeds[e] ^ TAG_COUNT);
        for (int32_t t = 0; t < n_steps; t++) row[t] = cdf_sample(&tab, sm_next(&sc));
        free(tab.thr);
    }
    return 0;
}

/* Absolute offsets [n_envs][n_steps+1] of an env-major contiguous layout. */
int64_t mbogen_offsets(int64_t n_envs, int32_t n_steps, const int32_t *counts, int64_t *offsets_out) {
    int64_t acc = 0;
    for (int64_t e = 0; e < n_envs; e++) {
        for (int32_t t = 0; t < n_steps; t++) {
            offsets_out[e * (int64_t)(n_steps + 1) + t] = acc;
            acc += counts[e * (int64_t)n_steps + t];
        }
        offsets_out[e * (int64_t)(n_steps + 1) + n_steps] = acc;
    }
    return acc;
}

int mbogen_generate(const mbogen_params *p, int64_t n_envs, const uint64_t *env_seeds,
                    int32_t n_steps, const int32_t *counts, const int64_t *offsets,
                    void *out_msgs, int32_t n_threads, int32_t *mids_out) {
    shared_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = p; c.env_seeds = env_seeds; c.n_envs = n_envs; c.n_steps = n_steps;
    c.counts = counts; c.offsets = offsets; c.out = (mbo_msg *)out_msgs; c.mids = mids_out;
    double tot = p->mix_add + p->mix_partial + p->mix_delete + p->mix_market;
    if (!(tot > 0.0)) return -1;
    c.thr_move = prob_to_u64(p->p_move);
    c.thr_add = prob_to_u64(p->mix_add / tot);
    c.thr_partial = prob_to_u64((p->mix_add + p->mix_partial) / tot);
    c.thr_delete = prob_to_u64((p->mix_add + p->mix_partial + p->mix_delete) / tot);
    c.thr_burst = prob_to_u64(p->p_burst);
    if (build_geom(&c.geom_price, p->price_p, 0, 4096)) return -1;
    int rc = p->size_model == 0 ? build_geom(&c.size_tab, p->size_p, 0, 1 << 16)
                                : build_pareto(&c.size_tab, p->pareto_alpha, p->size_cap);
    if (rc) { free(c.geom_price.thr); return -1; }
    pthread_mutex_init(&c.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < n_threads; i++)
        if (pthread_create(&th[started], NULL, worker, &c) == 0) started++;
    worker(&c);
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&c.mu);
    free(c.geom_price.thr);
    free(c.size_tab.thr);
    return c.error;
}

/* Per-env book capacities drawn uniformly from a list of choices. */
void mbogen_env_caps(uint64_t seed, int64_t n_envs, const int32_t *choices, int32_t n_choices, int32_t *caps_out) {
    for (int64_t e = 0; e < n_envs; e++) {
        uint64_t s = sm_mix(mbogen_env_seed(seed, e) ^ TAG_CAPS);
        caps_out[e] = choices[lemire32(sm_next(&s), (uint32_t)n_choices)];
    }
}

/* The draw thresholds of a model, for the device generator (mbogen_gpu.cu)
 * to draw the same integers: scal = {move, add, partial, delete, burst};
 * geom (price gaps, <= 4096 entries) and size (<= 65536 entries) tables with
 * their lengths and the size table's base value.  Returns -1 on a bad model. */
int mbogen_tables(const mbogen_params *p, uint64_t *scal, uint64_t *geom, int32_t *geom_n, uint64_t *size,
                  int32_t *size_n, int32_t *size_base) {
    double tot = p->mix_add + p->mix_partial + p->mix_delete + p->mix_market;
    if (!(tot > 0.0)) return -1;
    scal[0] = prob_to_u64(p->p_move);
    scal[1] = prob_to_u64(p->mix_add / tot);
    scal[2] = prob_to_u64((p->mix_add + p->mix_partial) / tot);
    scal[3] = prob_to_u64((p->mix_add + p->mix_partial + p->mix_delete) / tot);
    scal[4] = prob_to_u64(p->p_burst);
    cdf_table g, s;
    if (build_geom(&g, p->price_p, 0, 4096)) return -1;
    int rc = p->size_model == 0 ? build_geom(&s, p->size_p, 0, 1 << 16) : build_pareto(&s, p->pareto_alpha, p->size_cap);
    if (rc || s.n > (1 << 16)) { free(g.thr); if (!rc) free(s.thr); return -1; }
    memcpy(geom, g.thr, sizeof(uint64_t) * (size_t)g.n);
    memcpy(size, s.thr, sizeof(uint64_t) * (size_t)s.n);
    *geom_n = g.n;
    *size_n = s.n;
    *size_base = s.base;
    free(g.thr);
    free(s.thr);
    return 0;
}
