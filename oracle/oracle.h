/*
 * oracle.h -- CPU oracle of the batched limit-order-book environment step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header, table or helper with the CUDA engine; both read the same
 * message bytes written by the input generator.
 *
 * What it computes (JaxMARL-HFT, Sec. 4 "Design", the five stages of one
 * environment step): action conversion with carry-over cancels, a random
 * shuffle of the agents' new orders, concatenation (agent cancels, agent
 * orders, then the step's background messages), price-time-priority matching
 * (the continuous double auction of Sec. 2.1) and the step outcomes
 * (observations, portfolio-value rewards per Eq. 1, termination flags).
 * Points the paper leaves open are fixed by the readings listed beside each
 * function in oracle.cpp.
 */
#ifndef LOB_ORACLE_H
#define LOB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NCOUNTERS 16
#define ORC_MAX_PER_TYPE 16   /* agents per type (Table 1 runs 1, 5 and 10) */

typedef struct orc_config {
    int32_t n_envs;
    int32_t n_agents;     /* 0 (pure replay) or 2P: P execution agents (0..P-1), then P market
                             makers (P..2P-1), P <= ORC_MAX_PER_TYPE */
    int32_t cap;          /* book capacity per side when no per-env array is given */
    int32_t top_levels;   /* L aggregated levels per side in the observation */
    int32_t episode_len;  /* T */
    int32_t mm_lot;
    int32_t exec_target;
    int32_t exec_dir;     /* -1 sell task, +1 buy task, 0 drawn per env and episode (Table 2) */
    int32_t action_mode;  /* 0: actions given per step, 1: seeded uniform random policy */
    int32_t trace;        /* bit0: keep the step's fill log; bit1: book snapshot of env 0 after every message */
    int32_t start_px;     /* reference price before the first trade */
    int32_t n_threads;
    int32_t reward_mode;  /* 0: PV change (Eq. 1) for both agents; 1: BuySell (Eq. 4) and
                             2: Spooner (Eq. 3) for the market maker, in quarter-tick*qty */
    int32_t spooner_lambda_pct;  /* lambda of Eq. 3 in percent (0..100) */
    int32_t inv_penalty;  /* quadratic inventory penalty of the market maker, per unit^2 */
    int32_t exec_penalty_milli; /* end-of-episode penalty per unfilled unit of the execution
                             task, in thousandths of a tick; every reward is the floor of
                             its exact value */
    int32_t mm_space;     /* market maker's action space (Sec. 4.1): 0 the 12-way spread/skew
                             head, 1 Fixed Quantity (8 options), 2 directional trading (3) */
    int32_t pv_ref;       /* reference price of Eq. 1 (Table 2): 0 the touch one would liquidate
                             at (best price), 1 the mid price, PV then in half ticks */
} orc_config;

void   *orc_create(const orc_config *cfg, const int32_t *caps /* [n_envs] or NULL */);
void    orc_destroy(void *h);
void    orc_reset(void *h, const uint64_t *env_seeds);
/* One env step for every env.  Env e's background messages of this step are
 * msgs[offsets[e*stride + k] .. offsets[e*stride + k + 1]).  Returns 0, or -6
 * when some message was malformed (it is skipped and counted). */
int     orc_step(void *h, const int32_t *actions, const void *msgs, const int64_t *offsets,
                 int64_t stride, int32_t k);
/* Episodes over one shared message stream (Sec. 3, parallelisation over
 * episodes): all messages of the data set in one contiguous array `msgs`,
 * data step d covering msgs[step_off[d] .. step_off[d+1]).  An episode starts
 * at one of n_starts snapshots: starts[j] gives its first data step, the last
 * trade price at that time and its level counts; levels[j][side][i] = (price,
 * quantity) of level i, side 0 bids best-first, side 1 asks best-first, each
 * side of levels_per_side entries.  After this call orc_reset and
 * orc_step_episodes run in episode mode: at the start of episode k each env
 * draws its snapshot, the book is the snapshot's levels as resting orders,
 * and after the last step of an episode the env starts the next one.  The
 * arrays are copied; msgs must stay valid. */
typedef struct orc_start {
    int32_t data_step, last_px, n_bid, n_ask;
} orc_start;
void    orc_set_episodes(void *h, const void *msgs, const int64_t *step_off, int64_t n_data_steps,
                         const orc_start *starts, const int32_t *levels, int32_t levels_per_side,
                         int64_t n_starts);
int     orc_step_episodes(void *h, const int32_t *actions);
/* First data step of every env's current episode. */
void    orc_get_episode(void *h, int64_t *out);
void    orc_observe(void *h, float *obs, int64_t *rewards, uint8_t *done);
int32_t orc_obs_dim(void *h);
void    orc_get_book(void *h, int64_t env, int32_t *n2, int32_t *px, int32_t *qty, int64_t *id, int64_t *ts);
void    orc_get_counters(void *h, int64_t *out);
void    orc_get_agents(void *h, int64_t *out);
void    orc_get_env_misc(void *h, int64_t *out);
void    orc_get_actions(void *h, int32_t *out);
int64_t orc_get_fills(void *h, int64_t env, void *out, int64_t cap);
int64_t orc_get_snapshots(void *h, void *out, int64_t cap);
/* The random-policy action and shuffle draws, exposed so tests can pin them. */
uint64_t orc_draw(uint64_t env_seed, int64_t t, uint64_t tag, int64_t i);
uint32_t orc_lemire(uint64_t x, uint32_t n);
/* i-th (0-based) output of SplitMix64 started from `state`. */
uint64_t orc_splitmix(uint64_t state, int64_t i);

#ifdef __cplusplus
}
#endif
#endif
