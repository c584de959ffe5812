/*
 * lob.h -- C ABI of the GB300 batched limit-order-book environment (liblob.so).
 *
 * The library steps thousands of independent market environments at once, the
 * environment step of JaxMARL-HFT Sec. 4 ("Design"):
 *   1. action conversion: each agent's action becomes limit orders; the
 *      agent's unmatched orders from the previous step are cancelled unless a
 *      new order sits at the same price level (Sec. 4, "Action Conversion");
 *   2. the agents' new orders are randomly shuffled (Sec. 4, "Random shuffling");
 *   3. cancels, then the agents' orders, then the step's market-replay
 *      messages are concatenated in that order (Sec. 4, "Augment with
 *      market-replay messages");
 *   4. a price-time-priority matching engine (Sec. 2.1) processes them and
 *      records the trades (Sec. 4, "Processing by JAX-LOB");
 *   5. rewards, termination flags and observations are computed (Sec. 4,
 *      "Calculate step outcomes"; portfolio value per Eq. 1).
 * With n_agents = 2P, agents 0..P-1 are order-execution agents (Sec. 4.1.2,
 * 12 discrete actions: four reference prices x {1, 2, 5} lots) and agents
 * P..2P-1 market makers (Sec. 4.1.1; by default 12 discrete actions: one lot
 * at the best bid/ask -/+ {0,1,2} ticks, or one tick into the spread on either
 * side).  The benchmark pair is P = 1.  With n_agents = 0 the library is a
 * plain market-replay engine.
 *
 * Conventions (every entry point):
 *   - returns LOB_OK (0) or a negative LOB_E* code; lob_strerror() names it;
 *   - pointers prefixed d_ are device pointers (any CUDA allocation on the
 *     handle's device), h_ are host pointers; the caller owns every buffer it
 *     passes and keeps it alive while work using it may run;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     device work is enqueued on it and the call returns without waiting,
 *     except where a function says it synchronises;
 *   - errors found on the device (a malformed message, an invalid action, a
 *     bounded wait that expired, a failed check of the checked build) are
 *     recorded in the handle's status word and returned by the next
 *     lob_sync();
 *   - a handle is not thread-safe; handles are independent of each other.
 */
#ifndef LOB_H
#define LOB_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LOB_OK          0
#define LOB_EINVAL     (-1)  /* bad argument, or an action outside [0, 12) */
#define LOB_ENOMEM     (-2)  /* device allocation failed */
#define LOB_ECUDA      (-3)  /* a CUDA call failed */
#define LOB_ETIMEOUT   (-4)  /* a bounded device wait expired */
#define LOB_ECAPACITY  (-5)  /* a size exceeds what the handle or build supports */
#define LOB_EBADMSG    (-6)  /* a message with unknown type/side or non-positive size (skipped) */
#define LOB_ESTATE     (-7)  /* call out of order (no messages bound, window exhausted) */
#define LOB_ECHECK     (-8)  /* checked build only (compiled with LOB_CHECKED): an index bound
                                or a book invariant failed on the device */

/* message types and sides (LOBSTER-style event codes) */
#define LOB_ADD     1
#define LOB_PARTIAL 2
#define LOB_DELETE  3
#define LOB_MARKET  4
#define LOB_BUY     1
#define LOB_SELL   (-1)

/* action sources */
#define LOB_ACT_HOST   0  /* actions passed to lob_step per step */
#define LOB_ACT_RANDOM 1  /* seeded uniform random policy drawn on the device */

#define LOB_NCOUNTERS 16
/* per-env cumulative counters, in this order (int64 each):
 * msgs, agent_msgs, fills, fill_vol, add_vol, mkt_vol, mkt_discard_vol,
 * cancel_vol, cancel_miss, drop_vol, drop_cnt, evict_vol, evict_cnt,
 * bad_msgs, bg_cash, bg_inv */

/* 32-byte market-by-order message record (little endian). */
typedef struct lob_msg {
    int64_t ts;    /* source timestamp (not used by matching) */
    int64_t oid;   /* order id; background ids are >= 0 */
    int32_t px;    /* limit price in ticks (ignored for market orders) */
    int32_t qty;   /* size; cancelled amount for LOB_PARTIAL; ignored for LOB_DELETE */
    int16_t type;  /* LOB_ADD .. LOB_MARKET */
    int16_t side;  /* LOB_BUY or LOB_SELL */
    int32_t pad;
} lob_msg;

/* Compact 16-byte background record: px and qty as above, word = id << 4 |
 * (side == LOB_SELL) << 3 | type, with ids in [LOB_MSG16_ID_MIN,
 * LOB_MSG16_ID_MAX] and type 0 for a record whose type or side is invalid
 * (skipped and counted like any malformed message).  Half the bytes of
 * lob_msg for the same step results. */
typedef struct lob_msg16 {
    int32_t px;
    int32_t qty;
    int64_t word;
} lob_msg16;
#define LOB_MSG16_ID_MIN (-(1LL << 59))
#define LOB_MSG16_ID_MAX ((1LL << 59) - 1)

/* 32-byte trade record of the fill log. */
typedef struct lob_fill {
    int64_t maker_id;   /* resting order */
    int64_t taker_id;   /* incoming order */
    int32_t px;         /* trade price = resting order's price */
    int32_t qty;
    int32_t msg_idx;    /* index of the incoming message within the step's processing order */
    int32_t taker_side; /* LOB_BUY / LOB_SELL */
} lob_fill;

#define LOB_MAX_PER_TYPE 16   /* agents of each type per env (Table 1 runs 1, 5 and 10) */

typedef struct lob_config {
    int32_t n_envs;        /* >= 1 */
    int32_t n_agents;      /* 0 (replay only) or 2P, P <= LOB_MAX_PER_TYPE agents of each type (Sec. 3):
                              agents 0..P-1 execute (each its own task), P..2P-1 make markets;
                              P = 1 is the benchmark pair (execution agent 0, market maker 1) */
    int32_t cap_per_side;  /* book capacity per side, 1..LOB_MAX_CAP (Table 2: 100) */
    int32_t top_levels;    /* L aggregated levels per side in the observation, 1..64 */
    int32_t episode_len;   /* T steps per episode, >= 1 */
    int32_t mm_lot;        /* market maker's quote size, >= 1 */
    int32_t exec_target;   /* execution task size, >= 0 */
    int32_t exec_dir;      /* LOB_SELL or LOB_BUY: side of the execution task; 0 = drawn per env and
                              episode (Table 2: uniformly sampled) from the top bit of a SplitMix64
                              draw keyed (seed, episode, LOB_TAG_TASKDIR), set -> sell; the
                              remaining-target observation is then signed (+ buy, - sell) */
    int32_t action_mode;   /* LOB_ACT_HOST or LOB_ACT_RANDOM */
    int32_t trace;         /* bit0: fill log; bit1: env 0 book snapshot after every message */
    int32_t start_px;      /* reference price before the first trade (e.g. 10000) */
    int32_t warps_per_block; /* launch shape hint; 0 = library default */
    /* Reward of the market maker (Sec. 5):
     *   LOB_REWARD_PV       change of PV = Q_inv * P_ref + Cash (Eq. 1), ticks x qty;
     *   LOB_REWARD_BUYSELL  Psi_b + Psi_s (Eq. 4), in quarter ticks x qty;
     *   LOB_REWARD_SPOONER  Psi_b + Psi_s + Psi_INV - (1 - lambda) max(0, Psi_INV) (Eq. 3),
     *                       in quarter ticks x qty.
     * Psi_b = sum over this step's buys of (Mbar - P) Q, Psi_s = sum over its sells of
     * (P - Mbar) Q, Mbar = mean of the mids at the start and the end of the step,
     * Psi_INV = I (M_end - M_start) with I the inventory at the end of the step; a mid
     * is that of the reference touches (last trade price on an empty side).  The
     * execution agent's reward is always the Eq. 1 change.  Every reward is the floor
     * of its exact value. */
    int32_t reward_mode;
    int32_t spooner_lambda_pct;  /* lambda of Eq. 3 in percent, 0..100 */
    int32_t inv_penalty;         /* rho >= 0: market maker's reward -= rho * inventory^2 (Table 2) */
    int32_t exec_penalty_milli;  /* >= 0: at the last step of the episode the execution agent's
                                    reward -= this * unfilled units / 1000 (Table 2's unfilled
                                    order penalty, in thousandths of a tick per unit) */
    /* Market maker's action space (Sec. 4.1.1), each quote of mm_lot; bb / ba the touches:
     *   LOB_MM_SPREAD_SKEW  12 actions: 0 none; 1..9 bid bb - (a-1)/3, ask ba + (a-1)%3;
     *                       10 bid bb+1, ask ba; 11 bid bb, ask ba-1
     *   LOB_MM_FIXED_QUANT   8 actions: 0 none; 1 bb-2 / ba+2; 2 bb-4 / ba+4; 3 bb+1 / ba-1;
     *                       4 bid bb-2 only; 5 ask ba+2 only; 6 bb-5 / ba-1; 7 bb+1 / ba+5
     *   LOB_MM_DIRECTIONAL   3 actions: 0 none; 1 bid at bb; 2 ask at ba
     * The random policy draws the market maker's action over its space; host
     * actions outside it give LOB_EINVAL.  lob_rollout_policy (12 logits)
     * needs LOB_MM_SPREAD_SKEW. */
    int32_t mm_space;
    /* Reference price P_ref of Eq. 1 (Table 2's value reference price):
     *   LOB_PV_TOUCH  the touch one would liquidate at (best bid if long, best ask if short)
     *   LOB_PV_MID    the mid price; PV is then exact in half ticks and the Eq. 1 rewards
     *                 and the unfilled-task penalty are reported in half ticks x qty */
    int32_t pv_ref;
    int32_t reserved[2];         /* must be zero */
} lob_config;

#define LOB_PV_TOUCH 0
#define LOB_PV_MID   1

#define LOB_MM_SPREAD_SKEW 0
#define LOB_MM_FIXED_QUANT 1
#define LOB_MM_DIRECTIONAL 2

#define LOB_REWARD_PV      0
#define LOB_REWARD_BUYSELL 1
#define LOB_REWARD_SPOONER 2

#define LOB_MAX_CAP 1024   /* largest per-side capacity the library supports */

typedef struct lob_handle lob_handle;

/* Observation length per agent: 4 * top_levels + 5 (0 when n_agents == 0).
 * Layout per agent: [bid (px - anchor, qty) x L][ask (px - anchor, qty) x L],
 * inventory, cash, time left (T - t) / T, remaining execution target (execution agents)
 * or 0, the agent's own resting quantity.  anchor = floor((best bid + best
 * ask) / 2); an empty side's touch is the last trade price; missing levels
 * are (0, 0). */
int32_t lob_obs_dim(const lob_config *cfg);

/* Create a handle on the current CUDA device and allocate its state (books,
 * agent state, counters).  h_caps: optional host array [n_envs] of per-env
 * capacities (each 1..LOB_MAX_CAP) overriding cap_per_side.  The handle starts
 * unusable until lob_reset(). */
int lob_create(const lob_config *cfg, const int32_t *h_caps, lob_handle **out);
int lob_destroy(lob_handle *h);   /* frees device state; synchronises the device */

/* Bind a window of background messages (the contiguous store with start
 * indices of Sec. 4): env e's messages of window step k are
 * d_msgs[d_offsets[e * stride + k] .. d_offsets[e * stride + k + 1]).
 * Offsets are message indices; stride >= n_steps + 1.  The buffers are
 * borrowed and must stay alive while steps using them run.  Rebinding resets
 * the window cursor to 0 without touching env state. */
int lob_load_messages(lob_handle *h, const lob_msg *d_msgs, const int64_t *d_offsets,
                      int32_t n_steps, int64_t stride);
/* The same for a stream of compact 16-byte records (d_msgs 16-byte aligned,
 * like every bound message buffer: LOB_EINVAL otherwise). */
int lob_load_messages16(lob_handle *h, const lob_msg16 *d_msgs, const int64_t *d_offsets,
                        int32_t n_steps, int64_t stride);
/* Device-side conversion of n records to the compact form.  d_status
 * (optional, device int32) is set to LOB_EINVAL if an id does not fit (that
 * record becomes a malformed one). */
int lob_pack_messages16(const lob_msg *d_src, int64_t n, lob_msg16 *d_dst, int32_t *d_status, void *stream);

/* ---- Episodes over one shared message stream (Sec. 3: the whole data set
 * in one contiguous array, runtime indexing of episode starts, episodes free
 * to overlap; the book at an episode start initialised from the state of the
 * book at that time).
 *
 * d_msgs / d_step_offsets (device, borrowed, must stay alive): data step d
 * covers d_msgs[d_step_offsets[d] .. d_step_offsets[d + 1]), d < n_data_steps.
 * h_starts [n_starts] and h_levels [n_starts][2][levels_per_side][2] (host,
 * copied): snapshot j starts episodes at data step h_starts[j].data_step
 * (<= n_data_steps - T) with last trade price last_px; levels (price,
 * quantity) best first, side 0 bids (prices strictly falling), side 1 asks
 * (strictly rising), n_bid / n_ask of them (<= levels_per_side and <= the
 * capacity), quantities >= 1, best bid < best ask when both sides exist.
 *
 * In episode mode episode k of env e starts at snapshot
 * j = Lemire(SplitMix64 output 1 from key(seed_e, k, LOB_TAG_EPISODE), n_starts)
 * (key(s, k, tag) = mix(mix(s ^ tag) + GAMMA (k + 1)), the keying of the
 * shuffle and the random policy): its book is the snapshot's levels as one
 * resting order each, bids then asks, best first, arrival stamps 0, 1, ...,
 * ids LOB_INIT_ID + the same index; agents start flat.  Step t reads data
 * step start + (t mod T).  After an episode's last step the env starts the
 * next episode at once: that step reports its own rewards and done = 1 with
 * the new episode's first observation.  Steps never run out (no LOB_ESTATE
 * at t == T).  Requires one capacity for all envs (no h_caps at create).
 * The mode holds until lob_load_messages; either call requires lob_reset
 * before the next step.  LOB_EINVAL on a table that breaks the rules above. */
#define LOB_INIT_ID 0x4000000000000000LL
#define LOB_TAG_EPISODE 0x4550495344450003ULL
#define LOB_TAG_TASKDIR 0x5441534B44495204ULL
typedef struct lob_start {
    int32_t data_step;
    int32_t last_px;
    int32_t n_bid, n_ask;
} lob_start;
int lob_set_episodes(lob_handle *h, const lob_msg *d_msgs, const int64_t *d_step_offsets, int64_t n_data_steps,
                     const lob_start *h_starts, const int32_t *h_levels, int32_t levels_per_side,
                     int64_t n_starts);
/* Episode mode over a shared stream of compact 16-byte records. */
int lob_set_episodes16(lob_handle *h, const lob_msg16 *d_msgs, const int64_t *d_step_offsets, int64_t n_data_steps,
                       const lob_start *h_starts, const int32_t *h_levels, int32_t levels_per_side,
                       int64_t n_starts);
/* Device int32 [n_envs]: the first data step of every env's current episode
 * (episode mode; 0 otherwise). */
int lob_get_episode_starts(lob_handle *h, int32_t *d_out, void *stream);

/* Start a new episode in every env: zero agent state and counters, step
 * t = 0, and an empty book (episode mode: the book of the drawn snapshot).
 * d_env_seeds: device [n_envs] uint64 keys for the shuffle, the random policy
 * and the episode draws.  The observation buffer then holds the reset
 * observation (the starting book's levels -- all (0, 0) for an empty book --,
 * zero inventory and cash, time left 1, the full execution target for
 * the execution agents). */
int lob_reset(lob_handle *h, const uint64_t *d_env_seeds, void *stream);

/* One environment step for every env (stages 1-5 above), consuming the next
 * window step of bound messages.  d_actions: device int32 [n_envs][n_agents] in
 * LOB_ACT_HOST mode, ignored (may be NULL) otherwise.  Fails with LOB_ESTATE
 * when the episode is over (t == T) or the window is exhausted (outside
 * episode mode). */
int lob_step(lob_handle *h, const int32_t *d_actions, void *stream);

/* Outputs of the last step: d_obs float [n_envs][n_agents][obs_dim],
 * d_rewards int64 [n_envs][n_agents] (change of portfolio value, Eq. 1, in
 * tick * qty), d_done uint8 [n_envs].  Any pointer may be NULL. */
int lob_observe(lob_handle *h, float *d_obs, int64_t *d_rewards, uint8_t *d_done, void *stream);

/* Several steps in one persistent launch, the book kept on chip between
 * steps.  Outputs of step i go to d_obs + i * n_envs * n_agents * obs_dim etc.
 * (any may be NULL).  Actions: LOB_ACT_RANDOM, or LOB_ACT_HOST with
 * d_actions [n_steps][n_envs][n_agents]. */
int lob_rollout(lob_handle *h, int32_t n_steps, const int32_t *d_actions, float *d_obs,
                int64_t *d_rewards, uint8_t *d_done, void *stream);

/* ---- Actor-critic policy (IPPO networks, Sec. 4.2: separate weights per
 * agent).  Per agent: x = obs * s (fixed per-feature input scale: level
 * prices 1/10, level sizes 1/1000, inventory 1/100, cash 1e-6, time left 1,
 * remaining target and own resting quantity 1/100), h1 = tanh(W1 x + b1),
 * h2 = tanh(W2 h1 + b2), y = W3 h2 + b3 with 128 hidden units; y[0..11] are
 * the logits of the 12 actions, y[12] the value; the action is the argmax of
 * the logits (ties to the lowest index). */
#define LOB_POLICY_HIDDEN 128
#define LOB_PREC_FP32 0   /* FP32 FMAs on the CUDA cores */
#define LOB_PREC_BF16 1   /* BF16 operands, FP32 accumulation, tcgen05 tensor cores */
/* lob_rollout_policy only: the BF16 forward inside the step kernel, one
 * launch for the whole rollout (observations and actions stay on chip).
 * It takes the two-agent benchmark configuration on one capacity class of
 * 65..256 slots per side, obs_dim <= 48, the PV reward with the touch
 * reference and no penalties, a fixed task side (exec_dir +1 or -1), no
 * trace, no episode mode; anything else is LOB_EINVAL.  Its actions equal LOB_PREC_BF16's wherever the two forwards
 * round alike (the hidden layers are the same BF16 products; the head sums
 * in another order). */
#define LOB_PREC_BF16_FUSED 2
typedef struct lob_policy lob_policy;
/* Floats per agent in the parameter block: W1 [128][obs_dim], b1 [128],
 * W2 [128][128], b2 [128], W3 [13][128], b3 [13], in that order (row-major,
 * W[out][in]).  0 for an unsupported obs_dim (1..128). */
int64_t lob_policy_param_count(int32_t obs_dim);
/* Upload n_agents (1 .. 2 * LOB_MAX_PER_TYPE; every agent its own weights,
 * Sec. 4.2) consecutive parameter blocks from the host; the
 * library keeps an FP32 copy and a BF16 copy packed for the tensor cores. */
int lob_policy_create(int32_t n_agents, int32_t obs_dim, const float *h_params, lob_policy **out);
int lob_policy_destroy(lob_policy *pol);   /* synchronises the device */
/* Forward of every (env, agent) row: d_obs float [n_envs][n_agents][obs_dim];
 * outputs (any may be NULL) d_logits float [n_envs][n_agents][12], d_values
 * float [n_envs][n_agents], d_actions int32 [n_envs][n_agents]. */
int lob_policy_forward(lob_policy *pol, const float *d_obs, int32_t n_envs, int32_t precision, float *d_logits,
                       float *d_values, int32_t *d_actions, void *stream);
/* Wait for `stream` and report the policy's device status (LOB_ETIMEOUT if a
 * bounded tensor-core wait expired). */
int lob_policy_sync(lob_policy *pol, void *stream);
/* Rollout with the policy in the loop (the handle must use LOB_ACT_HOST):
 * for each of n_steps steps, the policy acts on the current observation
 * (after lob_reset: the reset observation) and lob_step runs with those
 * actions, all enqueued on `stream` with no host synchronisation, so the
 * sequence can be captured in a CUDA graph.  Per-step outputs (any may be
 * NULL): d_obs [n_steps][n_envs][n_agents][obs_dim] (observation after step
 * i), d_rewards [n_steps][n_envs][n_agents], d_done [n_steps][n_envs],
 * d_actions [n_steps][n_envs][n_agents] (the actions taken at step i).  The
 * policy has one network per agent of the handle; the market makers use the
 * 12-way head. */
int lob_rollout_policy(lob_handle *h, lob_policy *pol, int32_t n_steps, int32_t precision, float *d_obs,
                       int64_t *d_rewards, uint8_t *d_done, int32_t *d_actions, void *stream);
/* The FP32 parameter blocks of every agent (layout of lob_policy_param_count)
 * into d_out float [n_agents][P] (device, caller-owned). */
int lob_policy_get_params(lob_policy *pol, float *d_out, void *stream);

/* ---- IPPO update (Sec. 4.2: independent PPO, each agent's network updated
 * from its own data only; Sec. 6 runs rollouts and updates on the GPU).  The
 * paper fixes no algorithmic detail, so this is the textbook update:
 *   advantages by GAE (Schulman et al. 2016): delta_t = r_t + gamma (1 - d_t)
 *     V_{t+1} - V_t, A_t = delta_t + gamma lambda (1 - d_t) A_{t+1}, targets
 *     R_t = A_t + V_t, with r_t = reward_scale * reward;
 *   per minibatch the mean of -min(rho A', clip(rho, 1 - eps, 1 + eps) A')
 *     + vf_coef (V - R)^2 / 2 - ent_coef * entropy (Schulman et al. 2017),
 *     rho = exp(log pi(a) - logp_old), A' the advantage normalised over the
 *     minibatch (population std + 1e-8);
 *   its gradient through the network (forward and backward as BF16
 *     tensor-core contractions with FP32 accumulation), clipped to a global
 *     L2 norm of max_grad_norm, then one Adam step (Kingma & Ba 2015, bias
 *     corrected) on the FP32 weights, which are repacked for the forward.
 * One call = one epoch: each agent's samples in the order d_perm gives, cut
 * into n_minibatches equal consecutive parts, one Adam step per part. */
typedef struct lob_ppo_hparams {
    float gamma, gae_lambda, clip_eps, vf_coef, ent_coef;
    float lr, beta1, beta2, adam_eps, max_grad_norm, reward_scale;
    int32_t n_minibatches;
} lob_ppo_hparams;
typedef struct lob_ppo_batch {
    int32_t T, n_envs;            /* rollout length and envs; samples per agent N = T * n_envs */
    const float *d_obs;           /* [T][n_envs][A][D]: the observation each action was taken on */
    const int32_t *d_actions;     /* [T][n_envs][A] in [0, 12) */
    const float *d_logp_old;      /* [T][n_envs][A]: log-probability of the action under the rollout's policy */
    const float *d_values;        /* [T + 1][n_envs][A]: the critic's values, row T bootstraps */
    const int64_t *d_rewards;     /* [T][n_envs][A] */
    const uint8_t *d_done;        /* [T][n_envs]: 1 where step t ended the episode */
    const int32_t *d_perm;        /* [A][N]: each agent's sample order (sample t * n_envs + e) */
    float *d_grad_out;            /* NULL, or [n_minibatches][A][P]: each minibatch's gradient before clipping */
} lob_ppo_batch;
/* All pointers are device pointers owned by the caller and read on `stream`.
 * The first call allocates the optimiser state (Adam moments, step count)
 * and work buffers in the policy; later calls continue it.  LOB_EINVAL for a
 * bad argument or N not divisible by n_minibatches, LOB_ECAPACITY when
 * obs_dim + 1 > 48 (the update's operand tiles hold 48 input columns: up to
 * 10 observation levels), LOB_ENOMEM, LOB_ECUDA.  A bounded tensor-core wait
 * that expires is reported by lob_policy_sync. */
int lob_ppo_update(lob_policy *pol, const lob_ppo_batch *batch, const lob_ppo_hparams *hp, void *stream);

/* Host-buffer convenience step: copies this step's background messages
 * (h_msgs[h_offsets[e] .. h_offsets[e + 1]], h_offsets [n_envs + 1]) and
 * actions to the device, steps, and copies obs / rewards / done back to host
 * buffers (any output may be NULL).  Synchronises the stream. */
int lob_step_host(lob_handle *h, const lob_msg *h_msgs, const int64_t *h_offsets,
                  const int32_t *h_actions, float *h_obs, int64_t *h_rewards,
                  uint8_t *h_done, void *stream);
/* The same step, pipelined; returns without synchronising.  When every
 * buffer is page-locked host memory that the GPU maps at the same address
 * (cudaMallocHost, cudaHostAlloc, pinned torch tensors) and the messages are
 * 16-byte aligned, the step kernel itself reads the messages, offsets and
 * actions and writes the outputs in host memory over the coherent CPU-GPU
 * link (zero copy): one launch per call, and the handle's own output buffers
 * (lob_observe) are not updated by such a call.  Otherwise the inputs go up
 * on the handle's copy stream into one of two device staging slots (so they
 * overlap the previous step), and the outputs come back on `stream`.  The
 * caller keeps the input buffers unchanged until `stream` has run past this
 * step, and reads the outputs only after synchronising it.  h_offsets is read
 * during the call.  Same errors as lob_step_host. */
int lob_step_host_async(lob_handle *h, const lob_msg *h_msgs, const int64_t *h_offsets,
                        const int32_t *h_actions, float *h_obs, int64_t *h_rewards,
                        uint8_t *h_done, void *stream);

/* Book of every env in the canonical layout, per env a record of
 * 8 + 48 * C bytes (C = that env's capacity): int32 n[2]; int32 px[2][C];
 * int32 qty[2][C]; int64 id[2][C]; int64 ts[2][C]; side 0 = bids, 1 = asks,
 * each in priority order, unused slots zero.  Records are packed back to
 * back in env order.  d_out must hold lob_book_bytes() bytes. */
int64_t lob_book_bytes(const lob_handle *h);
int lob_get_book(lob_handle *h, void *d_out, void *stream);

/* d_out int64 [n_envs][LOB_NCOUNTERS]. */
int lob_get_counters(lob_handle *h, int64_t *d_out, void *stream);
/* d_out int64 [n_envs][n_agents][4]: inventory, cash, last portfolio value, executed volume. */
int lob_get_agents(lob_handle *h, int64_t *d_out, void *stream);
/* d_out int64 [n_envs][4]: next arrival stamp, next agent order sequence, last trade price, step t. */
int lob_get_env_misc(lob_handle *h, int64_t *d_out, void *stream);
/* d_out int32 [n_envs][n_agents]: the actions used in the last step. */
int lob_get_actions(lob_handle *h, int32_t *d_out, void *stream);
/* Statistics for byte accounting (no counterpart in the paper): adds the
 * number of resting orders of every env, bids plus asks, to the int64 at
 * d_acc (device, caller-owned, not cleared), on the stream, without a host
 * synchronisation; one small kernel.  LOB_EINVAL for a NULL argument. */
int lob_live_orders(lob_handle *h, int64_t *d_acc, void *stream);

/* Trace buffers (caller-owned, device): fill log of the last step for every
 * env, d_fills [n_envs][fill_cap] with d_fill_counts int32 [n_envs] (counts
 * beyond fill_cap are still counted); env 0's book after every message of
 * the last step, d_snaps [snap_cap] canonical records (see lob_get_book) with
 * d_snap_count int64.  Pass NULL to disable either. */
int lob_set_trace(lob_handle *h, lob_fill *d_fills, int32_t fill_cap, int32_t *d_fill_counts,
                  void *d_snaps, int64_t snap_cap, int64_t *d_snap_count);

/* Wait for the handle's work on `stream`, then return and clear the device
 * status: LOB_ETIMEOUT, else LOB_ECHECK (checked build), else LOB_EINVAL (an
 * invalid action), else LOB_EBADMSG (a malformed message), else LOB_OK. */
int lob_sync(lob_handle *h, void *stream);
/* Launch-shape control used by the autotuner: warps per block for the step
 * kernels (1..8) and whether they take envs from a work queue. */
int lob_set_launch(lob_handle *h, int32_t warps_per_block, int32_t persistent);
/* Launch mode persistent = 2 (set by lob_set_launch or by this call): one
 * persistent kernel runs the envs of every capacity class up to 512 slots per
 * side (a handle with larger books keeps one launch per class).  Each block
 * holds warps_per_class[k] warps of class k (k = 0 .. 4: 32 .. 512 slots;
 * LOB_NCLASSES entries, class 5 must be 0; 1 .. 8 warps in all, their shared
 * memory within one block's); a warp takes envs of its own class from that
 * class's queue and, when it is empty, envs of smaller classes.  Every class
 * with envs needs a warp of its class or of a larger one.  LOB_EINVAL or
 * LOB_ECAPACITY otherwise.  lob_set_launch(h, w, 2) derives a split from the
 * classes' env counts. */
#define LOB_NCLASSES 6
int lob_set_multi_split(lob_handle *h, const int32_t *warps_per_class);
/* Threads per env: 32 (default, one warp runs both sides of an env's book) or
 * 64: the plain step -- the benchmark pair or no agents, a fixed task side,
 * the PV reward, no trace, capacity classes of 33..256 slots per side, no
 * work queue (persistent 0) -- runs with one warp per book side.  Each warp
 * handles the messages that change its side (its rests and cancels, and the
 * takes of the other side's incoming orders); a limit add that may cross
 * waits for the opposite warp's take to post its unfilled remainder; arrival
 * stamps and the per-owner totals are merged at every staged chunk and every
 * step's end.  Results are identical to 32; launches that do not qualify run
 * one warp per env.  On the 1,024-env benchmark workload it measured about
 * twice the step time of 32 (more instructions in all and two code paths per
 * SM), so 32 stays the default.  LOB_EINVAL for other values. */
int lob_set_threads_per_env(lob_handle *h, int32_t threads);
/* Message-tile size: each env's messages of a step are copied from device
 * memory into shared memory `records` at a time (16, 32 -- the default -- or
 * 64), double-buffered, and the step processes one staged tile while the next
 * is in flight.  It applies to launches of the plain step (the benchmark pair
 * or no agents, a fixed task side, the PV reward, device-resident 32-byte
 * records, no trace), which has an instance per size; 64-record tiles take
 * (2 x 64 + 1) x 32 bytes of shared memory per warp beyond its block, so
 * fewer warps may fit a block of the larger capacity classes.  Every other
 * launch (extended, traced, several agents per type, the one-kernel
 * multi-class form, the fused policy rollout, 64 threads per env) stages 32.
 * Results do not depend on it.  LOB_EINVAL for other values. */
int lob_set_tile_records(lob_handle *h, int32_t records);
/* Failure-detection hook.  `cycles` bounds every wait of the step kernels on
 * a message tile, in SM cycles (0 = the default, about one second).  hold = 1
 * makes the next step or rollout launch leave each env's first message tile
 * unrequested (device-resident messages only), so that the wait for it runs
 * out: the launch stops every env at that point, its outputs and env state
 * are not written (counters may have advanced), and lob_sync reports
 * LOB_ETIMEOUT.  The hold applies to that one launch; continue with lob_reset
 * (or lob_load of a checkpoint).  Returns LOB_EINVAL for cycles < 0 or hold
 * not 0/1. */
int lob_debug_wait(lob_handle *h, int64_t cycles, int32_t hold);
/* ---- Checkpoint / resume of every env (books, per-env scalars, counters,
 * seeds, the last step's outputs, the step t and the window cursor).  The
 * bound message window is not part of it: bind the same window before
 * continuing.  dst / src may be host or device memory (copied with
 * cudaMemcpyDefault semantics on `stream`; host memory should be pinned).
 * lob_load requires a handle created with the same configuration and
 * capacities; it returns LOB_EINVAL for a checkpoint of another shape.  Both
 * calls synchronise `stream`. */
int64_t lob_checkpoint_bytes(const lob_handle *h);
int lob_save(lob_handle *h, void *dst, void *stream);
int lob_load(lob_handle *h, const void *src, void *stream);

/* Work hint for the persistent (work-queue) launches: h_cost [n_envs] host
 * floats, larger = more work; each capacity class then hands out its envs
 * longest first.  NULL restores env order. */
int lob_set_env_costs(lob_handle *h, const float *h_cost);
/* Number of kernels the library launched since creation (for accounting). */
int64_t lob_kernel_launches(const lob_handle *h);

/* ---- Allocation-free step (the paper has no counterpart) ------------------
 * For callers that cannot call cudaMalloc: code embedded in a host program
 * whose device memory is all reserved up front by its own allocator or a fixed
 * memory budget, and loops that must not pay cudaMalloc's implicit device-wide
 * synchronisation.  No handle is used: the caller passes every input and
 * output buffer, and the work queue plus the env tables the step kernel
 * needs live in one file-scope static device array of this library
 * (LOB_NOALLOC_MAX_ENVS entries, about 256 KB, held by every GPU that loads
 * the library until the process exits).  The function calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  Every call shares the array and overwrites it (the
 * queue counter is cleared at the start of each call), so calls that overlap
 * on the GPU -- on two streams, or on two host threads -- race: serialise
 * them.
 *
 * It runs one env step for every env (the same stages, kernel and results as
 * lob_step in persistent mode) on caller-owned state:
 *   cfg           uniform capacity cap_per_side, trace must be 0,
 *                 warps_per_block 0..8 (0 = 4, fewer where a block's shared
 *                 memory cannot hold that many books); n_envs <= LOB_NOALLOC_MAX_ENVS;
 *                 n_agents 0 or 2 with the defaults of every other option
 *                 (LOB_REWARD_PV, no penalties, LOB_MM_SPREAD_SKEW, LOB_PV_TOUCH,
 *                 exec_dir LOB_SELL or LOB_BUY), else LOB_EINVAL
 *   d_books       n_envs book blocks, each 48*S bytes rounded up to a multiple
 *                 of 256, S = the smallest power of two >= max(cap, 32);
 *                 256-byte aligned.  At t == 0 their contents are ignored
 *                 (any bytes will do); afterwards they are the library's.
 *   d_env_state   n_envs * 128 bytes of per-env scalars (opaque), 16-byte aligned
 *   d_counters    int64 [n_envs][LOB_NCOUNTERS]
 *   d_env_seeds   uint64 [n_envs]
 *   d_msgs, d_offsets, stride, k   as lob_load_messages: this step uses
 *                 window step k; d_msgs 16-byte aligned
 *   t             episode step; t == 0 first resets every env (empty books,
 *                 zero agents and counters), as lob_reset does
 *   d_actions     int32 [n_envs][2] in LOB_ACT_HOST mode, else ignored
 *   d_obs, d_rewards, d_done   outputs as lob_observe (any may be NULL)
 *   d_status      int32, OR-ed with 1 (malformed message), 2 (invalid action),
 *                 4 (bounded wait expired); the caller clears it
 * Returns LOB_EINVAL for a bad argument (including a pointer off the
 * alignment stated above, refused before anything is launched), LOB_ECAPACITY
 * when n_envs or the capacity exceeds the limits above, LOB_ECUDA if a CUDA
 * call fails. */
#define LOB_NOALLOC_MAX_ENVS 16384
typedef struct lob_noalloc_args {
    const lob_config *cfg;
    void *d_books;
    void *d_env_state;
    int64_t *d_counters;
    const uint64_t *d_env_seeds;
    const lob_msg *d_msgs;
    const int64_t *d_offsets;
    int64_t stride;
    int32_t k;
    int32_t t;
    const int32_t *d_actions;
    float *d_obs;
    int64_t *d_rewards;
    uint8_t *d_done;
    int32_t *d_status;
} lob_noalloc_args;
int lob_step_noalloc(const lob_noalloc_args *args, void *stream);

const char *lob_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LOB_H */
