// oracle.cpp -- plain, slow CPU oracle of the batched LOB environment step.
//
// TEST INFRASTRUCTURE ONLY (see oracle.h).  Written for a reader checking it
// against the paper: one std::map of FIFO price levels per side, one env at a
// time, every stage of Sec. 4's environment step in the paper's order.
//
// Readings of points the paper leaves open (JaxMARL-HFT defers matching to the
// JAX-LOB simulator, which is not part of the paper):
//   * priority: best price first, FIFO (arrival stamp) within a price; a trade
//     executes at the resting order's price (Sec. 2.1, continuous double
//     auction with price and time priority);
//   * arrival stamp: a per-env counter, taken when an order comes to rest;
//   * a marketable limit order matches up to its limit price, then rests;
//     a market order's unfilled remainder is discarded;
//   * partial cancel removes min(c, qty) and keeps time priority; delete and
//     partial cancel look up (side, price level, id); a miss is a no-op;
//   * full side (capacity C, Table 2 "book capacity 100 orders"): an incoming
//     remainder strictly better than the worst resting price evicts the
//     worst-priced, latest-arrived order; otherwise the remainder is dropped;
//   * agent order ids are negative: id = -(1 + agent + A * seq);
//   * carry-over (Sec. 4, Action Conversion): an agent's resting order at the
//     same (side, price) as one of its new orders is kept; the new order sends
//     only the quantity beyond what is kept; every other resting order of the
//     agent is cancelled;
//   * shuffle (Sec. 4, Random shuffling): Fisher-Yates over the agents' new
//     orders with SplitMix64 draws keyed by (env seed, step);
//   * concatenation (Sec. 4, Augment with market-replay messages): agent
//     cancels (agent 0, then agent 1; bids, then asks; book order), the
//     shuffled new orders, then the step's background messages in order;
//   * reward: change of portfolio value PV = Q_inv * P_ref + Cash (Eq. 1) with
//     P_ref the touch one would liquidate at (best bid if long, best ask if
//     short); an empty side's touch is the last trade price;
//   * episodes (Sec. 3, parallelisation over episodes): one contiguous message
//     array with per-data-step start indices; episode k of an env starts at
//     the snapshot drawn with a SplitMix64 draw keyed by (env seed, k); the
//     snapshot's levels become resting orders (one per level, bids then asks,
//     best first, arrival stamps 0, 1, ...; ids INIT_ID + the same index);
//     agents start flat; after the episode's last step the env starts the
//     next episode and reports that episode's first observation, with the
//     finished step's rewards and done flag.
#include "oracle.h"

#include <algorithm>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <thread>
#include <vector>

namespace {

enum { ADD = 1, PARTIAL = 2, DELETE = 3, MARKET = 4 };
enum { BUY = 1, SELL = -1 };
enum {
    C_MSGS, C_AGENT_MSGS, C_FILLS, C_FILL_VOL, C_ADD_VOL, C_MKT_VOL, C_MKT_DISCARD,
    C_CANCEL_VOL, C_CANCEL_MISS, C_DROP_VOL, C_DROP_CNT, C_EVICT_VOL, C_EVICT_CNT,
    C_BAD_MSGS, C_BG_CASH, C_BG_INV
};

struct Msg {  // the generator's 32-byte record
    int64_t ts, oid;
    int32_t px, qty;
    int16_t type, side;
    int32_t pad;
};
static_assert(sizeof(Msg) == 32, "message record is 32 bytes");

struct Fill {
    int64_t maker_id, taker_id;
    int32_t px, qty, msg_idx, taker_side;
};
static_assert(sizeof(Fill) == 32, "fill record is 32 bytes");

struct Order {
    int64_t id, ts;
    int32_t px, qty;
};

// Wrapping int64 arithmetic (two's complement), written without signed overflow.
inline int64_t wadd(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
inline int64_t wsub(int64_t a, int64_t b) { return (int64_t)((uint64_t)a - (uint64_t)b); }
inline int64_t wmul(int64_t a, int64_t b) { return (int64_t)((uint64_t)a * (uint64_t)b); }

// One side of the book: price -> FIFO queue of resting orders.
struct Side {
    bool is_bid = true;
    std::map<int32_t, std::deque<Order>> levels;
    int count = 0;

    bool better(int32_t a, int32_t b) const { return is_bid ? a > b : a < b; }
    std::map<int32_t, std::deque<Order>>::iterator best() {
        return is_bid ? std::prev(levels.end()) : levels.begin();
    }
    std::map<int32_t, std::deque<Order>>::iterator worst() {
        return is_bid ? levels.begin() : std::prev(levels.end());
    }
    // Orders in priority order (best price first, then arrival).
    std::vector<Order> ordered() const {
        std::vector<Order> out;
        if (is_bid) {
            for (auto it = levels.rbegin(); it != levels.rend(); ++it)
                for (const Order &o : it->second) out.push_back(o);
        } else {
            for (auto it = levels.begin(); it != levels.end(); ++it)
                for (const Order &o : it->second) out.push_back(o);
        }
        return out;
    }
    // Aggregated levels in priority order: (price, total quantity).
    std::vector<std::pair<int32_t, int64_t>> aggregated() const {
        std::vector<std::pair<int32_t, int64_t>> out;
        auto add = [&](const std::pair<const int32_t, std::deque<Order>> &lv) {
            int64_t q = 0;
            for (const Order &o : lv.second) q += o.qty;
            out.push_back({lv.first, q});
        };
        if (is_bid) for (auto it = levels.rbegin(); it != levels.rend(); ++it) add(*it);
        else for (auto it = levels.begin(); it != levels.end(); ++it) add(*it);
        return out;
    }
};

struct Agent {
    int64_t inv = 0, cash = 0, pv_prev = 0, exec_done = 0;
    // this step's fills, split by direction (for the Eq. 3 / Eq. 4 rewards)
    int64_t buy_q = 0, buy_n = 0, sell_q = 0, sell_n = 0;
};

// ---- SplitMix64 (Steele, Lea & Flood 2014) and Lemire's bounded map ------
const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;
uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// The i-th (0-based) output of a SplitMix64 generator whose state starts at
// key(t) = mix64(mix64(env_seed ^ tag) + GAMMA * (t + 1)).
uint64_t draw(uint64_t env_seed, int64_t t, uint64_t tag, int64_t i) {
    uint64_t key = mix64(mix64(env_seed ^ tag) + GAMMA * (uint64_t)(t + 1));
    return mix64(key + GAMMA * (uint64_t)(i + 1));
}
uint32_t lemire(uint64_t x, uint32_t n) {
    return (uint32_t)(((uint64_t)(uint32_t)(x >> 32) * (uint64_t)n) >> 32);
}
const uint64_t TAG_SHUFFLE = 0x5348554646000001ULL;
const uint64_t TAG_POLICY = 0x504F4C4943590002ULL;
const uint64_t TAG_EPISODE = 0x4550495344450003ULL;
const uint64_t TAG_TASKDIR = 0x5441534B44495204ULL;
const int64_t INIT_ID = 0x4000000000000000LL;   // ids of a snapshot's resting orders

// Number of market-maker actions of each action space (Sec. 4.1.1).
int mm_actions(int space) { return space == 1 ? 8 : space == 2 ? 3 : 12; }

int64_t floor_half(int64_t s) { return s >= 0 ? s / 2 : -((-s + 1) / 2); }
int64_t ceil_half(int64_t s) { return -floor_half(-s); }

struct Config {
    orc_config c;
    int obs_dim() const { return c.n_agents > 0 ? 4 * c.top_levels + 5 : 0; }
};

struct Env {
    Side bids, asks;
    int32_t cap = 0;
    int64_t ts_next = 0, seq_next = 0;
    int32_t last_px = 0;
    uint64_t seed = 0;
    std::vector<Agent> ag;              // A agents: execution 0..P-1, market making P..2P-1
    int64_t cnt[ORC_NCOUNTERS] = {};
    std::vector<Fill> fills;
    std::vector<float> obs;
    std::vector<int64_t> rew;
    uint8_t done = 0;
    std::vector<int32_t> act;
    bool bad = false;
    int32_t msg_idx = 0;                // processing index within the current step
    int64_t ep_start = 0;               // episode mode: first data step of the current episode
    int exec_dir = SELL;                // the execution task's side in this episode
    std::vector<unsigned char> *snaps = nullptr;  // env 0 book after every message
};

// Owner of an order id: agents 0..A-1 for negative ids, A (background) else.
int owner(int64_t id, int A) {
    if (id >= 0 || A == 0) return A;
    return (int)((-(id + 1)) % A);
}

struct Engine {
    Config cfg;
    std::vector<Env> envs;
    int64_t t = 0;  // steps taken since reset
    std::vector<unsigned char> snaps;
    // episode mode
    bool ep_mode = false;
    const Msg *ep_msgs = nullptr;
    std::vector<int64_t> ep_off;
    std::vector<orc_start> ep_starts;
    std::vector<int32_t> ep_levels;   // [n_starts][2][ep_ls][2]
    int32_t ep_ls = 0;

    Side &side_book(Env &E, int side) { return side == BUY ? E.bids : E.asks; }

    // Touch prices with the empty-side rule.
    int64_t ref_bid(Env &E) { return E.bids.count ? E.bids.best()->first : E.last_px; }
    int64_t ref_ask(Env &E) { return E.asks.count ? E.asks.best()->first : E.last_px; }

    void snapshot(Env &E) {
        if (!E.snaps) return;
        const int C = E.cap;
        std::vector<int32_t> n(2), px(2 * C, 0), qty(2 * C, 0);
        std::vector<int64_t> id(2 * C, 0), ts(2 * C, 0);
        const Side *sides[2] = {&E.bids, &E.asks};
        for (int s = 0; s < 2; s++) {
            std::vector<Order> v = sides[s]->ordered();
            n[s] = (int32_t)v.size();
            for (size_t j = 0; j < v.size(); j++) {
                px[s * C + j] = v[j].px; qty[s * C + j] = v[j].qty;
                id[s * C + j] = v[j].id; ts[s * C + j] = v[j].ts;
            }
        }
        auto put = [&](const void *p, size_t b) {
            const unsigned char *q = (const unsigned char *)p;
            E.snaps->insert(E.snaps->end(), q, q + b);
        };
        put(n.data(), 8); put(px.data(), 8 * C); put(qty.data(), 8 * C);
        put(id.data(), 16 * C); put(ts.data(), 16 * C);
    }

    // A trade of f units at the maker's price between a resting order and the
    // incoming order: cash and inventory move between their owners.
    void fill(Env &E, const Order &maker, int64_t taker_id, int taker_side, int32_t f) {
        const int A = cfg.c.n_agents;
        int om = owner(maker.id, A), ot = owner(taker_id, A);
        int buyer = taker_side == BUY ? ot : om;
        int seller = taker_side == BUY ? om : ot;
        int64_t notional = wmul(maker.px, f);
        auto credit = [&](int who, int64_t dcash, int64_t dinv) {
            if (who == A) {
                E.cnt[C_BG_CASH] = wadd(E.cnt[C_BG_CASH], dcash);
                E.cnt[C_BG_INV] = wadd(E.cnt[C_BG_INV], dinv);
            } else {
                E.ag[who].cash = wadd(E.ag[who].cash, dcash);
                E.ag[who].inv = wadd(E.ag[who].inv, dinv);
            }
        };
        credit(buyer, -notional, f);
        credit(seller, notional, -(int64_t)f);
        if (buyer != A) { E.ag[buyer].buy_q += f; E.ag[buyer].buy_n = wadd(E.ag[buyer].buy_n, notional); }
        if (seller != A) { E.ag[seller].sell_q += f; E.ag[seller].sell_n = wadd(E.ag[seller].sell_n, notional); }
        if (A > 0) {
            // the side of the execution task: its owner, if an execution agent, progresses
            int task_owner = E.exec_dir == SELL ? seller : buyer;
            if (task_owner < A / 2) E.ag[task_owner].exec_done += f;
        }
        E.last_px = maker.px;
        E.cnt[C_FILLS] += 1;
        E.cnt[C_FILL_VOL] += f;
        if (cfg.c.trace & 1)
            E.fills.push_back(Fill{maker.id, taker_id, maker.px, f, E.msg_idx, taker_side});
    }

    // Take liquidity from the opposite side: best price first, FIFO within a
    // price, stopping at the limit price (or never, for a market order).
    int32_t take(Env &E, int side, bool has_limit, int32_t limit, int32_t q, int64_t taker_id) {
        Side &opp = side_book(E, -side);
        while (q > 0 && opp.count > 0) {
            auto lv = opp.best();
            if (has_limit && (side == BUY ? lv->first > limit : lv->first < limit)) break;
            Order &o = lv->second.front();
            int32_t f = std::min(q, o.qty);
            fill(E, o, taker_id, side, f);
            o.qty -= f;
            q -= f;
            if (o.qty == 0) {
                lv->second.pop_front();
                opp.count--;
                if (lv->second.empty()) opp.levels.erase(lv);
            }
        }
        return q;
    }

    // Rest a remainder on its own side, applying the capacity rule.
    void rest(Env &E, int side, int32_t px, int32_t q, int64_t id) {
        Side &own = side_book(E, side);
        if (own.count >= E.cap) {
            auto wl = own.worst();
            if (own.better(px, wl->first)) {
                Order victim = wl->second.back();
                wl->second.pop_back();
                own.count--;
                if (wl->second.empty()) own.levels.erase(wl);
                E.cnt[C_EVICT_VOL] += victim.qty;
                E.cnt[C_EVICT_CNT] += 1;
            } else {
                E.cnt[C_DROP_VOL] += q;
                E.cnt[C_DROP_CNT] += 1;
                return;
            }
        }
        own.levels[px].push_back(Order{id, E.ts_next++, px, q});
        own.count++;
    }

    // Find a resting order by (side, price level, id).
    bool locate(Env &E, int side, int32_t px, int64_t id, std::deque<Order> **q, size_t *pos) {
        Side &own = side_book(E, side);
        auto lv = own.levels.find(px);
        if (lv == own.levels.end()) return false;
        for (size_t i = 0; i < lv->second.size(); i++)
            if (lv->second[i].id == id) { *q = &lv->second; *pos = i; return true; }
        return false;
    }

    void remove_at(Env &E, int side, int32_t px, size_t pos) {
        Side &own = side_book(E, side);
        auto lv = own.levels.find(px);
        lv->second.erase(lv->second.begin() + (long)pos);
        own.count--;
        if (lv->second.empty()) own.levels.erase(lv);
    }

    void process(Env &E, const Msg &m, bool is_agent) {
        E.cnt[C_MSGS] += 1;
        if (is_agent) E.cnt[C_AGENT_MSGS] += 1;
        bool ok = m.type >= ADD && m.type <= MARKET && (m.side == BUY || m.side == SELL);
        if (ok && m.type != DELETE && m.qty <= 0) ok = false;
        if (!ok) {
            E.cnt[C_BAD_MSGS] += 1;
            E.bad = true;
        } else if (m.type == ADD) {
            E.cnt[C_ADD_VOL] += m.qty;
            int32_t left = take(E, m.side, true, m.px, m.qty, m.oid);
            if (left > 0) rest(E, m.side, m.px, left, m.oid);
        } else if (m.type == MARKET) {
            E.cnt[C_MKT_VOL] += m.qty;
            int32_t left = take(E, m.side, false, 0, m.qty, m.oid);
            E.cnt[C_MKT_DISCARD] += left;
        } else {
            std::deque<Order> *q = nullptr;
            size_t pos = 0;
            if (!locate(E, m.side, m.px, m.oid, &q, &pos)) {
                E.cnt[C_CANCEL_MISS] += 1;
            } else if (m.type == PARTIAL) {
                Order &o = (*q)[pos];
                int32_t c = std::min(m.qty, o.qty);
                o.qty -= c;
                E.cnt[C_CANCEL_VOL] += c;
                if (o.qty == 0) remove_at(E, m.side, m.px, pos);
            } else {
                E.cnt[C_CANCEL_VOL] += (*q)[pos].qty;
                remove_at(E, m.side, m.px, pos);
            }
        }
        snapshot(E);
        E.msg_idx++;
    }

    // The execution task's side in episode k (Table 2: uniformly sampled when
    // exec_dir is 0): the top bit of a keyed SplitMix64 draw, set -> sell.
    int task_dir(const Env &E, int64_t k) const {
        if (cfg.c.exec_dir != 0) return cfg.c.exec_dir;
        return (draw(E.seed, k, TAG_TASKDIR, 0) >> 63) ? SELL : BUY;
    }

    // Start episode k of env E from its drawn snapshot (episode mode).
    void begin_episode(Env &E, int64_t k) {
        const uint32_t j = lemire(draw(E.seed, k, TAG_EPISODE, 0), (uint32_t)ep_starts.size());
        const orc_start &st = ep_starts[j];
        E.bids.levels.clear(); E.bids.count = 0;
        E.asks.levels.clear(); E.asks.count = 0;
        E.ts_next = 0;
        E.seq_next = 0;
        for (Agent &g : E.ag) g = Agent();
        E.last_px = st.last_px;
        E.ep_start = st.data_step;
        E.exec_dir = task_dir(E, k);
        int64_t idx = 0;
        for (int s = 0; s < 2; s++) {
            Side &side = s == 0 ? E.bids : E.asks;
            const int n = s == 0 ? st.n_bid : st.n_ask;
            for (int i = 0; i < n; i++) {
                const int32_t *lv = ep_levels.data() + (((size_t)j * 2 + s) * ep_ls + i) * 2;
                side.levels[lv[0]].push_back(Order{INIT_ID + idx, E.ts_next++, lv[0], lv[1]});
                side.count++;
                idx++;
            }
        }
    }

    // Observation of every agent (Sec. 4.1.1): top-L aggregated levels per
    // side relative to the anchor, inventory, cash, time left, remaining
    // execution target, own resting quantity.
    void write_obs(Env &E, float tl) {
        const orc_config &c = cfg.c;
        const int A = c.n_agents, L = c.top_levels, D = cfg.obs_dim();
        int64_t bb = ref_bid(E), ba = ref_ask(E);
        int64_t anchor = floor_half(bb + ba);
        E.obs.assign((size_t)A * D, 0.0f);
        std::vector<std::pair<int32_t, int64_t>> lv[2] = {E.bids.aggregated(), E.asks.aggregated()};
        std::vector<int64_t> own_rest(A, 0);
        for (int s = 0; s < 2; s++)
            for (const Order &o : (s == 0 ? E.bids : E.asks).ordered())
                if (o.id < 0) own_rest[owner(o.id, A)] += o.qty;
        for (int a = 0; a < A; a++) {
            float *ob = E.obs.data() + (size_t)a * D;
            for (int s = 0; s < 2; s++)
                for (int i = 0; i < L && i < (int)lv[s].size(); i++) {
                    ob[s * 2 * L + 2 * i] = (float)(lv[s][i].first - anchor);
                    ob[s * 2 * L + 2 * i + 1] = (float)lv[s][i].second;
                }
            const Agent &g = E.ag[a];
            ob[4 * L + 0] = (float)g.inv;
            ob[4 * L + 1] = (float)g.cash;
            ob[4 * L + 2] = tl;
            // remaining target; signed by the task's side (+ buy, - sell) when the side is drawn
            const int64_t rem = (int64_t)c.exec_target - g.exec_done;
            ob[4 * L + 3] = a < A / 2 ? (float)(c.exec_dir == 0 && E.exec_dir == SELL ? -rem : rem) : 0.0f;
            ob[4 * L + 4] = (float)own_rest[a];
        }
    }

    struct NewOrder { int agent, side; int32_t px, qty; };

    void env_step(Env &E, int64_t e, const int32_t *actions, const Msg *bg, int64_t nbg) {
        const orc_config &c = cfg.c;
        const int A = c.n_agents;
        E.fills.clear();
        E.msg_idx = 0;
        if (E.snaps) E.snaps->clear();
        for (Agent &g : E.ag) g.buy_q = g.buy_n = g.sell_q = g.sell_n = 0;
        const int64_t mid2_start = ref_bid(E) + ref_ask(E);   // twice the mid when the step begins
        std::vector<NewOrder> want;
        std::vector<Msg> cancels;
        if (A > 0) {
            // -- Action conversion (Sec. 4): actions -> new orders.  Agents
            // 0..P-1 execute, P..2P-1 make markets (P agents per type).
            const int P = A / 2;
            for (int a = 0; a < A; a++) {
                const uint32_t n_act = a < P ? 12u : (uint32_t)mm_actions(c.mm_space);
                if (c.action_mode == 1)
                    E.act[a] = (int32_t)lemire(draw(E.seed, t, TAG_POLICY, a), n_act);
                else
                    E.act[a] = actions[e * A + a];
            }
            int64_t bb = ref_bid(E), ba = ref_ask(E);
            // execution agents (Sec. 4.1.2): 4 reference prices x {1,2,5} lots
            for (int ag = 0; ag < P; ag++) {
                int64_t remaining = (int64_t)c.exec_target - E.ag[ag].exec_done;
                if (remaining <= 0) continue;
                int a = E.act[ag];
                int pi = a / 3;
                int64_t mult = a % 3 == 0 ? 1 : a % 3 == 1 ? 2 : 5;
                int64_t q0 = std::max<int64_t>(1, ((int64_t)c.exec_target + c.episode_len - 1) / c.episode_len);
                int64_t qty = std::min(mult * q0, remaining);
                int64_t px;
                if (E.exec_dir == SELL) {
                    const int64_t p4[4] = {bb, ceil_half(bb + ba), ba, ba + 2};
                    px = p4[pi];
                } else {
                    const int64_t p4[4] = {ba, floor_half(bb + ba), bb, bb - 2};
                    px = p4[pi];
                }
                want.push_back({ag, E.exec_dir, (int32_t)px, (int32_t)qty});
            }
            // market makers (Sec. 4.1.1): quotes of mm_lot around the touch
            for (int ag = P; ag < A; ag++) {
                int a = E.act[ag];
                int64_t bid = 0, ask = 0;
                bool has_bid = false, has_ask = false;
                if (c.mm_space == 0) {
                    // 12-way head: bid / ask each 0, 1 or 2 ticks behind the touch,
                    // or one tick into the spread on one side
                    has_bid = has_ask = a >= 1 && a <= 11;
                    if (a >= 1 && a <= 9) { bid = bb - (a - 1) / 3; ask = ba + (a - 1) % 3; }
                    else if (a == 10) { bid = bb + 1; ask = ba; }
                    else if (a == 11) { bid = bb; ask = ba - 1; }
                } else if (c.mm_space == 1) {
                    // Fixed Quantity, 8 options: none; 2 / 4 ticks behind both
                    // touches; one tick into the spread on both; 2 ticks behind on
                    // the bid only / the ask only; 5 ticks behind on one side with
                    // one tick into the spread on the other
                    switch (a) {
                        case 1: bid = bb - 2; ask = ba + 2; has_bid = has_ask = true; break;
                        case 2: bid = bb - 4; ask = ba + 4; has_bid = has_ask = true; break;
                        case 3: bid = bb + 1; ask = ba - 1; has_bid = has_ask = true; break;
                        case 4: bid = bb - 2; has_bid = true; break;
                        case 5: ask = ba + 2; has_ask = true; break;
                        case 6: bid = bb - 5; ask = ba - 1; has_bid = has_ask = true; break;
                        case 7: bid = bb + 1; ask = ba + 5; has_bid = has_ask = true; break;
                        default: break;
                    }
                } else {
                    // directional trading: a bid at the best bid, an ask at the best ask, or nothing
                    if (a == 1) { bid = bb; has_bid = true; }
                    if (a == 2) { ask = ba; has_ask = true; }
                }
                if (has_bid) want.push_back({ag, BUY, (int32_t)bid, c.mm_lot});
                if (has_ask) want.push_back({ag, SELL, (int32_t)ask, c.mm_lot});
            }
            // -- carry-over: keep same-(side, price) resting orders, cancel the rest
            std::vector<int64_t> kept(want.size(), 0);
            for (int ag = 0; ag < A; ag++) {
                for (int s = 0; s < 2; s++) {
                    int side = s == 0 ? BUY : SELL;
                    for (const Order &o : side_book(E, side).ordered()) {
                        if (o.id >= 0 || owner(o.id, A) != ag) continue;
                        int match = -1;
                        for (size_t i = 0; i < want.size(); i++)
                            if (want[i].agent == ag && want[i].side == side && want[i].px == o.px) match = (int)i;
                        if (match >= 0) {
                            kept[match] += o.qty;
                        } else {
                            Msg m{};
                            m.type = DELETE; m.side = (int16_t)side; m.px = o.px; m.oid = o.id; m.qty = o.qty;
                            cancels.push_back(m);
                        }
                    }
                }
            }
            std::vector<NewOrder> send;
            for (size_t i = 0; i < want.size(); i++) {
                int64_t q = want[i].qty - kept[i];
                if (q > 0) send.push_back({want[i].agent, want[i].side, want[i].px, (int32_t)q});
            }
            // -- Random shuffling (Sec. 4): Fisher-Yates, SplitMix64 + Lemire
            int n = (int)send.size();
            for (int i = n - 1, d = 0; i >= 1; i--, d++) {
                uint32_t j = lemire(draw(E.seed, t, TAG_SHUFFLE, d), (uint32_t)(i + 1));
                std::swap(send[i], send[j]);
            }
            // -- Augment (Sec. 4): cancels, then the agents' orders ...
            for (const Msg &m : cancels) process(E, m, true);
            for (const NewOrder &o : send) {
                Msg m{};
                m.type = ADD; m.side = (int16_t)o.side; m.px = o.px; m.qty = o.qty;
                m.oid = -(1 + (int64_t)o.agent + (int64_t)A * E.seq_next);
                E.seq_next++;
                process(E, m, true);
            }
        }
        // ... then the background messages (Processing by JAX-LOB)
        for (int64_t i = 0; i < nbg; i++) process(E, bg[i], false);

        // -- Step outcomes (Sec. 4): observation, reward, termination
        // (te: step within the episode; episodes restart only in episode mode)
        const int64_t te = ep_mode ? t % c.episode_len : t;
        const bool last = te + 1 == c.episode_len;
        if (A > 0) {
            int64_t bb = ref_bid(E), ba = ref_ask(E);
            write_obs(E, (float)(c.episode_len - (te + 1)) / (float)c.episode_len);
            for (int a = 0; a < A; a++) {
                Agent &g = E.ag[a];
                // PV = Q_inv * P_ref + Cash (Eq. 1), P_ref the liquidation touch,
                // or the mid price with PV counted in half ticks (2 PV exact)
                int64_t pref = g.inv > 0 ? bb : g.inv < 0 ? ba : 0;
                int64_t pv = c.pv_ref == 1 ? wadd(wmul(g.inv, bb + ba), wmul(2, g.cash))
                                           : wadd(wmul(g.inv, pref), g.cash);
                E.rew[a] = wsub(pv, g.pv_prev);
                g.pv_prev = pv;
                const bool mm = a >= A / 2;
                if (mm && c.reward_mode != 0) {
                    // Sec. 5: trading PnL against the average mid over the step,
                    // read as the mean of its start and end mids, so 4*Mbar is
                    // an integer and the reward is exact in quarter-tick*qty.
                    const int64_t mid2_end = bb + ba;
                    const int64_t m4 = mid2_start + mid2_end;
                    const int64_t psi_b4 = wsub(wmul(m4, g.buy_q), wmul(4, g.buy_n));      // 4 * Psi_b
                    const int64_t psi_s4 = wsub(wmul(4, g.sell_n), wmul(m4, g.sell_q));    // 4 * Psi_s
                    int64_t r4 = wadd(psi_b4, psi_s4);                                   // Eq. 4
                    if (c.reward_mode == 2) {
                        // Eq. 3: + Psi_INV - (1 - lambda) max(0, Psi_INV), Psi_INV = I_t (M_t - M_{t-1})
                        const int64_t psi_inv4 = wmul(wmul(2, g.inv), mid2_end - mid2_start);
                        // the damping is rounded up, so the reward is the floor of its exact value
                        const int64_t damp =
                            (wmul(100 - c.spooner_lambda_pct, std::max<int64_t>(0, psi_inv4)) + 99) / 100;
                        r4 = wsub(wadd(r4, psi_inv4), damp);
                    }
                    E.rew[a] = r4;
                }
                if (mm && c.inv_penalty != 0)   // quadratic inventory penalty
                    E.rew[a] = wsub(E.rew[a], wmul(c.inv_penalty, wmul(g.inv, g.inv)));
                if (!mm && c.exec_penalty_milli != 0 && last) {
                    // Table 2: penalty on the part of the task still unfilled at the end
                    const int64_t unfilled = std::max<int64_t>(0, (int64_t)c.exec_target - g.exec_done);
                    // rounded up; in half ticks with the mid reference
                    const int64_t milli = wmul(c.exec_penalty_milli, unfilled) * (c.pv_ref == 1 ? 2 : 1);
                    E.rew[a] = wsub(E.rew[a], (milli + 999) / 1000);
                }
            }
        }
        E.done = (uint8_t)last;
        if (ep_mode && last) {
            // the next episode begins; its first observation is what the agents see
            begin_episode(E, t / c.episode_len + 1);
            if (A > 0) write_obs(E, (float)c.episode_len / (float)c.episode_len);
        }
    }
};

}  // namespace

extern "C" {

void *orc_create(const orc_config *cfg, const int32_t *caps) {
    if (!cfg || cfg->n_envs < 0 || cfg->n_agents < 0 || cfg->n_agents % 2 != 0 || cfg->n_agents > 2 * ORC_MAX_PER_TYPE)
        return nullptr;
    Engine *g = new Engine();
    g->cfg.c = *cfg;
    g->envs.resize((size_t)cfg->n_envs);
    for (int64_t e = 0; e < cfg->n_envs; e++) {
        Env &E = g->envs[(size_t)e];
        E.cap = caps ? caps[e] : cfg->cap;
        E.bids.is_bid = true;
        E.asks.is_bid = false;
        E.ag.assign((size_t)cfg->n_agents, Agent());
        E.rew.assign((size_t)cfg->n_agents, 0);
        E.act.assign((size_t)cfg->n_agents, 0);
    }
    if (cfg->n_envs > 0 && (cfg->trace & 2)) g->envs[0].snaps = &g->snaps;
    return g;
}

void orc_destroy(void *h) { delete (Engine *)h; }

void orc_reset(void *h, const uint64_t *env_seeds) {
    Engine *g = (Engine *)h;
    g->t = 0;
    for (size_t e = 0; e < g->envs.size(); e++) {
        Env &E = g->envs[e];
        std::vector<unsigned char> *sn = E.snaps;
        int32_t cap = E.cap;
        E = Env();
        E.snaps = sn;
        E.cap = cap;
        E.bids.is_bid = true;
        E.asks.is_bid = false;
        E.seed = env_seeds[e];
        E.last_px = g->cfg.c.start_px;
        E.exec_dir = g->task_dir(E, 0);
        E.ag.assign((size_t)g->cfg.c.n_agents, Agent());
        E.rew.assign((size_t)g->cfg.c.n_agents, 0);
        E.act.assign((size_t)g->cfg.c.n_agents, 0);
        if (g->ep_mode) g->begin_episode(E, 0);
        // reset observation: the starting book (empty outside episode mode),
        // nothing held, the whole episode and (for the execution agents) the
        // whole target still ahead
        g->write_obs(E, (float)g->cfg.c.episode_len / (float)g->cfg.c.episode_len);
    }
}

int orc_step(void *h, const int32_t *actions, const void *msgs, const int64_t *offsets, int64_t stride, int32_t k) {
    Engine *g = (Engine *)h;
    const Msg *all = (const Msg *)msgs;
    const int64_t n = (int64_t)g->envs.size();
    auto run = [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; e++) {
            int64_t b = offsets[e * stride + k], en = offsets[e * stride + k + 1];
            g->env_step(g->envs[(size_t)e], e, actions, all + b, en - b);
        }
    };
    int nt = std::max(1, g->cfg.c.n_threads);
    if (nt == 1 || n < 2) {
        run(0, n);
    } else {
        std::vector<std::thread> th;
        int64_t per = (n + nt - 1) / nt;
        for (int i = 0; i < nt; i++) {
            int64_t lo = i * per, hi = std::min(n, lo + per);
            if (lo < hi) th.emplace_back(run, lo, hi);
        }
        for (auto &x : th) x.join();
    }
    g->t++;
    int rc = 0;
    for (Env &E : g->envs) if (E.bad) { rc = -6; E.bad = false; }
    return rc;
}

void orc_set_episodes(void *h, const void *msgs, const int64_t *step_off, int64_t n_data_steps,
                      const orc_start *starts, const int32_t *levels, int32_t levels_per_side, int64_t n_starts) {
    Engine *g = (Engine *)h;
    g->ep_mode = true;
    g->ep_msgs = (const Msg *)msgs;
    g->ep_off.assign(step_off, step_off + n_data_steps + 1);
    g->ep_starts.assign(starts, starts + n_starts);
    g->ep_levels.assign(levels, levels + (size_t)n_starts * 2 * levels_per_side * 2);
    g->ep_ls = levels_per_side;
}

int orc_step_episodes(void *h, const int32_t *actions) {
    Engine *g = (Engine *)h;
    const int64_t n = (int64_t)g->envs.size(), T = g->cfg.c.episode_len;
    const int64_t te = g->t % T;
    auto run = [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; e++) {
            Env &E = g->envs[(size_t)e];
            const int64_t d = E.ep_start + te;   // this step's data step
            const int64_t b = g->ep_off[(size_t)d], en = g->ep_off[(size_t)d + 1];
            g->env_step(E, e, actions, g->ep_msgs + b, en - b);
        }
    };
    int nt = std::max(1, g->cfg.c.n_threads);
    if (nt == 1 || n < 2) {
        run(0, n);
    } else {
        std::vector<std::thread> th;
        int64_t per = (n + nt - 1) / nt;
        for (int i = 0; i < nt; i++) {
            int64_t lo = i * per, hi = std::min(n, lo + per);
            if (lo < hi) th.emplace_back(run, lo, hi);
        }
        for (auto &x : th) x.join();
    }
    g->t++;
    int rc = 0;
    for (Env &E : g->envs) if (E.bad) { rc = -6; E.bad = false; }
    return rc;
}

void orc_get_episode(void *h, int64_t *out) {
    Engine *g = (Engine *)h;
    for (size_t e = 0; e < g->envs.size(); e++) out[e] = g->envs[e].ep_start;
}

int32_t orc_obs_dim(void *h) { return ((Engine *)h)->cfg.obs_dim(); }

void orc_observe(void *h, float *obs, int64_t *rewards, uint8_t *done) {
    Engine *g = (Engine *)h;
    const int A = g->cfg.c.n_agents, D = g->cfg.obs_dim();
    for (size_t e = 0; e < g->envs.size(); e++) {
        Env &E = g->envs[e];
        if (obs && A) std::memcpy(obs + e * (size_t)A * D, E.obs.data(), sizeof(float) * (size_t)A * D);
        if (rewards) for (int a = 0; a < A; a++) rewards[e * A + a] = E.rew[a];
        if (done) done[e] = E.done;
    }
}

void orc_get_book(void *h, int64_t env, int32_t *n2, int32_t *px, int32_t *qty, int64_t *id, int64_t *ts) {
    Engine *g = (Engine *)h;
    Env &E = g->envs[(size_t)env];
    const int C = E.cap;
    const Side *sides[2] = {&E.bids, &E.asks};
    for (int s = 0; s < 2; s++) {
        std::vector<Order> v = sides[s]->ordered();
        n2[s] = (int32_t)v.size();
        for (int j = 0; j < C; j++) {
            bool live = j < (int)v.size();
            px[s * C + j] = live ? v[j].px : 0;
            qty[s * C + j] = live ? v[j].qty : 0;
            id[s * C + j] = live ? v[j].id : 0;
            ts[s * C + j] = live ? v[j].ts : 0;
        }
    }
}

void orc_get_counters(void *h, int64_t *out) {
    Engine *g = (Engine *)h;
    for (size_t e = 0; e < g->envs.size(); e++)
        std::memcpy(out + e * ORC_NCOUNTERS, g->envs[e].cnt, sizeof(int64_t) * ORC_NCOUNTERS);
}

void orc_get_agents(void *h, int64_t *out) {
    Engine *g = (Engine *)h;
    const int A = g->cfg.c.n_agents;
    for (size_t e = 0; e < g->envs.size(); e++)
        for (int a = 0; a < A; a++) {
            const Agent &x = g->envs[e].ag[a];
            int64_t *o = out + (e * A + a) * 4;
            o[0] = x.inv; o[1] = x.cash; o[2] = x.pv_prev; o[3] = x.exec_done;
        }
}

void orc_get_env_misc(void *h, int64_t *out) {
    Engine *g = (Engine *)h;
    for (size_t e = 0; e < g->envs.size(); e++) {
        const Env &E = g->envs[e];
        out[e * 4 + 0] = E.ts_next;
        out[e * 4 + 1] = E.seq_next;
        out[e * 4 + 2] = E.last_px;
        out[e * 4 + 3] = g->t;
    }
}

void orc_get_actions(void *h, int32_t *out) {
    Engine *g = (Engine *)h;
    const int A = g->cfg.c.n_agents;
    for (size_t e = 0; e < g->envs.size(); e++)
        for (int a = 0; a < A; a++) out[e * A + a] = g->envs[e].act[a];
}

int64_t orc_get_fills(void *h, int64_t env, void *out, int64_t cap) {
    Engine *g = (Engine *)h;
    const std::vector<Fill> &f = g->envs[(size_t)env].fills;
    int64_t n = (int64_t)f.size();
    if (out) std::memcpy(out, f.data(), sizeof(Fill) * (size_t)std::min(n, cap));
    return n;
}

int64_t orc_get_snapshots(void *h, void *out, int64_t cap) {
    Engine *g = (Engine *)h;
    if (g->envs.empty()) return 0;
    const size_t rec = 8 + 48 * (size_t)g->envs[0].cap;
    int64_t n = (int64_t)(g->snaps.size() / rec);
    if (out) std::memcpy(out, g->snaps.data(), rec * (size_t)std::min(n, cap));
    return n;
}

uint64_t orc_draw(uint64_t env_seed, int64_t t, uint64_t tag, int64_t i) { return draw(env_seed, t, tag, i); }
uint32_t orc_lemire(uint64_t x, uint32_t n) { return lemire(x, n); }
uint64_t orc_splitmix(uint64_t state, int64_t i) { return mix64(state + GAMMA * (uint64_t)(i + 1)); }

}  // extern "C"
