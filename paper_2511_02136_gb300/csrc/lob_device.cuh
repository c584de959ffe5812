// lob_device.cuh -- sm_103a kernels of the batched limit-order-book env step.
//
// One warp runs one environment.  Each side of the book is a priority-sorted
// array (best price first, then arrival) held in REGISTERS in a blocked
// layout: lane l owns slots l*K .. l*K+K-1 of a side (capacity 32*K).  An
// insert or a removal is then one neighbour-lane shuffle plus per-lane
// selects; a lookup is a compare plus a ballot.  Messages are staged into
// shared memory tile by tile with cp.async.bulk (TMA bulk copy) completing on
// an mbarrier, and broadcast to the warp from there.  Agents, counters and
// all other per-env scalars are warp-uniform registers.
//
// The stages follow the environment step of JaxMARL-HFT Sec. 4: action
// conversion with carry-over cancels, random shuffle of the agents' orders,
// concatenation (cancels, agent orders, market-replay messages), price-time
// matching (Sec. 2.1) and the step outcomes (observation, Eq. 1 portfolio-
// value reward, termination flag).
#pragma once
#include <cstdint>
#include "lob.h"

namespace lobk {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TILE = 32;        // messages per staged tile
constexpr int LMAX = 64;        // max observation levels per side
constexpr int ST_BADMSG = 1, ST_BADACT = 2, ST_TIMEOUT = 4;

struct DevMsg {
    long long ts, oid;
    int px, qty;
    short type, side;
    int pad;
};
static_assert(sizeof(DevMsg) == 32, "message record");

// Per-env scalar state in HBM (128 bytes).
struct __align__(16) EnvState {
    long long ts_next, seq_next;
    long long inv[2], cash[2], pv_prev[2];
    long long exec_done;
    int last_px;
    int n[2];
    int act[2];
    int t;
    int pad[8];
};
static_assert(sizeof(EnvState) == 128, "env state");

struct KParams {
    unsigned char *books;
    const long long *book_off;
    const int *caps;
    EnvState *st;
    long long *counters;
    const unsigned long long *seeds;
    int *status;
    const DevMsg *msgs;
    const long long *offsets;
    long long off_stride;
    int k0;
    const int *actions;
    long long act_step_stride;
    int action_mode;
    float *obs;
    long long *rew;
    unsigned char *done;
    int *act_out;
    int n_envs, n_agents, L, T, mm_lot, exec_target, exec_dir, D;
    int t0, n_steps;
    lob_fill *fills;
    int fill_cap;
    int *fill_counts;
    unsigned char *snaps;
    long long snap_cap;
    long long *snap_count;
    const int *env_list;
    int n_list;
    int *queue;
    long long wait_budget;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1-D TMA bulk copy global -> shared, completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, unsigned bytes,
                                             unsigned long long *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `budget` SM cycles.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase, long long budget) {
    if (mbar_try_wait(bar, phase)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > budget) return false;
    return true;
}

// ---------------------------------------------------------------- RNG
// SplitMix64 (Steele, Lea & Flood 2014): the i-th output from state
// key(t) = mix(mix(seed ^ tag) + gamma * (t + 1)); Lemire's multiply-shift
// maps the high 32 bits onto [0, n).
constexpr unsigned long long GAMMA = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long TAG_SHUFFLE = 0x5348554646000001ull;
constexpr unsigned long long TAG_POLICY = 0x504F4C4943590002ull;
__device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long step_key(unsigned long long seed, long long t,
                                                      unsigned long long tag) {
    return sm_mix(sm_mix(seed ^ tag) + GAMMA * (unsigned long long)(t + 1));
}
__device__ __forceinline__ unsigned bounded(unsigned long long x, unsigned n) {
    return (unsigned)(((unsigned long long)(unsigned)(x >> 32) * n) >> 32);
}

// ---------------------------------------------------------------- book
template <int K>
struct Book {
    int px[K], qty[K];
    long long id[K], ts[K];
    int n;     // live orders (warp-uniform)
    int best;  // price of slot 0 when n > 0 (warp-uniform)
};

// "a has priority over (or ties with) a new order at p" on a side
template <bool BID>
__device__ __forceinline__ bool at_least(int a, int p) { return BID ? a >= p : a <= p; }

template <int K, bool BID>
__device__ __forceinline__ void book_load(Book<K> &S, const unsigned char *blk, int cap_slots, int lane, int n) {
    const int s = BID ? 0 : 1;
    const int *px = reinterpret_cast<const int *>(blk) + s * cap_slots + lane * K;
    const int *qt = reinterpret_cast<const int *>(blk) + 2 * cap_slots + s * cap_slots + lane * K;
    const long long *id = reinterpret_cast<const long long *>(blk + 16 * cap_slots) + s * cap_slots + lane * K;
    const long long *ts = reinterpret_cast<const long long *>(blk + 32 * cap_slots) + s * cap_slots + lane * K;
    S.n = n;
    if (lane * K < n) {
        if constexpr (K % 4 == 0) {
#pragma unroll
            for (int v = 0; v < K / 4; v++) {
                int4 a = reinterpret_cast<const int4 *>(px)[v];
                int4 b = reinterpret_cast<const int4 *>(qt)[v];
                S.px[4 * v] = a.x; S.px[4 * v + 1] = a.y; S.px[4 * v + 2] = a.z; S.px[4 * v + 3] = a.w;
                S.qty[4 * v] = b.x; S.qty[4 * v + 1] = b.y; S.qty[4 * v + 2] = b.z; S.qty[4 * v + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int r = 0; r < K; r++) { S.px[r] = px[r]; S.qty[r] = qt[r]; }
        }
        if constexpr (K % 2 == 0) {
#pragma unroll
            for (int v = 0; v < K / 2; v++) {
                longlong2 a = reinterpret_cast<const longlong2 *>(id)[v];
                longlong2 b = reinterpret_cast<const longlong2 *>(ts)[v];
                S.id[2 * v] = a.x; S.id[2 * v + 1] = a.y;
                S.ts[2 * v] = b.x; S.ts[2 * v + 1] = b.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < K; r++) { S.id[r] = id[r]; S.ts[r] = ts[r]; }
        }
    } else {
#pragma unroll
        for (int r = 0; r < K; r++) { S.px[r] = 0; S.qty[r] = 0; S.id[r] = 0; S.ts[r] = 0; }
    }
    S.best = __shfl_sync(FULL, S.px[0], 0);
}

template <int K, bool BID>
__device__ __forceinline__ void book_store(const Book<K> &S, unsigned char *blk, int cap_slots, int lane) {
    const int s = BID ? 0 : 1;
    int *px = reinterpret_cast<int *>(blk) + s * cap_slots + lane * K;
    int *qt = reinterpret_cast<int *>(blk) + 2 * cap_slots + s * cap_slots + lane * K;
    long long *id = reinterpret_cast<long long *>(blk + 16 * cap_slots) + s * cap_slots + lane * K;
    long long *ts = reinterpret_cast<long long *>(blk + 32 * cap_slots) + s * cap_slots + lane * K;
    if (lane * K >= S.n) return;
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int v = 0; v < K / 4; v++) {
            reinterpret_cast<int4 *>(px)[v] = make_int4(S.px[4 * v], S.px[4 * v + 1], S.px[4 * v + 2], S.px[4 * v + 3]);
            reinterpret_cast<int4 *>(qt)[v] = make_int4(S.qty[4 * v], S.qty[4 * v + 1], S.qty[4 * v + 2], S.qty[4 * v + 3]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < K; r++) { px[r] = S.px[r]; qt[r] = S.qty[r]; }
    }
    if constexpr (K % 2 == 0) {
#pragma unroll
        for (int v = 0; v < K / 2; v++) {
            reinterpret_cast<longlong2 *>(id)[v] = make_longlong2(S.id[2 * v], S.id[2 * v + 1]);
            reinterpret_cast<longlong2 *>(ts)[v] = make_longlong2(S.ts[2 * v], S.ts[2 * v + 1]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < K; r++) { id[r] = S.id[r]; ts[r] = S.ts[r]; }
    }
}

// Rest an order.  Returns 0 inserted, 1 inserted after evicting the last
// (worst price, latest arrival) order of a full side, 2 dropped (full and not
// strictly better than the worst resting price).
template <int K, bool BID>
__device__ __forceinline__ int book_insert(Book<K> &S, int cap, int p, int q, long long oid, long long tsn,
                                           int lane, long long &evict_vol) {
    bool pre[K];
    bool any_after = false;
#pragma unroll
    for (int r = 0; r < K; r++) {
        const bool v = lane * K + r < S.n;
        pre[r] = v && at_least<BID>(S.px[r], p);
        any_after |= v && !pre[r];
    }
    const int ppx = __shfl_up_sync(FULL, S.px[K - 1], 1);
    const int pq = __shfl_up_sync(FULL, S.qty[K - 1], 1);
    const long long pid = __shfl_up_sync(FULL, S.id[K - 1], 1);
    const long long pts = __shfl_up_sync(FULL, S.ts[K - 1], 1);
    const bool ppre = lane == 0 || (lane * K - 1 < S.n && at_least<BID>(ppx, p));
    int ret = 0;
    if (S.n >= cap) {
        if (__ballot_sync(FULL, any_after) == 0) return 2;
#pragma unroll
        for (int r = 0; r < K; r++)
            if (lane * K + r == S.n - 1) evict_vol += S.qty[r];
        ret = 1;
    }
#pragma unroll
    for (int r = K - 1; r >= 0; r--) {
        const bool pp = r == 0 ? ppre : pre[r - 1];
        if (!pre[r]) {
            if (pp) {
                S.px[r] = p; S.qty[r] = q; S.id[r] = oid; S.ts[r] = tsn;
            } else if (r == 0) {
                S.px[0] = ppx; S.qty[0] = pq; S.id[0] = pid; S.ts[0] = pts;
            } else {
                S.px[r] = S.px[r - 1]; S.qty[r] = S.qty[r - 1]; S.id[r] = S.id[r - 1]; S.ts[r] = S.ts[r - 1];
            }
        }
    }
    S.best = S.n == 0 ? p : (BID ? max(S.best, p) : min(S.best, p));
    if (ret == 0) S.n++;
    return ret;
}

// Remove the single slot marked in `hit` (bits r) of lane `first`.
template <int K>
__device__ __forceinline__ void book_remove(Book<K> &S, unsigned hit, int first, int lane) {
    const int nx = __shfl_down_sync(FULL, S.px[0], 1);
    const int nq = __shfl_down_sync(FULL, S.qty[0], 1);
    const long long nid = __shfl_down_sync(FULL, S.id[0], 1);
    const long long nts = __shfl_down_sync(FULL, S.ts[0], 1);
    bool after = lane > first;
#pragma unroll
    for (int r = 0; r < K; r++) {
        after = after || ((hit >> r) & 1u);
        if (after) {
            if (r == K - 1) {
                S.px[r] = nx; S.qty[r] = nq; S.id[r] = nid; S.ts[r] = nts;
            } else {
                S.px[r] = S.px[r + 1]; S.qty[r] = S.qty[r + 1]; S.id[r] = S.id[r + 1]; S.ts[r] = S.ts[r + 1];
            }
        }
    }
    S.n--;
    S.best = __shfl_sync(FULL, S.px[0], 0);
}

// First slot (priority order) with this (price, id); returns the lane holding
// it (or -1) and that lane's one-bit mask in `hit`.
template <int K>
__device__ __forceinline__ int book_find(const Book<K> &S, int p, long long oid, int lane, unsigned &hit) {
    unsigned h = 0;
#pragma unroll
    for (int r = 0; r < K; r++)
        if (lane * K + r < S.n && S.id[r] == oid && S.px[r] == p) h |= 1u << r;
    const unsigned lanes = __ballot_sync(FULL, h != 0);
    if (lanes == 0) { hit = 0; return -1; }
    const int first = __ffs(lanes) - 1;
    hit = lane == first ? (h & (0u - h)) : 0u;
    return first;
}

// ---------------------------------------------------------------- env context
// Warp-uniform per-env scalars of the running step.
struct Ctx {
    long long ts_next, seq_next;
    long long inv0, inv1, cash0, cash1, pv0, pv1, exec_done;
    long long bg_cash, bg_inv;
    int last_px;
    int A, exec_dir;
    // cumulative counters (uniform), plus per-lane partial sums
    long long c_msgs, c_agent, c_fills, c_fill_vol, c_add_vol, c_mkt_vol, c_mkt_disc;
    long long c_cancel_miss, c_drop_vol, c_drop_cnt, c_evict_cnt, c_bad;
    long long l_cancel_vol, l_evict_vol;  // per lane
    int msg_idx;
    int fill_n;
    int status;
    lob_fill *fill_log;
    int fill_cap;

    __device__ __forceinline__ void credit(int who, long long dcash, long long dinv) {
        if (who == 0) { cash0 += dcash; inv0 += dinv; }
        else if (who == 1) { cash1 += dcash; inv1 += dinv; }
        else { bg_cash += dcash; bg_inv += dinv; }
    }
    __device__ __forceinline__ int owner(long long id) const {
        return (id >= 0 || A == 0) ? 2 : (int)((~id) & 1);
    }
    // A trade at the resting order's price; cash and inventory move between
    // the owners of the two orders.
    __device__ __forceinline__ void fill(int px, int f, long long maker_id, long long taker_id, int taker_side,
                                         int lane) {
        const int om = owner(maker_id), ot = owner(taker_id);
        const int buyer = taker_side == LOB_BUY ? ot : om;
        const int seller = taker_side == LOB_BUY ? om : ot;
        const long long notional = (long long)((unsigned long long)(long long)px * (unsigned long long)(long long)f);
        credit(buyer, -notional, f);
        credit(seller, notional, -(long long)f);
        if (A > 0 && (exec_dir == LOB_SELL ? seller : buyer) == 0) exec_done += f;
        last_px = px;
        c_fills += 1;
        c_fill_vol += f;
        if (fill_log != nullptr && lane == 0 && fill_n < fill_cap) {
            lob_fill r;
            r.maker_id = maker_id; r.taker_id = taker_id; r.px = px; r.qty = f;
            r.msg_idx = msg_idx; r.taker_side = taker_side;
            fill_log[fill_n] = r;
        }
        fill_n++;
    }
};

// Take liquidity from resting side O (RBID: O holds bids), price first then
// time, up to the limit (if any).  Returns the unfilled quantity.
template <int K, bool RBID>
__device__ __forceinline__ int book_take(Book<K> &O, bool has_limit, int limit, int q, long long taker_id,
                                         int taker_side, Ctx &c, int lane) {
    if (O.n == 0 || (has_limit && !at_least<RBID>(O.best, limit))) return q;
    while (q > 0 && O.n > 0) {
        const int fpx = __shfl_sync(FULL, O.px[0], 0);
        const int fq = __shfl_sync(FULL, O.qty[0], 0);
        const long long fid = __shfl_sync(FULL, O.id[0], 0);
        if (has_limit && !at_least<RBID>(fpx, limit)) break;
        const int f = min(q, fq);
        c.fill(fpx, f, fid, taker_id, taker_side, lane);
        q -= f;
        if (f == fq) {
            const int nx = __shfl_down_sync(FULL, O.px[0], 1);
            const int nq = __shfl_down_sync(FULL, O.qty[0], 1);
            const long long nid = __shfl_down_sync(FULL, O.id[0], 1);
            const long long nts = __shfl_down_sync(FULL, O.ts[0], 1);
#pragma unroll
            for (int r = 0; r < K - 1; r++) {
                O.px[r] = O.px[r + 1]; O.qty[r] = O.qty[r + 1]; O.id[r] = O.id[r + 1]; O.ts[r] = O.ts[r + 1];
            }
            O.px[K - 1] = nx; O.qty[K - 1] = nq; O.id[K - 1] = nid; O.ts[K - 1] = nts;
            O.n--;
        } else if (lane == 0) {
            O.qty[0] -= f;
        }
    }
    O.best = __shfl_sync(FULL, O.px[0], 0);
    return q;
}

// Book of env 0 after a message, canonical layout (trace mode).
template <int K>
__device__ void write_snapshot(const Book<K> &B, const Book<K> &S, int C, unsigned char *rec, int lane) {
    int *n2 = reinterpret_cast<int *>(rec);
    int *px = n2 + 2;
    int *qt = px + 2 * C;
    long long *id = reinterpret_cast<long long *>(rec + 8 + 16 * (long long)C);
    long long *ts = id + 2 * C;
    if (lane == 0) { n2[0] = B.n; n2[1] = S.n; }
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int j = lane * K + r;
        if (j < C) {
            const bool vb = j < B.n, va = j < S.n;
            px[j] = vb ? B.px[r] : 0; qt[j] = vb ? B.qty[r] : 0; id[j] = vb ? B.id[r] : 0; ts[j] = vb ? B.ts[r] : 0;
            px[C + j] = va ? S.px[r] : 0; qt[C + j] = va ? S.qty[r] : 0;
            id[C + j] = va ? S.id[r] : 0; ts[C + j] = va ? S.ts[r] : 0;
        }
    }
}

// Partial cancel or delete on one side: lookup by (price, id); a miss is a no-op.
template <int K>
__device__ __forceinline__ void cancel_on(Book<K> &S, int type, int px, int qty, long long oid, Ctx &c, int lane) {
    unsigned hit;
    const int first = book_find<K>(S, px, oid, lane, hit);
    if (first < 0) {
        c.c_cancel_miss += 1;
        return;
    }
    bool zero = false;
#pragma unroll
    for (int r = 0; r < K; r++) {
        if ((hit >> r) & 1u) {
            const int cut = type == LOB_PARTIAL ? min(qty, S.qty[r]) : S.qty[r];
            c.l_cancel_vol += cut;
            S.qty[r] -= cut;
            zero = S.qty[r] == 0;
        }
    }
    zero = __shfl_sync(FULL, zero, first);
    if (zero) book_remove<K>(S, hit, first, lane);
}

// One message through the matching engine.
template <int K>
__device__ __forceinline__ void process_msg(Book<K> &bid, Book<K> &ask, int cap, int type, int side, int px,
                                            int qty, long long oid, bool agent, Ctx &c, int lane) {
    c.c_msgs += 1;
    if (agent) c.c_agent += 1;
    const bool ok = type >= LOB_ADD && type <= LOB_MARKET && (side == LOB_BUY || side == LOB_SELL) &&
                    (type == LOB_DELETE || qty > 0);
    if (!ok) {
        c.c_bad += 1;
        c.status |= ST_BADMSG;
    } else if (type == LOB_ADD) {
        c.c_add_vol += qty;
        int left;
        if (side == LOB_BUY) {
            left = book_take<K, false>(ask, true, px, qty, oid, side, c, lane);
            if (left > 0) {
                const int r = book_insert<K, true>(bid, cap, px, left, oid, c.ts_next, lane, c.l_evict_vol);
                if (r == 2) { c.c_drop_vol += left; c.c_drop_cnt += 1; }
                else { c.ts_next++; if (r == 1) c.c_evict_cnt += 1; }
            }
        } else {
            left = book_take<K, true>(bid, true, px, qty, oid, side, c, lane);
            if (left > 0) {
                const int r = book_insert<K, false>(ask, cap, px, left, oid, c.ts_next, lane, c.l_evict_vol);
                if (r == 2) { c.c_drop_vol += left; c.c_drop_cnt += 1; }
                else { c.ts_next++; if (r == 1) c.c_evict_cnt += 1; }
            }
        }
    } else if (type == LOB_MARKET) {
        c.c_mkt_vol += qty;
        const int left = side == LOB_BUY ? book_take<K, false>(ask, false, 0, qty, oid, side, c, lane)
                                         : book_take<K, true>(bid, false, 0, qty, oid, side, c, lane);
        c.c_mkt_disc += left;
    } else if (side == LOB_BUY) {
        cancel_on<K>(bid, type, px, qty, oid, c, lane);
    } else {
        cancel_on<K>(ask, type, px, qty, oid, c, lane);
    }
}

// Warp-wide int64 sum.
__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

// Aggregated top-L levels of one side into shared memory; returns level count.
template <int K, bool BID>
__device__ __forceinline__ int side_levels(const Book<K> &S, int L, int *lvl_px, long long *lvl_q, int lane) {
    const int ppx = __shfl_up_sync(FULL, S.px[K - 1], 1);
    bool start[K];
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int j = lane * K + r;
        const int prev = r == 0 ? ppx : S.px[r - 1];
        start[r] = j < S.n && (j == 0 || S.px[r] != prev);
        cnt += start[r];
    }
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    int lv = incl - cnt - 1;
#pragma unroll
    for (int r = 0; r < K; r++) {
        const int j = lane * K + r;
        if (start[r]) lv++;
        if (j < S.n && lv < L) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&lvl_q[lv]), (unsigned long long)(long long)S.qty[r]);
            if (start[r]) lvl_px[lv] = S.px[r];
        }
    }
    return __shfl_sync(FULL, incl, 31);
}

// Carry-over cancels of agent `a` on one side (Sec. 4, Action Conversion):
// every resting order of the agent not at a wanted (side, price) is deleted,
// in book order, each as one agent message.
template <int K, bool BID>
__device__ __forceinline__ void agent_cancels(Book<K> &S, const Book<K> &bid, const Book<K> &ask, int a,
                                              const int (&wa)[3], const int (&ws)[3], const int (&wp)[3], int nw,
                                              Ctx &c, int lane, bool snap_env, const KParams &p, int cap,
                                              long long &snap_n, long long snap_bytes) {
    const int side = BID ? LOB_BUY : LOB_SELL;
    for (;;) {
        unsigned h = 0;
#pragma unroll
        for (int r = 0; r < K; r++) {
            const int j = lane * K + r;
            if (j < S.n && S.id[r] < 0 && (int)((~S.id[r]) & 1) == a) {
                bool keep = false;
#pragma unroll
                for (int i = 0; i < 3; i++) keep |= i < nw && wa[i] == a && ws[i] == side && wp[i] == S.px[r];
                if (!keep) h |= 1u << r;
            }
        }
        const unsigned lanes = __ballot_sync(FULL, h != 0);
        if (lanes == 0) break;
        const int first = __ffs(lanes) - 1;
        h = lane == first ? (h & (0u - h)) : 0u;
        c.c_msgs += 1;
        c.c_agent += 1;
#pragma unroll
        for (int r = 0; r < K; r++)
            if ((h >> r) & 1u) c.l_cancel_vol += S.qty[r];
        book_remove<K>(S, h, first, lane);
        if (snap_env && snap_n < p.snap_cap) write_snapshot<K>(bid, ask, cap, p.snaps + snap_n * snap_bytes, lane);
        snap_n++;
        c.msg_idx++;
    }
}

// Per-warp shared memory.
struct WarpSmem {
    DevMsg tile[2][TILE];
    unsigned long long bar[2];
    long long lvl_q[2][LMAX];
    int lvl_px[2][LMAX];
};

// Message tile pipeline state of one warp.
struct MsgPipe {
    unsigned tiles;  // tiles issued so far by this warp (buffer = tiles & 1)
    unsigned waited; // tiles waited for
};

// Run n_steps env steps of env e with the book resident in registers.
template <int K>
__device__ void run_env(const KParams &p, int e, WarpSmem &sm, MsgPipe &pipe, int lane) {
    EnvState *st = p.st + e;
    const int cap = p.caps[e];
    const int CAPS = 32 * K;
    unsigned char *blk = p.books + p.book_off[e];
    const int A = p.n_agents;

    Ctx c;
    c.ts_next = st->ts_next; c.seq_next = st->seq_next;
    c.inv0 = st->inv[0]; c.inv1 = st->inv[1];
    c.cash0 = st->cash[0]; c.cash1 = st->cash[1];
    c.pv0 = st->pv_prev[0]; c.pv1 = st->pv_prev[1];
    c.exec_done = st->exec_done;
    c.last_px = st->last_px;
    c.A = A; c.exec_dir = p.exec_dir;
    long long *cnt = p.counters + (long long)e * LOB_NCOUNTERS;
    c.c_msgs = cnt[0]; c.c_agent = cnt[1]; c.c_fills = cnt[2]; c.c_fill_vol = cnt[3];
    c.c_add_vol = cnt[4]; c.c_mkt_vol = cnt[5]; c.c_mkt_disc = cnt[6];
    c.c_cancel_miss = cnt[8]; c.c_drop_vol = cnt[9]; c.c_drop_cnt = cnt[10]; c.c_evict_cnt = cnt[12];
    c.c_bad = cnt[13]; c.bg_cash = cnt[14]; c.bg_inv = cnt[15];
    c.l_cancel_vol = 0; c.l_evict_vol = 0;
    c.status = 0;
    c.fill_log = p.fills ? p.fills + (long long)e * p.fill_cap : nullptr;
    c.fill_cap = p.fill_cap;
    const unsigned long long seed = p.seeds[e];

    Book<K> bid, ask;
    const int nb0 = st->n[0], na0 = st->n[1];
    book_load<K, true>(bid, blk, CAPS, lane, nb0);
    book_load<K, false>(ask, blk, CAPS, lane, na0);

    const bool snap_env = p.snaps != nullptr && e == 0;
    long long snap_n = 0;
    const long long snap_bytes = 8 + 48 * (long long)cap;
    bool timed_out = false;

    for (int step = 0; step < p.n_steps && !timed_out; step++) {
        const int t = p.t0 + step;
        const int k = p.k0 + step;
        const long long mb = p.offsets[(long long)e * p.off_stride + k];
        const long long me = p.offsets[(long long)e * p.off_stride + k + 1];
        const int nmsg = (int)(me - mb);
        const int ntiles = (nmsg + TILE - 1) / TILE;
        const unsigned tile0 = pipe.tiles;
        if (ntiles > 0) {
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                const int cntm = min(TILE, nmsg);
                tma_bulk_g2s(sm.tile[pipe.tiles & 1], p.msgs + mb, (unsigned)cntm * 32u, &sm.bar[pipe.tiles & 1]);
            }
            pipe.tiles++;
        }
        c.msg_idx = 0;
        c.fill_n = 0;
        snap_n = 0;

        // ---- 1-3. action conversion, carry-over cancels, shuffle, agent orders
        int act0 = 0, act1 = 0;
        if (A == 2) {
            if (p.action_mode == LOB_ACT_RANDOM) {
                const unsigned long long key = step_key(seed, t, TAG_POLICY);
                act0 = (int)bounded(sm_mix(key + GAMMA), 12);
                act1 = (int)bounded(sm_mix(key + 2 * GAMMA), 12);
            } else {
                const int *ap = p.actions + (long long)step * p.act_step_stride + 2LL * e;
                act0 = ap[0];
                act1 = ap[1];
                if (act0 < 0 || act0 >= 12 || act1 < 0 || act1 >= 12) c.status |= ST_BADACT;
            }
            const long long bb = bid.n ? bid.best : c.last_px;
            const long long ba = ask.n ? ask.best : c.last_px;
            // wanted orders: (agent, side, px, qty); at most 3
            int wa[3] = {0, 0, 0}, ws[3] = {0, 0, 0}, wp[3] = {0, 0, 0};
            long long wq[3] = {0, 0, 0};
            int nw = 0;
            const long long remaining = (long long)p.exec_target - c.exec_done;
            if (remaining > 0 && act0 >= 0 && act0 < 12) {
                const int pi = act0 / 3, mi = act0 % 3;
                const long long mult = mi == 0 ? 1 : (mi == 1 ? 2 : 5);
                long long q0 = ((long long)p.exec_target + p.T - 1) / p.T;
                q0 = q0 < 1 ? 1 : q0;
                long long qty = mult * q0;
                qty = qty < remaining ? qty : remaining;
                const long long s2 = bb + ba;
                const long long fl = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
                const long long ce = -((s2 <= 0) ? (-s2) / 2 : -((s2 + 1) / 2));
                long long wpx;
                if (p.exec_dir == LOB_SELL) wpx = pi == 0 ? bb : pi == 1 ? ce : pi == 2 ? ba : ba + 2;
                else wpx = pi == 0 ? ba : pi == 1 ? fl : pi == 2 ? bb : bb - 2;
                wa[0] = 0; ws[0] = p.exec_dir; wp[0] = (int)wpx; wq[0] = qty;
                nw = 1;
            }
            if (act1 >= 1 && act1 < 12) {
                long long qb, qa;
                if (act1 <= 9) { qb = bb - (act1 - 1) / 3; qa = ba + (act1 - 1) % 3; }
                else if (act1 == 10) { qb = bb + 1; qa = ba; }
                else { qb = bb; qa = ba - 1; }
                if (nw == 0) {
                    wa[0] = 1; ws[0] = LOB_BUY; wp[0] = (int)qb; wq[0] = p.mm_lot;
                    wa[1] = 1; ws[1] = LOB_SELL; wp[1] = (int)qa; wq[1] = p.mm_lot;
                } else {
                    wa[1] = 1; ws[1] = LOB_BUY; wp[1] = (int)qb; wq[1] = p.mm_lot;
                    wa[2] = 1; ws[2] = LOB_SELL; wp[2] = (int)qa; wq[2] = p.mm_lot;
                }
                nw += 2;
            }
            // carry-over: resting agent orders at a wanted (agent, side, price) are kept
            long long kept[3] = {0, 0, 0};
#pragma unroll
            for (int r = 0; r < K; r++) {
                const int j = lane * K + r;
                if (j < bid.n && bid.id[r] < 0) {
                    const int a = (int)((~bid.id[r]) & 1);
                    int m = -1;
#pragma unroll
                    for (int i = 0; i < 3; i++)
                        if (i < nw && wa[i] == a && ws[i] == LOB_BUY && wp[i] == bid.px[r]) m = i;
#pragma unroll
                    for (int i = 0; i < 3; i++) if (m == i) kept[i] += bid.qty[r];
                }
                if (j < ask.n && ask.id[r] < 0) {
                    const int a = (int)((~ask.id[r]) & 1);
                    int m = -1;
#pragma unroll
                    for (int i = 0; i < 3; i++)
                        if (i < nw && wa[i] == a && ws[i] == LOB_SELL && wp[i] == ask.px[r]) m = i;
#pragma unroll
                    for (int i = 0; i < 3; i++) if (m == i) kept[i] += ask.qty[r];
                }
            }
#pragma unroll
            for (int i = 0; i < 3; i++) kept[i] = warp_sum(kept[i]);
            // cancels: agent 0 then 1, bids then asks, each in book order
            const bool snap_on = snap_env;
            agent_cancels<K, true>(bid, bid, ask, 0, wa, ws, wp, nw, c, lane, snap_on, p, cap, snap_n, snap_bytes);
            agent_cancels<K, false>(ask, bid, ask, 0, wa, ws, wp, nw, c, lane, snap_on, p, cap, snap_n, snap_bytes);
            agent_cancels<K, true>(bid, bid, ask, 1, wa, ws, wp, nw, c, lane, snap_on, p, cap, snap_n, snap_bytes);
            agent_cancels<K, false>(ask, bid, ask, 1, wa, ws, wp, nw, c, lane, snap_on, p, cap, snap_n, snap_bytes);
            // orders to send: wanted minus kept; then Fisher-Yates shuffle
            int sa[3], ss[3], sp[3], sq[3];
            int ns = 0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const long long q = wq[i] - kept[i];
                if (i < nw && q > 0) {
#pragma unroll
                    for (int u = 0; u < 3; u++)
                        if (u == ns) { sa[u] = wa[i]; ss[u] = ws[i]; sp[u] = wp[i]; sq[u] = (int)q; }
                    ns++;
                }
            }
            if (ns > 1) {
                const unsigned long long key = step_key(seed, t, TAG_SHUFFLE);
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    const int i = ns - 1 - d;
                    if (i >= 1) {
                        const int jj = (int)bounded(sm_mix(key + GAMMA * (unsigned long long)(d + 1)), (unsigned)(i + 1));
                        // swap entries i and jj (static indices only)
                        int ta = 0, ts_ = 0, tp = 0, tq = 0, ua = 0, us = 0, up = 0, uq = 0;
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            if (u == i) { ta = sa[u]; ts_ = ss[u]; tp = sp[u]; tq = sq[u]; }
                            if (u == jj) { ua = sa[u]; us = ss[u]; up = sp[u]; uq = sq[u]; }
                        }
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            if (u == i) { sa[u] = ua; ss[u] = us; sp[u] = up; sq[u] = uq; }
                            else if (u == jj) { sa[u] = ta; ss[u] = ts_; sp[u] = tp; sq[u] = tq; }
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 3; u++) {
                if (u < ns) {
                    const long long oid = -(1 + (long long)sa[u] + 2LL * c.seq_next);
                    c.seq_next++;
                    process_msg<K>(bid, ask, cap, LOB_ADD, ss[u], sp[u], sq[u], oid, true, c, lane);
                    if (snap_env && snap_n < p.snap_cap)
                        write_snapshot<K>(bid, ask, cap, p.snaps + snap_n * snap_bytes, lane);
                    snap_n++;
                    c.msg_idx++;
                }
            }
        }

        // ---- 4. market-replay messages, staged tile by tile
        for (int tix = 0; tix < ntiles; tix++) {
            const unsigned buf = (tile0 + tix) & 1u;
            const unsigned phase = ((tile0 + tix) >> 1) & 1u;
            if (!mbar_wait(&sm.bar[buf], phase, p.wait_budget)) {
                c.status |= ST_TIMEOUT;
                mbar_wait(&sm.bar[buf], phase, p.wait_budget);  // let the copy in flight land
                timed_out = true;
                break;
            }
            if (tix + 1 < ntiles) {
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async_smem();
                    const int cntm = min(TILE, nmsg - (tix + 1) * TILE);
                    tma_bulk_g2s(sm.tile[pipe.tiles & 1], p.msgs + mb + (long long)(tix + 1) * TILE,
                                 (unsigned)cntm * 32u, &sm.bar[pipe.tiles & 1]);
                }
                pipe.tiles++;
            }
            const int cnt_t = min(TILE, nmsg - tix * TILE);
            for (int i = 0; i < cnt_t; i++) {
                const int4 w0 = *reinterpret_cast<const int4 *>(&sm.tile[buf][i]);
                const int4 w1 = *(reinterpret_cast<const int4 *>(&sm.tile[buf][i]) + 1);
                const long long oid = ((long long)(unsigned)w0.w << 32) | (unsigned)w0.z;
                const int type = (short)(w1.z & 0xffff);
                const int side = (short)((unsigned)w1.z >> 16);
                process_msg<K>(bid, ask, cap, type, side, w1.x, w1.y, oid, false, c, lane);
                if (snap_env && snap_n < p.snap_cap)
                    write_snapshot<K>(bid, ask, cap, p.snaps + snap_n * snap_bytes, lane);
                snap_n++;
                c.msg_idx++;
            }
        }
        if (timed_out) break;

        // ---- 5. step outcomes
        const long long obs_base = ((long long)step * p.n_envs + e);
        if (A > 0) {
            const int L = p.L;
            for (int i = lane; i < 2 * LMAX; i += 32) {
                (&sm.lvl_q[0][0])[i] = 0;
                (&sm.lvl_px[0][0])[i] = 0;
            }
            __syncwarp();
            const int nlb = side_levels<K, true>(bid, L, sm.lvl_px[0], sm.lvl_q[0], lane);
            const int nla = side_levels<K, false>(ask, L, sm.lvl_px[1], sm.lvl_q[1], lane);
            __syncwarp();
            const long long bb = bid.n ? bid.best : c.last_px;
            const long long ba = ask.n ? ask.best : c.last_px;
            const long long s2 = bb + ba;
            const long long anchor = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
            long long own0 = 0, own1 = 0;
#pragma unroll
            for (int r = 0; r < K; r++) {
                const int j = lane * K + r;
                if (j < bid.n && bid.id[r] < 0) { if ((~bid.id[r]) & 1) own1 += bid.qty[r]; else own0 += bid.qty[r]; }
                if (j < ask.n && ask.id[r] < 0) { if ((~ask.id[r]) & 1) own1 += ask.qty[r]; else own0 += ask.qty[r]; }
            }
            own0 = warp_sum(own0);
            own1 = warp_sum(own1);
            // Eq. 1: PV = Q_inv * P_ref + Cash, P_ref the liquidation touch
            const long long pref0 = c.inv0 > 0 ? bb : (c.inv0 < 0 ? ba : 0);
            const long long pref1 = c.inv1 > 0 ? bb : (c.inv1 < 0 ? ba : 0);
            const long long pv0 = (long long)((unsigned long long)c.inv0 * (unsigned long long)pref0 + (unsigned long long)c.cash0);
            const long long pv1 = (long long)((unsigned long long)c.inv1 * (unsigned long long)pref1 + (unsigned long long)c.cash1);
            const long long r0 = (long long)((unsigned long long)pv0 - (unsigned long long)c.pv0);
            const long long r1 = (long long)((unsigned long long)pv1 - (unsigned long long)c.pv1);
            c.pv0 = pv0; c.pv1 = pv1;
            const float tl = __fdiv_rn((float)(p.T - (t + 1)), (float)p.T);
            const int D = p.D;
            float *ob = p.obs ? p.obs + obs_base * A * D : nullptr;
            if (ob) {
                for (int idx = lane; idx < A * D; idx += 32) {
                    const int a = idx / D, f = idx % D;
                    float v;
                    if (f < 4 * L) {
                        const int s = f / (2 * L);
                        const int i = (f % (2 * L)) >> 1;
                        const int nl = s == 0 ? nlb : nla;
                        if (i >= nl) v = 0.0f;
                        else if (f & 1) v = __ll2float_rn(sm.lvl_q[s][i]);
                        else v = __ll2float_rn((long long)sm.lvl_px[s][i] - anchor);
                    } else {
                        const int g = f - 4 * L;
                        if (g == 0) v = __ll2float_rn(a == 0 ? c.inv0 : c.inv1);
                        else if (g == 1) v = __ll2float_rn(a == 0 ? c.cash0 : c.cash1);
                        else if (g == 2) v = tl;
                        else if (g == 3) v = a == 0 ? __ll2float_rn((long long)p.exec_target - c.exec_done) : 0.0f;
                        else v = __ll2float_rn(a == 0 ? own0 : own1);
                    }
                    ob[idx] = v;
                }
            }
            if (lane == 0) {
                if (p.rew) { p.rew[obs_base * A] = r0; p.rew[obs_base * A + 1] = r1; }
                if (p.act_out) { p.act_out[2LL * e] = act0; p.act_out[2LL * e + 1] = act1; }
            }
        }
        if (lane == 0 && p.done) p.done[obs_base] = (unsigned char)(t + 1 == p.T);
        if (lane == 0 && p.fill_counts) p.fill_counts[e] = c.fill_n;
        if (lane == 0 && snap_env && p.snap_count) *p.snap_count = snap_n;
        if (lane == 0) { st->act[0] = act0; st->act[1] = act1; }
    }

    // ---- write back: counters, env scalars, book
    const long long cv = warp_sum(c.l_cancel_vol);
    const long long ev = warp_sum(c.l_evict_vol);
    const int any_status = __reduce_or_sync(FULL, (unsigned)c.status);
    if (lane == 0) {
        if (any_status) atomicOr(p.status, any_status);
        cnt[0] = c.c_msgs; cnt[1] = c.c_agent; cnt[2] = c.c_fills; cnt[3] = c.c_fill_vol;
        cnt[4] = c.c_add_vol; cnt[5] = c.c_mkt_vol; cnt[6] = c.c_mkt_disc; cnt[7] += cv;
        cnt[8] = c.c_cancel_miss; cnt[9] = c.c_drop_vol; cnt[10] = c.c_drop_cnt; cnt[11] += ev;
        cnt[12] = c.c_evict_cnt; cnt[13] = c.c_bad; cnt[14] = c.bg_cash; cnt[15] = c.bg_inv;
    }
    if (timed_out) return;
    if (lane == 0) {
        st->ts_next = c.ts_next; st->seq_next = c.seq_next;
        st->inv[0] = c.inv0; st->inv[1] = c.inv1; st->cash[0] = c.cash0; st->cash[1] = c.cash1;
        st->pv_prev[0] = c.pv0; st->pv_prev[1] = c.pv1; st->exec_done = c.exec_done;
        st->last_px = c.last_px; st->n[0] = bid.n; st->n[1] = ask.n;
        st->t = p.t0 + p.n_steps;
    }
    book_store<K, true>(bid, blk, CAPS, lane);
    book_store<K, false>(ask, blk, CAPS, lane);
}

template <int K>
__global__ void __launch_bounds__(256) k_env_steps(const KParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[wib];
    if (lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    MsgPipe pipe{0u, 0u};
    if (p.queue == nullptr) {
        const int w = blockIdx.x * (blockDim.x >> 5) + wib;
        if (w < p.n_list) run_env<K>(p, p.env_list[w], sm, pipe, lane);
    } else {
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(p.queue, 1);
            w = __shfl_sync(FULL, w, 0);
            if (w >= p.n_list) break;
            run_env<K>(p, p.env_list[w], sm, pipe, lane);
        }
    }
}

}  // namespace lobk
