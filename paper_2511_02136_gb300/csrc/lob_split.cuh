// lob_split.cuh -- the env step with two warps per env, one per book side
// (the plain benchmark configuration: the benchmark pair or no agents, a
// fixed task side, the PV reward, no trace; register-pool classes K = 2..8).
//
// A side's book changes only through messages its own warp handles: the
// side's own rests and cancels, and the takes of incoming orders of the other
// side.  So each warp walks the whole message sequence and acts on the
// messages of its side; the only hand-over is the remainder of a limit add
// that may cross: the opposite warp runs the take and posts the unfilled
// quantity, which the add's own warp then rests.  A buy add at price p cannot
// cross when p is below a lower bound of the best ask at its position -- the
// ask front at the chunk's start and the prices of the sell adds before it in
// the chunk (only a resting sell lowers the best ask) -- and the mirror holds
// for sells; both warps derive the same bound from the staged chunk, so
// those adds need no hand-over at all.
//
// Everything else is merged without a hand-over:
//  * fills move cash and inventory between owners additively; each warp keeps
//    its own deltas and both add the two at the step's end (the last trade
//    price is the fill of the later message);
//  * arrival stamps count the rests of both sides in message order: a rest
//    gets a provisional stamp, and at the chunk's end, when both warps' rest
//    masks of the chunk are known, the stamp becomes the step's rest count
//    before it (stamps only order orders of one price, which the priority
//    index already does, so the provisional values change no decision);
//  * counters are sums of the two warps' counts.
// The two warps meet at a named barrier at the end of every staged chunk and
// at the step's start and end; every wait is bounded.
#pragma once
#include "lob_device.cuh"

namespace lobk {

constexpr long long PROV_TS = 1LL << 62;   // provisional arrival stamp base (real stamps stay below it)

// The per-step scalars the two warps add up: agent inventory, cash and
// executed volume, and the counters that change inside a step.
constexpr int NACC = 19;
__device__ __forceinline__ void acc_store(const Ctx &c, long long *d) {
    d[0] = c.inv0; d[1] = c.inv1; d[2] = c.cash0; d[3] = c.cash1; d[4] = c.exec_done;
    d[5] = c.c_msgs; d[6] = c.c_agent; d[7] = c.c_fills; d[8] = c.c_fill_vol; d[9] = c.c_add_vol;
    d[10] = c.c_mkt_vol; d[11] = c.c_mkt_disc; d[12] = c.c_cancel_vol; d[13] = c.c_cancel_miss;
    d[14] = c.c_drop_vol; d[15] = c.c_drop_cnt; d[16] = c.c_evict_vol; d[17] = c.c_evict_cnt; d[18] = c.c_bad;
}
// c = a + b - base, field by field, in wrapping 64-bit arithmetic (both
// warps start a step from the same values, base).
__device__ __forceinline__ void acc_merge(Ctx &c, const long long *a, const long long *b, const long long *base) {
    typedef unsigned long long u64;
    long long v[NACC];
#pragma unroll
    for (int i = 0; i < NACC; i++) v[i] = (long long)((u64)a[i] + (u64)b[i] - (u64)base[i]);
    c.inv0 = v[0]; c.inv1 = v[1]; c.cash0 = v[2]; c.cash1 = v[3]; c.exec_done = v[4];
    c.c_msgs = v[5]; c.c_agent = v[6]; c.c_fills = v[7]; c.c_fill_vol = v[8]; c.c_add_vol = v[9];
    c.c_mkt_vol = v[10]; c.c_mkt_disc = v[11]; c.c_cancel_vol = v[12]; c.c_cancel_miss = v[13];
    c.c_drop_vol = v[14]; c.c_drop_cnt = v[15]; c.c_evict_vol = v[16]; c.c_evict_cnt = v[17]; c.c_bad = v[18];
}

// What one warp tells the other at the step's end.
struct SplitSummary {
    long long acc[NACC];          // this warp's copy of the summed scalars
    long long lf_pos;             // launch position of this warp's last fill, or -1
    long long own0, own1;         // the agents' resting quantity on this side
    int last_px;                  // this warp's last-trade price
    int n, fpx;                   // live orders and front price of this side
    int status, tmo;
    int nlev;                     // levels of this side (top L)
    int pad[2];
};

// Per env pair, after the block's WarpSmem array.
struct __align__(16) SplitSmem {
    DevMsg amsg[2][4];            // each warp's copy of the step's agent orders
    int rem[TILE + 3];            // the remainder of each add of the chunk that may cross
    int prog[2];                  // per side: 1 + launch position of the last remainder posted (volatile use)
    long long front[2][2];        // [chunk parity][side]: front price at the chunk's start (or an empty mark)
    unsigned rmask[2][2];         // [chunk parity][side]: records of the chunk that came to rest
    long long kept[2][3];         // carry-over: kept quantity of each wanted order, per side
    long long base[2][NACC];      // per side: its scalars at the step's start
    SplitSummary sum[2][2];       // [step parity][side], at the step's end
};
static_assert(sizeof(SplitSmem) % 16 == 0, "keeps the pairs' areas 16-byte aligned");

constexpr long long SPLIT_NO_BID = -(1LL << 40), SPLIT_NO_ASK = 1LL << 40;   // fronts of empty sides

__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// side_rest with an explicit arrival stamp: returns whether the order was
// inserted (not dropped) and, through f_out, its slot.
template <int K, bool BID>
__device__ __forceinline__ bool split_rest(Side<K> &S, PoolSmem<K> &P, int cap, int p, int q, long long oid,
                                           long long ts, Ctx &c, int lane, int &f_out) {
    const int vic = LOB_CHK(slot_at<K>(S, S.n > 0 ? S.n - 1 : 0), 32 * K, c.status);
    const int vic_q = P.qty[vic];
    const unsigned fr = ~S.occ & Side<K>::KMASK;
    const unsigned flanes = __ballot_sync(FULL, fr != 0);
    const int free_slot = __shfl_sync(FULL, slot_of<K>(lane, 31 - __clz(fr)), 31 - __clz(flanes));
    int pos = 0;
#pragma unroll
    for (int r = 0; r < K; r++)
        pos += __popc(__ballot_sync(FULL, ((S.occ >> r) & 1u) && at_least<BID>(S.px[r], p)));
    const bool full = S.n >= cap;
    const bool ins = !(full && pos >= S.n);
    const bool ev = full && ins;
    if (full) {
        c.c_drop_vol += ins ? 0 : q;
        c.c_drop_cnt += ins ? 0 : 1;
        c.c_evict_vol += ev ? vic_q : 0;
        c.c_evict_cnt += ev ? 1 : 0;
    }
    const int f = full ? vic : LOB_CHK(free_slot, 32 * K, c.status);
    const int fl = slot_lane<K>(f), fr_ = slot_r<K>(f);
    if (ins && lane == fl) S.occ |= 1u << fr_;
#pragma unroll
    for (int r = 0; r < K; r++)
        if (ins && lane == fl && r == fr_) { S.px[r] = p; S.id[r] = oid; }
    if (ins) { P.px[f] = p; P.qty[f] = q; P.id[f] = oid; P.ts[f] = ts; }
    unsigned nix[Side<K>::NW];
    ix_inserted<K>(S, pos, f, lane, nix);
#pragma unroll
    for (int w = 0; w < Side<K>::NW; w++) S.ix[w] = ins ? nix[w] : S.ix[w];
    S.n += (ins && !full) ? 1 : 0;
    const bool front = ins && pos == 0;
    S.fpx = front ? p : S.fpx;
    S.fqty = front ? q : S.fqty;
    S.fid = front ? oid : S.fid;
    S.fslot = front ? f : S.fslot;
    f_out = f;
    return ins;
}

// A bounded wait until the other warp has posted the remainder of launch
// position `want - 1`.
__device__ __forceinline__ bool split_wait(const int *prog, int want, long long budget) {
    const long long t0 = clock64();
    for (;;) {
        const int v = *reinterpret_cast<const volatile int *>(prog);
        if ((int)(v - want) >= 0) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// n_steps steps of env e on one side: BID = the warp of the bids.  Both warps
// of the pair run this with the same arguments; `bar` is the pair's barrier.
template <int K, bool BID>
__device__ void run_env_split(const KParams &p, int e, WarpSmem<K> &sm, SplitSmem &sx, MsgPipe &pipe, int lane,
                              int bar) {
    constexpr int SD = BID ? 0 : 1, OD = 1 - SD;
    // dispatch codes (type - 1) * 2 + (side is sell): this side's limit add,
    // the other side's (taken against this side), this side's cancels, and
    // the other side's market order (taken against this side)
    constexpr int OWN_ADD = BID ? 0 : 1, OPP_ADD = 1 - OWN_ADD;
    constexpr int OWN_PART = BID ? 2 : 3, OWN_DEL = BID ? 4 : 5, OPP_MKT = BID ? 7 : 6;
    constexpr int TAKER_SIDE = BID ? LOB_SELL : LOB_BUY;
    typedef unsigned long long u64;
    PoolSmem<K> &P = sm.pool[SD];
    EnvState *st = p.st + e;
    const bool uni = p.uni_cap > 0;
    const int cap = uni ? p.uni_cap : p.caps[e];
    unsigned char *blk = p.books + (uni ? (long long)e * p.uni_block : p.book_off[e]);
    if (BID && p.book_prefetch && lane == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(blk), "r"((unsigned)(48 * 32 * K)) : "memory");
    const int A = p.n_agents;
    const unsigned long long seed = p.seeds[e];
    long long *cnt = p.counters + (long long)e * LOB_NCOUNTERS;
    const char *msg_base = reinterpret_cast<const char *>(p.msgs);
    const long long d0 = (long long)e * p.off_stride + p.k0;
    long long mb = p.offsets[d0];
    long long me = p.offsets[d0 + 1];

    Side<K> S;
    Ctx c;
    c.ts_next = st->ts_next; c.seq_next = st->seq_next;
    c.inv0 = st->inv[0]; c.inv1 = st->inv[1];
    c.cash0 = st->cash[0]; c.cash1 = st->cash[1];
    c.pv0 = st->pv_prev[0]; c.pv1 = st->pv_prev[1];
    c.exec_done = st->exec_done;
    c.last_px = st->last_px;
    const int n_load = st->n[SD];
    c.A = A;
    c.exec_dir = p.exec_dir;
    c.c_msgs = cnt[0]; c.c_agent = cnt[1]; c.c_fills = cnt[2]; c.c_fill_vol = cnt[3];
    c.c_add_vol = cnt[4]; c.c_mkt_vol = cnt[5]; c.c_mkt_disc = cnt[6]; c.c_cancel_vol = cnt[7];
    c.c_cancel_miss = cnt[8]; c.c_drop_vol = cnt[9]; c.c_drop_cnt = cnt[10]; c.c_evict_vol = cnt[11];
    c.c_evict_cnt = cnt[12]; c.c_bad = cnt[13]; c.bg_cash = cnt[14]; c.bg_inv = cnt[15];
    c.status = 0;
    c.fill_log = nullptr;
    c.fill_cap = 0;
    c.ag = nullptr;
    c.msg_idx = 0;
    c.fill_n = 0;

    bool timed_out = false;
    unsigned kc = 0;            // exchanges so far in this launch (parity of the exchange slots)
    long long pos_base = 0;     // launch position of the current chunk's first record
    long long lf_pos = -1;      // launch position of this warp's last fill
    int rslot = 0;              // the slot of this lane's record if it came to rest in the current chunk
    int n_other = 0;            // live orders of the other side at the last step's end
    int act0 = 0, act1 = 0;

    for (int step = 0; step < p.n_steps; step++) {
        const int t = p.t0 + step;
        if (step > 0) {
            mb = p.offsets[d0 + step];
            me = p.offsets[d0 + step + 1];
        }
        const int nmsg = (int)(me - mb);
        const int ntiles = (nmsg + TILE - 1) / TILE;
        const unsigned tile0 = pipe.tiles;
        if (ntiles > 0) {   // the bid warp requests the tiles; both count them
            __syncwarp();
            if (BID && lane == 0 && !timed_out) {
                fence_proxy_async_smem();
                tma_bulk_g2s(sm.tile[pipe.tiles & 1], msg_base + mb * 32, (unsigned)(min(TILE, nmsg) * 32),
                             &sm.bar[pipe.tiles & 1]);
            }
            pipe.tiles++;
        }
        if (step == 0) {
            __syncwarp();
            side_load<K, BID>(S, P, blk, lane);
            side_set_count<K>(S, n_load, lane);
            __syncwarp();
            front_refresh<K>(S, P);
            if (lane == 0) sx.front[kc & 1][SD] = S.n > 0 ? (long long)S.fpx : (BID ? SPLIT_NO_BID : SPLIT_NO_ASK);
            pair_sync(bar);
        }
        // the step's start: both warps hold the same scalars
        if (lane == 0) acc_store(c, sx.base[SD]);
        const u64 pair_cash0 = (u64)c.cash0 + (u64)c.cash1, pair_inv0 = (u64)c.inv0 + (u64)c.inv1;
        long long ts_base = c.ts_next;

        // ---- 1-3. action conversion, carry-over cancels, shuffle (both warps
        // derive the same orders; each cancels on its own side)
        int ns = 0;
        if (A == 2) {
            if (p.action_mode == LOB_ACT_RANDOM) {
                const unsigned long long key = step_key(seed, t, TAG_POLICY);
                act0 = (int)bounded(sm_mix(key + GAMMA), 12);
                act1 = (int)bounded(sm_mix(key + 2 * GAMMA), 12u);
            } else {
                const int *ap = p.actions + (long long)step * p.act_step_stride + 2LL * e;
                act0 = ap[0];
                act1 = ap[1];
                if (act0 < 0 || act0 >= 12 || act1 < 0 || act1 >= 12) c.status |= ST_BADACT;
            }
            const long long fb = sx.front[kc & 1][0], fa = sx.front[kc & 1][1];
            const long long bb = fb != SPLIT_NO_BID ? fb : c.last_px;
            const long long ba = fa != SPLIT_NO_ASK ? fa : c.last_px;
            int wa[3] = {0, 0, 0}, ws[3] = {0, 0, 0}, wp[3] = {0, 0, 0};
            long long wq[3] = {0, 0, 0};
            int nw = 0;
            const long long remaining = (long long)p.exec_target - c.exec_done;
            if (remaining > 0 && act0 >= 0 && act0 < 12) {
                const int pi = act0 / 3, mi = act0 % 3;
                const long long mult = mi == 0 ? 1 : (mi == 1 ? 2 : 5);
                long long qty = mult * p.exec_q0;
                qty = qty < remaining ? qty : remaining;
                const long long s2 = bb + ba;
                const long long fl = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
                const long long ce = s2 <= 0 ? -((-s2) / 2) : (s2 + 1) / 2;
                long long wpx;
                if (c.exec_dir == LOB_SELL) wpx = pi == 0 ? bb : pi == 1 ? ce : pi == 2 ? ba : ba + 2;
                else wpx = pi == 0 ? ba : pi == 1 ? fl : pi == 2 ? bb : bb - 2;
                wa[0] = 0; ws[0] = c.exec_dir; wp[0] = (int)wpx; wq[0] = qty;
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
            unsigned kept_u[3] = {0u, 0u, 0u};
            const unsigned cmask = side_carry<K>(S, P, sm.cand[SD], BID ? LOB_BUY : LOB_SELL, wa, ws, wp, nw, kept_u, lane);
            long long kept_own[3];
#pragma unroll
            for (int i = 0; i < 3; i++) kept_own[i] = (long long)__reduce_add_sync(FULL, kept_u[i]);
            side_cancel_set<K>(S, P, cmask, c, lane);
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 3; i++) sx.kept[SD][i] = kept_own[i];
                sx.front[(kc + 1) & 1][SD] = S.n > 0 ? (long long)S.fpx : (BID ? SPLIT_NO_BID : SPLIT_NO_ASK);
            }
            pair_sync(bar);
            kc++;
            long long kept[3];
#pragma unroll
            for (int i = 0; i < 3; i++) kept[i] = sx.kept[0][i] + sx.kept[1][i];
            int sa[3] = {0, 0, 0}, ss[3] = {0, 0, 0}, sp[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
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
                        int ta = 0, tb = 0, tp = 0, tq = 0, ua = 0, ub = 0, up = 0, uq = 0;
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            if (u == i) { ta = sa[u]; tb = ss[u]; tp = sp[u]; tq = sq[u]; }
                            if (u == jj) { ua = sa[u]; ub = ss[u]; up = sp[u]; uq = sq[u]; }
                        }
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            if (u == i) { sa[u] = ua; ss[u] = ub; sp[u] = up; sq[u] = uq; }
                            else if (u == jj) { sa[u] = ta; ss[u] = tb; sp[u] = tp; sq[u] = tq; }
                        }
                    }
                }
            }
            if (lane < ns) {
                int ma = 0, ms = 0, mp = 0, mq = 0;
#pragma unroll
                for (int u = 0; u < 3; u++)
                    if (u == lane) { ma = sa[u]; ms = ss[u]; mp = sp[u]; mq = sq[u]; }
                DevMsg r;
                r.ts = 0;
                r.oid = -(1 + (long long)ma + 2LL * (c.seq_next + lane));
                r.px = mp; r.qty = mq; r.type = (short)LOB_ADD; r.side = (short)ms; r.pad = 0;
                sx.amsg[SD][lane] = r;
            }
            c.seq_next += ns;
            __syncwarp();
        }

        // ---- 4. the agents' orders, then the market-replay messages
        for (int ch = ns > 0 ? -1 : 0; ch < ntiles; ch++) {
            const DevMsg *base;
            int cnt_ch;
            if (ch < 0) {
                base = sx.amsg[SD];
                cnt_ch = ns;
            } else {
                const unsigned buf = (tile0 + ch) & 1u;
                const unsigned phase = ((tile0 + ch) >> 1) & 1u;
                if (!timed_out && !mbar_wait(&sm.bar[buf], phase, p.wait_budget)) {
                    c.status |= ST_TIMEOUT;
                    mbar_wait(&sm.bar[buf], phase, p.drain_budget);   // let the copy in flight land
                    timed_out = true;
                }
                if (ch + 1 < ntiles) {
                    __syncwarp();
                    if (BID && lane == 0 && !timed_out) {
                        fence_proxy_async_smem();
                        tma_bulk_g2s(sm.tile[pipe.tiles & 1], msg_base + (mb + (long long)(ch + 1) * TILE) * 32,
                                     (unsigned)(min(TILE, nmsg - (ch + 1) * TILE) * 32), &sm.bar[pipe.tiles & 1]);
                    }
                    pipe.tiles++;
                }
                base = sm.tile[buf];
                cnt_ch = min(TILE, nmsg - ch * TILE);
            }
            const int4 *rp = reinterpret_cast<const int4 *>(base);
            if (BID) {
                c.c_msgs += cnt_ch;
                c.c_agent += ch < 0 ? cnt_ch : 0;
            }
            // each record's dispatch code (lane r = record r) and the
            // no-cross bounds: the other side's front at the chunk's start
            // and the prices of the adds before the record that could improve it
            const bool has = lane < cnt_ch;
            int d = 8, rpx = 0;
            if (has) {
                const int4 w = rp[2 * lane + 1];
                const int ty = w.z & 0xffff, sd = w.z >> 16;
                const bool ok = ty >= LOB_ADD && ty <= LOB_MARKET && (sd == 1 || sd == -1) && (w.y > 0 || ty == LOB_DELETE);
                d = ok ? ((ty - 1) << 1) | (sd < 0 ? 1 : 0) : 8;
                rpx = w.x;
            }
            unsigned char *dx = sm.cand[SD];
            if (has) dx[lane] = (unsigned char)d;
            int lo = d == 1 ? rpx : 0x7fffffff;          // sell adds: the ask side's best can fall to them
            int hi = d == 0 ? rpx : -0x7fffffff - 1;     // buy adds: the bid side's best can rise to them
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const int l2 = __shfl_up_sync(FULL, lo, k), h2 = __shfl_up_sync(FULL, hi, k);
                if (lane >= k) { lo = min(lo, l2); hi = max(hi, h2); }
            }
            int lo_ex = __shfl_up_sync(FULL, lo, 1), hi_ex = __shfl_up_sync(FULL, hi, 1);
            if (lane == 0) { lo_ex = 0x7fffffff; hi_ex = -0x7fffffff - 1; }
            const long long ask_lb = min(sx.front[kc & 1][1], (long long)lo_ex);
            const long long bid_ub = max(sx.front[kc & 1][0], (long long)hi_ex);
            const bool pas = (d == 0 && (long long)rpx < ask_lb) || (d == 1 && (long long)rpx > bid_ub);
            const unsigned passive = __ballot_sync(FULL, has && pas);
            const unsigned m_own_add = __ballot_sync(FULL, has && d == OWN_ADD);
            const unsigned m_opp_add = __ballot_sync(FULL, has && d == OPP_ADD);
            const unsigned m_other = __ballot_sync(FULL, has && (d == OWN_PART || d == OWN_DEL || d == OPP_MKT));
            if (BID) {
                const unsigned bad = __ballot_sync(FULL, has && d == 8);
                c.c_bad += __popc(bad);
                if (bad) c.status |= ST_BADMSG;
            }
            unsigned todo = timed_out ? 0u : (m_own_add | (m_opp_add & ~passive) | m_other);
            unsigned rested = 0;
            __syncwarp();
            int r = todo ? __ffs(todo) - 1 : cnt_ch;
            todo &= todo - 1;
            int4 w0 = rp[2 * r], w1 = rp[2 * r + 1];
            int dcur = dx[r];
            while (r < cnt_ch) {
                const int rn = todo ? __ffs(todo) - 1 : cnt_ch;
                todo &= todo - 1;
                const int4 n0 = rp[2 * rn], n1 = rp[2 * rn + 1];   // one ahead (stays in this pair's space)
                const int dn = dx[rn];
                const long long oid = ((long long)(unsigned)w0.w << 32) | (unsigned)w0.z;
                const int px = w1.x;
                const int qty = w1.y;
                const long long gpos = pos_base + r;
                if (dcur == OWN_ADD) {
                    c.c_add_vol += qty;
                    int q = qty;
                    if (!((passive >> r) & 1u)) {   // the other warp takes first and posts the rest
                        if (timed_out || !split_wait(&sx.prog[OD], (int)(gpos + 1), p.wait_budget)) {
                            c.status |= ST_TIMEOUT;
                            timed_out = true;
                        } else {
                            __threadfence_block();
                            q = *reinterpret_cast<const volatile int *>(&sx.rem[r]);
                        }
                    }
                    if (q > 0) {
                        int f = 0;
                        if (split_rest<K, BID>(S, P, cap, px, q, oid, PROV_TS + r, c, lane, f)) {
                            rested |= 1u << r;
                            if (lane == r) rslot = f;
                        }
                    }
                } else if (dcur == OPP_ADD) {
                    int q = qty;
                    if (S.n > 0 && at_least<BID>(S.fpx, px)) {
                        const long long f0 = c.c_fills;
                        q = side_take<K, BID, false, false>(S, P, true, px, qty, oid, TAKER_SIDE, c, lane);
                        if (c.c_fills != f0) lf_pos = gpos;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        sx.rem[r] = q;
                        __threadfence_block();
                        *reinterpret_cast<volatile int *>(&sx.prog[SD]) = (int)(gpos + 1);
                    }
                } else if (dcur == OPP_MKT) {
                    c.c_mkt_vol += qty;
                    const long long f0 = c.c_fills;
                    c.c_mkt_disc += side_take<K, BID, false, false>(S, P, false, 0, qty, oid, TAKER_SIDE, c, lane);
                    if (c.c_fills != f0) lf_pos = gpos;
                } else {
                    side_cancel<K>(S, P, (dcur >> 1) + 1, px, qty, oid, c, lane);
                }
                w0 = n0;
                w1 = n1;
                dcur = dn;
                r = rn;
            }
            // the chunk's end: fronts for the next chunk's bounds, rest masks for the stamps
            if (lane == 0) {
                sx.front[(kc + 1) & 1][SD] = S.n > 0 ? (long long)S.fpx : (BID ? SPLIT_NO_BID : SPLIT_NO_ASK);
                sx.rmask[kc & 1][SD] = rested;
            }
            pair_sync(bar);
            const unsigned all = rested | sx.rmask[kc & 1][OD];
            kc++;
            if ((rested >> lane) & 1u) {
                if (P.ts[rslot] == PROV_TS + lane) P.ts[rslot] = ts_base + __popc(all & ((1u << lane) - 1u));
            }
            ts_base += __popc(all);
            pos_base += cnt_ch;
            __syncwarp();
        }
        c.ts_next = ts_base;

        // ---- 5. step outcomes: each warp its side's levels, then both merge
        const int L = p.L;
        for (int i = lane; i < LMAX; i += 32) {
            sm.lvl_q[SD][i] = 0;
            sm.lvl_px[SD][i] = 0;
        }
        __syncwarp();
        long long own0 = 0, own1 = 0;
        int nlev = 0;
        if (A > 0) nlev = side_levels<K>(S, P, L, sm.lvl_px[SD], sm.lvl_q[SD], own0, own1, lane);
        const int any_status = (int)__reduce_or_sync(FULL, (unsigned)c.status);
        if (lane == 0) {
            SplitSummary &m = sx.sum[step & 1][SD];
            acc_store(c, m.acc);
            m.lf_pos = lf_pos;
            m.own0 = own0;
            m.own1 = own1;
            m.last_px = c.last_px;
            m.n = S.n;
            m.fpx = S.fpx;
            m.status = any_status;
            m.tmo = timed_out ? 1 : 0;
            m.nlev = nlev;
        }
        pair_sync(bar);
        const SplitSummary &mb_ = sx.sum[step & 1][0], &ma_ = sx.sum[step & 1][1];
        acc_merge(c, mb_.acc, ma_.acc, sx.base[SD]);
        c.last_px = ma_.lf_pos > mb_.lf_pos ? ma_.last_px : mb_.last_px;
        c.status = mb_.status | ma_.status;
        timed_out = (mb_.tmo | ma_.tmo) != 0;
        const int nb = mb_.n, na = ma_.n;
        const int nlb = mb_.nlev, nla = ma_.nlev;
        n_other = BID ? na : nb;
        // the background gained what the pair lost this step
        c.bg_cash = (long long)((u64)c.bg_cash - ((u64)c.cash0 + (u64)c.cash1 - pair_cash0));
        c.bg_inv = (long long)((u64)c.bg_inv - ((u64)c.inv0 + (u64)c.inv1 - pair_inv0));
        const long long step_base = (long long)step * p.n_envs + e;
        const long long obs_base = p.ow_obs ? (long long)e : step_base;
        const long long rew_base = p.ow_rew ? (long long)e : step_base;
        const long long done_base = p.ow_done ? (long long)e : step_base;
        if (A > 0) {
            const long long bb = nb ? (long long)mb_.fpx : c.last_px;
            const long long ba = na ? (long long)ma_.fpx : c.last_px;
            const long long s2 = bb + ba;
            const long long anchor = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
            const long long own0_all = mb_.own0 + ma_.own0, own1_all = mb_.own1 + ma_.own1;
            // Eq. 1: PV = Q_inv * P_ref + Cash, P_ref the liquidation touch
            const long long pref0 = c.inv0 > 0 ? bb : (c.inv0 < 0 ? ba : 0);
            const long long pref1 = c.inv1 > 0 ? bb : (c.inv1 < 0 ? ba : 0);
            const long long pv0 = (long long)((u64)c.inv0 * (u64)pref0 + (u64)c.cash0);
            const long long pv1 = (long long)((u64)c.inv1 * (u64)pref1 + (u64)c.cash1);
            const long long r0 = (long long)((u64)pv0 - (u64)c.pv0);
            const long long r1 = (long long)((u64)pv1 - (u64)c.pv1);
            c.pv0 = pv0; c.pv1 = pv1;
            if (BID) {
                const float tl = __fdiv_rn((float)(p.T - (t + 1)), (float)p.T);
                const int D = p.D;
                float *ob = p.obs ? p.obs + obs_base * A * D : nullptr;
                if (ob) {
                    for (int idx = lane; idx < 4 * L; idx += 32) {
                        const int sd = idx >= 2 * L ? 1 : 0;
                        const int i = (idx - sd * 2 * L) >> 1;
                        const long long lq = sm.lvl_q[sd][i];
                        const int nl = sd == 0 ? nlb : nla;
                        const long long lp = (long long)sm.lvl_px[sd][i] - anchor;
                        const float v = i >= nl ? 0.0f : __ll2float_rn((idx & 1) ? lq : lp);
                        ob[idx] = v;
                        ob[D + idx] = v;
                    }
                    if (lane < 10) {
                        const int a = lane >= 5 ? 1 : 0;
                        const int g = lane - 5 * a;
                        const long long iv = a == 0 ? c.inv0 : c.inv1;
                        const long long cs = a == 0 ? c.cash0 : c.cash1;
                        const long long rem = a == 0 ? (long long)p.exec_target - c.exec_done : 0;
                        const long long own = a == 0 ? own0_all : own1_all;
                        const long long x = g == 0 ? iv : g == 1 ? cs : g == 3 ? rem : own;
                        ob[a * D + 4 * L + g] = g == 2 ? tl : __ll2float_rn(x);
                    }
                }
                if (lane == 0) {
                    if (p.rew) { p.rew[rew_base * A] = r0; p.rew[rew_base * A + 1] = r1; }
                    if (p.act_out) { p.act_out[2LL * e] = act0; p.act_out[2LL * e + 1] = act1; }
                }
            }
        }
        if (BID && lane == 0) {
            if (p.done) p.done[done_base] = (unsigned char)(t + 1 == p.T);
            st->act[0] = act0;
            st->act[1] = act1;
        }
        if (step + 1 == p.n_steps && !timed_out) side_store<K, BID>(S, P, blk, lane);
        __syncwarp();
    }

    // ---- counters and env scalars (the bid warp)
    if (!BID) return;
    if (lane == 0) {
        if (c.status) atomicOr(p.status, c.status);
        cnt[0] = c.c_msgs; cnt[1] = c.c_agent; cnt[2] = c.c_fills; cnt[3] = c.c_fill_vol;
        cnt[4] = c.c_add_vol; cnt[5] = c.c_mkt_vol; cnt[6] = c.c_mkt_disc; cnt[7] = c.c_cancel_vol;
        cnt[8] = c.c_cancel_miss; cnt[9] = c.c_drop_vol; cnt[10] = c.c_drop_cnt; cnt[11] = c.c_evict_vol;
        cnt[12] = c.c_evict_cnt; cnt[13] = c.c_bad; cnt[14] = c.bg_cash; cnt[15] = c.bg_inv;
    }
    if (timed_out) return;
    if (lane == 0) {
        st->ts_next = c.ts_next; st->seq_next = c.seq_next;
        st->inv[0] = c.inv0; st->inv[1] = c.inv1; st->cash[0] = c.cash0; st->cash[1] = c.cash1;
        st->pv_prev[0] = c.pv0; st->pv_prev[1] = c.pv1; st->exec_done = c.exec_done;
        st->last_px = c.last_px;
        st->n[0] = S.n;
        st->n[1] = n_other;
        st->t = p.t0 + p.n_steps;
    }
}


// Two warps per env (even warp: bids, odd warp: asks), pairs of warps side by
// side in the block; each pair has its own named barrier.  128 registers: the
// register file is split between the SM's four schedulers, and 1,024 envs
// (2,048 warps) fit one wave only with four warps per scheduler.
template <int K>
__global__ void __maxnreg__(128) k_env_steps_split(const KParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pair = wib >> 1;
    const int npairs = blockDim.x >> 6;
    WarpSmem<K> &sm = reinterpret_cast<WarpSmem<K> *>(smem_raw)[pair];
    SplitSmem &sx = reinterpret_cast<SplitSmem *>(smem_raw + npairs * sizeof(WarpSmem<K>))[pair];
    if ((wib & 1) == 0 && lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        sx.prog[0] = 0;
        sx.prog[1] = 0;
    }
    __syncthreads();
    const int w = blockIdx.x * npairs + pair;
    if (w >= p.n_list) return;
    const int e = p.env_list ? p.env_list[w] : w;
    MsgPipe pipe{0u};
    if ((wib & 1) == 0) run_env_split<K, true>(p, e, sm, sx, pipe, lane, 1 + pair);
    else run_env_split<K, false>(p, e, sm, sx, pipe, lane, 1 + pair);
}

}  // namespace lobk
