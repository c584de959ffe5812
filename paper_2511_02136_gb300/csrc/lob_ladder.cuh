// lob_ladder.cuh -- price-ladder book primitives of the step kernel.
//
// The same price-time priority book as the slot pool + sorted index of
// lob_device.cuh (Sec. 2.1: best price first, FIFO by arrival within a price;
// trades at the resting order's price), kept in a form whose frequent
// operations need no insertion-position search and no index shift:
//
//   * each side's live prices span fewer than LW ticks, so a price p owns
//     level p mod LW of a circular ladder;
//   * each level is a FIFO of pool slots in arrival order -- a doubly linked
//     list in shared memory (head / tail per level, next / prev per slot) --
//     with the level's resting quantity and order count beside it;
//   * a bitmap of non-empty levels sits in warp-uniform registers, and the
//     front (best) order and the worst price are cached in them as well.
//
// Resting an order appends it at its level's tail, taking the front order
// pops a level head, evicting the worst order (capacity rule) unlinks the
// worst level's tail, and the top-L observation levels are the first L set
// bits of the bitmap with their stored sums.  Cancels find their order by a
// lane-parallel (price, id) compare over the pool, as in the sorted form.
//
// When an order would stretch a side's price span to LW ticks or more, the
// env converts both sides to the sorted-index form (the positions of every
// order in priority order are recovered by walking the levels) and the step
// continues there: results are the same either way.  Books are loaded from
// and stored to HBM in priority order, so every other kernel and the host
// see one layout.
#pragma once

namespace lobk {

constexpr int LW = 128;            // ladder levels per side (price window in ticks)
constexpr int LWW = LW / 32;       // 32-level passes over the ring
constexpr short LNIL = -1;

// Ladder arrays of one side.
template <int K>
struct __align__(16) LadSide {
    long long lqty[LW];            // resting quantity per level
    int lcnt[LW];                  // orders per level
    short head[LW], tail[LW];      // FIFO ends per level (slot numbers)
    short next[32 * K], prev[32 * K];   // FIFO links per slot
};

// Per-warp ladder block (after the block's WarpSmem array): both sides and a
// position -> slot table used by stores and by the conversion.
template <int K>
struct __align__(16) LadBlock {
    LadSide<K> s[2];
    unsigned short inv[32 * K];
};
static_assert(sizeof(LadBlock<1>) % 16 == 0 && sizeof(LadBlock<4>) % 16 == 0 && sizeof(LadBlock<8>) % 16 == 0,
              "ladder block keeps 16-byte alignment");

// Classes that run the ladder form (none at present: on the 1,024-env
// benchmark its linked-list pops put dependent shared-memory round trips on
// the taker's chain and measured slower than the sorted index; see the
// design notes).  The register-pool classes K <= 8 can take it.
template <int K>
__host__ __device__ constexpr bool ladder_class() { return false; }
template <int K>
__host__ __device__ constexpr size_t ladder_bytes() { return ladder_class<K>() ? sizeof(LadBlock<K>) : 0; }

// ---------------------------------------------------------------- bitmap
// The 128-level ring's bitmap is two 64-bit words (levels 0..63 in lo,
// 64..127 in hi) held in registers; every access picks a word with a select,
// so nothing is indexed at run time.
__device__ __forceinline__ bool bm_test(const Bm128 &b, int d) {
    const unsigned long long x = d < 64 ? b.lo : b.hi;
    return (x >> (d & 63)) & 1ull;
}
__device__ __forceinline__ void bm_set(Bm128 &b, int d) {
    const unsigned long long m = 1ull << (d & 63);
    b.lo |= d < 64 ? m : 0ull;
    b.hi |= d < 64 ? 0ull : m;
}
__device__ __forceinline__ void bm_clear(Bm128 &b, int d) {
    const unsigned long long m = 1ull << (d & 63);
    b.lo &= d < 64 ? ~m : ~0ull;
    b.hi &= d < 64 ? ~0ull : ~m;
}
// Nearest set bit at index d or below, wrapping around the ring (the bitmap
// must have one): this word at or below d, else the other word, else this
// word above d -- all three computed and selected, with no branch.
__device__ __forceinline__ int bm_scan_down(const Bm128 &b, int d) {
    const bool in_lo = d < 64;
    const int bit = d & 63, base = in_lo ? 0 : 64, obase = 64 - base;
    const unsigned long long x = in_lo ? b.lo : b.hi, o = in_lo ? b.hi : b.lo;
    const unsigned long long below = (2ull << bit) - 1ull;   // bits 0..bit (all for bit 63)
    const unsigned long long m = x & below;
    const int r1 = base + 63 - __clzll((long long)m);
    const int r2 = obase + 63 - __clzll((long long)o);
    const int r3 = base + 63 - __clzll((long long)(x & ~below));
    return m ? r1 : (o ? r2 : r3);
}
// Nearest set bit at index d or above, wrapping around the ring.
__device__ __forceinline__ int bm_scan_up(const Bm128 &b, int d) {
    const bool in_lo = d < 64;
    const int bit = d & 63, base = in_lo ? 0 : 64, obase = 64 - base;
    const unsigned long long x = in_lo ? b.lo : b.hi, o = in_lo ? b.hi : b.lo;
    const unsigned long long above = ~0ull << bit;
    const unsigned long long m = x & above;
    const int r1 = base + __ffsll((long long)m) - 1;
    const int r2 = obase + __ffsll((long long)o) - 1;
    const int r3 = base + __ffsll((long long)(x & ~above)) - 1;
    return m ? r1 : (o ? r2 : r3);
}
__device__ __forceinline__ int lvl_of(int px) { return (int)((unsigned)px & (unsigned)(LW - 1)); }

// The nearest non-empty price strictly worse (BID: lower) than px.
template <bool BID>
__device__ __forceinline__ int lad_worse(const Bm128 &bm, int px) {
    if constexpr (BID) {
        const int p1 = (int)((unsigned)px - 1u);
        const int d1 = lvl_of(p1);
        const int f = bm_scan_down(bm, d1);
        return (int)((unsigned)p1 - (unsigned)((d1 - f) & (LW - 1)));
    } else {
        const int p1 = (int)((unsigned)px + 1u);
        const int d1 = lvl_of(p1);
        const int f = bm_scan_up(bm, d1);
        return (int)((unsigned)p1 + (unsigned)((f - d1) & (LW - 1)));
    }
}
// The nearest non-empty price strictly better (BID: higher) than px.
template <bool BID>
__device__ __forceinline__ int lad_better(const Bm128 &bm, int px) {
    return lad_worse<!BID>(bm, px);
}

// ---------------------------------------------------------------- build (after a load)
// Builds one side's ladder from the pool loaded in priority order (slot q =
// position q, q < n).  Returns false, leaving the sorted-index form to the
// caller, when the side's prices span LW ticks or more.
template <int K, bool BID>
__device__ __forceinline__ bool lad_build(Side<K> &S, const PoolSmem<K> &P, LadSide<K> &D, int lane) {
    const int n = S.n;
    S.bm.lo = 0ull;
    S.bm.hi = 0ull;
    if (n == 0) return true;
    const int p0 = P.px[0], pl = P.px[n - 1];
    if ((BID ? (long long)p0 - pl : (long long)pl - p0) >= LW) return false;
    for (int i = lane; i < LW; i += 32) {
        D.lqty[i] = 0;
        D.lcnt[i] = 0;
    }
    __syncwarp();
    Bm128 m;
    m.lo = 0ull;
    m.hi = 0ull;
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;   // position = slot after a load
        if (q < n) {
            const int px = P.px[q];
            const int pp = q > 0 ? P.px[q - 1] : px;
            const int pn = q + 1 < n ? P.px[q + 1] : px;
            const bool first = q == 0 || pp != px, last = q + 1 == n || pn != px;
            const int d = lvl_of(px);
            D.prev[q] = first ? LNIL : (short)(q - 1);
            D.next[q] = last ? LNIL : (short)(q + 1);
            if (first) D.head[d] = (short)q;
            if (last) D.tail[d] = (short)q;
            atomicAdd(reinterpret_cast<unsigned long long *>(&D.lqty[d]), (unsigned long long)(long long)P.qty[q]);
            atomicAdd(&D.lcnt[d], 1);
            bm_set(m, d);
        }
    }
    S.bm.lo = ((unsigned long long)__reduce_or_sync(FULL, (unsigned)(m.lo >> 32)) << 32) |
              __reduce_or_sync(FULL, (unsigned)m.lo);
    S.bm.hi = ((unsigned long long)__reduce_or_sync(FULL, (unsigned)(m.hi >> 32)) << 32) |
              __reduce_or_sync(FULL, (unsigned)m.hi);
    S.wpx = pl;
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------- front refresh
// The front order is the head of the front level at price S.fpx.
template <int K>
__device__ __forceinline__ void lad_front_from(Side<K> &S, const PoolSmem<K> &P, const LadSide<K> &D) {
    const int s = D.head[lvl_of(S.fpx)];
    S.fslot = s;
    S.fqty = P.qty[s];
    S.fid = P.id[s];
}

// ---------------------------------------------------------------- remove
// Remove occupied slot s (any position) from its level and the pool, moving
// the cached front and worst price as needed.
template <int K, bool BID>
__device__ __forceinline__ void lad_remove(Side<K> &S, const PoolSmem<K> &P, LadSide<K> &D, int s, int lane) {
    const int px = P.px[s];
    const int d = lvl_of(px);
    const int q = P.qty[s];
    const int pv = D.prev[s], nx = D.next[s];
    const long long lq = D.lqty[d];
    const int lc = D.lcnt[d];
    __syncwarp();   // every lane has read before any lane writes
    D.lqty[d] = lq - q;
    D.lcnt[d] = lc - 1;
    if (pv == LNIL) D.head[d] = (short)nx;
    else D.next[pv] = (short)nx;
    if (nx == LNIL) D.tail[d] = (short)pv;
    else D.prev[nx] = (short)pv;
    slot_clear<K>(S, s, lane);
    S.n--;
    __syncwarp();
    if (pv == LNIL && nx == LNIL) {   // the level is empty now
        bm_clear(S.bm, d);
        if (S.n > 0) {
            if (px == S.fpx) {
                S.fpx = lad_worse<BID>(S.bm, px);
                lad_front_from<K>(S, P, D);
            } else if (px == S.wpx) {
                S.wpx = lad_better<BID>(S.bm, px);
            }
        }
    } else if (s == S.fslot) {        // the front order left a non-empty level: its successor leads
        S.fslot = nx;
        S.fqty = P.qty[nx];
        S.fid = P.id[nx];
    }
}

// ---------------------------------------------------------------- take
// Take liquidity from resting side O (RBID: O holds bids), price first then
// time, up to the limit (if any); returns the unfilled quantity.
template <int K, bool RBID, bool TRACE, bool MA>
__device__ __forceinline__ int lad_take(Side<K> &O, PoolSmem<K> &P, LadSide<K> &D, bool has_limit, int limit, int q,
                                        long long taker_id, int taker_side, Ctx &c, int lane) {
    while (q > 0 && O.n > 0 && (!has_limit || at_least<RBID>(O.fpx, limit))) {
        const int s = O.fslot;
        const int fq = O.fqty;
        const int d = lvl_of(O.fpx);
        const int nx = D.next[s];            // fetched before we know whether it is needed
        const long long lq = D.lqty[d];
        const int lc = D.lcnt[d];
        const int f = min(q, fq);
        do_fill<TRACE, MA>(c, O.fpx, f, O.fid, taker_id, taker_side, lane);
        q -= f;
        __syncwarp();                         // every lane has read before any lane writes
        D.lqty[d] = lq - f;
        if (f == fq) {                        // the front order is gone
            D.lcnt[d] = lc - 1;
            slot_clear<K>(O, s, lane);
            O.n--;
            if (nx != LNIL) {
                D.head[d] = (short)nx;
                D.prev[nx] = LNIL;
                __syncwarp();
                O.fslot = nx;
                O.fqty = P.qty[nx];
                O.fid = P.id[nx];
            } else {
                bm_clear(O.bm, d);
                __syncwarp();
                if (O.n > 0) {
                    O.fpx = lad_worse<RBID>(O.bm, O.fpx);
                    lad_front_from<K>(O, P, D);
                }
            }
        } else {
            O.fqty = fq - f;
            P.qty[s] = fq - f;                // every lane stores the same value
            __syncwarp();
        }
    }
    return q;
}

// ---------------------------------------------------------------- rest
// Whether an order at price p may rest on side S without stretching the
// side's price span to LW ticks or more (checked against the current worst,
// so conservative when the order would evict or be dropped).
template <int K, bool BID>
__device__ __forceinline__ bool lad_fits(const Side<K> &S, int p) {
    const int best = BID ? max(S.fpx, p) : min(S.fpx, p);
    const int worst = BID ? min(S.wpx, p) : max(S.wpx, p);
    const unsigned span = BID ? (unsigned)best - (unsigned)worst : (unsigned)worst - (unsigned)best;
    return S.n == 0 || span < (unsigned)LW;
}

// Rest an order on its own side with the capacity rule (reading 6: on a full
// side an order strictly better than the worst price evicts the worst-priced,
// latest-arrived order; otherwise it is dropped).  The price must fit the
// ladder (lad_fits).
template <int K, bool BID>
__device__ __forceinline__ void lad_rest(Side<K> &S, PoolSmem<K> &P, LadSide<K> &D, int cap, int p, int q,
                                         long long oid, Ctx &c, int lane) {
    const bool full = S.n >= cap;
    if (full && !(BID ? p > S.wpx : p < S.wpx)) {   // not strictly better than the worst: dropped
        c.c_drop_vol += q;
        c.c_drop_cnt += 1;
        return;
    }
    int f;
    if (full) {   // evict the tail of the worst level and reuse its slot
        const int v = D.tail[lvl_of(S.wpx)];
        c.c_evict_vol += P.qty[v];
        c.c_evict_cnt += 1;
        lad_remove<K, BID>(S, P, D, v, lane);
        f = v;
    } else {
        const unsigned fr = ~S.occ & Side<K>::KMASK;
        const unsigned flanes = __ballot_sync(FULL, fr != 0);
        f = __shfl_sync(FULL, slot_of<K>(lane, 31 - __clz(fr)), 31 - __clz(flanes));
    }
    const int fl = slot_lane<K>(f), fr_ = slot_r<K>(f);
    if (lane == fl) S.occ |= 1u << fr_;
    if constexpr (Side<K>::REG) {
#pragma unroll
        for (int r = 0; r < K; r++)
            if (lane == fl && r == fr_) { S.px[r] = p; S.id[r] = oid; }
    }
    const int d = lvl_of(p);
    const bool had = bm_test(S.bm, d);
    const int t = D.tail[d];
    const long long lq = had ? D.lqty[d] : 0;
    const int lc = had ? D.lcnt[d] : 0;
    __syncwarp();
    P.px[f] = p; P.qty[f] = q; P.id[f] = oid; P.ts[f] = c.ts_next;   // same value from every lane
    if (had) D.next[t] = (short)f;
    else D.head[d] = (short)f;
    D.prev[f] = had ? (short)t : LNIL;
    D.next[f] = LNIL;
    D.tail[d] = (short)f;
    D.lqty[d] = lq + q;
    D.lcnt[d] = lc + 1;
    __syncwarp();
    bm_set(S.bm, d);
    c.ts_next += 1;
    if (S.n == 0) {
        S.fpx = p; S.fqty = q; S.fid = oid; S.fslot = f;
        S.wpx = p;
    } else {
        if (BID ? p > S.fpx : p < S.fpx) { S.fpx = p; S.fqty = q; S.fid = oid; S.fslot = f; }
        if (BID ? p < S.wpx : p > S.wpx) S.wpx = p;
    }
    S.n++;
}

// ---------------------------------------------------------------- cancel
// Repeated (price, id) matches (this lane's slots in m): the slot of the
// match that arrived first (smallest stamp).  Out of line: ids repeat only in
// unusual streams.
template <int K>
__device__ __noinline__ int lad_dup_slot(const long long *ts, unsigned m, int lane) {
    long long bts = 0x7fffffffffffffffLL;
    int bs = -1;
    for (int r = 0; r < K; r++)
        if ((m >> r) & 1u) {
            const int sl = slot_of<K>(lane, r);
            if (ts[sl] < bts) { bts = ts[sl]; bs = sl; }
        }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const long long ots = __shfl_xor_sync(FULL, bts, o);
        const int os = __shfl_xor_sync(FULL, bs, o);
        if (ots < bts || (ots == bts && os >= 0 && (bs < 0 || os < bs))) { bts = ots; bs = os; }
    }
    return bs;
}

// Partial cancel or delete: lookup by (price, id) over the pool; a miss is a
// no-op; with repeated ids the earliest-arrived match is hit.
template <int K, bool BID>
__device__ __forceinline__ void lad_cancel(Side<K> &S, PoolSmem<K> &P, LadSide<K> &D, int type, int p, int qty,
                                           long long oid, Ctx &c, int lane) {
    unsigned m = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++)
        if (((S.occ >> r) & 1u) && spx<K>(S, P, r, lane) == p && sid<K>(S, P, r, lane) == oid) m |= 1u << r;
    const unsigned lanes = __ballot_sync(FULL, m != 0);
    if (lanes == 0) {
        c.c_cancel_miss += 1;
        return;
    }
    int s;
    if (__popc(lanes) == 1 && __ballot_sync(FULL, __popc(m) > 1) == 0) {
        const int L = 31 - __clz(lanes);
        s = __shfl_sync(FULL, slot_of<K>(lane, 31 - __clz(m)), L);
    } else {
        s = lad_dup_slot<K>(P.ts, m, lane);
    }
    s = LOB_CHK(s, 32 * K, c.status);
    const int q0 = P.qty[s];
    const int cut = type == LOB_PARTIAL ? min(qty, q0) : q0;
    c.c_cancel_vol += cut;
    if (q0 - cut == 0) {
        lad_remove<K, BID>(S, P, D, s, lane);
    } else {
        const int d = lvl_of(p);
        const long long lq = D.lqty[d];
        __syncwarp();
        P.qty[s] = q0 - cut;   // same value from every lane
        D.lqty[d] = lq - cut;
        __syncwarp();
        if (s == S.fslot) S.fqty = q0 - cut;
    }
}

// Delete the flagged agent orders of one side (carry-over cancels; the final
// book does not depend on their order); one agent message per cancel.
template <int K, bool BID>
__device__ __forceinline__ void lad_cancel_set(Side<K> &S, PoolSmem<K> &P, LadSide<K> &D, unsigned cmask, Ctx &c,
                                               int lane) {
    unsigned vol = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++)
        if ((cmask >> r) & 1u) vol += (unsigned)P.qty[slot_of<K>(lane, r)];
    const int ncan = (int)__reduce_add_sync(FULL, (unsigned)__popc(cmask));
    if (ncan == 0) return;
    c.c_cancel_vol += (long long)__reduce_add_sync(FULL, vol);
    c.c_msgs += ncan;
    c.c_agent += ncan;
    c.msg_idx += ncan;
    for (;;) {
        const unsigned lanes = __ballot_sync(FULL, cmask != 0);
        if (lanes == 0) break;
        const int L = __ffs(lanes) - 1;
        const int s = __shfl_sync(FULL, slot_of<K>(lane, __ffs(cmask) - 1), L);
        if (lane == L) cmask &= cmask - 1;
        lad_remove<K, BID>(S, P, D, s, lane);
    }
}

// ---------------------------------------------------------------- positions
// The pool slot of every position 0..n-1 in priority order, written to inv:
// lanes take the levels at offsets 0..31, 32..63, ... from the front, place
// each level by an exclusive scan of the level counts, and walk its FIFO.
template <int K, bool BID>
__device__ __forceinline__ void lad_positions(const Side<K> &S, const LadSide<K> &D, unsigned short *inv, int lane) {
    const int n = S.n;
    int st = 0;   // checked build: a link out of range is clamped (the book check then fails)
    (void)st;
    int base = 0;
#pragma unroll 1
    for (int pass = 0; pass < LWW && base < n; pass++) {
        const int off = pass * 32 + lane;
        const int price = BID ? (int)((unsigned)S.fpx - (unsigned)off) : (int)((unsigned)S.fpx + (unsigned)off);
        const int d = lvl_of(price);
        const bool ne = bm_test(S.bm, d);
        const int cnt = ne ? D.lcnt[d] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (ne) {
            int pos = base + incl - cnt;
            int s = D.head[d];
            for (int k = 0; k < cnt && pos < 32 * K; k++, pos++) {
                s = LOB_CHK(s, 32 * K, st);
                inv[pos] = (unsigned short)s;
                if (k + 1 < cnt) s = D.next[s];
            }
        }
        base += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
}

// Store one side in priority order from the ladder (positions from
// lad_positions), with the vector stores of side_store.
template <int K, bool BID>
__device__ __forceinline__ void lad_store(const Side<K> &S, const PoolSmem<K> &P, const LadSide<K> &D,
                                          unsigned short *inv, unsigned char *blk, int lane) {
    lad_positions<K, BID>(S, D, inv, lane);
    constexpr int SL = 32 * K;
    const int sd = BID ? 0 : 1;
    int *gpx = reinterpret_cast<int *>(blk) + sd * SL + lane * K;
    int *gqt = reinterpret_cast<int *>(blk) + 2 * SL + sd * SL + lane * K;
    long long *gid = reinterpret_cast<long long *>(blk + 16 * SL) + sd * SL + lane * K;
    long long *gts = reinterpret_cast<long long *>(blk + 32 * SL) + sd * SL + lane * K;
    constexpr int G = K < 4 ? K : 4;
#pragma unroll
    for (int g = 0; g < K; g += G) {
        if (lane * K + g >= S.n) break;
        int px[G], qt[G];
        long long id[G], ts[G];
#pragma unroll
        for (int u = 0; u < G; u++) {
            // positions >= n of a vector group were not written by the walk:
            // store slot 0's values there (never read back)
            const int q = lane * K + g + u;
            const int s = q < S.n ? (int)inv[q] : 0;
            px[u] = P.px[s]; qt[u] = P.qty[s]; id[u] = P.id[s]; ts[u] = P.ts[s];
        }
        if constexpr (G == 4) {
            *reinterpret_cast<int4 *>(gpx + g) = make_int4(px[0], px[1], px[2], px[3]);
            *reinterpret_cast<int4 *>(gqt + g) = make_int4(qt[0], qt[1], qt[2], qt[3]);
            *reinterpret_cast<longlong2 *>(gid + g) = make_longlong2(id[0], id[1]);
            *reinterpret_cast<longlong2 *>(gid + g + 2) = make_longlong2(id[2], id[3]);
            *reinterpret_cast<longlong2 *>(gts + g) = make_longlong2(ts[0], ts[1]);
            *reinterpret_cast<longlong2 *>(gts + g + 2) = make_longlong2(ts[2], ts[3]);
        } else {
#pragma unroll
            for (int u = 0; u < G; u++) { gpx[g + u] = px[u]; gqt[g + u] = qt[u]; gid[g + u] = id[u]; gts[g + u] = ts[u]; }
        }
    }
    __syncwarp();
}

// Conversion to the sorted-index form: the index entries of this lane's
// positions from the ladder's priority order (the pool, occupancy and front
// cache are shared by both forms).
template <int K, bool BID>
__device__ __forceinline__ void lad_to_index(Side<K> &S, const LadSide<K> &D, unsigned short *inv, int lane) {
    lad_positions<K, BID>(S, D, inv, lane);
#pragma unroll
    for (int w = 0; w < Side<K>::NW; w++) {
        unsigned v = 0;
#pragma unroll
        for (int b = 0; b < Side<K>::BPW; b++) {
            const int q = lane * K + Side<K>::EPW * w + b;
            const unsigned e = q < S.n ? (unsigned)inv[q] : 0u;
            v |= (e & Side<K>::EMASK) << (Side<K>::IXB * b);
        }
        S.ix[w] = v;
    }
    // positions >= n hold the free slots, as the sorted form expects: any order
    // of them will do, so they are listed after the live ones by slot number
    const unsigned fr = ~S.occ & Side<K>::KMASK;
    int before = 0;
    {
        int cnt = __popc(fr), incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        before = incl - cnt;
    }
    __syncwarp();
    {
        unsigned f = fr;
        int k = 0;
        while (f) {
            const int r = __ffs(f) - 1;
            f &= f - 1;
            if (S.n + before + k < 32 * K) inv[S.n + before + k] = (unsigned short)slot_of<K>(lane, r);
            k++;
        }
    }
    __syncwarp();
#pragma unroll
    for (int w = 0; w < Side<K>::NW; w++) {
        unsigned v = S.ix[w];
#pragma unroll
        for (int b = 0; b < Side<K>::BPW; b++) {
            const int q = lane * K + Side<K>::EPW * w + b;
            if (q >= S.n && q < 32 * K) {
                const unsigned e = (unsigned)inv[q];
                v = (v & ~(Side<K>::EMASK << (Side<K>::IXB * b))) | ((e & Side<K>::EMASK) << (Side<K>::IXB * b));
            }
        }
        S.ix[w] = v;
    }
    __syncwarp();
}

// ---------------------------------------------------------------- observation levels
// Aggregated top-L levels of one side straight from the ladder (level sums
// are kept per level), plus each agent's resting quantity on this side from
// a scan of the pool.  Returns the level count.
template <int K, bool BID>
__device__ __forceinline__ int lad_levels(const Side<K> &S, const PoolSmem<K> &P, const LadSide<K> &D, int L,
                                          int *lvl_px, long long *lvl_q, long long &own0, long long &own1, int lane) {
    long long o0 = 0, o1 = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++) {
        const long long id = sid<K>(S, P, r, lane);
        if (((S.occ >> r) & 1u) && id < 0) {
            const int qt = P.qty[slot_of<K>(lane, r)];
            if ((~id) & 1) o1 += qt; else o0 += qt;
        }
    }
    own0 += warp_sum(o0);
    own1 += warp_sum(o1);
    int found = 0;
    if (S.n > 0) {
#pragma unroll 1
        for (int pass = 0; pass < LWW && found < L; pass++) {
            const int off = pass * 32 + lane;
            const int price = BID ? (int)((unsigned)S.fpx - (unsigned)off) : (int)((unsigned)S.fpx + (unsigned)off);
            const int d = lvl_of(price);
            const bool ne = bm_test(S.bm, d);
            const unsigned b = __ballot_sync(FULL, ne);
            const int idx = found + __popc(b & ((1u << lane) - 1u));
            if (ne && idx < L) {
                lvl_px[idx] = price;
                lvl_q[idx] = D.lqty[d];
            }
            found += __popc(b);
        }
    }
    __syncwarp();
    return found < L ? found : L;
}

#ifdef LOB_CHECKED
// Checked build: the ladder's invariants after a step -- the positions walked
// from the levels name n distinct occupied slots in strict price-time
// priority with positive quantities, the level sums match, and the cached
// front and worst price agree.  Warp-uniform result.
template <int K, bool BID>
__device__ bool lad_ok(const Side<K> &S, const PoolSmem<K> &P, const LadSide<K> &D, unsigned short *inv, int cap,
                       int lane) {
    const int n = S.n;
    const int occ_n = (int)__reduce_add_sync(FULL, (unsigned)__popc(S.occ & Side<K>::KMASK));
    bool ok = n >= 0 && n <= cap && occ_n == n;
    if (!__all_sync(FULL, ok)) return false;
    lad_positions<K, BID>(S, D, inv, lane);
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;
        if (q < n) {
            const int s = inv[q];
            const bool in_range = s < 32 * K;
            const int ss = in_range ? s : 0;
            ok = ok && in_range && P.qty[ss] > 0;
            if (q > 0 && in_range) {
                const int sp = inv[q - 1] < 32 * K ? inv[q - 1] : 0;
                const bool order = BID ? (P.px[sp] > P.px[ss] || (P.px[sp] == P.px[ss] && P.ts[sp] < P.ts[ss]))
                                       : (P.px[sp] < P.px[ss] || (P.px[sp] == P.px[ss] && P.ts[sp] < P.ts[ss]));
                ok = ok && order;
            }
        }
    }
    if (n > 0) {
        const int f = inv[0] < 32 * K ? inv[0] : 0;
        const int w = inv[n - 1] < 32 * K ? inv[n - 1] : 0;
        ok = ok && f == S.fslot && P.px[f] == S.fpx && P.qty[f] == S.fqty && P.id[f] == S.fid && P.px[w] == S.wpx;
    }
    return __all_sync(FULL, ok);
}
#endif

}  // namespace lobk
