// lob_device.cuh -- sm_103a kernels of the batched limit-order-book env step.
//
// One warp runs one environment.  Each side of the book is a POOL of S = 32*K
// order slots plus a priority INDEX:
//   * pool slot s belongs to lane s / K (register r = s % K); that lane keeps
//     the slot's price and id in registers so that "how many resting orders
//     rank ahead of price p" and "which slot holds (price, id)" are one
//     compare per register plus one warp reduction / ballot;
//   * every slot's price, size, id and arrival stamp are also in shared memory
//     (written once when the order comes to rest);
//   * the index lists slot numbers in priority order (best price first, then
//     arrival), one byte per position, positions lane*K .. lane*K+K-1 packed
//     four to a 32-bit register of that lane.  Resting an order or removing
//     one shifts only these bytes: one neighbour-lane shuffle and a few
//     byte-mask operations, whatever the number of fields per order;
//   * the front order (position 0) is cached in warp-uniform registers.
// Messages are staged into shared memory 32 records at a time by
// cp.async.bulk (TMA bulk copy) completing on an mbarrier, and the next record
// is always read one message ahead.
//
// The stages follow the environment step of JaxMARL-HFT Sec. 4: action
// conversion with carry-over cancels, random shuffle of the agents' orders,
// concatenation (cancels, agent orders, market-replay messages), price-time
// matching (Sec. 2.1) and the step outcomes (observation, Eq. 1 portfolio-
// value reward, termination flag).
#pragma once
#include <cstddef>
#include <cstdint>
#include "lob.h"

namespace lobk {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TILE = 32;        // messages per staged tile in the per-warp block (the default)
constexpr int TILE_MAX = 64;    // the largest staged tile (its buffers then follow the per-warp blocks)
constexpr int LMAX = 64;        // max observation levels per side
constexpr int SMAX = 256;       // max pool slots per side (byte-wide index)
constexpr int ST_BADMSG = 1, ST_BADACT = 2, ST_TIMEOUT = 4, ST_CHECK = 8;

// Checked build (-DLOB_CHECKED, compute-sanitizer being unavailable): every
// slot number and position taken from the priority index is bounds-checked
// before it addresses shared memory, and each step ends with a check of both
// books' invariants; a violation records ST_CHECK (the index is clamped into
// range) instead of faulting.  The regular build compiles none of it.
#ifdef LOB_CHECKED
__device__ __forceinline__ int lob_chk(int x, int hi, int &st) {
    if ((unsigned)x < (unsigned)hi) return x;
    st |= ST_CHECK;
    return 0;
}
#define LOB_CHK(x, hi, st) lob_chk((x), (hi), (st))
#else
#define LOB_CHK(x, hi, st) (x)
#endif

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
    int ep_start;          // episode mode: first data step of the current episode
    int exec_dir;          // the execution task's side in this episode (drawn when configured 0)
    int pad[6];
};
static_assert(sizeof(EnvState) == 128, "env state");

// Several agents per type (Sec. 3, Table 1): per-agent state in HBM, one
// record per (env, agent), agents 0..P-1 executing and P..2P-1 market making.
constexpr int AMAX = 2 * LOB_MAX_PER_TYPE;
struct __align__(16) AgentState {
    long long inv, cash, pv_prev, exec_done;
    int act;
    int pad[3];
};
static_assert(sizeof(AgentState) == 48, "agent state");

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
    const int *env_list;   // NULL: env = list position (identity)
    int n_list;
    int *queue;
    long long wait_budget;      // bound of a wait on a message tile (SM cycles)
    long long drain_budget;     // bound of the wait for a copy in flight after a timeout
    int hold_first;             // test hook: the launch's first tile per env is never requested
    int book_prefetch;          // one-wave launches: each env's book block is requested into L2 at entry
    // uniform layout: when uni_cap > 0 every env has capacity uni_cap and its
    // book block at env * uni_block; book_off / caps are not read
    int uni_cap;
    long long uni_block;
    long long exec_q0;     // max(1, ceil(exec_target / T)), computed on the host
    int reward_mode, lam_pct;        // market maker's reward (Eq. 1, 4 or 3), lambda in percent
    long long inv_penalty;           // rho of the quadratic inventory penalty
    long long exec_pen_milli;        // unfilled-task penalty, thousandths of a tick per unit
    int mm_space;                    // market maker's action space (Sec. 4.1.1)
    int pv_ref;                      // P_ref of Eq. 1: liquidation touch, or mid (PV in half ticks)
    // episode mode (one shared stream; offsets index data steps): start table,
    // prebuilt book images (ep_block bytes each) and first observations
    int ep_mode;
    int n_starts;
    long long ep_block;
    const lob_start *ep_starts;
    const unsigned char *ep_images;
    const float *ep_obs;
    AgentState *agents;              // several agents per type: [n_envs][n_agents]
    int msgs_sysmem;                 // messages (and offsets) in page-locked host memory
    int msg16;                       // background messages are 16-byte compact records
    int tile;                        // records per staged tile the launch was sized for (0 = TILE)
    int ow_obs, ow_rew, ow_done;     // that output overwrites env e's slot every step (else one slot per step)
    int *act_steps;                  // fused rollout: the actions taken at each step [n_steps][n_envs][2], or NULL
    const float *obs_in;             // fused rollout: every env's current observation [n_envs][2][D]
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
// 16-byte asynchronous copies global -> shared through the SM's load path
// (any address the GPU maps, including page-locked host memory read over the
// coherent CPU-GPU link), completed per thread by a commit group.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
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
// The execution task's side of an env in episode k when it is drawn (Table 2:
// uniformly sampled): the top bit of a keyed SplitMix64 draw, set -> sell.
constexpr unsigned long long TAG_TASKDIR = 0x5441534B44495204ull;
__device__ __forceinline__ int drawn_task_side(unsigned long long seed, long long k);
__device__ __forceinline__ unsigned bounded(unsigned long long x, unsigned n) {
    return (unsigned)(((unsigned long long)(unsigned)(x >> 32) * n) >> 32);
}
__device__ __forceinline__ int drawn_task_side(unsigned long long seed, long long k) {
    return (sm_mix(step_key(seed, k, TAG_TASKDIR) + GAMMA) >> 63) ? LOB_SELL : LOB_BUY;
}

// ---------------------------------------------------------------- shared memory
// Pool copies of one side (slot-indexed), S = 32*K slots.
template <int K>
struct PoolSmem {
    long long id[32 * K];
    long long ts[32 * K];
    int px[32 * K];
    int qty[32 * K];
};

// Per-warp shared memory.  Warps index an array of these, so the size is a
// multiple of 16 bytes: each warp's message tiles stay on the 16-byte boundary
// that bulk copies need.
template <int K>
struct __align__(16) WarpSmem {
    DevMsg tile[2][TILE];
    DevMsg amsg[4];                // the step's agent orders, after the shuffle
    unsigned long long bar[2];
    PoolSmem<K> pool[2];           // 0 = bids, 1 = asks
    long long lvl_q[2][LMAX];
    int lvl_px[2][LMAX];
    unsigned char cand[2][32 * K]; // carry-over cancel flags per slot
    long long rw[3];               // step start: twice the mid, MM inventory, MM cash (lane 0)
};
static_assert(sizeof(WarpSmem<1>) % 16 == 0 && sizeof(WarpSmem<2>) % 16 == 0 && sizeof(WarpSmem<4>) % 16 == 0 &&
                  sizeof(WarpSmem<8>) % 16 == 0 && sizeof(WarpSmem<16>) % 16 == 0 && sizeof(WarpSmem<32>) % 16 == 0,
              "per-warp shared memory must keep 16-byte alignment across warps");
static_assert(offsetof(WarpSmem<1>, tile) == 0 && offsetof(WarpSmem<32>, tile) == 0, "tiles lead the block");

// Per-warp agent block of the several-agents kernel, after the WarpSmem
// array: the step's agent orders (3 per agent pair at most, plus the record
// read ahead), the agents' running state and the step's wanted orders.
constexpr int AMSG_MA = 3 * LOB_MAX_PER_TYPE + 1;
// the message loop keeps a chunk's dispatch indices in the carry-over flags'
// space: a tile or the agents' orders, plus the one-ahead read
static_assert(sizeof(WarpSmem<1>::cand) >= AMSG_MA + 1 && sizeof(WarpSmem<1>::cand) >= TILE_MAX,
              "dispatch indices fit the carry-over flags");
static_assert(offsetof(WarpSmem<1>, rw) == offsetof(WarpSmem<1>, cand) + sizeof(WarpSmem<1>::cand),
              "the dispatch index read one past a full tile stays in the warp's block");
struct __align__(16) AgentSmem {
    DevMsg amsg[AMSG_MA];
    long long inv[AMAX], cash[AMAX], pv[AMAX], done[AMAX];
    long long inv0[AMAX], cash0[AMAX];   // at the start of the step (reward variants)
    long long own[AMAX];                 // resting quantity (observation)
    long long kept[AMAX][2];             // carried-over quantity per wanted order
    int want_px[AMAX][2], want_q[AMAX][2];   // [agent][0 bid, 1 ask]; q 0 = none
    int act[AMAX];
};
static_assert(sizeof(AgentSmem) % 16 == 0, "agent block keeps 16-byte alignment");

// A 128-bit bitmap as two words (the price ladder's non-empty levels).
struct Bm128 {
    unsigned long long lo, hi;
};

// ---------------------------------------------------------------- book side
// Pool slot s of a side belongs to one lane, which scans it in its register
// index r:  K <= 8: s = lane*K + r, with the slot's price and id kept in
// registers;  K >= 16: s = r*32 + lane, price and id read from shared memory
// (consecutive lanes -> consecutive banks).  Index entries (slot numbers) are
// 8 bits wide for pools of up to 256 slots, 16 bits beyond.
template <int K>
struct Side {
    static constexpr bool REG = K <= 8;
    static constexpr int IXB = K <= 8 ? 8 : 16;           // bits per index entry
    static constexpr int EPW = 32 / IXB;                  // entries per 32-bit word
    static constexpr int NW = (K + EPW - 1) / EPW;        // index words per lane
    static constexpr int BPW = K < EPW ? K : EPW;         // entries used per word
    static constexpr unsigned EMASK = (1u << IXB) - 1u;
    static constexpr unsigned ALLB = BPW * IXB == 32 ? 0xffffffffu : ((1u << (BPW * IXB)) - 1u);
    static constexpr unsigned REP = IXB == 8 ? 0x01010101u : 0x00010001u;
    static constexpr unsigned KMASK = K == 32 ? 0xffffffffu : ((1u << K) - 1u);
    static constexpr int RK = REG ? K : 1;
    // unroll factor of loops over a lane's slots that touch no register array:
    // for the largest books partial unrolling keeps the kernel's code small
    // (instruction fetch bounds that class); smaller ones unroll fully
    static constexpr int SU = K >= 32 ? 4 : K;
    int px[RK];         // price of slot (lane, r) (registers mode only)
    long long id[RK];   // id of slot (lane, r) (registers mode only)
    unsigned occ;       // occupied slots of this lane (bit r)
    unsigned ix[NW];    // index entries for positions lane*K .. lane*K+K-1
    int n;              // live orders (warp-uniform)
    int fpx, fqty, fslot;  // front order (position 0), valid when n > 0
    long long fid;
    // price-ladder form (lob_ladder.cuh): bitmap of non-empty levels and the
    // worst resting price, warp-uniform, valid when n > 0
    Bm128 bm;
    int wpx;
};

template <int K> __device__ __forceinline__ int slot_of(int lane, int r) {
    return Side<K>::REG ? lane * K + r : r * 32 + lane;
}
template <int K> __device__ __forceinline__ int slot_lane(int s) { return Side<K>::REG ? s / K : (s & 31); }
template <int K> __device__ __forceinline__ int slot_r(int s) { return Side<K>::REG ? s % K : (s >> 5); }
template <int K>
__device__ __forceinline__ int spx(const Side<K> &S, const PoolSmem<K> &P, int r, int lane) {
    if constexpr (Side<K>::REG) return S.px[r];
    else return P.px[r * 32 + lane];
}
template <int K>
__device__ __forceinline__ long long sid(const Side<K> &S, const PoolSmem<K> &P, int r, int lane) {
    if constexpr (Side<K>::REG) return S.id[r];
    else return P.id[r * 32 + lane];
}

template <bool BID>
__device__ __forceinline__ bool at_least(int a, int p) { return BID ? a >= p : a <= p; }

// Index entry (slot number) at local position j of this lane.
template <int K>
__device__ __forceinline__ int ix_ent(const Side<K> &S, int j) {
    constexpr int EPW = Side<K>::EPW, IXB = Side<K>::IXB;
    return (S.ix[j / EPW] >> (IXB * (j % EPW))) & Side<K>::EMASK;
}

// Slot number at uniform position q (q < 32*K).
template <int K>
__device__ __forceinline__ int slot_at(const Side<K> &S, int q) {
    constexpr int EPW = Side<K>::EPW, IXB = Side<K>::IXB;
    const int j = q % K;
    unsigned w = S.ix[0];
#pragma unroll
    for (int i = 1; i < Side<K>::NW; i++)
        if (j / EPW == i) w = S.ix[i];
    w = __shfl_sync(FULL, w, q / K);
    return (w >> (IXB * (j % EPW))) & Side<K>::EMASK;
}

// Per-word mask of the entries at positions below `lim` (positions of word w
// of this lane start at lane*K + EPW*w).
template <int K>
__device__ __forceinline__ unsigned ix_below(int lim, int lane, int w) {
    constexpr int BPW = Side<K>::BPW, IXB = Side<K>::IXB;
    const int d = lim - (lane * K + Side<K>::EPW * w);
    return d <= 0 ? 0u : (d >= BPW ? Side<K>::ALLB : ((1u << (IXB * d)) - 1u));
}

// Remove position q; positions > q move down by one.
template <int K>
__device__ __forceinline__ void ix_remove(Side<K> &S, int q, int lane) {
    constexpr int NW = Side<K>::NW, BPW = Side<K>::BPW, IXB = Side<K>::IXB;
    constexpr unsigned ALLB = Side<K>::ALLB, EMASK = Side<K>::EMASK;
    const unsigned nxt = __shfl_down_sync(FULL, S.ix[0] & EMASK, 1);
    unsigned shifted[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const unsigned in = w + 1 < NW ? (S.ix[w + 1] & EMASK) : nxt;
        shifted[w] = ((S.ix[w] >> IXB) | (in << (IXB * (BPW - 1)))) & ALLB;
    }
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const unsigned keep = ix_below<K>(q, lane, w);
        S.ix[w] = (S.ix[w] & keep) | (shifted[w] & ~keep);
    }
}

// The index words after removing position q, without modifying the side.
template <int K>
__device__ __forceinline__ void ix_removed(const Side<K> &S, int q, int lane, unsigned (&out)[Side<K>::NW]) {
    constexpr int NW = Side<K>::NW, BPW = Side<K>::BPW, IXB = Side<K>::IXB;
    constexpr unsigned ALLB = Side<K>::ALLB, EMASK = Side<K>::EMASK;
    const unsigned nxt = __shfl_down_sync(FULL, S.ix[0] & EMASK, 1);
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const unsigned in = w + 1 < NW ? (S.ix[w + 1] & EMASK) : nxt;
        const unsigned shifted = ((S.ix[w] >> IXB) | (in << (IXB * (BPW - 1)))) & ALLB;
        const unsigned keep = ix_below<K>(q, lane, w);
        out[w] = (S.ix[w] & keep) | (shifted & ~keep);
    }
}

// The index words after inserting slot f at position pos (positions >= pos
// move up by one; the top entry of the last lane falls off).
template <int K>
__device__ __forceinline__ void ix_inserted(const Side<K> &S, int pos, int f, int lane, unsigned (&out)[Side<K>::NW]) {
    constexpr int NW = Side<K>::NW, BPW = Side<K>::BPW, IXB = Side<K>::IXB, EPW = Side<K>::EPW;
    constexpr unsigned ALLB = Side<K>::ALLB, EMASK = Side<K>::EMASK;
    const unsigned top = (S.ix[NW - 1] >> (IXB * (BPW - 1))) & EMASK;
    const unsigned carry = __shfl_up_sync(FULL, top, 1);
    const unsigned fb = (unsigned)f * Side<K>::REP;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const unsigned in = w == 0 ? carry : (S.ix[w - 1] >> (IXB * (BPW - 1)));
        const unsigned shifted = ((S.ix[w] << IXB) | in) & ALLB;
        const int d = pos - (lane * K + EPW * w);
        const unsigned keep = ix_below<K>(pos, lane, w);
        const unsigned fm = (d >= 0 && d < BPW) ? (EMASK << (IXB * d)) : 0u;
        out[w] = (S.ix[w] & keep) | (fb & fm) | (shifted & ~(keep | fm));
    }
}

// Position of slot s among the n live positions.
template <int K>
__device__ __forceinline__ int ix_find(const Side<K> &S, int s, int lane) {
    constexpr int NW = Side<K>::NW, IXB = Side<K>::IXB, EPW = Side<K>::EPW;
    int local = -1;
#pragma unroll
    for (int w = NW - 1; w >= 0; w--) {
        const unsigned key = (unsigned)s * Side<K>::REP;
        const unsigned eq = IXB == 8 ? __vcmpeq4(S.ix[w], key) : __vcmpeq2(S.ix[w], key);
        const unsigned m = eq & ix_below<K>(S.n, lane, w);
        if (m) local = EPW * w + (31 - __clz(m)) / IXB;   // s occurs once: any set bit of its entry
    }
    const unsigned lanes = __ballot_sync(FULL, local >= 0);
    const int L = 31 - __clz(lanes);
    return __shfl_sync(FULL, lane * K + local, L);
}

template <int K>
__device__ __forceinline__ void slot_clear(Side<K> &S, int s, int lane) {
    if (lane == slot_lane<K>(s)) S.occ &= ~(1u << slot_r<K>(s));
}

// Refresh the cached front order from position 0.
template <int K>
__device__ __forceinline__ void front_refresh(Side<K> &S, const PoolSmem<K> &P) {
    if (S.n > 0) {
        const int s = slot_at<K>(S, 0);
        S.fslot = s;
        S.fpx = P.px[s];
        S.fqty = P.qty[s];
        S.fid = P.id[s];
    }
}

#ifdef LOB_CHECKED
// Checked build: one side's invariants after a step -- live count within the
// capacity and equal to the occupied slots; positions 0..n-1 name occupied
// slots in priority order (better price first, earlier stamp first at a
// price), each with a positive quantity; register copies and the cached front
// order agree with shared memory.  Warp-uniform result.
template <int K, bool BID>
__device__ bool book_ok(const Side<K> &S, const PoolSmem<K> &P, int cap, int lane) {
    const int n = S.n;
    const int occ_n = (int)__reduce_add_sync(FULL, (unsigned)__popc(S.occ & Side<K>::KMASK));
    bool ok = n >= 0 && n <= cap && n <= 32 * K && occ_n == n;
    const int last = min(ix_ent<K>(S, K - 1), 32 * K - 1);
    int ppx = __shfl_up_sync(FULL, P.px[last], 1);
    long long pts = __shfl_up_sync(FULL, P.ts[last], 1);
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;
        const int s = ix_ent<K>(S, j);
        const bool in_range = s < 32 * K;
        const int ss = in_range ? s : 0;
        const unsigned o = __shfl_sync(FULL, S.occ, slot_lane<K>(ss));
        const bool occupied = (o >> slot_r<K>(ss)) & 1u;
        const int px = P.px[ss];
        const long long ts = P.ts[ss];
        const bool order = q == 0 || (BID ? (ppx > px || (ppx == px && pts < ts)) : (ppx < px || (ppx == px && pts < ts)));
        if (q < n) ok = ok && in_range && occupied && order && P.qty[ss] > 0;
        if constexpr (Side<K>::REG) {
            if ((S.occ >> j) & 1u) ok = ok && S.px[j] == P.px[slot_of<K>(lane, j)] && S.id[j] == P.id[slot_of<K>(lane, j)];
        }
        ppx = px;
        pts = ts;
    }
    if (n > 0) {
        const int f = min(slot_at<K>(S, 0), 32 * K - 1);
        ok = ok && f == S.fslot && P.px[f] == S.fpx && P.qty[f] == S.fqty && P.id[f] == S.fid;
    }
    return __all_sync(FULL, ok);
}
#endif

// ---------------------------------------------------------------- env context
// Warp-uniform per-env scalars of the running step.
struct Ctx {
    long long ts_next, seq_next;
    long long inv0, inv1, cash0, cash1, pv0, pv1, exec_done;
    long long bg_cash, bg_inv;
    int last_px;
    int A, exec_dir;
    long long c_msgs, c_agent, c_fills, c_fill_vol, c_add_vol, c_mkt_vol, c_mkt_disc, c_cancel_vol;
    long long c_cancel_miss, c_drop_vol, c_drop_cnt, c_evict_vol, c_evict_cnt, c_bad;
    int msg_idx;
    int fill_n;
    int status;
    lob_fill *fill_log;
    int fill_cap;
    AgentSmem *ag;   // several agents per type only

    __device__ __forceinline__ int owner(long long id) const {
        return (id >= 0 || A == 0) ? 2 : (int)((~id) & 1);
    }
};

static __device__ __noinline__ void log_fill(lob_fill *log, int idx, long long maker, long long taker, int px, int f,
                                      int msg_idx, int side) {
    lob_fill r;
    r.maker_id = maker; r.taker_id = taker; r.px = px; r.qty = f; r.msg_idx = msg_idx; r.taker_side = side;
    log[idx] = r;
}

// A trade at the resting order's price; cash and inventory move between the
// owners of the two orders (0, 1 = agents, 2 = background).
template <bool TRACE, bool MA = false>
__device__ __forceinline__ void do_fill(Ctx &c, int px, int f, long long maker_id, long long taker_id,
                                        int taker_side, int lane) {
    if constexpr (MA) {
        // owners: agent (-id - 1) mod A of a negative id, else background (A);
        // agent state lives in shared memory, written by lane 0
        const int A = c.A;
        const int om = maker_id >= 0 ? A : (int)((unsigned long long)(~maker_id) % (unsigned)A);
        const int ot = taker_id >= 0 ? A : (int)((unsigned long long)(~taker_id) % (unsigned)A);
        const int buyer = taker_side == LOB_BUY ? ot : om;
        const int seller = taker_side == LOB_BUY ? om : ot;
        typedef unsigned long long u64;
        const long long notional = (long long)((u64)(long long)px * (u64)(long long)f);
        if (buyer == A) { c.bg_cash -= notional; c.bg_inv += f; }
        if (seller == A) { c.bg_cash += notional; c.bg_inv -= f; }
        if (lane == 0) {
            AgentSmem &g = *c.ag;
            if (buyer < A) { g.cash[buyer] = (long long)((u64)g.cash[buyer] - (u64)notional); g.inv[buyer] += f; }
            if (seller < A) { g.cash[seller] = (long long)((u64)g.cash[seller] + (u64)notional); g.inv[seller] -= f; }
            const int task = c.exec_dir == LOB_SELL ? seller : buyer;   // its owner, if executing, progresses
            if (task < (A >> 1)) g.done[task] += f;
        }
        c.last_px = px;
        c.c_fills += 1;
        c.c_fill_vol += f;
        if constexpr (TRACE) {
            if (c.fill_log != nullptr) {
                if (lane == 0 && c.fill_n < c.fill_cap)
                    log_fill(c.fill_log, c.fill_n, maker_id, taker_id, px, f, c.msg_idx, taker_side);
                c.fill_n++;
            }
        }
        return;
    }
    // Only agent ids are negative, so a fill between two background orders
    // (the common case) moves nothing tracked per owner and skips this
    // block; the background's totals are the negated agents' totals over the
    // step (every notional and quantity changes hands), settled once per step.
    if ((maker_id | taker_id) < 0 && c.A > 0) {
        const int om = c.owner(maker_id), ot = c.owner(taker_id);
        const int buyer = taker_side == LOB_BUY ? ot : om;
        const int seller = taker_side == LOB_BUY ? om : ot;
        const long long notional = (long long)((unsigned long long)(long long)px * (unsigned long long)(long long)f);
        const long long ff = f;
        c.cash0 += (buyer == 0 ? -notional : 0) + (seller == 0 ? notional : 0);
        c.inv0 += (buyer == 0 ? ff : 0) - (seller == 0 ? ff : 0);
        c.cash1 += (buyer == 1 ? -notional : 0) + (seller == 1 ? notional : 0);
        c.inv1 += (buyer == 1 ? ff : 0) - (seller == 1 ? ff : 0);
        c.exec_done += ((c.exec_dir == LOB_SELL ? seller : buyer) == 0) ? ff : 0;
    }
    c.last_px = px;
    c.c_fills += 1;
    c.c_fill_vol += f;
    if constexpr (TRACE) {
        if (c.fill_log != nullptr) {
            if (lane == 0 && c.fill_n < c.fill_cap)
                log_fill(c.fill_log, c.fill_n, maker_id, taker_id, px, f, c.msg_idx, taker_side);
            c.fill_n++;
        }
    }
}

// Take liquidity from resting side O (RBID: O holds bids), price first then
// time, up to the limit (if any).  Returns the unfilled quantity.
template <int K, bool RBID, bool TRACE, bool MA = false>
__device__ __forceinline__ int side_take(Side<K> &O, PoolSmem<K> &P, bool has_limit, int limit, int q,
                                         long long taker_id, int taker_side, Ctx &c, int lane) {
    while (q > 0 && O.n > 0 && (!has_limit || at_least<RBID>(O.fpx, limit))) {
        // the order behind the front, fetched before we know whether it is needed
        const int s1 = LOB_CHK(slot_at<K>(O, 1), 32 * K, c.status);
        const int npx = P.px[s1], nqt = P.qty[s1];
        const long long nid = P.id[s1];
        unsigned popped[Side<K>::NW];
        ix_removed<K>(O, 0, lane, popped);
        const int f = min(q, O.fqty);
        do_fill<TRACE, MA>(c, O.fpx, f, O.fid, taker_id, taker_side, lane);
        q -= f;
        const bool gone = f == O.fqty;
        const int left = O.fqty - f;
        P.qty[O.fslot] = left;          // every lane stores the same value
        if (gone && lane == slot_lane<K>(O.fslot)) O.occ &= ~(1u << slot_r<K>(O.fslot));
#pragma unroll
        for (int w = 0; w < Side<K>::NW; w++) O.ix[w] = gone ? popped[w] : O.ix[w];
        O.n -= gone ? 1 : 0;
        O.fpx = gone ? npx : O.fpx;
        O.fqty = gone ? nqt : left;
        O.fid = gone ? nid : O.fid;
        O.fslot = gone ? s1 : O.fslot;
    }
    return q;
}

// Rest an order on its own side, applying the capacity rule.  Branch-free:
// every outcome (drop, evict and insert, insert) is computed and selected.
template <int K, bool BID>
__device__ __forceinline__ void side_rest(Side<K> &S, PoolSmem<K> &P, int cap, int p, int q, long long oid,
                                          Ctx &c, int lane) {
    // independent of p: the worst order (evicted if the side is full) and a free slot
    const int vic = LOB_CHK(slot_at<K>(S, S.n > 0 ? S.n - 1 : 0), 32 * K, c.status);
    const int vic_q = P.qty[vic];
    const unsigned fr = ~S.occ & Side<K>::KMASK;
    const unsigned flanes = __ballot_sync(FULL, fr != 0);
    // any free slot will do: the highest set bits (one instruction each)
    const int free_slot = __shfl_sync(FULL, slot_of<K>(lane, 31 - __clz(fr)), 31 - __clz(flanes));
    int pos;
    if constexpr (Side<K>::REG) {
        // one warp sum of the lanes' counts (fewer instructions than a ballot per register)
        int cnt = 0;
#pragma unroll
        for (int r = 0; r < K; r++) cnt += (int)(((S.occ >> r) & 1u) && at_least<BID>(S.px[r], p));
        pos = (int)__reduce_add_sync(FULL, (unsigned)cnt);
    } else {
        int cnt = 0;
#pragma unroll (Side<K>::SU)
        for (int r = 0; r < K; r++) cnt += (int)(((S.occ >> r) & 1u) && at_least<BID>(spx<K>(S, P, r, lane), p));
        pos = (int)__reduce_add_sync(FULL, (unsigned)cnt);
    }
    const bool full = S.n >= cap;
    const bool ins = !(full && pos >= S.n);   // a full side keeps only strictly better prices
    const bool ev = full && ins;
    if (full) {   // the capacity counters move only on a full side
        c.c_drop_vol += ins ? 0 : q;
        c.c_drop_cnt += ins ? 0 : 1;
        c.c_evict_vol += ev ? vic_q : 0;
        c.c_evict_cnt += ev ? 1 : 0;
    }
    const int f = full ? vic : LOB_CHK(free_slot, 32 * K, c.status);
    const int fl = slot_lane<K>(f), fr_ = slot_r<K>(f);
    if (ins && lane == fl) S.occ |= 1u << fr_;   // a reused victim slot stays occupied
    if constexpr (Side<K>::REG) {
#pragma unroll
        for (int r = 0; r < K; r++)
            if (ins && lane == fl && r == fr_) { S.px[r] = p; S.id[r] = oid; }
    }
    if (ins) { P.px[f] = p; P.qty[f] = q; P.id[f] = oid; P.ts[f] = c.ts_next; }   // same value from every lane
    c.ts_next += ins ? 1 : 0;
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
}

// Remove slot s (any position) and fix the front if it was there.
template <int K>
__device__ __forceinline__ void side_remove_slot(Side<K> &S, PoolSmem<K> &P, int s, int lane, int &st) {
    const int q = LOB_CHK(ix_find<K>(S, s, lane), S.n, st);
    slot_clear<K>(S, s, lane);
    ix_remove<K>(S, q, lane);
    S.n--;
    if (q == 0) front_refresh<K>(S, P);
}

// First slot in priority order holding (price, id), when several do.
template <int K>
__device__ __forceinline__ int first_dup_slot(const Side<K> &S, const PoolSmem<K> &P, int p, long long oid, int lane) {
    int best = -1;
#pragma unroll
    for (int j = K - 1; j >= 0; j--) {
        const int q = lane * K + j;
        if (q < S.n) {
            const int s = ix_ent<K>(S, j);
            if (P.px[s] == p && P.id[s] == oid) best = j;
        }
    }
    const unsigned lanes = __ballot_sync(FULL, best >= 0);
    const int L = __ffs(lanes) - 1;
    const int j = __shfl_sync(FULL, best, L);
    return slot_at<K>(S, L * K + j);
}

// Partial cancel or delete: lookup by (price, id); a miss is a no-op.
template <int K>
__device__ __forceinline__ void side_cancel(Side<K> &S, PoolSmem<K> &P, int type, int p, int qty, long long oid,
                                            Ctx &c, int lane) {
    unsigned m = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++)
        if (((S.occ >> r) & 1u) && spx<K>(S, P, r, lane) == p && sid<K>(S, P, r, lane) == oid) m |= 1u << r;
    const unsigned lanes = __ballot_sync(FULL, m != 0);
    if (lanes == 0) {
        c.c_cancel_miss += 1;
        return;
    }
    const bool dup = __popc(lanes) > 1 || __ballot_sync(FULL, __popc(m) > 1) != 0;
    int s;
    if (!dup) {   // the single match: its lane and register by their highest set bits
        const int L = 31 - __clz(lanes);
        s = __shfl_sync(FULL, slot_of<K>(lane, 31 - __clz(m)), L);
    } else {
        s = first_dup_slot<K>(S, P, p, oid, lane);
    }
    s = LOB_CHK(s, 32 * K, c.status);
    const int q0 = P.qty[s];
    const int cut = type == LOB_PARTIAL ? min(qty, q0) : q0;
    c.c_cancel_vol += cut;
    if (q0 - cut == 0) {
        side_remove_slot<K>(S, P, s, lane, c.status);
    } else {
        P.qty[s] = q0 - cut;   // same value from every lane
        if (s == S.fslot) S.fqty = q0 - cut;
    }
}

// ---------------------------------------------------------------- load / store / gather
// Load one side's block (positions in priority order, lane l loading
// positions l*K .. l*K+K-1 with vector loads); position q goes to pool slot q,
// so the index starts as the identity.  Occupancy is set once n is known.
template <int K, bool BID>
__device__ __forceinline__ void side_load(Side<K> &S, PoolSmem<K> &P, const unsigned char *blk, int lane) {
    constexpr int SL = 32 * K;
    const int s = BID ? 0 : 1;
    const int *gpx = reinterpret_cast<const int *>(blk) + s * SL + lane * K;
    const int *gqt = reinterpret_cast<const int *>(blk) + 2 * SL + s * SL + lane * K;
    const long long *gid = reinterpret_cast<const long long *>(blk + 16 * SL) + s * SL + lane * K;
    const long long *gts = reinterpret_cast<const long long *>(blk + 32 * SL) + s * SL + lane * K;
    constexpr int G = K < 4 ? K : 4;   // positions per vector group
#pragma unroll
    for (int g = 0; g < K; g += G) {
        int px[G], qt[G];
        long long id[G], ts[G];
        if constexpr (G == 4) {
            const int4 a = *reinterpret_cast<const int4 *>(gpx + g);
            const int4 b = *reinterpret_cast<const int4 *>(gqt + g);
            px[0] = a.x; px[1] = a.y; px[2] = a.z; px[3] = a.w;
            qt[0] = b.x; qt[1] = b.y; qt[2] = b.z; qt[3] = b.w;
            const longlong2 c0 = *reinterpret_cast<const longlong2 *>(gid + g);
            const longlong2 c1 = *reinterpret_cast<const longlong2 *>(gid + g + 2);
            const longlong2 d0 = *reinterpret_cast<const longlong2 *>(gts + g);
            const longlong2 d1 = *reinterpret_cast<const longlong2 *>(gts + g + 2);
            id[0] = c0.x; id[1] = c0.y; id[2] = c1.x; id[3] = c1.y;
            ts[0] = d0.x; ts[1] = d0.y; ts[2] = d1.x; ts[3] = d1.y;
        } else {
#pragma unroll
            for (int u = 0; u < G; u++) { px[u] = gpx[g + u]; qt[u] = gqt[g + u]; id[u] = gid[g + u]; ts[u] = gts[g + u]; }
        }
#pragma unroll
        for (int u = 0; u < G; u++) {
            const int slot = lane * K + g + u;
            P.px[slot] = px[u]; P.qty[slot] = qt[u]; P.id[slot] = id[u]; P.ts[slot] = ts[u];
            if constexpr (Side<K>::REG) { S.px[g + u] = px[u]; S.id[g + u] = id[u]; }
        }
    }
#pragma unroll
    for (int w = 0; w < Side<K>::NW; w++) {
        unsigned v = 0;
#pragma unroll
        for (int b = 0; b < Side<K>::BPW; b++)
            v |= (unsigned)(lane * K + Side<K>::EPW * w + b) << (Side<K>::IXB * b);
        S.ix[w] = v;
    }
}

// Mark slots 0 .. n-1 occupied (the identity index after a load).
template <int K>
__device__ __forceinline__ void side_set_count(Side<K> &S, int n, int lane) {
    S.n = n;
    S.occ = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++)
        if (slot_of<K>(lane, r) < n) S.occ |= 1u << r;
}

// Store one side in priority order (this lane's K positions, gathered from
// the pool), vector stores as in the load.
template <int K, bool BID>
__device__ __forceinline__ void side_store(const Side<K> &S, const PoolSmem<K> &P, unsigned char *blk, int lane) {
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
            const int s = ix_ent<K>(S, g + u);
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
}

// Book of env 0 after a message, canonical layout (trace mode only).
template <int K>
__device__ __forceinline__ void write_snapshot(const Side<K> &B, const Side<K> &A, const WarpSmem<K> &sm, int C,
                                               unsigned char *rec, int lane) {
    int *n2 = reinterpret_cast<int *>(rec);
    int *px = n2 + 2;
    int *qt = px + 2 * C;
    long long *id = reinterpret_cast<long long *>(rec + 8 + 16 * (long long)C);
    long long *ts = id + 2 * C;
    if (lane == 0) { n2[0] = B.n; n2[1] = A.n; }
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;
        if (q < C) {
            const bool vb = q < B.n, va = q < A.n;
            const int sb = ix_ent<K>(B, j), sa = ix_ent<K>(A, j);
            px[q] = vb ? sm.pool[0].px[sb] : 0; qt[q] = vb ? sm.pool[0].qty[sb] : 0;
            id[q] = vb ? sm.pool[0].id[sb] : 0; ts[q] = vb ? sm.pool[0].ts[sb] : 0;
            px[C + q] = va ? sm.pool[1].px[sa] : 0; qt[C + q] = va ? sm.pool[1].qty[sa] : 0;
            id[C + q] = va ? sm.pool[1].id[sa] : 0; ts[C + q] = va ? sm.pool[1].ts[sa] : 0;
        }
    }
}

// Warp-wide int64 sum.
__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

// Aggregated top-L levels of one side, read from the pool in priority order
// in two passes over this lane's positions (level starts, then run sums into
// shared-memory int64 atomics).  Also returns the resting quantity of each
// agent on this side (own0 / own1, warp totals).  Returns the level count.
template <int K>
__device__ __forceinline__ int side_levels(const Side<K> &S, const PoolSmem<K> &P, int L, int *lvl_px,
                                           long long *lvl_q, long long &own0, long long &own1, int lane) {
    const int n = S.n;
    const int ppx = __shfl_up_sync(FULL, P.px[ix_ent<K>(S, K - 1)], 1);
    int cnt = 0, prev = ppx;
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;
        const int px = P.px[ix_ent<K>(S, j)];
        cnt += (q < n && (q == 0 || px != prev)) ? 1 : 0;
        prev = px;
    }
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    int lv = incl - cnt - 1;
    long long run = 0, o0 = 0, o1 = 0;
    int run_lv = -1;
    prev = ppx;
#pragma unroll
    for (int j = 0; j < K; j++) {
        const int q = lane * K + j;
        const int s = ix_ent<K>(S, j);
        const int px = P.px[s];
        if (q < n) {
            const int qt = P.qty[s];
            const long long id = P.id[s];
            if (q == 0 || px != prev) {
                if (run_lv >= 0 && run_lv < L)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&lvl_q[run_lv]), (unsigned long long)run);
                lv++;
                run = 0;
                if (lv < L) lvl_px[lv] = px;
            }
            run += qt;
            run_lv = lv;
            if (id < 0) { if ((~id) & 1) o1 += qt; else o0 += qt; }
        }
        prev = px;
    }
    if (run_lv >= 0 && run_lv < L && run != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&lvl_q[run_lv]), (unsigned long long)run);
    own0 += warp_sum(o0);
    own1 += warp_sum(o1);
    return __shfl_sync(FULL, incl, 31);
}

// Carry-over of one side (Sec. 4, Action Conversion): a resting order of an
// agent at one of that agent's wanted (side, price) is kept (its quantity
// added to `kept`); every other resting agent order is flagged for
// cancellation -- per slot in `cand` (1 + agent) and as this lane's bit mask.
template <int K>
__device__ __forceinline__ unsigned side_carry(const Side<K> &S, const PoolSmem<K> &P, unsigned char *cand, int side,
                                               const int (&wa)[3], const int (&ws)[3], const int (&wp)[3], int nw,
                                               unsigned (&kept)[3], int lane) {
    unsigned cmask = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++) {
        const int slot = slot_of<K>(lane, r);
        unsigned char flag = 0;
        const long long oid = sid<K>(S, P, r, lane);
        if (((S.occ >> r) & 1u) && oid < 0) {
            const int a = (int)((~oid) & 1);
            const int opx = spx<K>(S, P, r, lane);
            int m = -1;
#pragma unroll
            for (int i = 0; i < 3; i++)
                if (i < nw && wa[i] == a && ws[i] == side && wp[i] == opx) m = i;
            if (m < 0) {
                flag = (unsigned char)(1 + a);
                cmask |= 1u << r;
            } else {
                const unsigned q = (unsigned)P.qty[slot];
#pragma unroll
                for (int i = 0; i < 3; i++) if (m == i) kept[i] += q;
            }
        }
        cand[slot] = flag;
    }
    return cmask;
}

// Delete the flagged agent orders of one side in any order (the final book
// does not depend on it); counts one agent message per cancel.
template <int K>
__device__ __forceinline__ void side_cancel_set(Side<K> &S, PoolSmem<K> &P, unsigned cmask, Ctx &c, int lane) {
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
        side_remove_slot<K>(S, P, s, lane, c.status);
    }
}

// Delete, in priority order, agent a's flagged orders on one side.
template <int K>
__device__ __forceinline__ void side_agent_cancels(Side<K> &S, PoolSmem<K> &P, unsigned char *cand, int a, Ctx &c,
                                                   int lane, const Side<K> &B, const Side<K> &A2,
                                                   const WarpSmem<K> &sm, bool snap_env, const KParams &p, int cap,
                                                   long long &snap_n, long long snap_bytes) {
    for (;;) {
        __syncwarp();
        int first = -1;
#pragma unroll
        for (int j = K - 1; j >= 0; j--)
            if (lane * K + j < S.n && cand[ix_ent<K>(S, j)] == 1 + a) first = j;
        const unsigned lanes = __ballot_sync(FULL, first >= 0);
        if (lanes == 0) break;
        const int L = __ffs(lanes) - 1;
        const int q = L * K + __shfl_sync(FULL, first, L);
        const int s = LOB_CHK(slot_at<K>(S, q), 32 * K, c.status);
        c.c_msgs += 1;
        c.c_agent += 1;
        c.c_cancel_vol += P.qty[s];
        __syncwarp();
        if (lane == 0) cand[s] = 0;
        slot_clear<K>(S, s, lane);
        ix_remove<K>(S, q, lane);
        S.n--;
        if (q == 0) front_refresh<K>(S, P);
        if (snap_env && snap_n < p.snap_cap) write_snapshot<K>(B, A2, sm, cap, p.snaps + snap_n * snap_bytes, lane);
        snap_n++;
        c.msg_idx++;
    }
}

// Sec. 5 rewards of the market maker and the Table 2 penalties, in wrapping
// 64-bit arithmetic.  With Mbar the step's average mid, Psi_b + Psi_s (Eq. 4)
// sums (Mbar - P) Q over buys and (P - Mbar) Q over sells, which is
// Mbar * (inventory change) + (cash change) of the step, so it is formed from
// the step-start inventory and cash without a per-fill record.  Values are in
// quarter ticks (4 Mbar = start + end of twice the mid); the lambda damping of
// Eq. 3 and the unfilled-task penalty round up, so each reward is the floor of
// its exact value.  Arguments pass by value, so none of the caller's register
// state is addressed.
static __device__ __noinline__ longlong2 reward_variants(int mode, int lam_pct, long long rho, long long pen_milli,
                                                         bool last_step, long long unfilled, long long mid2_start,
                                                         long long mid2_end, long long inv_start, long long cash_start,
                                                         long long inv1, long long cash1, long long r0, long long r1) {
    typedef unsigned long long u64;
    if (mode != LOB_REWARD_PV) {
        const u64 m4 = (u64)mid2_start + (u64)mid2_end;
        const u64 dinv = (u64)inv1 - (u64)inv_start;
        const u64 dcash = (u64)cash1 - (u64)cash_start;
        u64 r4 = m4 * dinv + 4ull * dcash;
        if (mode == LOB_REWARD_SPOONER) {
            const long long psi_inv4 = (long long)(2ull * (u64)inv1 * ((u64)mid2_end - (u64)mid2_start));
            const long long pos = psi_inv4 > 0 ? psi_inv4 : 0;
            const long long damp = (long long)((u64)(100 - lam_pct) * (u64)pos + 99ull) / 100;
            r4 = r4 + (u64)psi_inv4 - (u64)damp;
        }
        r1 = (long long)r4;
    }
    r1 = (long long)((u64)r1 - (u64)rho * ((u64)inv1 * (u64)inv1));
    if (last_step && pen_milli != 0) {
        unfilled = unfilled > 0 ? unfilled : 0;
        const long long pen = (long long)((u64)pen_milli * (u64)unfilled + 999ull) / 1000;
        r0 = (long long)((u64)r0 - (u64)pen);
    }
    return make_longlong2(r0, r1);
}

// ---------------------------------------------------------------- several agents per type
// Carry-over of one side for A agents: a resting agent order is kept when
// its owner wants an order at its (side, price) -- its quantity adds to that
// order's kept amount -- and flagged for cancellation (1 + owner) otherwise.
template <int K>
__device__ __forceinline__ unsigned side_carry_ma(const Side<K> &S, const PoolSmem<K> &P, unsigned char *cand, int sd,
                                                  AgentSmem &ag, int A, int lane) {
    unsigned cmask = 0;
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++) {
        const int slot = slot_of<K>(lane, r);
        unsigned char flag = 0;
        const long long oid = sid<K>(S, P, r, lane);
        if (((S.occ >> r) & 1u) && oid < 0) {
            const int a = (int)((unsigned long long)(~oid) % (unsigned)A);
            if (ag.want_q[a][sd] > 0 && ag.want_px[a][sd] == spx<K>(S, P, r, lane)) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&ag.kept[a][sd]), (unsigned long long)P.qty[slot]);
            } else {
                flag = (unsigned char)(1 + a);
                cmask |= 1u << r;
            }
        }
        cand[slot] = flag;
    }
    return cmask;
}

// Resting quantity of every agent on one side (shared-memory atomics).
template <int K>
__device__ __forceinline__ void side_own_ma(const Side<K> &S, const PoolSmem<K> &P, AgentSmem &ag, int A, int lane) {
#pragma unroll (Side<K>::SU)
    for (int r = 0; r < K; r++) {
        const long long oid = sid<K>(S, P, r, lane);
        if (((S.occ >> r) & 1u) && oid < 0)
            atomicAdd(reinterpret_cast<unsigned long long *>(&ag.own[(unsigned long long)(~oid) % (unsigned)A]),
                      (unsigned long long)P.qty[slot_of<K>(lane, r)]);
    }
}

// Action conversion of A = 2P agents (Sec. 4 with Sec. 3's agents of each
// type), lanes over agents: the action (host or random policy), the
// step-start state for the reward variants, and each agent's wanted orders
// -- an execution agent one order at one of four reference prices times
// {1, 2, 5} q0 while its task is unfinished, a market maker its space's
// quotes of mm_lot.
__device__ __forceinline__ void agent_wants_ma(const KParams &p, int e, int t, int step, unsigned long long seed,
                                               long long bb, long long ba, AgentSmem &ag, Ctx &c, int lane) {
    const int A = p.n_agents, P = A >> 1;
    const int n_mm = p.mm_space == LOB_MM_FIXED_QUANT ? 8 : p.mm_space == LOB_MM_DIRECTIONAL ? 3 : 12;
    const unsigned long long pkey = step_key(seed, t, TAG_POLICY);
    for (int a = lane; a < A; a += 32) {
        const int n_act = a < P ? 12 : n_mm;
        int act;
        if (p.action_mode == LOB_ACT_RANDOM) {
            act = (int)bounded(sm_mix(pkey + GAMMA * (unsigned long long)(a + 1)), (unsigned)n_act);
        } else {
            act = p.actions[(long long)step * p.act_step_stride + (long long)e * A + a];
            if (act < 0 || act >= n_act) c.status |= ST_BADACT;
        }
        ag.act[a] = act;
        ag.inv0[a] = ag.inv[a];
        ag.cash0[a] = ag.cash[a];
        long long bpx = 0, apx = 0;
        int bq = 0, aq = 0;
        if (act >= 0 && act < n_act) {
            if (a < P) {
                const long long remaining = (long long)p.exec_target - ag.done[a];
                if (remaining > 0) {
                    const int pi = act / 3, mi = act % 3;
                    const long long mult = mi == 0 ? 1 : (mi == 1 ? 2 : 5);
                    long long qty = mult * p.exec_q0;
                    qty = qty < remaining ? qty : remaining;
                    const long long s2 = bb + ba;
                    const long long fl = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
                    const long long ce = s2 <= 0 ? -((-s2) / 2) : (s2 + 1) / 2;
                    if (c.exec_dir == LOB_SELL) {
                        apx = pi == 0 ? bb : pi == 1 ? ce : pi == 2 ? ba : ba + 2;
                        aq = (int)qty;
                    } else {
                        bpx = pi == 0 ? ba : pi == 1 ? fl : pi == 2 ? bb : bb - 2;
                        bq = (int)qty;
                    }
                }
            } else if (p.mm_space == LOB_MM_SPREAD_SKEW) {
                if (act >= 1) {
                    if (act <= 9) { bpx = bb - (act - 1) / 3; apx = ba + (act - 1) % 3; }
                    else if (act == 10) { bpx = bb + 1; apx = ba; }
                    else { bpx = bb; apx = ba - 1; }
                    bq = aq = p.mm_lot;
                }
            } else if (p.mm_space == LOB_MM_FIXED_QUANT) {
                switch (act) {
                    case 1: bpx = bb - 2; apx = ba + 2; bq = aq = p.mm_lot; break;
                    case 2: bpx = bb - 4; apx = ba + 4; bq = aq = p.mm_lot; break;
                    case 3: bpx = bb + 1; apx = ba - 1; bq = aq = p.mm_lot; break;
                    case 4: bpx = bb - 2; bq = p.mm_lot; break;
                    case 5: apx = ba + 2; aq = p.mm_lot; break;
                    case 6: bpx = bb - 5; apx = ba - 1; bq = aq = p.mm_lot; break;
                    case 7: bpx = bb + 1; apx = ba + 5; bq = aq = p.mm_lot; break;
                    default: break;
                }
            } else {
                if (act == 1) { bpx = bb; bq = p.mm_lot; }
                if (act == 2) { apx = ba; aq = p.mm_lot; }
            }
        }
        ag.want_px[a][0] = (int)bpx; ag.want_q[a][0] = bq;
        ag.want_px[a][1] = (int)apx; ag.want_q[a][1] = aq;
        ag.kept[a][0] = 0;
        ag.kept[a][1] = 0;
    }
}

// The orders the agents send after carry-over (wanted minus kept), in agent
// order (an execution agent's order; a market maker's bid, then ask),
// Fisher-Yates shuffled with the step's SplitMix64 draws, then given ids
// -(1 + agent + A seq) in processing order.  Lane 0 writes them as message
// records; returns their count on every lane.
__device__ __forceinline__ int agent_orders_ma(const KParams &p, int t, unsigned long long seed, AgentSmem &ag,
                                               Ctx &c, int lane) {
    const int A = p.n_agents;
    int ns = 0;
    if (lane == 0) {
        for (int a = 0; a < A; a++)
            for (int sd = 0; sd < 2; sd++) {
                const long long q = (long long)ag.want_q[a][sd] - ag.kept[a][sd];
                if (ag.want_q[a][sd] > 0 && q > 0) {
                    DevMsg r;
                    r.ts = 0;
                    r.oid = a;   // the owner until the ids are given
                    r.px = ag.want_px[a][sd];
                    r.qty = (int)q;
                    r.type = (short)LOB_ADD;
                    r.side = (short)(sd == 0 ? LOB_BUY : LOB_SELL);
                    r.pad = 0;
                    ag.amsg[ns++] = r;
                }
            }
        const unsigned long long key = step_key(seed, t, TAG_SHUFFLE);
        for (int i = ns - 1, d = 0; i >= 1; i--, d++) {
            const int j = (int)bounded(sm_mix(key + GAMMA * (unsigned long long)(d + 1)), (unsigned)(i + 1));
            const DevMsg x = ag.amsg[i];
            ag.amsg[i] = ag.amsg[j];
            ag.amsg[j] = x;
        }
        for (int u = 0; u < ns; u++)
            ag.amsg[u].oid = -(1 + ag.amsg[u].oid + (long long)A * (c.seq_next + u));
    }
    return __shfl_sync(FULL, ns, 0);
}

// Quotes of the Fixed Quantity (8 options) and directional (3) market-maker
// spaces (Sec. 4.1.1) around touches bb / ba: {bid, ask, bit 0 = bid quoted,
// bit 1 = ask quoted}.  Out of line: the benchmark's head never calls it.
static __device__ __noinline__ int4 mm_other_quotes(int space, int act, int bb, int ba) {
    int qb = 0, qa = 0, f = 0;
    if (space == LOB_MM_FIXED_QUANT) {
        switch (act) {
            case 1: qb = bb - 2; qa = ba + 2; f = 3; break;
            case 2: qb = bb - 4; qa = ba + 4; f = 3; break;
            case 3: qb = bb + 1; qa = ba - 1; f = 3; break;
            case 4: qb = bb - 2; f = 1; break;
            case 5: qa = ba + 2; f = 2; break;
            case 6: qb = bb - 5; qa = ba - 1; f = 3; break;
            case 7: qb = bb + 1; qa = ba + 5; f = 3; break;
            default: break;
        }
    } else {
        if (act == 1) { qb = bb; f = 1; }
        if (act == 2) { qa = ba; f = 2; }
    }
    return make_int4(qb, qa, f, 0);
}

// One message tile (up to TILE_MAX records) copied by the warp's lanes, one
// record per lane per pass, as one commit group.
__device__ __forceinline__ void tile_copy_lanes(void *dst, const void *src, int count, int rec_bytes, int lane) {
    for (int r = lane; r < count; r += 32) {
        char *d = reinterpret_cast<char *>(dst) + (long long)r * rec_bytes;
        const char *g = reinterpret_cast<const char *>(src) + (long long)r * rec_bytes;
        cp_async16(d, g);
        if (rec_bytes == 32) cp_async16(d + 16, g + 16);
    }
    cp_async_commit();
}

// A tile of compact records {px, qty, word = id << 4 | sell << 3 | type},
// landed in the upper half of a tile buffer, rewritten in place as 32-byte
// records (all lanes read before any lane writes).
__device__ __forceinline__ DevMsg widen_record(int4 w) {
    const long long word = ((long long)(unsigned)w.w << 32) | (unsigned)w.z;
    DevMsg r;
    r.ts = 0;
    r.oid = word >> 4;
    r.px = w.x;
    r.qty = w.y;
    r.type = (short)(word & 7);
    r.side = (short)((word & 8) ? LOB_SELL : LOB_BUY);
    r.pad = 0;
    return r;
}
__device__ __forceinline__ void widen_tile(DevMsg *tile, int count, int T, int lane) {
    const int4 *src = reinterpret_cast<const int4 *>(reinterpret_cast<const char *>(tile) + 16 * T);
    // up to two records per lane (T <= 64), all read before any is written
    int4 w0 = make_int4(0, 0, 0, 0), w1 = make_int4(0, 0, 0, 0);
    if (lane < count) w0 = src[lane];
    if (lane + 32 < count) w1 = src[lane + 32];
    __syncwarp();
    if (lane < count) tile[lane] = widen_record(w0);
    if (lane + 32 < count) tile[lane + 32] = widen_record(w1);
    __syncwarp();
}

}  // namespace lobk
#include "lob_ladder.cuh"
#include "fused.cuh"
namespace lobk {

// The fused rollout's per-warp handle on its CTA's policy tile.
struct FusedCtx {
    FusedSmem *fz;
    const FusedParams *f;
    unsigned phase;
    int nw, tid, row;   // warps in the CTA, thread index, this warp's row (env) in the tile
};
static_assert(LW == 128, "Side<K>::bm holds the ladder bitmap");

// Book operations at the step's edges in the env's current form: the price
// ladder while `lad` holds (LADC: the instance has a ladder), else the sorted
// index.  The message loops of the two forms are separate (msgs_ladder,
// msgs_index) so that each keeps a compact body.
template <int K, bool BID, bool LADC>
__device__ __forceinline__ void book_cancel_set(Side<K> &S, PoolSmem<K> &P, LadBlock<K> *lb, bool lad,
                                                unsigned cmask, Ctx &c, int lane) {
    if constexpr (LADC) {
        if (lad) {
            lad_cancel_set<K, BID>(S, P, lb->s[BID ? 0 : 1], cmask, c, lane);
            return;
        }
    }
    side_cancel_set<K>(S, P, cmask, c, lane);
}
template <int K, bool BID, bool LADC>
__device__ __forceinline__ int book_levels(const Side<K> &S, const PoolSmem<K> &P, LadBlock<K> *lb, bool lad, int L,
                                           int *lvl_px, long long *lvl_q, long long &own0, long long &own1, int lane) {
    if constexpr (LADC) {
        if (lad) return lad_levels<K, BID>(S, P, lb->s[BID ? 0 : 1], L, lvl_px, lvl_q, own0, own1, lane);
    }
    return side_levels<K>(S, P, L, lvl_px, lvl_q, own0, own1, lane);
}
template <int K, bool BID, bool LADC>
__device__ __forceinline__ void book_store(const Side<K> &S, const PoolSmem<K> &P, LadBlock<K> *lb, bool lad,
                                           unsigned char *blk, int lane) {
    if constexpr (LADC) {
        if (lad) {
            lad_store<K, BID>(S, P, lb->s[BID ? 0 : 1], lb->inv, blk, lane);
            return;
        }
    }
    side_store<K, BID>(S, P, blk, lane);
}

// The message loop of one chunk in the sorted-index form, from record i0 to
// cnt (the next record is always read one ahead; a read past the chunk end
// stays inside this warp's shared memory and is unused).
template <int K, bool TRACE, bool MA>
__device__ __forceinline__ void msgs_index(const KParams &p, WarpSmem<K> &sm, Side<K> &bid, Side<K> &ask, Ctx &c,
                                           int cap, const int4 *rp, const unsigned char *dx, int i0, int cnt,
                                           bool snap_env, long long &snap_n, long long snap_bytes, int lane) {
    int4 w0 = rp[2 * i0], w1 = rp[2 * i0 + 1];
    int dcur = dx[i0];
    for (int i = i0; i < cnt; i++) {
        const int4 n0 = rp[2 * i + 2], n1 = rp[2 * i + 3];
        const int dnext = dx[i + 1];   // read one ahead, like the record (stays in this warp's space)
        const long long oid = ((long long)(unsigned)w0.w << 32) | (unsigned)w0.z;
        const int px = w1.x;
        int qty = w1.y;
        const int didx = dcur;
        const int type = (didx >> 1) + 1;   // cancels: LOB_PARTIAL or LOB_DELETE
        if constexpr (K >= 32) {
            // the largest books: one call site per side for taking
            // liquidity and for resting, to keep the kernel's code small
            if (didx == 0 || didx == 6) {          // buy: limit add or market
                const bool lim = didx == 0;
                if (lim) c.c_add_vol += qty; else c.c_mkt_vol += qty;
                if (!lim || (ask.n > 0 && px >= ask.fpx))
                    qty = side_take<K, false, TRACE, MA>(ask, sm.pool[1], lim, px, qty, oid, LOB_BUY, c, lane);
                if (!lim) c.c_mkt_disc += qty;
                else if (qty > 0) side_rest<K, true>(bid, sm.pool[0], cap, px, qty, oid, c, lane);
            } else if (didx == 1 || didx == 7) {   // sell: limit add or market
                const bool lim = didx == 1;
                if (lim) c.c_add_vol += qty; else c.c_mkt_vol += qty;
                if (!lim || (bid.n > 0 && px <= bid.fpx))
                    qty = side_take<K, true, TRACE, MA>(bid, sm.pool[0], lim, px, qty, oid, LOB_SELL, c, lane);
                if (!lim) c.c_mkt_disc += qty;
                else if (qty > 0) side_rest<K, false>(ask, sm.pool[1], cap, px, qty, oid, c, lane);
            } else if (didx == 2 || didx == 4) {
                side_cancel<K>(bid, sm.pool[0], type, px, qty, oid, c, lane);
            } else if (didx == 3 || didx == 5) {
                side_cancel<K>(ask, sm.pool[1], type, px, qty, oid, c, lane);
            } else {
                c.c_bad += 1;
                c.status |= ST_BADMSG;
            }
        } else {
            // uniform branches in order of frequency: adds, cancels, market orders
            if (didx < 2) {
                c.c_add_vol += qty;
                if (didx == 0) {
                    if (ask.n > 0 && px >= ask.fpx)
                        qty = side_take<K, false, TRACE, MA>(ask, sm.pool[1], true, px, qty, oid, LOB_BUY, c, lane);
                    if (qty > 0) side_rest<K, true>(bid, sm.pool[0], cap, px, qty, oid, c, lane);
                } else {
                    if (bid.n > 0 && px <= bid.fpx)
                        qty = side_take<K, true, TRACE, MA>(bid, sm.pool[0], true, px, qty, oid, LOB_SELL, c, lane);
                    if (qty > 0) side_rest<K, false>(ask, sm.pool[1], cap, px, qty, oid, c, lane);
                }
            } else if (didx < 6) {
                if ((didx & 1) == 0) side_cancel<K>(bid, sm.pool[0], type, px, qty, oid, c, lane);
                else side_cancel<K>(ask, sm.pool[1], type, px, qty, oid, c, lane);
            } else if (didx < 8) {
                c.c_mkt_vol += qty;
                if (didx == 6)
                    c.c_mkt_disc += side_take<K, false, TRACE, MA>(ask, sm.pool[1], false, 0, qty, oid, LOB_BUY, c, lane);
                else
                    c.c_mkt_disc += side_take<K, true, TRACE, MA>(bid, sm.pool[0], false, 0, qty, oid, LOB_SELL, c, lane);
            } else {
                c.c_bad += 1;
                c.status |= ST_BADMSG;
            }
        }
        if (TRACE && snap_env) {
            __syncwarp();
            if (snap_n < p.snap_cap) write_snapshot<K>(bid, ask, sm, cap, p.snaps + snap_n * snap_bytes, lane);
            snap_n++;
        }
        c.msg_idx++;
        w0 = n0;
        w1 = n1;
        dcur = dnext;
    }
}

// The message loop of one chunk in the price-ladder form, from record i0:
// one call site per (operation, side).  Returns the first record it did not
// process -- cnt, or a limit order whose price would stretch its own side past
// the ladder (the caller then converts the env to the sorted form and goes on
// from that record there).
template <int K, bool MA>
__device__ __forceinline__ int msgs_ladder(WarpSmem<K> &sm, LadBlock<K> *lb, Side<K> &bid, Side<K> &ask, Ctx &c,
                                           int cap, const int4 *rp, const unsigned char *dx, int i0, int cnt,
                                           int lane) {
    int4 w0 = rp[2 * i0], w1 = rp[2 * i0 + 1];
    int dcur = dx[i0];
    for (int i = i0; i < cnt; i++) {
        const int4 n0 = rp[2 * i + 2], n1 = rp[2 * i + 3];
        const int dnext = dx[i + 1];
        const long long oid = ((long long)(unsigned)w0.w << 32) | (unsigned)w0.z;
        const int px = w1.x;
        int qty = w1.y;
        const int didx = dcur;
        if (didx < 2 || didx == 6 || didx == 7) {   // limit add or market order
            const bool sell = (didx & 1) != 0, lim = didx < 2;
            if (lim) {
                if (!(sell ? lad_fits<K, false>(ask, px) : lad_fits<K, true>(bid, px))) return i;
                c.c_add_vol += qty;
            } else {
                c.c_mkt_vol += qty;
            }
            if (!sell) {
                if (!lim || (ask.n > 0 && px >= ask.fpx))
                    qty = lad_take<K, false, false, MA>(ask, sm.pool[1], lb->s[1], lim, px, qty, oid, LOB_BUY, c, lane);
            } else {
                if (!lim || (bid.n > 0 && px <= bid.fpx))
                    qty = lad_take<K, true, false, MA>(bid, sm.pool[0], lb->s[0], lim, px, qty, oid, LOB_SELL, c, lane);
            }
            if (!lim) {
                c.c_mkt_disc += qty;
            } else if (qty > 0) {
                if (!sell) lad_rest<K, true>(bid, sm.pool[0], lb->s[0], cap, px, qty, oid, c, lane);
                else lad_rest<K, false>(ask, sm.pool[1], lb->s[1], cap, px, qty, oid, c, lane);
            }
        } else if (didx < 6) {
            const int type = (didx >> 1) + 1;   // LOB_PARTIAL or LOB_DELETE
            if ((didx & 1) == 0) lad_cancel<K, true>(bid, sm.pool[0], lb->s[0], type, px, qty, oid, c, lane);
            else lad_cancel<K, false>(ask, sm.pool[1], lb->s[1], type, px, qty, oid, c, lane);
        } else {
            c.c_bad += 1;
            c.status |= ST_BADMSG;
        }
        c.msg_idx++;
        w0 = n0;
        w1 = n1;
        dcur = dnext;
    }
    return cnt;
}

// Message pipeline state of one warp (tiles issued so far).
struct MsgPipe {
    unsigned tiles;
    DevMsg *buf;   // tiles larger than TILE: this warp's two buffers (plus one record read ahead)
};

// Run n_steps env steps of env e with the book resident on chip.  EXT
// compiles in episode mode, the reward variants and the other action spaces;
// without it those settings are ignored, so the host launches EXT whenever
// one is set.  MA (which implies EXT) runs 2P agents with their state in the
// warp's agent block agp; without it the agents are the benchmark pair.
template <int K, bool TRACE, bool EXT, bool MA, bool FUSED = false, int TT = TILE>
__device__ void run_env(const KParams &p, int e, WarpSmem<K> &sm, AgentSmem *agp, LadBlock<K> *lb, MsgPipe &pipe,
                        int lane, FusedCtx *fc = nullptr) {
    // TT records per staged message tile: up to TILE in the per-warp block's
    // buffers, more in the warp's own buffers after every per-warp block
    static_assert(TT == 16 || TT == 32 || TT == 64, "staged tiles of 16, 32 or 64 records");
    constexpr int T = TT;
    constexpr int lgT = TT == 16 ? 4 : (TT == 64 ? 6 : 5);
    DevMsg *const tb = TT > TILE ? pipe.buf : &sm.tile[0][0];
    constexpr bool XT = EXT || MA;
    // the price-ladder form for every untraced instance of the register-pool
    // classes (traces record the book after every message in the sorted form)
    constexpr bool LADC = !TRACE && ladder_class<K>();
    bool lad = false;
    EnvState *st = p.st + e;
    const bool uni = p.uni_cap > 0;
    const int cap = uni ? p.uni_cap : p.caps[e];
    unsigned char *blk = p.books + (uni ? (long long)e * p.uni_block : p.book_off[e]);
    // one-wave launches: the env's book block heads for L2 while the offsets
    // and the env state are read, so the first book load finds it there
    if (p.book_prefetch && lane == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(blk), "r"((unsigned)(48 * 32 * K)) : "memory");
    const int A = p.n_agents;
    const unsigned long long seed = p.seeds[e];
    long long *cnt = p.counters + (long long)e * LOB_NCOUNTERS;

    // first message window, issued before anything waits on memory.  The
    // offsets index of a step's data is the env's window position, or in
    // episode mode (dcur) its episode's first data step plus the step within it.
    const bool ep_mode = XT && p.ep_mode;
    const bool sysm = XT && p.msgs_sysmem;   // message tiles by lane copies instead of bulk copies
    const bool m16 = XT && p.msg16;          // compact 16-byte background records
    const int rec = m16 ? 16 : 32;
    const char *msg_base = reinterpret_cast<const char *>(p.msgs);
    int ep_start = ep_mode ? st->ep_start : 0;
    long long dcur = ep_mode ? (long long)ep_start + p.t0 % p.T : 0;
    const long long d0 = ep_mode ? dcur : (long long)e * p.off_stride + p.k0;
    long long mb = p.offsets[d0];
    long long me = p.offsets[d0 + 1];

    Side<K> bid, ask;

    Ctx c;
    c.ts_next = st->ts_next; c.seq_next = st->seq_next;
    c.inv0 = st->inv[0]; c.inv1 = st->inv[1];
    c.cash0 = st->cash[0]; c.cash1 = st->cash[1];
    c.pv0 = st->pv_prev[0]; c.pv1 = st->pv_prev[1];
    c.exec_done = st->exec_done;
    c.last_px = st->last_px;
    const int nb0 = st->n[0], na0 = st->n[1];
    c.A = A;
    c.exec_dir = (XT && p.exec_dir == 0) ? st->exec_dir : p.exec_dir;
    c.c_msgs = cnt[0]; c.c_agent = cnt[1]; c.c_fills = cnt[2]; c.c_fill_vol = cnt[3];
    c.c_add_vol = cnt[4]; c.c_mkt_vol = cnt[5]; c.c_mkt_disc = cnt[6]; c.c_cancel_vol = cnt[7];
    c.c_cancel_miss = cnt[8]; c.c_drop_vol = cnt[9]; c.c_drop_cnt = cnt[10]; c.c_evict_vol = cnt[11];
    c.c_evict_cnt = cnt[12]; c.c_bad = cnt[13]; c.bg_cash = cnt[14]; c.bg_inv = cnt[15];
    c.status = 0;
    c.fill_log = (TRACE && p.fills) ? p.fills + (long long)e * p.fill_cap : nullptr;
    c.fill_cap = p.fill_cap;
    c.ag = agp;
    if constexpr (MA) {
        for (int a = lane; a < A; a += 32) {
            const AgentState x = p.agents[(long long)e * A + a];
            agp->inv[a] = x.inv; agp->cash[a] = x.cash; agp->pv[a] = x.pv_prev; agp->done[a] = x.exec_done;
            agp->act[a] = x.act;
        }
    }
    // The book is loaded at the top of the first step, after its first
    // message tile is requested (the two fetches overlap), and in episode
    // mode again after a reset, from the snapshot image; live counts come
    // with the state.
    const unsigned char *load_src = blk;
    int load_nb = nb0, load_na = na0;
    bool need_load = true;

    const bool snap_env = TRACE && p.snaps != nullptr && e == 0;
    long long snap_n = 0;
    const long long snap_bytes = 8 + 48 * (long long)cap;
    bool timed_out = false;

    for (int step = 0; step < p.n_steps && (FUSED || !timed_out); step++) {
        if constexpr (FUSED) {   // after a timeout the warp only keeps its CTA's policy in step
            if (timed_out) {
                fused_policy(*fc->fz, *fc->f, fc->phase, fc->nw, fc->tid);
                continue;
            }
        }
        const int t = p.t0 + step;
        const int te = ep_mode ? t % p.T : t;   // step within the episode
        if (step > 0) {
            const long long d = ep_mode ? dcur : (long long)e * p.off_stride + p.k0 + step;
            mb = p.offsets[d];
            me = p.offsets[d + 1];
        }
        const int nmsg = (int)(me - mb);
        const int ntiles = (nmsg + T - 1) >> lgT;
        const unsigned tile0 = pipe.tiles;
        // failure-detection test hook: the launch's first tile is not requested,
        // so the wait for it runs out (bulk-copy path only)
        const bool held = p.hold_first && step == 0 && !sysm;
        if (ntiles > 0) {
            __syncwarp();
            // compact tiles land in the upper half of the buffer and are widened on arrival
            char *dst = reinterpret_cast<char *>(tb + (pipe.tiles & 1) * T) + (m16 ? 16 * T : 0);
            if (sysm) {
                tile_copy_lanes(dst, msg_base + mb * rec, min(T, nmsg), rec, lane);
            } else if (lane == 0 && !held) {
                fence_proxy_async_smem();
                tma_bulk_g2s(dst, msg_base + mb * rec, (unsigned)(min(T, nmsg) * rec), &sm.bar[pipe.tiles & 1]);
            }
            pipe.tiles++;
        }
        if (need_load) {
            __syncwarp();
            side_load<K, true>(bid, sm.pool[0], load_src, lane);
            side_load<K, false>(ask, sm.pool[1], load_src, lane);
            side_set_count<K>(bid, load_nb, lane);
            side_set_count<K>(ask, load_na, lane);
            __syncwarp();
            front_refresh<K>(bid, sm.pool[0]);
            front_refresh<K>(ask, sm.pool[1]);
            if constexpr (LADC) {
                const bool okb = lad_build<K, true>(bid, sm.pool[0], lb->s[0], lane);
                const bool oka = lad_build<K, false>(ask, sm.pool[1], lb->s[1], lane);
                lad = okb && oka;   // else both sides keep the sorted index of the load
            }
            need_load = false;
        }
        c.msg_idx = 0;
        c.fill_n = 0;
        snap_n = 0;
        // the pair's totals at the step start (the background settles against them)
        typedef unsigned long long u64;
        const u64 pair_cash0 = (u64)c.cash0 + (u64)c.cash1, pair_inv0 = (u64)c.inv0 + (u64)c.inv1;

        // ---- 1-3. action conversion, carry-over cancels, shuffle
        int act0 = 0, act1 = 0, ns = 0;
        if constexpr (MA) {
            AgentSmem &ag = *agp;
            const long long bb = bid.n ? bid.fpx : c.last_px;
            const long long ba = ask.n ? ask.fpx : c.last_px;
            if (lane == 0) sm.rw[0] = bb + ba;   // twice the mid at the start of the step
            __syncwarp();
            agent_wants_ma(p, e, t, step, seed, bb, ba, ag, c, lane);
            __syncwarp();
            const unsigned cm_b = side_carry_ma<K>(bid, sm.pool[0], sm.cand[0], 0, ag, A, lane);
            const unsigned cm_a = side_carry_ma<K>(ask, sm.pool[1], sm.cand[1], 1, ag, A, lane);
            __syncwarp();
            if (TRACE && snap_env) {
                // trace mode: cancels one by one in the paper's order, a snapshot after each
                for (int a = 0; a < A; a++) {
                    side_agent_cancels<K>(bid, sm.pool[0], sm.cand[0], a, c, lane, bid, ask, sm, snap_env, p, cap,
                                          snap_n, snap_bytes);
                    side_agent_cancels<K>(ask, sm.pool[1], sm.cand[1], a, c, lane, bid, ask, sm, snap_env, p, cap,
                                          snap_n, snap_bytes);
                }
            } else {
                book_cancel_set<K, true, LADC>(bid, sm.pool[0], lb, lad, cm_b, c, lane);
                book_cancel_set<K, false, LADC>(ask, sm.pool[1], lb, lad, cm_a, c, lane);
            }
            ns = agent_orders_ma(p, t, seed, ag, c, lane);
            c.seq_next += ns;
            __syncwarp();
        } else if (A == 2) {
            // market maker's action count: 12, or (extended kernel) 8 / 3
            const int n_mm = !XT ? 12 : p.mm_space == LOB_MM_FIXED_QUANT ? 8 : p.mm_space == LOB_MM_DIRECTIONAL ? 3 : 12;
            if constexpr (FUSED) {   // the CTA's policy acted on the last observation
                act0 = fc->fz->acts[fc->row][0];
                act1 = fc->fz->acts[fc->row][1];
                if (p.act_steps && lane < 2) p.act_steps[((long long)step * p.n_envs + e) * 2 + lane] = lane ? act1 : act0;
            } else if (p.action_mode == LOB_ACT_RANDOM) {
                const unsigned long long key = step_key(seed, t, TAG_POLICY);
                act0 = (int)bounded(sm_mix(key + GAMMA), 12);
                act1 = (int)bounded(sm_mix(key + 2 * GAMMA), (unsigned)n_mm);
            } else {
                const int *ap = p.actions + (long long)step * p.act_step_stride + 2LL * e;
                act0 = ap[0];
                act1 = ap[1];
                if (act0 < 0 || act0 >= 12 || act1 < 0 || act1 >= n_mm) c.status |= ST_BADACT;
            }
            const long long bb = bid.n ? bid.fpx : c.last_px;
            const long long ba = ask.n ? ask.fpx : c.last_px;
            if (XT && p.reward_mode != LOB_REWARD_PV && lane == 0) {
                sm.rw[0] = bb + ba; sm.rw[1] = c.inv1; sm.rw[2] = c.cash1;
            }
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
            if (!XT || p.mm_space == LOB_MM_SPREAD_SKEW) {
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
            } else {
                // Fixed Quantity (8 options) or directional (3): quotes that may be one-sided
                const int4 mq = mm_other_quotes(p.mm_space, act1, (int)bb, (int)ba);
                const bool hb = (mq.z & 1) != 0, ha = (mq.z & 2) != 0;
                const long long qb = mq.x, qa = mq.y;
                // constant array indices only, so the wanted orders stay in registers
                const int q1s = ha ? LOB_SELL : LOB_BUY;      // a one-sided quote
                const int q1p = (int)(ha ? qa : qb);
                if (hb && ha) {
                    if (nw == 0) {
                        wa[0] = 1; ws[0] = LOB_BUY; wp[0] = (int)qb; wq[0] = p.mm_lot;
                        wa[1] = 1; ws[1] = LOB_SELL; wp[1] = (int)qa; wq[1] = p.mm_lot;
                    } else {
                        wa[1] = 1; ws[1] = LOB_BUY; wp[1] = (int)qb; wq[1] = p.mm_lot;
                        wa[2] = 1; ws[2] = LOB_SELL; wp[2] = (int)qa; wq[2] = p.mm_lot;
                    }
                } else if (hb || ha) {
                    if (nw == 0) { wa[0] = 1; ws[0] = q1s; wp[0] = q1p; wq[0] = p.mm_lot; }
                    else { wa[1] = 1; ws[1] = q1s; wp[1] = q1p; wq[1] = p.mm_lot; }
                }
                nw += (hb ? 1 : 0) + (ha ? 1 : 0);
            }
            // carry-over: keep resting orders at a wanted (agent, side, price)
            unsigned kept_u[3] = {0u, 0u, 0u};
            const unsigned cm_b = side_carry<K>(bid, sm.pool[0], sm.cand[0], LOB_BUY, wa, ws, wp, nw, kept_u, lane);
            const unsigned cm_a = side_carry<K>(ask, sm.pool[1], sm.cand[1], LOB_SELL, wa, ws, wp, nw, kept_u, lane);
            long long kept[3];
#pragma unroll
            for (int i = 0; i < 3; i++) kept[i] = (long long)__reduce_add_sync(FULL, kept_u[i]);
            if (TRACE && snap_env) {
                // trace mode: cancels one by one in the paper's order, a snapshot after each
#pragma unroll
                for (int a = 0; a < 2; a++) {
                    side_agent_cancels<K>(bid, sm.pool[0], sm.cand[0], a, c, lane, bid, ask, sm, snap_env, p, cap,
                                          snap_n, snap_bytes);
                    side_agent_cancels<K>(ask, sm.pool[1], sm.cand[1], a, c, lane, bid, ask, sm, snap_env, p, cap,
                                          snap_n, snap_bytes);
                }
            } else {
                book_cancel_set<K, true, LADC>(bid, sm.pool[0], lb, lad, cm_b, c, lane);
                book_cancel_set<K, false, LADC>(ask, sm.pool[1], lb, lad, cm_a, c, lane);
            }
            // orders to send (wanted minus kept), Fisher-Yates shuffled
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
            // the agents' orders become the first records of the step
            if (lane < ns) {
                int ma = 0, ms = 0, mp = 0, mq = 0;
#pragma unroll
                for (int u = 0; u < 3; u++)
                    if (u == lane) { ma = sa[u]; ms = ss[u]; mp = sp[u]; mq = sq[u]; }
                DevMsg r;
                r.ts = 0;
                r.oid = -(1 + (long long)ma + 2LL * (c.seq_next + lane));
                r.px = mp; r.qty = mq; r.type = (short)LOB_ADD; r.side = (short)ms; r.pad = 0;
                sm.amsg[lane] = r;
            }
            c.seq_next += ns;
            __syncwarp();
        }

        // ---- 4. the agents' orders, then the market-replay messages.  Chunk -1
        // is the agents' records, chunk j >= 0 the j-th staged tile; inside a
        // chunk the next record is read one message ahead (a read past the
        // chunk end stays inside this warp's shared memory and is unused).
        for (int ch = ns > 0 ? -1 : 0; ch < ntiles && !timed_out; ch++) {
            const DevMsg *base;
            int cnt_ch;
            const int agent = ch < 0 ? 1 : 0;
            if (ch < 0) {
                base = MA ? agp->amsg : sm.amsg;
                cnt_ch = ns;
            } else {
                const unsigned buf = (tile0 + ch) & 1u;
                const unsigned phase = ((tile0 + ch) >> 1) & 1u;
                if (sysm) {
                    cp_async_wait_all();   // this tile is the only group in flight
                    __syncwarp();
                } else if (!mbar_wait(&sm.bar[buf], phase, p.wait_budget)) {
                    c.status |= ST_TIMEOUT;
                    if (!(held && ch == 0))
                        mbar_wait(&sm.bar[buf], phase, p.drain_budget);  // let the copy in flight land
                    timed_out = true;
                    break;
                }
                if (ch + 1 < ntiles) {
                    __syncwarp();
                    const char *src = msg_base + (mb + (long long)(ch + 1) * T) * rec;
                    char *dst = reinterpret_cast<char *>(tb + (pipe.tiles & 1) * T) + (m16 ? 16 * T : 0);
                    if (sysm) {
                        tile_copy_lanes(dst, src, min(T, nmsg - (ch + 1) * T), rec, lane);
                    } else if (lane == 0) {
                        fence_proxy_async_smem();
                        tma_bulk_g2s(dst, src, (unsigned)(min(T, nmsg - (ch + 1) * T) * rec),
                                     &sm.bar[pipe.tiles & 1]);
                    }
                    pipe.tiles++;
                }
                base = tb + buf * T;
                cnt_ch = min(T, nmsg - ch * T);
                if (m16) widen_tile(tb + buf * T, cnt_ch, T, lane);
            }
            const int4 *rp = reinterpret_cast<const int4 *>(base);
            c.c_msgs += cnt_ch;                 // a started chunk is always finished
            c.c_agent += agent ? cnt_ch : 0;
            // each record's dense dispatch index, (type - 1) * 2 + (side is sell)
            // or 8 = malformed, decoded one record per lane into a byte array
            // (the carry-over flags' space, free during the message loop and
            // rewritten by the next step's carry-over), off the serial chain
            unsigned char *dx = &sm.cand[0][0];
            for (int r = lane; r < cnt_ch; r += 32) {   // a tile, or up to 3 orders per agent
                const int4 w = rp[2 * r + 1];
                const int ty = w.z & 0xffff, sd = w.z >> 16;
                const bool ok = ty >= LOB_ADD && ty <= LOB_MARKET && (sd == 1 || sd == -1) && (w.y > 0 || ty == LOB_DELETE);
                dx[r] = (unsigned char)(ok ? ((ty - 1) << 1) | (sd < 0 ? 1 : 0) : 8);
            }
            __syncwarp();
            int i0 = 0;
            if constexpr (LADC) {
                if (lad) {
                    i0 = msgs_ladder<K, MA>(sm, lb, bid, ask, c, cap, rp, dx, 0, cnt_ch, lane);
                    if (i0 < cnt_ch) {   // an order the ladder cannot hold: both sides to the sorted form
                        lad_to_index<K, true>(bid, lb->s[0], lb->inv, lane);
                        lad_to_index<K, false>(ask, lb->s[1], lb->inv, lane);
                        lad = false;
                    }
                }
            }
            if (i0 < cnt_ch)
                msgs_index<K, TRACE, MA>(p, sm, bid, ask, c, cap, rp, dx, i0, cnt_ch, snap_env, snap_n, snap_bytes, lane);
        }
        if (timed_out) {
            if constexpr (FUSED) {
                fused_policy(*fc->fz, *fc->f, fc->phase, fc->nw, fc->tid);
                continue;
            } else {
                break;
            }
        }
#ifdef LOB_CHECKED
        {
            bool ok;
            if constexpr (LADC) {
                ok = lad ? (lad_ok<K, true>(bid, sm.pool[0], lb->s[0], lb->inv, cap, lane) &&
                            lad_ok<K, false>(ask, sm.pool[1], lb->s[1], lb->inv, cap, lane))
                         : (book_ok<K, true>(bid, sm.pool[0], cap, lane) && book_ok<K, false>(ask, sm.pool[1], cap, lane));
            } else {
                ok = book_ok<K, true>(bid, sm.pool[0], cap, lane) && book_ok<K, false>(ask, sm.pool[1], cap, lane);
            }
            if (bid.n > 0 && ask.n > 0 && bid.fpx >= ask.fpx) ok = false;   // never crossed after a message
            if (!ok) c.status |= ST_CHECK;
        }
#endif
        if constexpr (!MA) {   // the background gained what the pair lost this step
            c.bg_cash = (long long)((u64)c.bg_cash - ((u64)c.cash0 + (u64)c.cash1 - pair_cash0));
            c.bg_inv = (long long)((u64)c.bg_inv - ((u64)c.inv0 + (u64)c.inv1 - pair_inv0));
        }

        // ---- 5. step outcomes (and, after the last step, the book write-back)
        // Episode mode: after the episode's last step the env starts the next
        // episode from snapshot ep_j; the step reports that episode's first
        // observation with its own rewards and done flag.
        const bool ep_end = ep_mode && te + 1 == p.T;
        const unsigned ep_j =
            ep_end ? bounded(sm_mix(step_key(seed, t / p.T + 1, LOB_TAG_EPISODE) + GAMMA), (unsigned)p.n_starts) : 0u;
        // a drawn task side is signed into the remaining-target observation
        // (+ buy, - sell); the next episode draws its own side
        const bool side_drawn = XT && p.exec_dir == 0;
        const int ep_dir = (ep_end && side_drawn) ? drawn_task_side(seed, t / p.T + 1) : c.exec_dir;
        __syncwarp();
        const long long step_base = (long long)step * p.n_envs + e;
        const long long obs_base = p.ow_obs ? (long long)e : step_base;
        const long long rew_base = p.ow_rew ? (long long)e : step_base;
        const long long done_base = p.ow_done ? (long long)e : step_base;
        if (A > 0) {
            const int L = p.L;
            for (int i = lane; i < 2 * LMAX; i += 32) {
                (&sm.lvl_q[0][0])[i] = 0;
                (&sm.lvl_px[0][0])[i] = 0;
            }
            __syncwarp();
            long long own0 = 0, own1 = 0;
            const int nlb = book_levels<K, true, LADC>(bid, sm.pool[0], lb, lad, L, sm.lvl_px[0], sm.lvl_q[0], own0, own1, lane);
            const int nla = book_levels<K, false, LADC>(ask, sm.pool[1], lb, lad, L, sm.lvl_px[1], sm.lvl_q[1], own0, own1, lane);
            const long long bb = bid.n ? bid.fpx : c.last_px;
            const long long ba = ask.n ? ask.fpx : c.last_px;
            const long long s2 = bb + ba;
            const long long anchor = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
            if constexpr (MA) {
                AgentSmem &ag = *agp;
                const int P = A >> 1;
                for (int a = lane; a < A; a += 32) ag.own[a] = 0;
                __syncwarp();
                side_own_ma<K>(bid, sm.pool[0], ag, A, lane);
                side_own_ma<K>(ask, sm.pool[1], ag, A, lane);
                __syncwarp();
                const float tl = __fdiv_rn((float)(p.T - (te + 1)), (float)p.T);
                const int D = p.D;
                float *ob = p.obs ? p.obs + obs_base * A * D : nullptr;
                if (ob && ep_end) {
                    const float *src = p.ep_obs + (long long)ep_j * A * D;
                    const bool flip = side_drawn && ep_dir == LOB_SELL;
                    for (int i = lane; i < A * D; i += 32)
                        ob[i] = (flip && i % D == 4 * L + 3 && i / D < P) ? -src[i] : src[i];
                } else if (ob) {
                    for (int idx = lane; idx < 4 * L; idx += 32) {
                        const int sd = idx >= 2 * L ? 1 : 0;
                        const int i = (idx - sd * 2 * L) >> 1;
                        const int nl = sd == 0 ? nlb : nla;
                        const long long lq = sm.lvl_q[sd][i];
                        const long long lp = (long long)sm.lvl_px[sd][i] - anchor;
                        const float v = i >= nl ? 0.0f : __ll2float_rn((idx & 1) ? lq : lp);
                        for (int a = 0; a < A; a++) ob[a * D + idx] = v;
                    }
                    for (int i = lane; i < 5 * A; i += 32) {
                        const int a = i / 5, g = i - 5 * a;
                        const long long rem = a < P ? (long long)p.exec_target - ag.done[a] : 0;
                        const long long x = g == 0 ? ag.inv[a] : g == 1 ? ag.cash[a]
                                          : g == 3 ? ((side_drawn && c.exec_dir == LOB_SELL) ? -rem : rem) : ag.own[a];
                        ob[a * D + 4 * L + g] = g == 2 ? tl : __ll2float_rn(x);
                    }
                }
                // Eq. 1 per agent, then the variants and penalties of its type
                __syncwarp();
                for (int a = lane; a < A; a += 32) {
                    typedef unsigned long long u64;
                    const long long iv = ag.inv[a], cs = ag.cash[a];
                    const bool pvm = p.pv_ref == LOB_PV_MID;   // 2 PV in half ticks
                    const long long pref = pvm ? s2 : (iv > 0 ? bb : (iv < 0 ? ba : 0));
                    const long long pv = (long long)((u64)iv * (u64)pref + (u64)cs * (pvm ? 2ull : 1ull));
                    long long r = (long long)((u64)pv - (u64)ag.pv[a]);
                    ag.pv[a] = pv;
                    if (p.reward_mode != LOB_REWARD_PV || p.inv_penalty != 0 || p.exec_pen_milli != 0) {
                        const longlong2 rr = reward_variants(p.reward_mode, p.lam_pct, p.inv_penalty,
                                                             p.exec_pen_milli * (pvm ? 2 : 1), te + 1 == p.T,
                                                             (long long)p.exec_target - ag.done[a],
                                                             sm.rw[0], s2, ag.inv0[a], ag.cash0[a], iv, cs, r, r);
                        r = a < P ? rr.x : rr.y;
                    }
                    if (p.rew) p.rew[rew_base * A + a] = r;
                    if (p.act_out) p.act_out[(long long)e * A + a] = ag.act[a];
                }
            } else {
            // Eq. 1: PV = Q_inv * P_ref + Cash, P_ref the liquidation touch
            const long long pref0 = c.inv0 > 0 ? bb : (c.inv0 < 0 ? ba : 0);
            const long long pref1 = c.inv1 > 0 ? bb : (c.inv1 < 0 ? ba : 0);
            // with the mid reference, 2 PV = Q_inv (bb + ba) + 2 Cash, exact in half ticks
            const bool pvm = XT && p.pv_ref == LOB_PV_MID;
            const long long pv0 = (long long)((unsigned long long)c.inv0 * (unsigned long long)(pvm ? s2 : pref0) +
                                              (unsigned long long)c.cash0 * (pvm ? 2ull : 1ull));
            const long long pv1 = (long long)((unsigned long long)c.inv1 * (unsigned long long)(pvm ? s2 : pref1) +
                                              (unsigned long long)c.cash1 * (pvm ? 2ull : 1ull));
            long long r0 = (long long)((unsigned long long)pv0 - (unsigned long long)c.pv0);
            long long r1 = (long long)((unsigned long long)pv1 - (unsigned long long)c.pv1);
            c.pv0 = pv0; c.pv1 = pv1;
            const float tl = __fdiv_rn((float)(p.T - (te + 1)), (float)p.T);
            const int D = p.D;
            __syncwarp();
            float *ob = p.obs ? p.obs + obs_base * A * D : nullptr;
            if (ob && ep_end) {
                const float *src = p.ep_obs + (long long)ep_j * A * D;
                const bool flip = side_drawn && ep_dir == LOB_SELL;
                for (int i = lane; i < A * D; i += 32) ob[i] = (flip && i == 4 * L + 3) ? -src[i] : src[i];
            } else if (ob) {
                // level entries: the same for both agents
                for (int idx = lane; idx < 4 * L; idx += 32) {
                    const int sd = idx >= 2 * L ? 1 : 0;
                    const int i = (idx - sd * 2 * L) >> 1;
                    const int nl = sd == 0 ? nlb : nla;
                    const long long lq = sm.lvl_q[sd][i];
                    const long long lp = (long long)sm.lvl_px[sd][i] - anchor;
                    const float v = i >= nl ? 0.0f : __ll2float_rn((idx & 1) ? lq : lp);
                    ob[idx] = v;
                    ob[D + idx] = v;
                }
                // five agent scalars per agent: lanes 0..9
                if (lane < 10) {
                    const int a = lane >= 5 ? 1 : 0;
                    const int g = lane - 5 * a;
                    const long long iv = a == 0 ? c.inv0 : c.inv1;
                    const long long cs = a == 0 ? c.cash0 : c.cash1;
                    long long rem = a == 0 ? (long long)p.exec_target - c.exec_done : 0;
                    if (side_drawn && c.exec_dir == LOB_SELL) rem = -rem;
                    const long long own = a == 0 ? own0 : own1;
                    const long long x = g == 0 ? iv : g == 1 ? cs : g == 3 ? rem : own;
                    const float v = g == 2 ? tl : __ll2float_rn(x);
                    ob[a * D + 4 * L + g] = v;
                }
            }
            if constexpr (FUSED) {
                // the observation rows of both agents into the CTA's policy tile
                FusedSmem &fz = *fc->fz;
                for (int idx = lane; idx < 4 * L; idx += 32) {
                    const int sd = idx >= 2 * L ? 1 : 0;
                    const int i = (idx - sd * 2 * L) >> 1;
                    const int nl = sd == 0 ? nlb : nla;
                    const long long lq = sm.lvl_q[sd][i];
                    const long long lp = (long long)sm.lvl_px[sd][i] - anchor;
                    const float v = i >= nl ? 0.0f : __ll2float_rn((idx & 1) ? lq : lp);
                    fused_put_obs(fz, *fc->f, 0, fc->row, idx, v);
                    fused_put_obs(fz, *fc->f, 1, fc->row, idx, v);
                }
                if (lane < 10) {
                    const int a = lane >= 5 ? 1 : 0;
                    const int g = lane - 5 * a;
                    const long long iv = a == 0 ? c.inv0 : c.inv1;
                    const long long cs = a == 0 ? c.cash0 : c.cash1;
                    long long rem = a == 0 ? (long long)p.exec_target - c.exec_done : 0;
                    if (side_drawn && c.exec_dir == LOB_SELL) rem = -rem;
                    const long long own = a == 0 ? own0 : own1;
                    const long long x = g == 0 ? iv : g == 1 ? cs : g == 3 ? rem : own;
                    fused_put_obs(fz, *fc->f, a, fc->row, 4 * L + g, g == 2 ? tl : __ll2float_rn(x));
                }
                __syncwarp();
            }
            if (lane == 0) {
                if (XT && (p.reward_mode != LOB_REWARD_PV || p.inv_penalty != 0 || p.exec_pen_milli != 0)) {
                    const longlong2 r = reward_variants(p.reward_mode, p.lam_pct, p.inv_penalty,
                                                        p.exec_pen_milli * (pvm ? 2 : 1), te + 1 == p.T,
                                                        (long long)p.exec_target - c.exec_done,
                                                        sm.rw[0], s2, sm.rw[1], sm.rw[2], c.inv1, c.cash1, r0, r1);
                    r0 = r.x; r1 = r.y;
                }
                if (p.rew) { p.rew[rew_base * A] = r0; p.rew[rew_base * A + 1] = r1; }
                if (p.act_out) { p.act_out[2LL * e] = act0; p.act_out[2LL * e + 1] = act1; }
            }
            }  // the benchmark pair
        }
        if (lane == 0 && p.done) p.done[done_base] = (unsigned char)(te + 1 == p.T);
        if (TRACE && lane == 0 && p.fill_counts) p.fill_counts[e] = c.fill_n;
        if (TRACE && lane == 0 && snap_env && p.snap_count) *p.snap_count = snap_n;
        if (lane == 0) { st->act[0] = act0; st->act[1] = act1; }
        if (ep_end) {
            // the next episode: its snapshot book (loaded at the next step's
            // top, or copied to the env's block if this launch ends here),
            // flat agents, its first data step
            const lob_start S = p.ep_starts[ep_j];
            load_src = p.ep_images + (long long)ep_j * p.ep_block;
            load_nb = S.n_bid;
            load_na = S.n_ask;
            need_load = true;
            c.ts_next = S.n_bid + S.n_ask;
            c.seq_next = 0;
            c.inv0 = 0; c.inv1 = 0; c.cash0 = 0; c.cash1 = 0; c.pv0 = 0; c.pv1 = 0; c.exec_done = 0;
            c.last_px = S.last_px;
            c.exec_dir = ep_dir;
            if constexpr (MA) {
                __syncwarp();
                for (int a = lane; a < A; a += 32) { agp->inv[a] = 0; agp->cash[a] = 0; agp->pv[a] = 0; agp->done[a] = 0; }
                __syncwarp();
            }
            ep_start = S.data_step;
            dcur = S.data_step;
        } else if (ep_mode) {
            dcur++;
        }
        if constexpr (FUSED) fused_policy(*fc->fz, *fc->f, fc->phase, fc->nw, fc->tid);
        if (step + 1 == p.n_steps) {
            if (XT && need_load) {
                // an episode ended with the launch: the env's block becomes the image
                const int4 *src = reinterpret_cast<const int4 *>(load_src);
                int4 *dst = reinterpret_cast<int4 *>(blk);
                for (long long i = lane; i < p.ep_block / 16; i += 32) dst[i] = src[i];
            } else {
                book_store<K, true, LADC>(bid, sm.pool[0], lb, lad, blk, lane);
                book_store<K, false, LADC>(ask, sm.pool[1], lb, lad, blk, lane);
            }
        }
    }

    // ---- counters and env scalars
    const int any_status = __reduce_or_sync(FULL, (unsigned)c.status);
    if (lane == 0) {
        if (any_status) atomicOr(p.status, any_status);
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
        st->n[0] = (XT && need_load) ? load_nb : bid.n;
        st->n[1] = (XT && need_load) ? load_na : ask.n;
        st->t = p.t0 + p.n_steps;
        if (XT) st->ep_start = ep_start;
        if (XT) st->exec_dir = c.exec_dir;
    }
    if constexpr (MA) {
        __syncwarp();
        for (int a = lane; a < A; a += 32) {
            AgentState x;
            x.inv = agp->inv[a]; x.cash = agp->cash[a]; x.pv_prev = agp->pv[a]; x.exec_done = agp->done[a];
            x.act = agp->act[a];
            x.pad[0] = x.pad[1] = x.pad[2] = 0;
            p.agents[(long long)e * A + a] = x;
        }
    }
}

// One warp per env; with a work queue (p.queue) warps take envs until none is left.
template <int K, bool TRACE, bool EXT, bool MA, int TT = TILE>
__device__ __forceinline__ void env_steps_body(const KParams &p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpSmem<K> &sm = reinterpret_cast<WarpSmem<K> *>(smem_raw)[wib];
    // after the block's WarpSmem array: the warps' ladder blocks (register-pool
    // classes), then (several agents) the warps' agent blocks
    const int nw = blockDim.x >> 5;
    unsigned char *after = smem_raw + nw * sizeof(WarpSmem<K>);
    LadBlock<K> *lb = ladder_class<K>() ? reinterpret_cast<LadBlock<K> *>(after) + wib : nullptr;
    after += nw * ladder_bytes<K>();
    AgentSmem *agp = MA ? reinterpret_cast<AgentSmem *>(after) + wib : nullptr;
    after += MA ? nw * sizeof(AgentSmem) : 0;
    // tiles of more than TILE records: the warps' buffers after every other
    // per-warp block (two tiles and the record read one past the second)
    DevMsg *tbuf = TT > TILE ? reinterpret_cast<DevMsg *>(after) + wib * (2 * TT + 1) : nullptr;
    if (lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    MsgPipe pipe{0u, tbuf};
    if (p.queue == nullptr) {
        const int w = blockIdx.x * (blockDim.x >> 5) + wib;
        if (w < p.n_list)
            run_env<K, TRACE, EXT, MA, false, TT>(p, p.env_list ? p.env_list[w] : w, sm, agp, lb, pipe, lane);
    } else {
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(p.queue, 1);
            w = __shfl_sync(FULL, w, 0);
            if (w >= p.n_list) break;
            run_env<K, TRACE, EXT, MA, false, TT>(p, p.env_list ? p.env_list[w] : w, sm, agp, lb, pipe, lane);
        }
    }
}

// The step kernel in two register budgets.  k_env_steps leaves the budget
// to the compiler, which keeps two blocks' worth of warps resident (better
// for launches of several waves of small books); k_env_steps_wide may use the
// whole register file (one block per SM minimum): fewer spills and a shorter
// per-message path, the better choice when the launch fits one wave or when
// shared memory bounds residency anyway (K >= 8).
template <int K, bool TRACE, bool EXT, bool MA = false>
__global__ void __launch_bounds__(256) k_env_steps(const KParams p) {
    env_steps_body<K, TRACE, EXT, MA>(p);
}
template <int K, bool TRACE, bool EXT, bool MA = false, int TT = TILE>
__global__ void __launch_bounds__(256, 1) k_env_steps_wide(const KParams p) {
    env_steps_body<K, TRACE, EXT, MA, TT>(p);
}
// A fixed register budget of NREG per thread, for launches of several waves
// where resident warps per SM set the throughput: e.g. 168 keeps three 4-warp
// blocks resident (3 x 128 threads x 168 registers fit the 64 K register
// file), where ptxas left to itself may take a few registers more and leave
// room for two.
template <int K, bool TRACE, bool EXT, bool MA, int NREG>
__global__ void __maxnreg__(NREG) k_env_steps_nreg(const KParams p) {
    env_steps_body<K, TRACE, EXT, MA>(p);
}

}  // namespace lobk
