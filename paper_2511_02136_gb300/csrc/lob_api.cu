// lob_api.cu -- host side of the C ABI declared in include/lob.h.
//
// Owns the device state of a handle (books, per-env scalars, counters, the
// last step's outputs), validates every argument on the host, groups envs by
// book-capacity class (32, 64, 128 or 256 slots per side) and launches the
// warp-per-env step kernels of lob_device.cuh on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lob.h"
#include "lob_device.cuh"
#include "lob_steps.h"
#include "policy_internal.h"

using namespace lobk;

namespace {

constexpr int NCLASS = 6;                 // K = 1, 2, 4, 8, 16, 32 (32 .. 1024 slots per side)
constexpr int CLASS_K[NCLASS] = {1, 2, 4, 8, 16, 32};
constexpr size_t SMEM_PER_BLOCK_MAX = 227 * 1024;
constexpr long long DEFAULT_WAIT_BUDGET = 2000000000LL;  // ~1 s of SM cycles

int class_of(int cap) {
    for (int i = 0; i < NCLASS; i++)
        if (cap <= 32 * CLASS_K[i]) return i;
    return -1;
}

// Execution agent's base lot q0 = max(1, ceil(target / T)) (Sec. 4.1.2).
long long exec_lot(const lob_config &c) {
    const long long q0 = ((long long)c.exec_target + c.episode_len - 1) / c.episode_len;
    return q0 < 1 ? 1 : q0;
}

// Reward selection and penalties of the agents (Sec. 5, Eqs. 3-4, Table 2).
static void set_rewards(KParams &p, const lob_config &c) {
    p.reward_mode = c.reward_mode;
    p.lam_pct = c.spooner_lambda_pct;
    p.inv_penalty = c.inv_penalty;
    p.exec_pen_milli = c.exec_penalty_milli;
    p.mm_space = c.mm_space;
    p.pv_ref = c.pv_ref;
}

// Shared memory of one warp (env): its WarpSmem plus, for the register-pool
// classes, its price-ladder block.
size_t warp_smem_bytes(int K) {
    switch (K) {
        case 1: return sizeof(WarpSmem<1>) + ladder_bytes<1>();
        case 2: return sizeof(WarpSmem<2>) + ladder_bytes<2>();
        case 4: return sizeof(WarpSmem<4>) + ladder_bytes<4>();
        case 8: return sizeof(WarpSmem<8>) + ladder_bytes<8>();
        case 16: return sizeof(WarpSmem<16>) + ladder_bytes<16>();
        default: return sizeof(WarpSmem<32>) + ladder_bytes<32>();
    }
}

// Per-warp buffers of staged tiles larger than the per-warp block's own
// (two tiles and one record read past the second).
size_t tile_ext_bytes(int T) { return T > TILE ? (size_t)(2 * T + 1) * sizeof(DevMsg) : 0; }

// Most warps (envs) per block whose shared memory fits one block.
int max_wpb(int K, int T = TILE) {
    const int m = (int)(SMEM_PER_BLOCK_MAX / (warp_smem_bytes(K) + tile_ext_bytes(T)));
    return m < 8 ? m : 8;
}
// The same for the several-agents kernel (each warp also holds an agent block).
int max_wpb_ma(int K) {
    const int m = (int)(SMEM_PER_BLOCK_MAX / (warp_smem_bytes(K) + sizeof(AgentSmem)));
    return m < 8 ? m : 8;
}

// Every launch shape's shared memory stays within SMEM_PER_BLOCK_MAX, which
// the step kernels are opted into (the tile size changes a shape's bytes).
cudaError_t optin_k(int K) {
    const size_t smem = SMEM_PER_BLOCK_MAX;
    const size_t smem_ma = SMEM_PER_BLOCK_MAX;
    cudaError_t e;
    switch (K) {
        case 1: e = optin_steps_1(smem); return e == cudaSuccess ? optin_steps_ma_1(smem_ma) : e;
        case 2: e = optin_steps_2(smem); return e == cudaSuccess ? optin_steps_ma_2(smem_ma) : e;
        case 4: e = optin_steps_4(smem); return e == cudaSuccess ? optin_steps_ma_4(smem_ma) : e;
        case 8: e = optin_steps_8(smem); return e == cudaSuccess ? optin_steps_ma_8(smem_ma) : e;
        case 16: e = optin_steps_16(smem); return e == cudaSuccess ? optin_steps_ma_16(smem_ma) : e;
        default: e = optin_steps_32(smem); return e == cudaSuccess ? optin_steps_ma_32(smem_ma) : e;
    }
}

// Opt every step-kernel class into the shared memory of its widest launch
// shape, once per device; done when a handle is created so that launches
// themselves never change function attributes.
cudaError_t ensure_optin() {
    static bool done[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    for (int k = 0; k < NCLASS; k++)
        if ((e = optin_k(CLASS_K[k])) != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

// Resident blocks per SM of the wide step kernel, per (class, extended,
// warps per block); queried once (the launch shape fixes the shared memory).
int wide_blocks_per_sm(int K, bool ext, int wpb, size_t smem, int T) {
    static int cache[NCLASS][2][9][3];   // 0 = not queried yet; last index: tile 16, 32, 64
    const int k = class_of(32 * K);
    int &c = cache[k][ext ? 1 : 0][wpb][T == 16 ? 0 : (T == 64 ? 2 : 1)];
    if (c == 0) {
        int nb = 0;
        switch (K) {
            case 1: nb = wide_blocks_per_sm_1(ext, 32 * wpb, smem); break;
            case 2: nb = wide_blocks_per_sm_2(ext, 32 * wpb, smem); break;
            case 4: nb = wide_blocks_per_sm_4(ext, 32 * wpb, smem); break;
            case 8: nb = wide_blocks_per_sm_8(ext, 32 * wpb, smem); break;
            case 16: nb = wide_blocks_per_sm_16(ext, 32 * wpb, smem); break;
            default: nb = wide_blocks_per_sm_32(ext, 32 * wpb, smem); break;
        }
        c = nb > 0 ? nb : -1;
    }
    return c > 0 ? c : 0;
}

// Launch the step kernel of class K (shared memory opted in by ensure_optin);
// the warps per block are capped by what one block's shared memory holds.
// Whether a launch needs the extended kernel (episode mode, a reward
// variant, another action space, host-memory or compact messages, a drawn
// task side).
bool kernel_ext(const KParams &p) {
    return p.ep_mode != 0 || p.reward_mode != LOB_REWARD_PV || p.inv_penalty != 0 || p.exec_pen_milli != 0 ||
           p.mm_space != LOB_MM_SPREAD_SKEW || p.msgs_sysmem != 0 || p.msg16 != 0 || p.pv_ref != LOB_PV_TOUCH ||
           p.exec_dir == 0;
}

cudaError_t launch_k(int K, bool trace, int n_list, int wpb, bool persistent, int n_sm, cudaStream_t s,
                     const KParams &p) {
    if (p.n_agents > 2) {
        // several agents per type: the wide kernel with a per-warp agent block
        // (messages staged TILE records at a time)
        wpb = wpb < max_wpb_ma(K) ? wpb : max_wpb_ma(K);
        int blocks = (n_list + wpb - 1) / wpb;
        if (persistent) blocks = std::min(blocks, n_sm * std::max(1, 32 / wpb));
        const size_t smem = (size_t)wpb * (warp_smem_bytes(K) + sizeof(AgentSmem));
        switch (K) {
            case 1: return launch_steps_ma_1(trace, blocks, 32 * wpb, smem, s, p);
            case 2: return launch_steps_ma_2(trace, blocks, 32 * wpb, smem, s, p);
            case 4: return launch_steps_ma_4(trace, blocks, 32 * wpb, smem, s, p);
            case 8: return launch_steps_ma_8(trace, blocks, 32 * wpb, smem, s, p);
            case 16: return launch_steps_ma_16(trace, blocks, 32 * wpb, smem, s, p);
            default: return launch_steps_ma_32(trace, blocks, 32 * wpb, smem, s, p);
        }
    }
    // the extended kernel when episode mode, a reward variant or another
    // action space is on
    const bool ext = kernel_ext(p);
    // message tiles of 16 or 64 records: the plain kernel's own instances
    // (wide register budget); every other launch stages TILE records
    const int T = (!trace && !ext && p.tile != 0 && p.tile != TILE) ? p.tile : TILE;
    wpb = wpb < max_wpb(K, T) ? wpb : max_wpb(K, T);
    int blocks = (n_list + wpb - 1) / wpb;
    if (persistent) blocks = std::min(blocks, n_sm * std::max(1, 32 / wpb));
    const size_t smem = (size_t)wpb * (warp_smem_bytes(K) + tile_ext_bytes(T));
    // the wide register budget when every block is resident at once (one wave)
    const bool one_wave = blocks <= wide_blocks_per_sm(K, ext, wpb, smem, T) * n_sm;
    const bool wide = one_wave || T != TILE;
    KParams q = p;
    q.tile = T;
    q.book_prefetch = one_wave ? 1 : 0;   // every env starts at once: fetch the books early
    switch (K) {
        case 1: return launch_steps_1(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
        case 2: return launch_steps_2(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
        case 4: return launch_steps_4(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
        case 8: return launch_steps_8(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
        case 16: return launch_steps_16(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
        default: return launch_steps_32(trace, ext, wide, blocks, 32 * wpb, smem, s, q);
    }
}

}  // namespace

struct lob_handle {
    lob_config cfg;
    int dev = 0;
    int D = 0;
    std::vector<int> caps;
    // device state
    unsigned char *d_books = nullptr;
    long long *d_book_off = nullptr;
    long long *d_canon_off = nullptr;
    int *d_caps = nullptr;
    EnvState *d_state = nullptr;
    long long *d_counters = nullptr;
    unsigned long long *d_seeds = nullptr;
    int *d_status = nullptr;
    float *d_obs = nullptr;
    long long *d_rew = nullptr;
    unsigned char *d_done = nullptr;
    int *d_act = nullptr;
    int *d_env_list = nullptr;
    int *d_queue = nullptr;
    bool uniform_cap = false;
    bool custom_order = false;
    long long uni_block = 0;
    std::vector<int> env_list_h;
    int class_begin[NCLASS] = {0, 0, 0, 0};
    int class_count[NCLASS] = {0, 0, 0, 0};
    long long book_bytes = 0, canon_bytes = 0;
    // bound messages
    const lob_msg *msgs = nullptr;
    const int64_t *offsets = nullptr;
    int32_t win_steps = 0;
    int64_t stride = 0;
    int32_t cursor = 0;
    int32_t t = 0;
    bool reset_done = false;
    // trace
    lob_fill *d_fills = nullptr;
    int32_t fill_cap = 0;
    int32_t *d_fill_counts = nullptr;
    unsigned char *d_snaps = nullptr;
    int64_t snap_cap = 0;
    int64_t *d_snap_count = nullptr;
    // launch shape
    int wpb = 4;
    int persistent = 0;
    int tpe = 32;                // threads per env: 64 runs the plain step with one warp per book side
    int tile = TILE;             // records per staged message tile (16, 32 or 64)
    long long wait_budget = 0;   // 0: the default bound
    int hold_first = 0;          // failure-detection test hook (next launch only)
    int n_sm = 0;
    int64_t launches = 0;
    int multi_split[NCLASS] = {0, 0, 0, 0, 0, 0};   // persistent == 2: warps per block of each class (0: derived)
    // per-class streams: several capacity classes run concurrently (fork/join
    // with events, so the pattern also captures into a CUDA graph)
    cudaStream_t cls_stream[NCLASS] = {};
    cudaEvent_t ev_fork = nullptr, cls_done[NCLASS] = {};
    int n_active_classes = 0;
    // host-step staging
    lob_msg *d_stage_msgs = nullptr;
    size_t stage_cap = 0;
    int64_t *d_stage_off = nullptr;
    int32_t *d_stage_act = nullptr;
    // pipelined host steps: two staging slots filled on a copy stream
    struct AsyncSlot {
        lob_msg *d_msgs = nullptr;
        size_t cap = 0;
        int64_t *d_off = nullptr;
        int32_t *d_act = nullptr;
        int64_t *h_off = nullptr;              // pinned, the rebased offsets
        cudaEvent_t in_ready = nullptr;        // copies of this slot done
        cudaEvent_t free = nullptr;            // the step that read this slot done
    } aslot[2];
    cudaStream_t copy_stream = nullptr;
    int64_t async_calls = 0;
    const void *mapped_ok[6] = {};   // last host pointers found mapped, per argument
    bool msg16 = false;   // the bound background stream holds 16-byte compact records
    // several agents per type: per-agent state [n_envs][n_agents]
    AgentState *d_agents = nullptr;
    // episode mode (one shared stream, snapshot table, auto-reset)
    bool ep_mode = false;
    const int64_t *ep_off = nullptr;
    int64_t n_data_steps = 0;
    int32_t n_starts = 0;
    lob_start *d_ep_starts = nullptr;
    int32_t *d_ep_levels = nullptr;
    unsigned char *d_ep_images = nullptr;
    float *d_ep_obs = nullptr;
};

static int cuda_ok(cudaError_t e) { return e == cudaSuccess ? LOB_OK : LOB_ECUDA; }

static void free_all(lob_handle *h) {
    for (auto &a : h->aslot) {
        if (a.d_msgs) cudaFree(a.d_msgs);
        if (a.d_off) cudaFree(a.d_off);
        if (a.d_act) cudaFree(a.d_act);
        if (a.h_off) cudaFreeHost(a.h_off);
        if (a.in_ready) cudaEventDestroy(a.in_ready);
        if (a.free) cudaEventDestroy(a.free);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (int k = 0; k < NCLASS; k++) {
        if (h->cls_stream[k]) cudaStreamDestroy(h->cls_stream[k]);
        if (h->cls_done[k]) cudaEventDestroy(h->cls_done[k]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    void *ptrs[] = {h->d_books, h->d_book_off, h->d_canon_off, h->d_caps, h->d_state, h->d_counters,
                    h->d_seeds, h->d_status, h->d_obs, h->d_rew, h->d_done, h->d_act, h->d_env_list,
                    h->d_queue, h->d_stage_msgs, h->d_stage_off, h->d_stage_act, h->d_ep_starts,
                    h->d_ep_levels, h->d_ep_images, h->d_ep_obs, h->d_agents};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

extern "C" {

int32_t lob_obs_dim(const lob_config *cfg) {
    if (!cfg) return 0;
    return cfg->n_agents > 0 ? 4 * cfg->top_levels + 5 : 0;
}

const char *lob_strerror(int code) {
    switch (code) {
        case LOB_OK: return "ok";
        case LOB_EINVAL: return "invalid argument or action";
        case LOB_ENOMEM: return "device allocation failed";
        case LOB_ECUDA: return "CUDA call failed";
        case LOB_ETIMEOUT: return "bounded device wait expired";
        case LOB_ECAPACITY: return "size exceeds supported capacity";
        case LOB_EBADMSG: return "malformed message (skipped)";
        case LOB_ESTATE: return "call out of order";
        case LOB_ECHECK: return "checked build: an index bound or book invariant failed";
        default: return "unknown status";
    }
}

int lob_create(const lob_config *cfg, const int32_t *h_caps, lob_handle **out) {
    if (!cfg || !out) return LOB_EINVAL;
    *out = nullptr;
    const lob_config &c = *cfg;
    if (c.n_envs < 1 || c.n_agents < 0 || c.n_agents % 2 != 0 || c.n_agents > 2 * LOB_MAX_PER_TYPE ||
        c.top_levels < 1 || c.top_levels > LMAX ||
        c.episode_len < 1 || c.mm_lot < 1 || c.exec_target < 0 ||
        (c.exec_dir != LOB_SELL && c.exec_dir != LOB_BUY && c.exec_dir != 0) ||
        (c.action_mode != LOB_ACT_HOST && c.action_mode != LOB_ACT_RANDOM) || c.trace < 0 || c.trace > 3 ||
        c.warps_per_block < 0 || c.warps_per_block > 8)
        return LOB_EINVAL;
    if (c.reward_mode < LOB_REWARD_PV || c.reward_mode > LOB_REWARD_SPOONER || c.spooner_lambda_pct < 0 ||
        c.spooner_lambda_pct > 100 || c.inv_penalty < 0 || c.exec_penalty_milli < 0 ||
        c.mm_space < LOB_MM_SPREAD_SKEW || c.mm_space > LOB_MM_DIRECTIONAL || c.pv_ref < LOB_PV_TOUCH ||
        c.pv_ref > LOB_PV_MID)
        return LOB_EINVAL;
    for (int i = 0; i < 2; i++)
        if (c.reserved[i] != 0) return LOB_EINVAL;
    std::vector<int> caps((size_t)c.n_envs);
    for (int e = 0; e < c.n_envs; e++) {
        const int cp = h_caps ? h_caps[e] : c.cap_per_side;
        if (cp < 1) return LOB_EINVAL;
        if (cp > LOB_MAX_CAP) return LOB_ECAPACITY;
        caps[(size_t)e] = cp;
    }
    lob_handle *h = new (std::nothrow) lob_handle();
    if (!h) return LOB_ENOMEM;
    h->cfg = c;
    h->caps = caps;
    h->D = lob_obs_dim(cfg);
    if (c.warps_per_block > 0) h->wpb = c.warps_per_block;
    if (cudaGetDevice(&h->dev) != cudaSuccess || ensure_optin() != cudaSuccess) { delete h; return LOB_ECUDA; }
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev);

    // group envs by capacity class; book blocks are 256-byte aligned
    std::vector<int> list;
    std::vector<long long> off((size_t)c.n_envs), coff((size_t)c.n_envs);
    long long acc = 0, cacc = 0;
    for (int k = 0; k < NCLASS; k++) {
        h->class_begin[k] = (int)list.size();
        for (int e = 0; e < c.n_envs; e++)
            if (class_of(caps[(size_t)e]) == k) list.push_back(e);
        h->class_count[k] = (int)list.size() - h->class_begin[k];
    }
    for (int e = 0; e < c.n_envs; e++) {
        const int slots = 32 * CLASS_K[class_of(caps[(size_t)e])];
        off[(size_t)e] = acc;
        acc += ((48LL * slots + 255) / 256) * 256;
        coff[(size_t)e] = cacc;
        cacc += 8 + 48LL * caps[(size_t)e];
    }
    h->book_bytes = acc;
    h->canon_bytes = cacc;
    h->uniform_cap = !h_caps;
    h->uni_block = ((48LL * 32 * CLASS_K[class_of(c.cap_per_side < 1 ? 1 : (c.cap_per_side > LOB_MAX_CAP ? LOB_MAX_CAP : c.cap_per_side))] + 255) / 256) * 256;
    const size_t n = (size_t)c.n_envs;
    const int A = c.n_agents;
    bool fail = false;
    auto alloc = [&](void **p, size_t b) {
        if (fail) return;
        if (cudaMalloc(p, b ? b : 1) != cudaSuccess) fail = true;
    };
    alloc((void **)&h->d_books, (size_t)acc);
    alloc((void **)&h->d_book_off, n * 8);
    alloc((void **)&h->d_canon_off, n * 8);
    alloc((void **)&h->d_caps, n * 4);
    alloc((void **)&h->d_state, n * sizeof(EnvState));
    alloc((void **)&h->d_counters, n * 8 * LOB_NCOUNTERS);
    alloc((void **)&h->d_seeds, n * 8);
    alloc((void **)&h->d_status, 4);
    alloc((void **)&h->d_obs, n * (size_t)(A * h->D) * 4);
    alloc((void **)&h->d_rew, n * (size_t)A * 8);
    alloc((void **)&h->d_done, n);
    alloc((void **)&h->d_act, n * (size_t)(A > 2 ? A : 2) * 4);
    if (A > 2) alloc((void **)&h->d_agents, n * (size_t)A * sizeof(AgentState));
    alloc((void **)&h->d_env_list, n * 4);
    alloc((void **)&h->d_queue, NCLASS * 4);
    if (fail) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return LOB_ENOMEM;
    }
    int rc = LOB_OK;
    rc |= cuda_ok(cudaMemcpy(h->d_book_off, off.data(), n * 8, cudaMemcpyHostToDevice));
    rc |= cuda_ok(cudaMemcpy(h->d_canon_off, coff.data(), n * 8, cudaMemcpyHostToDevice));
    rc |= cuda_ok(cudaMemcpy(h->d_caps, caps.data(), n * 4, cudaMemcpyHostToDevice));
    rc |= cuda_ok(cudaMemcpy(h->d_env_list, list.data(), n * 4, cudaMemcpyHostToDevice));
    h->env_list_h = list;
    for (int k = 0; k < NCLASS; k++) h->n_active_classes += h->class_count[k] > 0;
    if (h->n_active_classes > 1) {
        rc |= cuda_ok(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        // larger classes (longer per-message chains) on higher-priority streams:
        // the block scheduler places their blocks first
        int prio_least = 0, prio_greatest = 0;
        rc |= cuda_ok(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
        for (int k = 0; k < NCLASS; k++) {
            if (h->class_count[k] == 0) continue;
            const int prio = std::max(prio_greatest, prio_least - k);
            rc |= cuda_ok(cudaStreamCreateWithPriority(&h->cls_stream[k], cudaStreamNonBlocking, prio));
            rc |= cuda_ok(cudaEventCreateWithFlags(&h->cls_done[k], cudaEventDisableTiming));
        }
    }
    rc |= cuda_ok(cudaMemset(h->d_status, 0, 4));
    rc |= cuda_ok(cudaMemset(h->d_obs, 0, n * (size_t)(A * h->D) * 4));
    rc |= cuda_ok(cudaMemset(h->d_rew, 0, n * (size_t)A * 8 + (A == 0)));
    rc |= cuda_ok(cudaMemset(h->d_done, 0, n));
    if (rc != LOB_OK) {
        free_all(h);
        delete h;
        return LOB_ECUDA;
    }
    *out = h;
    return LOB_OK;
}

int lob_destroy(lob_handle *h) {
    if (!h) return LOB_EINVAL;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return LOB_OK;
}

static int load_messages(lob_handle *h, const void *d_msgs, const int64_t *d_offsets, int32_t n_steps, int64_t stride,
                         bool msg16) {
    if (!h || !d_offsets || n_steps < 0 || stride < (int64_t)n_steps + 1) return LOB_EINVAL;
    if (((uintptr_t)d_msgs & 15u) != 0) return LOB_EINVAL;   // bulk copies start on 16-byte boundaries
    if (!d_msgs && n_steps > 0) {
        // an all-empty window may pass a NULL message pointer; offsets still needed
    }
    if (h->ep_mode) h->reset_done = false;   // leaving episode mode: the books need a reset
    h->ep_mode = false;
    h->msg16 = msg16;
    h->msgs = static_cast<const lob_msg *>(d_msgs);
    h->offsets = d_offsets;
    h->win_steps = n_steps;
    h->stride = stride;
    h->cursor = 0;
    return LOB_OK;
}

int lob_load_messages(lob_handle *h, const lob_msg *d_msgs, const int64_t *d_offsets, int32_t n_steps,
                      int64_t stride) {
    return load_messages(h, d_msgs, d_offsets, n_steps, stride, false);
}

int lob_load_messages16(lob_handle *h, const lob_msg16 *d_msgs, const int64_t *d_offsets, int32_t n_steps,
                        int64_t stride) {
    return load_messages(h, d_msgs, d_offsets, n_steps, stride, true);
}

}  // extern "C"

// zero the state of every env
__global__ void k_reset(EnvState *st, long long *cnt, unsigned long long *seeds_dst,
                        const unsigned long long *seeds_src, int n, int start_px, float *obs, int A, int D,
                        int L, int exec_target, int exec_dir) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    // the task's side: configured, or drawn (then signed into the remaining target)
    const int dir = exec_dir != 0 ? exec_dir : drawn_task_side(seeds_src[e], 0);
    const long long rem = (exec_dir == 0 && dir == LOB_SELL) ? -(long long)exec_target : exec_target;
    for (int a = 0; a < A; a++) {
        float *o = obs + ((long long)e * A + a) * D;
        for (int f = 0; f < D; f++) o[f] = 0.0f;
        o[4 * L + 2] = 1.0f;                                   // time left T / T
        if (a < (A >> 1)) o[4 * L + 3] = __ll2float_rn(rem);  // remaining target (execution agents)
    }
    EnvState z;
    memset(&z, 0, sizeof(z));
    z.last_px = start_px;
    z.exec_dir = dir;
    st[e] = z;
    for (int i = 0; i < LOB_NCOUNTERS; i++) cnt[(long long)e * LOB_NCOUNTERS + i] = 0;
    seeds_dst[e] = seeds_src[e];
}

// Episode-start book images in the book block layout (priority order: px,
// qty int32 [2][S], then id, ts int64 [2][S]); one block per snapshot.
__global__ void k_ep_images(const lob_start *starts, const int *levels, int ls, int slots, long long block,
                            unsigned char *images) {
    const int j = blockIdx.x;
    const lob_start st = starts[j];
    unsigned char *blk = images + (long long)j * block;
    int *px = reinterpret_cast<int *>(blk);
    int *qt = px + 2 * slots;
    long long *id = reinterpret_cast<long long *>(blk + 16LL * slots);
    long long *ts = id + 2 * slots;
    for (int i = threadIdx.x; i < 2 * slots; i += blockDim.x) {
        const int sd = i / slots, q = i % slots;
        const int n = sd == 0 ? st.n_bid : st.n_ask;
        const bool live = q < n;
        const int *lv = levels + (((long long)j * 2 + sd) * ls + (live ? q : 0)) * 2;
        const long long idx = (sd == 0 ? 0 : st.n_bid) + q;   // bids, then asks, best first
        px[i] = live ? lv[0] : 0;
        qt[i] = live ? lv[1] : 0;
        id[i] = live ? LOB_INIT_ID + idx : 0;
        ts[i] = live ? idx : 0;
    }
}

// First observation of an episode started at each snapshot: its levels
// against anchor floor((bb + ba) / 2) (an empty side's touch is the last
// trade price), flat agents, time left 1, the full target for agent 0.
__global__ void k_ep_obs(const lob_start *starts, const int *levels, int ls, int A, int D, int L, int exec_target,
                         float *obs) {
    const int j = blockIdx.x;
    const lob_start st = starts[j];
    const int *bl = levels + (long long)j * 2 * ls * 2;
    const int *al = bl + ls * 2;
    const long long bb = st.n_bid > 0 ? bl[0] : st.last_px;
    const long long ba = st.n_ask > 0 ? al[0] : st.last_px;
    const long long s2 = bb + ba;
    const long long anchor = s2 >= 0 ? s2 / 2 : -((-s2 + 1) / 2);
    for (int i = threadIdx.x; i < A * D; i += blockDim.x) {
        const int a = i / D, f = i % D;
        float v = 0.0f;
        if (f < 4 * L) {
            const int sd = f >= 2 * L ? 1 : 0;
            const int lvl = (f - sd * 2 * L) >> 1;
            const int n = sd == 0 ? st.n_bid : st.n_ask;
            const int *lv = (sd == 0 ? bl : al) + lvl * 2;
            if (lvl < n) v = __ll2float_rn((f & 1) ? (long long)lv[1] : (long long)lv[0] - anchor);
        } else if (f == 4 * L + 2) {
            v = 1.0f;
        } else if (f == 4 * L + 3 && a < (A >> 1)) {
            v = __ll2float_rn(exec_target);
        }
        obs[(long long)j * A * D + i] = v;
    }
}

// Episode-mode reset: each env draws its first snapshot, copies its image
// into the env's book block and starts from it.
__global__ void k_reset_ep(EnvState *st, long long *cnt, unsigned long long *seeds_dst,
                           const unsigned long long *seeds_src, int n, unsigned char *books,
                           const long long *book_off, const unsigned char *images, long long block,
                           const lob_start *starts, int n_starts, const float *ep_obs, float *obs, int A, int D,
                           int L, int exec_dir) {
    const int e = blockIdx.x;
    if (e >= n) return;
    const unsigned long long seed = seeds_src[e];
    const unsigned j = bounded(sm_mix(step_key(seed, 0, LOB_TAG_EPISODE) + GAMMA), (unsigned)n_starts);
    const int dir = exec_dir != 0 ? exec_dir : drawn_task_side(seed, 0);
    const bool flip = exec_dir == 0 && dir == LOB_SELL;   // a drawn sell task: negative remaining target
    const int4 *src = reinterpret_cast<const int4 *>(images + (long long)j * block);
    int4 *dst = reinterpret_cast<int4 *>(books + book_off[e]);
    for (long long i = threadIdx.x; i < block / 16; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < A * D; i += blockDim.x) {
        const float v = ep_obs[(long long)j * A * D + i];
        obs[(long long)e * A * D + i] = (flip && i % D == 4 * L + 3 && i / D < (A >> 1)) ? -v : v;
    }
    if (threadIdx.x < LOB_NCOUNTERS) cnt[(long long)e * LOB_NCOUNTERS + threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        const lob_start S = starts[j];
        EnvState z;
        memset(&z, 0, sizeof(z));
        z.ts_next = S.n_bid + S.n_ask;
        z.last_px = S.last_px;
        z.n[0] = S.n_bid;
        z.n[1] = S.n_ask;
        z.ep_start = S.data_step;
        z.exec_dir = dir;
        st[e] = z;
        seeds_dst[e] = seed;
    }
}

__global__ void k_get_ep_start(const EnvState *st, int *out, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = st[e].ep_start;
}

// Several agents per type: [inv, cash, pv_prev, exec_done] per (env, agent).
__global__ void k_get_agents_ma(const AgentState *ag, long long *out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const AgentState x = ag[i];
    out[4 * i + 0] = x.inv; out[4 * i + 1] = x.cash; out[4 * i + 2] = x.pv_prev; out[4 * i + 3] = x.exec_done;
}

// 32-byte records -> 16-byte compact records; an id outside the 60-bit range
// sets *status to LOB_EINVAL (that record is written as malformed).
__global__ void k_pack16(const lob_msg *src, lob_msg16 *dst, long long n, int *status) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const lob_msg m = src[i];
    const bool valid = m.type >= LOB_ADD && m.type <= LOB_MARKET && (m.side == LOB_BUY || m.side == LOB_SELL);
    const bool fits = m.oid >= LOB_MSG16_ID_MIN && m.oid <= LOB_MSG16_ID_MAX;
    if (!fits && status) atomicExch(status, LOB_EINVAL);
    lob_msg16 r;
    r.px = m.px;
    r.qty = m.qty;
    const unsigned long long code = (valid && fits) ? (unsigned long long)m.type | (m.side == LOB_SELL ? 8ull : 0ull) : 0ull;
    r.word = (long long)(((unsigned long long)(fits ? m.oid : 0) << 4) | code);
    dst[i] = r;
}

// internal blocked layout -> canonical priority-ordered record per env
__global__ void k_get_book(const unsigned char *books, const long long *book_off, const long long *canon_off,
                           const int *caps, const EnvState *st, unsigned char *out, int n) {
    const int e = blockIdx.x;
    if (e >= n) return;
    const int C = caps[e];
    int slots = 32;
    while (slots < C) slots *= 2;
    const unsigned char *blk = books + book_off[e];
    unsigned char *rec = out + canon_off[e];
    int *n2 = reinterpret_cast<int *>(rec);
    int *px = n2 + 2;
    int *qt = px + 2 * C;
    long long *id = reinterpret_cast<long long *>(rec + 8 + 16LL * C);
    long long *ts = id + 2 * C;
    const int *ipx = reinterpret_cast<const int *>(blk);
    const int *iqt = ipx + 2 * slots;
    const long long *iid = reinterpret_cast<const long long *>(blk + 16LL * slots);
    const long long *its = reinterpret_cast<const long long *>(blk + 32LL * slots);
    if (threadIdx.x == 0) { n2[0] = st[e].n[0]; n2[1] = st[e].n[1]; }
    for (int i = threadIdx.x; i < 2 * C; i += blockDim.x) {
        const int s = i / C, j = i % C;
        const bool live = j < st[e].n[s];
        px[i] = live ? ipx[s * slots + j] : 0;
        qt[i] = live ? iqt[s * slots + j] : 0;
        id[i] = live ? iid[s * slots + j] : 0;
        ts[i] = live ? its[s * slots + j] : 0;
    }
}

// Resting orders of all envs (both sides) added to *acc: a block-wide sum,
// then one atomic per block.
__global__ void k_live_orders(const EnvState *st, int n, long long *acc) {
    long long v = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        v += (long long)st[e].n[0] + st[e].n[1];
    v = warp_sum(v);
    __shared__ long long part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        atomicAdd(reinterpret_cast<unsigned long long *>(acc), (unsigned long long)t);
    }
}

__global__ void k_get_agents(const EnvState *st, long long *out, int n, int A, int misc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const EnvState &s = st[e];
    if (misc) {
        out[e * 4 + 0] = s.ts_next; out[e * 4 + 1] = s.seq_next;
        out[e * 4 + 2] = s.last_px; out[e * 4 + 3] = s.t;
        return;
    }
    for (int a = 0; a < A; a++) {
        long long *o = out + ((long long)e * A + a) * 4;
        o[0] = s.inv[a]; o[1] = s.cash[a]; o[2] = s.pv_prev[a]; o[3] = a == 0 ? s.exec_done : 0;
    }
}

// Whether n more steps may run: episode mode never runs out; otherwise the
// bound window and the episode bound the steps.
static bool steps_left(const lob_handle *h, int n) {
    if (!h->reset_done) return false;
    if (h->ep_mode) return (int64_t)h->t + n <= 0x7fffffffLL;
    return h->offsets && h->cursor + n <= h->win_steps && h->t + n <= h->cfg.episode_len;
}
static const int64_t *step_offsets(const lob_handle *h) { return h->ep_mode ? h->ep_off : h->offsets; }

// The step kernel's parameters for n_steps steps from the handle's state.
static KParams base_params(lob_handle *h, const lob_msg *msgs, const int64_t *offsets, int64_t stride, int k0,
                           int n_steps, const int32_t *d_actions, long long act_step_stride, float *obs,
                           long long *rew, unsigned char *done, bool msgs_sysmem, bool msg16) {
    const lob_config &c = h->cfg;
    KParams p;
    memset(&p, 0, sizeof(p));
    p.books = h->d_books; p.book_off = h->d_book_off; p.caps = h->d_caps; p.st = h->d_state;
    p.counters = h->d_counters; p.seeds = h->d_seeds; p.status = h->d_status;
    p.msgs = reinterpret_cast<const DevMsg *>(msgs); p.offsets = reinterpret_cast<const long long *>(offsets);
    p.off_stride = stride; p.k0 = k0;
    p.actions = d_actions; p.act_step_stride = act_step_stride; p.action_mode = c.action_mode;
    p.obs = obs; p.rew = rew; p.done = done; p.act_out = nullptr;
    p.n_envs = c.n_envs; p.n_agents = c.n_agents; p.L = c.top_levels; p.T = c.episode_len;
    p.mm_lot = c.mm_lot; p.exec_target = c.exec_target; p.exec_dir = c.exec_dir; p.D = h->D;
    p.t0 = h->t; p.n_steps = n_steps;
    p.fills = (c.trace & 1) ? h->d_fills : nullptr; p.fill_cap = h->fill_cap;
    p.fill_counts = (c.trace & 1) ? h->d_fill_counts : nullptr;
    p.snaps = (c.trace & 2) ? h->d_snaps : nullptr; p.snap_cap = h->snap_cap;
    p.snap_count = (c.trace & 2) ? reinterpret_cast<long long *>(h->d_snap_count) : nullptr;
    p.wait_budget = h->wait_budget > 0 ? h->wait_budget : DEFAULT_WAIT_BUDGET;
    p.drain_budget = DEFAULT_WAIT_BUDGET;
    p.hold_first = h->hold_first;
    h->hold_first = 0;   // one launch only
    p.exec_q0 = exec_lot(c);
    set_rewards(p, c);
    p.agents = h->d_agents;
    p.msgs_sysmem = msgs_sysmem ? 1 : 0;
    p.msg16 = msg16 ? 1 : 0;
    p.tile = h->tile;
    if (h->ep_mode) {
        p.ep_mode = 1;
        p.n_starts = h->n_starts;
        p.ep_block = h->uni_block;
        p.ep_starts = h->d_ep_starts;
        p.ep_images = h->d_ep_images;
        p.ep_obs = h->d_ep_obs;
    }
    return p;
}

static int launch_steps(lob_handle *h, const lob_msg *msgs, const int64_t *offsets, int64_t stride, int k0,
                        int n_steps, const int32_t *d_actions, long long act_step_stride, float *obs,
                        long long *rew, unsigned char *done, cudaStream_t s, bool msgs_sysmem = false,
                        bool msg16 = false) {
    const lob_config &c = h->cfg;
    KParams p = base_params(h, msgs, offsets, stride, k0, n_steps, d_actions, act_step_stride, obs, rew, done,
                            msgs_sysmem, msg16);
    const int wpb = h->wpb;
    if (h->persistent) {
        if (cudaMemsetAsync(h->d_queue, 0, NCLASS * 4, s) != cudaSuccess) return LOB_ECUDA;
    }
    if (h->persistent == 2 && p.fills == nullptr && p.snaps == nullptr && c.n_agents <= 2 && !kernel_ext(p) &&
        h->class_count[NCLASS - 1] == 0) {
        // one persistent kernel over every class (steps_multi.cu)
        MultiLayout m;
        memset(&m, 0, sizeof(m));
        int nw = 0;
        size_t off = 0;
        for (int k = MULTI_CLASSES - 1; k >= 0; k--)   // largest carve-outs first
            for (int i = 0; i < h->multi_split[k] && nw < 8; i++) {
                m.cls[nw] = k;
                m.off[nw] = (int)off;
                off += warp_smem_bytes(CLASS_K[k]);
                nw++;
            }
        m.off[nw] = (int)off;
        for (int k = 0; k < MULTI_CLASSES; k++) {
            m.begin[k] = h->class_begin[k];
            m.count[k] = h->class_count[k];
        }
        m.steal = 1;
        static bool opted[64];
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !opted[dev]) {
            if (optin_steps_multi(SMEM_PER_BLOCK_MAX) != cudaSuccess) return LOB_ECUDA;
            opted[dev] = true;
        }
        const int per_sm = std::max(1, multi_blocks_per_sm(32 * nw, off));
        p.env_list = h->d_env_list;
        p.uni_cap = 0;
        p.uni_block = 0;
        p.queue = h->d_queue;
        p.n_list = c.n_envs;
        h->launches++;
        return launch_steps_multi(per_sm * h->n_sm, 32 * nw, off, s, p, m) == cudaSuccess ? LOB_OK : LOB_ECUDA;
    }
    const bool fork = h->n_active_classes > 1;
    if (fork && cudaEventRecord(h->ev_fork, s) != cudaSuccess) return LOB_ECUDA;
    // the largest class first: its envs have the longest per-message chains
    for (int k = NCLASS - 1; k >= 0; k--) {
        const int cnt = h->class_count[k];
        if (cnt == 0) continue;
        cudaStream_t ks = s;
        if (fork) {
            ks = h->cls_stream[k];
            if (cudaStreamWaitEvent(ks, h->ev_fork, 0) != cudaSuccess) return LOB_ECUDA;
        }
        const bool uniform = cnt == c.n_envs && h->uniform_cap && !h->custom_order;
        p.env_list = uniform ? nullptr : h->d_env_list + h->class_begin[k];
        p.uni_cap = uniform ? c.cap_per_side : 0;
        p.uni_block = uniform ? h->uni_block : 0;
        p.n_list = cnt;
        p.queue = h->persistent ? h->d_queue + k : nullptr;
        h->launches++;
        const int K = CLASS_K[k];
        if (h->tpe == 64 && !h->persistent && p.fills == nullptr && p.snaps == nullptr && !kernel_ext(p) &&
            (c.n_agents == 0 || c.n_agents == 2) && (K == 2 || K == 4 || K == 8) && !p.hold_first) {
            // two warps per env, one block per env (lob_split.cuh)
            static bool opted[3][64];
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LOB_ECUDA;
            const int ki = K == 2 ? 0 : (K == 4 ? 1 : 2);
            const size_t smem = split_pair_bytes(K);
            if (!opted[ki][dev]) {
                if (optin_steps_split(K, smem) != cudaSuccess) return LOB_ECUDA;
                opted[ki][dev] = true;
            }
            KParams q = p;
            q.book_prefetch = cnt <= 7 * h->n_sm ? 1 : 0;   // one wave: fetch the books early
            if (launch_steps_split(K, cnt, 64, smem, ks, q) != cudaSuccess) return LOB_ECUDA;
        } else if (launch_k(K, p.fills != nullptr || p.snaps != nullptr, cnt, wpb, h->persistent != 0, h->n_sm, ks,
                            p) != cudaSuccess) {
            return LOB_ECUDA;
        }
        if (fork && cudaEventRecord(h->cls_done[k], ks) != cudaSuccess) return LOB_ECUDA;
    }
    if (fork)
        for (int k = 0; k < NCLASS; k++)
            if (h->class_count[k] && cudaStreamWaitEvent(s, h->cls_done[k], 0) != cudaSuccess) return LOB_ECUDA;
    return LOB_OK;
}

extern "C" {

static int set_episodes(lob_handle *h, const void *d_msgs, const int64_t *d_step_offsets, int64_t n_data_steps,
                        const lob_start *h_starts, const int32_t *h_levels, int32_t levels_per_side, int64_t n_starts,
                        bool msg16) {
    if (!h || !d_step_offsets || !h_starts || !h_levels || levels_per_side < 1 || n_starts < 1 ||
        n_starts > 0x7fffffffLL || n_data_steps < h->cfg.episode_len || !h->uniform_cap ||
        ((uintptr_t)d_msgs & 15u) != 0)
        return LOB_EINVAL;
    const int cap = h->cfg.cap_per_side, T = h->cfg.episode_len;
    const int ls = levels_per_side;
    for (int64_t j = 0; j < n_starts; j++) {
        const lob_start &S = h_starts[j];
        if (S.data_step < 0 || (int64_t)S.data_step + T > n_data_steps) return LOB_EINVAL;
        if (S.n_bid < 0 || S.n_ask < 0 || S.n_bid > ls || S.n_ask > ls || S.n_bid > cap || S.n_ask > cap)
            return LOB_EINVAL;
        const int32_t *bl = h_levels + (size_t)j * 2 * ls * 2, *al = bl + (size_t)ls * 2;
        for (int i = 0; i < S.n_bid; i++)
            if (bl[2 * i + 1] < 1 || (i > 0 && bl[2 * i] >= bl[2 * i - 2])) return LOB_EINVAL;
        for (int i = 0; i < S.n_ask; i++)
            if (al[2 * i + 1] < 1 || (i > 0 && al[2 * i] <= al[2 * i - 2])) return LOB_EINVAL;
        if (S.n_bid > 0 && S.n_ask > 0 && bl[0] >= al[0]) return LOB_EINVAL;
    }
    void *old[] = {h->d_ep_starts, h->d_ep_levels, h->d_ep_images, h->d_ep_obs};
    if (cudaDeviceSynchronize() != cudaSuccess) return LOB_ECUDA;
    for (void *p : old)
        if (p) cudaFree(p);
    h->d_ep_starts = nullptr; h->d_ep_levels = nullptr; h->d_ep_images = nullptr; h->d_ep_obs = nullptr;
    h->ep_mode = false;
    h->reset_done = false;
    const size_t A = (size_t)h->cfg.n_agents, D = (size_t)h->D;
    const size_t lv_bytes = (size_t)n_starts * 2 * ls * 2 * 4;
    if (cudaMalloc(&h->d_ep_starts, (size_t)n_starts * sizeof(lob_start)) != cudaSuccess ||
        cudaMalloc(&h->d_ep_levels, lv_bytes) != cudaSuccess ||
        cudaMalloc(&h->d_ep_images, (size_t)n_starts * (size_t)h->uni_block) != cudaSuccess ||
        cudaMalloc(&h->d_ep_obs, (size_t)n_starts * (A * D > 0 ? A * D : 1) * 4) != cudaSuccess)
        return LOB_ENOMEM;
    if (cudaMemcpy(h->d_ep_starts, h_starts, (size_t)n_starts * sizeof(lob_start), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(h->d_ep_levels, h_levels, lv_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return LOB_ECUDA;
    const int slots = 32 * CLASS_K[class_of(cap)];   // pool slots per side of this capacity
    k_ep_images<<<(unsigned)n_starts, 128>>>(h->d_ep_starts, h->d_ep_levels, ls, slots, h->uni_block,
                                              h->d_ep_images);
    h->launches++;
    if (A > 0) {
        k_ep_obs<<<(unsigned)n_starts, 128>>>(h->d_ep_starts, h->d_ep_levels, ls, (int)A, (int)D,
                                               h->cfg.top_levels, h->cfg.exec_target, h->d_ep_obs);
        h->launches++;
    }
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return LOB_ECUDA;
    h->ep_mode = true;
    h->msg16 = msg16;
    h->msgs = static_cast<const lob_msg *>(d_msgs);
    h->ep_off = d_step_offsets;
    h->n_data_steps = n_data_steps;
    h->n_starts = (int32_t)n_starts;
    return LOB_OK;
}

int lob_set_episodes(lob_handle *h, const lob_msg *d_msgs, const int64_t *d_step_offsets, int64_t n_data_steps,
                     const lob_start *h_starts, const int32_t *h_levels, int32_t levels_per_side,
                     int64_t n_starts) {
    return set_episodes(h, d_msgs, d_step_offsets, n_data_steps, h_starts, h_levels, levels_per_side, n_starts, false);
}

int lob_set_episodes16(lob_handle *h, const lob_msg16 *d_msgs, const int64_t *d_step_offsets, int64_t n_data_steps,
                       const lob_start *h_starts, const int32_t *h_levels, int32_t levels_per_side,
                       int64_t n_starts) {
    return set_episodes(h, d_msgs, d_step_offsets, n_data_steps, h_starts, h_levels, levels_per_side, n_starts, true);
}

int lob_get_episode_starts(lob_handle *h, int32_t *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    const int n = h->cfg.n_envs;
    k_get_ep_start<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(h->d_state, d_out, n);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_reset(lob_handle *h, const uint64_t *d_env_seeds, void *stream) {
    if (!h || !d_env_seeds) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->cfg.n_envs;
    // a fresh episode has earned nothing and is not done (the reset observation's reward and flag)
    if ((h->cfg.n_agents > 0 &&
         cudaMemsetAsync(h->d_rew, 0, (size_t)n * h->cfg.n_agents * 8, s) != cudaSuccess) ||
        cudaMemsetAsync(h->d_done, 0, (size_t)n, s) != cudaSuccess)
        return LOB_ECUDA;
    if (h->ep_mode) {
        k_reset_ep<<<n, 128, 0, s>>>(h->d_state, h->d_counters, h->d_seeds,
                                     reinterpret_cast<const unsigned long long *>(d_env_seeds), n, h->d_books,
                                     h->d_book_off, h->d_ep_images, h->uni_block, h->d_ep_starts, h->n_starts,
                                     h->d_ep_obs, h->d_obs, h->cfg.n_agents, h->D, h->cfg.top_levels,
                                     h->cfg.exec_dir);
        h->launches++;
        if (cudaGetLastError() != cudaSuccess) return LOB_ECUDA;
        if (h->d_agents &&
            cudaMemsetAsync(h->d_agents, 0, (size_t)n * h->cfg.n_agents * sizeof(AgentState), s) != cudaSuccess)
            return LOB_ECUDA;
        h->t = 0;
        h->reset_done = true;
        return LOB_OK;
    }
    if (h->d_agents &&
        cudaMemsetAsync(h->d_agents, 0, (size_t)n * h->cfg.n_agents * sizeof(AgentState), s) != cudaSuccess)
        return LOB_ECUDA;
    k_reset<<<(n + 127) / 128, 128, 0, s>>>(h->d_state, h->d_counters, h->d_seeds,
                                             reinterpret_cast<const unsigned long long *>(d_env_seeds), n,
                                             h->cfg.start_px, h->d_obs, h->cfg.n_agents, h->D, h->cfg.top_levels,
                                             h->cfg.exec_target, h->cfg.exec_dir);
    h->launches++;
    if (cudaGetLastError() != cudaSuccess) return LOB_ECUDA;
    h->t = 0;
    h->reset_done = true;
    return LOB_OK;
}

int lob_step(lob_handle *h, const int32_t *d_actions, void *stream) {
    if (!h) return LOB_EINVAL;
    if (!steps_left(h, 1)) return LOB_ESTATE;
    if (h->cfg.n_agents > 0 && h->cfg.action_mode == LOB_ACT_HOST && !d_actions) return LOB_EINVAL;
    int rc = launch_steps(h, h->msgs, step_offsets(h), h->stride, h->cursor, 1, d_actions, 0, h->d_obs, h->d_rew,
                          h->d_done, (cudaStream_t)stream, false, h->msg16);
    if (rc != LOB_OK) return rc;
    h->cursor++;
    h->t++;
    return LOB_OK;
}

int lob_rollout(lob_handle *h, int32_t n_steps, const int32_t *d_actions, float *d_obs, int64_t *d_rewards,
                uint8_t *d_done, void *stream) {
    if (!h || n_steps < 1) return LOB_EINVAL;
    if (!steps_left(h, n_steps)) return LOB_ESTATE;
    if (h->cfg.n_agents > 0 && h->cfg.action_mode == LOB_ACT_HOST && !d_actions) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_steps(h, h->msgs, step_offsets(h), h->stride, h->cursor, n_steps, d_actions,
                          (long long)h->cfg.n_agents * h->cfg.n_envs, d_obs, reinterpret_cast<long long *>(d_rewards),
                          d_done, s, false, h->msg16);
    if (rc != LOB_OK) return rc;
    // keep the last step's outputs for lob_observe
    const size_t n = (size_t)h->cfg.n_envs, A = (size_t)h->cfg.n_agents, D = (size_t)h->D;
    const size_t last = (size_t)(n_steps - 1);
    if (d_obs && A) cudaMemcpyAsync(h->d_obs, d_obs + last * n * A * D, n * A * D * 4, cudaMemcpyDeviceToDevice, s);
    if (d_rewards && A) cudaMemcpyAsync(h->d_rew, d_rewards + last * n * A, n * A * 8, cudaMemcpyDeviceToDevice, s);
    if (d_done) cudaMemcpyAsync(h->d_done, d_done + last * n, n, cudaMemcpyDeviceToDevice, s);
    h->cursor += n_steps;
    h->t += n_steps;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_observe(lob_handle *h, float *d_obs, int64_t *d_rewards, uint8_t *d_done, void *stream) {
    if (!h) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->cfg.n_envs, A = (size_t)h->cfg.n_agents, D = (size_t)h->D;
    int rc = LOB_OK;
    if (d_obs && A) rc |= cuda_ok(cudaMemcpyAsync(d_obs, h->d_obs, n * A * D * 4, cudaMemcpyDeviceToDevice, s));
    if (d_rewards && A) rc |= cuda_ok(cudaMemcpyAsync(d_rewards, h->d_rew, n * A * 8, cudaMemcpyDeviceToDevice, s));
    if (d_done) rc |= cuda_ok(cudaMemcpyAsync(d_done, h->d_done, n, cudaMemcpyDeviceToDevice, s));
    return rc ? LOB_ECUDA : LOB_OK;
}

int lob_step_host(lob_handle *h, const lob_msg *h_msgs, const int64_t *h_offsets, const int32_t *h_actions,
                  float *h_obs, int64_t *h_rewards, uint8_t *h_done, void *stream) {
    if (!h || !h_offsets) return LOB_EINVAL;
    if (!h->reset_done || h->ep_mode || h->t >= h->cfg.episode_len) return LOB_ESTATE;
    const lob_config &c = h->cfg;
    if (c.n_agents > 0 && c.action_mode == LOB_ACT_HOST && !h_actions) return LOB_EINVAL;
    const int n = c.n_envs;
    const size_t na = (size_t)(c.n_agents > 2 ? c.n_agents : 2);   // action slots per env
    const int64_t base = h_offsets[0], total = h_offsets[n] - base;
    if (total < 0) return LOB_EINVAL;
    for (int e = 0; e < n; e++)
        if (h_offsets[e + 1] < h_offsets[e]) return LOB_EINVAL;
    if (total > 0 && !h_msgs) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if ((size_t)total > h->stage_cap) {
        if (h->d_stage_msgs) cudaFree(h->d_stage_msgs);
        h->d_stage_msgs = nullptr;
        size_t want = std::max((size_t)total, h->stage_cap * 2);
        if (cudaMalloc(&h->d_stage_msgs, want * sizeof(lob_msg)) != cudaSuccess) {
            h->stage_cap = 0;
            return LOB_ENOMEM;
        }
        h->stage_cap = want;
    }
    if (!h->d_stage_off) {
        if (cudaMalloc(&h->d_stage_off, ((size_t)n + 1) * 8) != cudaSuccess) return LOB_ENOMEM;
        if (cudaMalloc(&h->d_stage_act, (size_t)n * na * 4) != cudaSuccess) return LOB_ENOMEM;
    }
    int rc = LOB_OK;
    if (total > 0)
        rc |= cuda_ok(cudaMemcpyAsync(h->d_stage_msgs, h_msgs + base, (size_t)total * sizeof(lob_msg),
                                      cudaMemcpyHostToDevice, s));
    // offsets relative to the staged slice
    std::vector<int64_t> rel((size_t)n + 1);
    for (int e = 0; e <= n; e++) rel[(size_t)e] = h_offsets[e] - base;
    rc |= cuda_ok(cudaMemcpyAsync(h->d_stage_off, rel.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (c.n_agents > 0 && c.action_mode == LOB_ACT_HOST)
        rc |= cuda_ok(cudaMemcpyAsync(h->d_stage_act, h_actions, (size_t)n * c.n_agents * 4, cudaMemcpyHostToDevice,
                                      s));
    if (rc != LOB_OK) return LOB_ECUDA;
    rc = launch_steps(h, h->d_stage_msgs, h->d_stage_off, 1, 0, 1, h->d_stage_act, 0, h->d_obs, h->d_rew,
                      h->d_done, s);
    if (rc != LOB_OK) return rc;
    h->t++;
    const size_t A = (size_t)c.n_agents, D = (size_t)h->D;
    if (h_obs && A) rc |= cuda_ok(cudaMemcpyAsync(h_obs, h->d_obs, (size_t)n * A * D * 4, cudaMemcpyDeviceToHost, s));
    if (h_rewards && A) rc |= cuda_ok(cudaMemcpyAsync(h_rewards, h->d_rew, (size_t)n * A * 8, cudaMemcpyDeviceToHost, s));
    if (h_done) rc |= cuda_ok(cudaMemcpyAsync(h_done, h->d_done, (size_t)n, cudaMemcpyDeviceToHost, s));
    rc |= cuda_ok(cudaStreamSynchronize(s));
    if (rc != LOB_OK) return LOB_ECUDA;
    return LOB_OK;
}

// Whether p is page-locked host memory mapped at the same device address;
// the last answer per argument slot is remembered.
static bool host_mapped(lob_handle *h, int slot, const void *p) {
    if (!p) return false;
    if (h->mapped_ok[slot] == p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const bool ok = at.type == cudaMemoryTypeHost && at.devicePointer == p;
    if (ok) h->mapped_ok[slot] = p;
    return ok;
}

// The pipelined form of lob_step_host: inputs go up on the handle's copy
// stream into one of two staging slots while the previous step runs; the
// step waits for its slot's copies, and the outputs come back on `stream`.
int lob_step_host_async(lob_handle *h, const lob_msg *h_msgs, const int64_t *h_offsets, const int32_t *h_actions,
                        float *h_obs, int64_t *h_rewards, uint8_t *h_done, void *stream) {
    if (!h || !h_offsets) return LOB_EINVAL;
    if (!h->reset_done || h->ep_mode || h->t >= h->cfg.episode_len) return LOB_ESTATE;
    const lob_config &c = h->cfg;
    if (c.n_agents > 0 && c.action_mode == LOB_ACT_HOST && !h_actions) return LOB_EINVAL;
    const int n = c.n_envs;
    const int64_t base = h_offsets[0], total = h_offsets[n] - base;
    if (total < 0) return LOB_EINVAL;
    for (int e = 0; e < n; e++)
        if (h_offsets[e + 1] < h_offsets[e]) return LOB_EINVAL;
    if (total > 0 && !h_msgs) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    auto &a = h->aslot[h->async_calls & 1];
    const size_t na = (size_t)(c.n_agents > 2 ? c.n_agents : 2);
    const size_t A = (size_t)c.n_agents, D = (size_t)h->D;
    const bool want_act = c.n_agents > 0 && c.action_mode == LOB_ACT_HOST;
    // Zero-copy: when every buffer is page-locked host memory the GPU maps at
    // the same address, the step reads the messages, offsets and actions and
    // writes the outputs in host memory itself (over the coherent CPU-GPU
    // link), so a call costs one launch instead of a chain of copies.
    const bool zc = (total == 0 || (host_mapped(h, 0, h_msgs + base) && host_mapped(h, 1, h_msgs + h_offsets[n] - 1) &&
                                    ((uintptr_t)(h_msgs + base) & 15u) == 0)) &&
                    (!want_act || host_mapped(h, 2, h_actions)) && (!h_obs || !A || host_mapped(h, 3, h_obs)) &&
                    (!h_rewards || !A || host_mapped(h, 4, h_rewards)) && (!h_done || host_mapped(h, 5, h_done));
    if (!a.h_off) {
        if (cudaMallocHost(&a.h_off, ((size_t)n + 1) * 8) != cudaSuccess ||
            cudaEventCreateWithFlags(&a.in_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&a.free, cudaEventDisableTiming) != cudaSuccess)
            return LOB_ENOMEM;
    }
    // the step two calls back has used this slot (its offsets, read directly
    // or through their upload) once it is done
    if (cudaEventSynchronize(a.free) != cudaSuccess) return LOB_ECUDA;
    if (zc) {
        for (int e = 0; e <= n; e++) a.h_off[e] = h_offsets[e] - base;
        int rc = launch_steps(h, total > 0 ? h_msgs + base : nullptr, a.h_off, 1, 0, 1, want_act ? h_actions : nullptr,
                              0, A ? h_obs : nullptr, A ? reinterpret_cast<long long *>(h_rewards) : nullptr, h_done,
                              s, true);
        if (rc != LOB_OK) return rc;
        if (cudaEventRecord(a.free, s) != cudaSuccess) return LOB_ECUDA;
        h->t++;
        h->async_calls++;
        return LOB_OK;
    }
    if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return LOB_ECUDA;
    if (!a.d_off) {
        if (cudaMalloc(&a.d_off, ((size_t)n + 1) * 8) != cudaSuccess || cudaMalloc(&a.d_act, (size_t)n * na * 4) !=
            cudaSuccess)
            return LOB_ENOMEM;
    }
    if ((size_t)total > a.cap) {
        if (a.d_msgs) cudaFree(a.d_msgs);
        a.d_msgs = nullptr;
        const size_t want = std::max((size_t)total, a.cap * 2);
        if (cudaMalloc(&a.d_msgs, want * sizeof(lob_msg)) != cudaSuccess) {
            a.cap = 0;
            return LOB_ENOMEM;
        }
        a.cap = want;
    }
    for (int e = 0; e <= n; e++) a.h_off[e] = h_offsets[e] - base;
    int rc = LOB_OK;
    rc |= cuda_ok(cudaStreamWaitEvent(h->copy_stream, a.free, 0));
    if (total > 0)
        rc |= cuda_ok(cudaMemcpyAsync(a.d_msgs, h_msgs + base, (size_t)total * sizeof(lob_msg), cudaMemcpyHostToDevice,
                                      h->copy_stream));
    rc |= cuda_ok(cudaMemcpyAsync(a.d_off, a.h_off, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, h->copy_stream));
    if (c.n_agents > 0 && c.action_mode == LOB_ACT_HOST)
        rc |= cuda_ok(cudaMemcpyAsync(a.d_act, h_actions, (size_t)n * c.n_agents * 4, cudaMemcpyHostToDevice,
                                      h->copy_stream));
    rc |= cuda_ok(cudaEventRecord(a.in_ready, h->copy_stream));
    rc |= cuda_ok(cudaStreamWaitEvent(s, a.in_ready, 0));
    if (rc != LOB_OK) return LOB_ECUDA;
    rc = launch_steps(h, a.d_msgs, a.d_off, 1, 0, 1, a.d_act, 0, h->d_obs, h->d_rew, h->d_done, s);
    if (rc != LOB_OK) return rc;
    if (cudaEventRecord(a.free, s) != cudaSuccess) return LOB_ECUDA;
    h->t++;
    h->async_calls++;
    if (h_obs && A) rc |= cuda_ok(cudaMemcpyAsync(h_obs, h->d_obs, (size_t)n * A * D * 4, cudaMemcpyDeviceToHost, s));
    if (h_rewards && A) rc |= cuda_ok(cudaMemcpyAsync(h_rewards, h->d_rew, (size_t)n * A * 8, cudaMemcpyDeviceToHost, s));
    if (h_done) rc |= cuda_ok(cudaMemcpyAsync(h_done, h->d_done, (size_t)n, cudaMemcpyDeviceToHost, s));
    return rc == LOB_OK ? LOB_OK : LOB_ECUDA;
}

int lob_pack_messages16(const lob_msg *d_src, int64_t n, lob_msg16 *d_dst, int32_t *d_status, void *stream) {
    if (n < 0 || (n > 0 && (!d_src || !d_dst))) return LOB_EINVAL;
    if (n == 0) return LOB_OK;
    k_pack16<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_src, d_dst, n, d_status);
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int64_t lob_book_bytes(const lob_handle *h) { return h ? h->canon_bytes : 0; }

int lob_get_book(lob_handle *h, void *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    k_get_book<<<h->cfg.n_envs, 128, 0, (cudaStream_t)stream>>>(h->d_books, h->d_book_off, h->d_canon_off, h->d_caps,
                                                                 h->d_state, (unsigned char *)d_out, h->cfg.n_envs);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_get_counters(lob_handle *h, int64_t *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    return cuda_ok(cudaMemcpyAsync(d_out, h->d_counters, (size_t)h->cfg.n_envs * 8 * LOB_NCOUNTERS,
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

int lob_get_agents(lob_handle *h, int64_t *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    if (h->cfg.n_agents == 0) return LOB_OK;
    const int n = h->cfg.n_envs;
    if (h->d_agents) {
        const long long m = (long long)n * h->cfg.n_agents;
        k_get_agents_ma<<<(unsigned)((m + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
            h->d_agents, reinterpret_cast<long long *>(d_out), m);
        h->launches++;
        return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
    }
    k_get_agents<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(h->d_state, reinterpret_cast<long long *>(d_out),
                                                                     n, h->cfg.n_agents, 0);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_get_env_misc(lob_handle *h, int64_t *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    const int n = h->cfg.n_envs;
    k_get_agents<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(h->d_state, reinterpret_cast<long long *>(d_out),
                                                                     n, 0, 1);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_live_orders(lob_handle *h, int64_t *d_acc, void *stream) {
    if (!h || !d_acc) return LOB_EINVAL;
    const int n = h->cfg.n_envs;
    const int blocks = std::min((n + 255) / 256, 4 * std::max(h->n_sm, 1));
    k_live_orders<<<blocks, 256, 0, (cudaStream_t)stream>>>(h->d_state, n, reinterpret_cast<long long *>(d_acc));
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int lob_get_actions(lob_handle *h, int32_t *d_out, void *stream) {
    if (!h || !d_out) return LOB_EINVAL;
    if (h->cfg.n_agents == 0) return LOB_OK;
    if (h->d_agents)
        return cuda_ok(cudaMemcpy2DAsync(d_out, 4, reinterpret_cast<const char *>(h->d_agents) + offsetof(AgentState, act),
                                         sizeof(AgentState), 4, (size_t)h->cfg.n_envs * h->cfg.n_agents,
                                         cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return cuda_ok(cudaMemcpy2DAsync(d_out, 8, reinterpret_cast<const char *>(h->d_state) + offsetof(EnvState, act),
                                     sizeof(EnvState), 8, (size_t)h->cfg.n_envs, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

int lob_set_trace(lob_handle *h, lob_fill *d_fills, int32_t fill_cap, int32_t *d_fill_counts, void *d_snaps,
                  int64_t snap_cap, int64_t *d_snap_count) {
    if (!h || fill_cap < 0 || snap_cap < 0) return LOB_EINVAL;
    if ((d_fills == nullptr) != (d_fill_counts == nullptr)) return LOB_EINVAL;
    if ((d_snaps == nullptr) != (d_snap_count == nullptr)) return LOB_EINVAL;
    h->d_fills = d_fills;
    h->fill_cap = d_fills ? fill_cap : 0;
    h->d_fill_counts = d_fill_counts;
    h->d_snaps = (unsigned char *)d_snaps;
    h->snap_cap = d_snaps ? snap_cap : 0;
    h->d_snap_count = d_snap_count;
    h->cfg.trace = (d_fills ? 1 : 0) | (d_snaps ? 2 : 0);
    return LOB_OK;
}

int lob_sync(lob_handle *h, void *stream) {
    if (!h) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LOB_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, h->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LOB_ECUDA;
    if (st) cudaMemset(h->d_status, 0, 4);
    if (st & ST_TIMEOUT) return LOB_ETIMEOUT;
    if (st & ST_CHECK) return LOB_ECHECK;
    if (st & ST_BADACT) return LOB_EINVAL;
    if (st & ST_BADMSG) return LOB_EBADMSG;
    return LOB_OK;
}

int lob_set_launch(lob_handle *h, int32_t warps_per_block, int32_t persistent) {
    if (!h || warps_per_block < 1 || warps_per_block > 8 || persistent < 0 || persistent > 2) return LOB_EINVAL;
    h->wpb = warps_per_block;
    h->persistent = persistent;
    if (persistent == 2) {
        // default split: every class with envs gets warps in proportion to its
        // envs, at least one, warps_per_block in all (fewer if a block's
        // shared memory cannot hold them)
        int total = 0, present = 0;
        for (int k = 0; k < MULTI_CLASSES; k++) present += h->class_count[k] > 0;
        if (present > warps_per_block) return LOB_EINVAL;
        for (int k = 0; k < MULTI_CLASSES; k++) {
            h->multi_split[k] = h->class_count[k] > 0 ? 1 : 0;
            total += h->multi_split[k];
        }
        while (total < warps_per_block) {   // hand the rest out by envs per warp
            int best = -1;
            double bv = -1.0;
            for (int k = 0; k < MULTI_CLASSES; k++)
                if (h->multi_split[k] > 0) {
                    const double v = (double)h->class_count[k] * CLASS_K[k] / h->multi_split[k];
                    if (v > bv) { bv = v; best = k; }
                }
            h->multi_split[best]++;
            total++;
        }
        size_t smem = 0;
        for (int k = 0; k < MULTI_CLASSES; k++) smem += (size_t)h->multi_split[k] * warp_smem_bytes(CLASS_K[k]);
        while (smem > SMEM_PER_BLOCK_MAX) {   // drop warps from the biggest share
            int best = -1;
            for (int k = 0; k < MULTI_CLASSES; k++)
                if (h->multi_split[k] > 1 && (best < 0 || h->multi_split[k] > h->multi_split[best])) best = k;
            if (best < 0) return LOB_ECAPACITY;
            h->multi_split[best]--;
            smem -= warp_smem_bytes(CLASS_K[best]);
        }
    }
    return LOB_OK;
}

int lob_set_threads_per_env(lob_handle *h, int32_t threads) {
    if (!h || (threads != 32 && threads != 64)) return LOB_EINVAL;
    h->tpe = threads;
    return LOB_OK;
}

int lob_set_tile_records(lob_handle *h, int32_t records) {
    if (!h || (records != 16 && records != 32 && records != TILE_MAX)) return LOB_EINVAL;
    h->tile = records;
    return LOB_OK;
}

int lob_set_multi_split(lob_handle *h, const int32_t *warps_per_class) {
    if (!h || !warps_per_class) return LOB_EINVAL;
    int total = 0;
    size_t smem = 0;
    for (int k = 0; k < NCLASS; k++) {
        if (warps_per_class[k] < 0) return LOB_EINVAL;
        if (k >= MULTI_CLASSES && warps_per_class[k] != 0) return LOB_EINVAL;
        total += warps_per_class[k];
        if (k < MULTI_CLASSES) smem += (size_t)warps_per_class[k] * warp_smem_bytes(CLASS_K[k]);
    }
    if (total < 1 || total > 8) return LOB_EINVAL;
    if (smem > SMEM_PER_BLOCK_MAX) return LOB_ECAPACITY;
    // every class with envs needs a warp of its class or a larger one
    for (int k = 0; k < MULTI_CLASSES; k++) {
        if (h->class_count[k] == 0) continue;
        int cover = 0;
        for (int j = k; j < MULTI_CLASSES; j++) cover += warps_per_class[j];
        if (cover == 0) return LOB_EINVAL;
    }
    for (int k = 0; k < NCLASS; k++) h->multi_split[k] = warps_per_class[k];
    h->persistent = 2;
    return LOB_OK;
}

int lob_debug_wait(lob_handle *h, int64_t cycles, int32_t hold) {
    if (!h || cycles < 0 || (hold != 0 && hold != 1)) return LOB_EINVAL;
    h->wait_budget = cycles;
    h->hold_first = hold;
    return LOB_OK;
}

int64_t lob_kernel_launches(const lob_handle *h) { return h ? h->launches : 0; }

int lob_set_env_costs(lob_handle *h, const float *h_cost) {
    if (!h) return LOB_EINVAL;
    std::vector<int> list = h->env_list_h;
    if (h_cost) {
        for (int k = 0; k < NCLASS; k++) {
            auto b = list.begin() + h->class_begin[k];
            std::stable_sort(b, b + h->class_count[k], [&](int x, int y) { return h_cost[x] > h_cost[y]; });
        }
    }
    if (cudaMemcpy(h->d_env_list, list.data(), list.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return LOB_ECUDA;
    h->custom_order = h_cost != nullptr;
    return LOB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free step.  Callers that cannot call cudaMalloc (a host program
// that reserves all device memory through its own allocator or a fixed
// budget, or a loop that must not take cudaMalloc's device-wide sync) pass
// every input and output; the scratch the persistent step kernel needs -- its
// work-queue counter and the env list / book offset / capacity tables --
// lives in this file-scope device array instead of a cudaMalloc'd buffer.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t NOALLOC_QUEUE_BYTES = 256;
constexpr size_t NOALLOC_LIST_OFF = NOALLOC_QUEUE_BYTES;
constexpr size_t NOALLOC_BOOKOFF_OFF = NOALLOC_LIST_OFF + 4 * (size_t)LOB_NOALLOC_MAX_ENVS;
constexpr size_t NOALLOC_CAPS_OFF = NOALLOC_BOOKOFF_OFF + 8 * (size_t)LOB_NOALLOC_MAX_ENVS;
constexpr size_t NOALLOC_BYTES = NOALLOC_CAPS_OFF + 4 * (size_t)LOB_NOALLOC_MAX_ENVS;
constexpr int NOALLOC_MAX_DEVICES = 64;
}  // namespace

// In host code this name is only a host-side stand-in for the symbol, not a
// device address: kernels receive the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static unsigned char *g_noalloc_dev_ptr[NOALLOC_MAX_DEVICES];
static int g_noalloc_n_sm[NOALLOC_MAX_DEVICES];

// Per-call preparation of the scratch tables (and the episode reset at t = 0).
__global__ void k_noalloc_prepare(unsigned char *scratch, int n, int cap, long long block_bytes, int reset,
                                  EnvState *st, long long *cnt, int start_px, int exec_dir) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) *reinterpret_cast<int *>(scratch) = 0;   // the work queue starts at zero every call
    if (e >= n) return;
    reinterpret_cast<int *>(scratch + NOALLOC_LIST_OFF)[e] = e;
    reinterpret_cast<long long *>(scratch + NOALLOC_BOOKOFF_OFF)[e] = (long long)e * block_bytes;
    reinterpret_cast<int *>(scratch + NOALLOC_CAPS_OFF)[e] = cap;
    if (reset) {
        EnvState z;
        memset(&z, 0, sizeof(z));
        z.last_px = start_px;
        z.exec_dir = exec_dir;   // the configured task side, as lob_reset stores it
        st[e] = z;
        for (int i = 0; i < LOB_NCOUNTERS; i++) cnt[(long long)e * LOB_NCOUNTERS + i] = 0;
    }
}

extern "C" int lob_step_noalloc(const lob_noalloc_args *a, void *stream) {
    if (!a || !a->cfg) return LOB_EINVAL;
    const lob_config &c = *a->cfg;
    if (c.n_envs < 1 || (c.n_agents != 0 && c.n_agents != 2) || c.top_levels < 1 || c.top_levels > LMAX ||
        c.episode_len < 1 || c.mm_lot < 1 || c.exec_target < 0 ||
        (c.exec_dir != LOB_SELL && c.exec_dir != LOB_BUY) ||
        (c.action_mode != LOB_ACT_HOST && c.action_mode != LOB_ACT_RANDOM) || c.trace != 0 ||
        c.warps_per_block < 0 || c.warps_per_block > 8 || c.cap_per_side < 1)
        return LOB_EINVAL;
    // the plain kernel only: the PV reward, no penalties, the 12-way market
    // maker, the touch as value reference, a fixed task side
    if (c.reward_mode != LOB_REWARD_PV || c.inv_penalty != 0 || c.exec_penalty_milli != 0 ||
        c.mm_space != LOB_MM_SPREAD_SKEW || c.pv_ref != LOB_PV_TOUCH)
        return LOB_EINVAL;
    if (c.n_envs > LOB_NOALLOC_MAX_ENVS || c.cap_per_side > LOB_MAX_CAP) return LOB_ECAPACITY;
    if (!a->d_books || !a->d_env_state || !a->d_counters || !a->d_env_seeds || !a->d_offsets || !a->d_status ||
        a->k < 0 || a->stride < (int64_t)a->k + 2 || a->t < 0 || a->t >= c.episode_len)
        return LOB_EINVAL;
    if (c.n_agents == 2 && c.action_mode == LOB_ACT_HOST && !a->d_actions) return LOB_EINVAL;
    // the kernel stages messages with bulk copies (16-byte boundaries), reads
    // the env state with 16-byte vector loads and each book block with 16-byte
    // vectors from 256-byte block boundaries: refuse what it could not read
    if (((uintptr_t)a->d_msgs & 15u) != 0 || ((uintptr_t)a->d_env_state & 15u) != 0 ||
        ((uintptr_t)a->d_books & 255u) != 0)
        return LOB_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LOB_ECUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LOB_ECAPACITY;
    if (g_noalloc_dev_ptr[dev] == nullptr) {   // once per device, with that device current
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return LOB_ECUDA;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LOB_ECUDA;
        if (ensure_optin() != cudaSuccess) return LOB_ECUDA;
        g_noalloc_n_sm[dev] = nsm;
        g_noalloc_dev_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *scratch = g_noalloc_dev_ptr[dev];
    const int cls = class_of(c.cap_per_side);
    const int K = CLASS_K[cls];
    const long long block_bytes = ((48LL * 32 * K + 255) / 256) * 256;
    const int n = c.n_envs;
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_prepare<<<(n + 127) / 128, 128, 0, s>>>(scratch, n, c.cap_per_side, block_bytes, a->t == 0 ? 1 : 0,
                                                       reinterpret_cast<EnvState *>(a->d_env_state),
                                                       reinterpret_cast<long long *>(a->d_counters), c.start_px,
                                                       c.exec_dir);
    if (cudaGetLastError() != cudaSuccess) return LOB_ECUDA;

    KParams p;
    memset(&p, 0, sizeof(p));
    p.books = static_cast<unsigned char *>(a->d_books);
    p.book_off = reinterpret_cast<const long long *>(scratch + NOALLOC_BOOKOFF_OFF);
    p.caps = reinterpret_cast<const int *>(scratch + NOALLOC_CAPS_OFF);
    p.st = reinterpret_cast<EnvState *>(a->d_env_state);
    p.counters = reinterpret_cast<long long *>(a->d_counters);
    p.seeds = reinterpret_cast<const unsigned long long *>(a->d_env_seeds);
    p.status = a->d_status;
    p.msgs = reinterpret_cast<const DevMsg *>(a->d_msgs);
    p.offsets = reinterpret_cast<const long long *>(a->d_offsets);
    p.off_stride = a->stride;
    p.k0 = a->k;
    p.actions = a->d_actions;
    p.act_step_stride = 0;
    p.action_mode = c.action_mode;
    p.obs = a->d_obs;
    p.rew = reinterpret_cast<long long *>(a->d_rewards);
    p.done = a->d_done;
    p.n_envs = n; p.n_agents = c.n_agents; p.L = c.top_levels; p.T = c.episode_len;
    p.mm_lot = c.mm_lot; p.exec_target = c.exec_target; p.exec_dir = c.exec_dir; p.D = lob_obs_dim(&c);
    p.t0 = a->t; p.n_steps = 1;
    p.env_list = reinterpret_cast<const int *>(scratch + NOALLOC_LIST_OFF);
    p.n_list = n;
    p.queue = reinterpret_cast<int *>(scratch);
    p.wait_budget = DEFAULT_WAIT_BUDGET;
    p.drain_budget = DEFAULT_WAIT_BUDGET;
    p.exec_q0 = exec_lot(c);
    set_rewards(p, c);
    const int wpb = c.warps_per_block > 0 ? c.warps_per_block : 4;
    if (launch_k(K, false, n, wpb, true, g_noalloc_n_sm[dev], s, p) != cudaSuccess) return LOB_ECUDA;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

// The fused BF16 rollout (rollout_fused.cuh): one launch for all n_steps steps
// when the handle is the plain benchmark pair on one capacity class of 128 or
// 256 slots; returns 1 when the configuration does not qualify.
static int fused_rollout(lob_handle *h, lob_policy *pol, int32_t n_steps, float *d_obs, int64_t *d_rewards,
                         uint8_t *d_done, int32_t *d_actions, cudaStream_t s) {
    const lob_config &c = h->cfg;
    const int K = CLASS_K[class_of(c.cap_per_side)];
    if (c.n_agents != 2 || !h->uniform_cap || h->custom_order || h->ep_mode || h->msg16 || c.trace != 0 ||
        (K != 4 && K != 8) || (h->D + 15) / 16 * 16 > FDMAX || c.reward_mode != LOB_REWARD_PV || c.inv_penalty != 0 ||
        c.exec_penalty_milli != 0 || c.pv_ref != LOB_PV_TOUCH || c.exec_dir == 0)
        return 1;
    const size_t per_warp = warp_smem_bytes(K);
    const int nw_fit = (int)((SMEM_PER_BLOCK_MAX - sizeof(FusedSmem)) / per_warp);
    const int nw_max = nw_fit < FWMAX ? nw_fit : FWMAX;
    if (nw_max < 4) return 1;
    // one CTA per SM (its tiles take half the shared memory): as few waves as
    // the widest CTA allows, then the envs spread evenly over every SM of them
    const long long slots = (long long)h->n_sm * nw_max;
    const long long waves = (c.n_envs + slots - 1) / slots;
    int nw = (int)((c.n_envs + waves * h->n_sm - 1) / (waves * h->n_sm));
    nw = nw < 4 ? 4 : (nw > nw_max ? nw_max : nw);
    const size_t smem = (size_t)nw * per_warp + sizeof(FusedSmem);
    static bool opted[2][64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LOB_ECUDA;
    if (!opted[K == 8][dev]) {
        // opt in at the widest shape of the class
        const size_t widest = (size_t)nw_max * per_warp + sizeof(FusedSmem);
        if ((K == 4 ? optin_fused_4(widest) : optin_fused_8(widest)) != cudaSuccess) return LOB_ECUDA;
        opted[K == 8][dev] = true;
    }
    const size_t n = (size_t)c.n_envs, D = (size_t)h->D;
    // each output goes to the caller's per-step buffer, else every step overwrites the handle's
    KParams p = base_params(h, h->msgs, step_offsets(h), h->stride, h->cursor, n_steps, nullptr, 0,
                            d_obs ? d_obs : h->d_obs, d_rewards ? reinterpret_cast<long long *>(d_rewards) : h->d_rew,
                            d_done ? d_done : h->d_done, false, false);
    if (kernel_ext(p)) return 1;   // the fused kernel is built on the plain step only
    p.ow_obs = d_obs ? 0 : 1;
    p.ow_rew = d_rewards ? 0 : 1;
    p.ow_done = d_done ? 0 : 1;
    p.act_steps = d_actions;
    p.obs_in = h->d_obs;
    p.env_list = nullptr;
    p.n_list = c.n_envs;
    p.uni_cap = c.cap_per_side;
    p.uni_block = h->uni_block;
    FusedParams f;
    policy_fused_params(pol, &f);
    const int blocks = (c.n_envs + nw - 1) / nw;
    h->launches++;
    policy_count_launch(pol);
    if ((K == 4 ? launch_fused_4(blocks, nw * 32, smem, s, p, f) : launch_fused_8(blocks, nw * 32, smem, s, p, f)) !=
        cudaSuccess)
        return LOB_ECUDA;
    // the handle keeps the last step's outputs (lob_observe, the next rollout's first actions)
    const size_t last = (size_t)(n_steps - 1);
    int rc = LOB_OK;
    if (d_obs) rc |= cuda_ok(cudaMemcpyAsync(h->d_obs, d_obs + last * n * 2 * D, n * 2 * D * 4, cudaMemcpyDeviceToDevice, s));
    if (d_rewards) rc |= cuda_ok(cudaMemcpyAsync(h->d_rew, d_rewards + last * n * 2, n * 2 * 8, cudaMemcpyDeviceToDevice, s));
    if (d_done) rc |= cuda_ok(cudaMemcpyAsync(h->d_done, d_done + last * n, n, cudaMemcpyDeviceToDevice, s));
    if (rc != LOB_OK) return LOB_ECUDA;
    h->cursor += n_steps;
    h->t += n_steps;
    return LOB_OK;
}

extern "C" int lob_rollout_policy(lob_handle *h, lob_policy *pol, int32_t n_steps, int32_t precision, float *d_obs,
                                  int64_t *d_rewards, uint8_t *d_done, int32_t *d_actions, void *stream) {
    if (!h || !pol || n_steps < 1) return LOB_EINVAL;
    if (h->cfg.n_agents < 2 || h->cfg.action_mode != LOB_ACT_HOST || h->cfg.mm_space != LOB_MM_SPREAD_SKEW)
        return LOB_EINVAL;
    if (policy_n_agents(pol) != h->cfg.n_agents || policy_obs_dim(pol) != h->D) return LOB_EINVAL;
    if (precision != LOB_PREC_FP32 && precision != LOB_PREC_BF16 && precision != LOB_PREC_BF16_FUSED) return LOB_EINVAL;
    if (!steps_left(h, n_steps)) return LOB_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == LOB_PREC_BF16_FUSED) {
        const int rc = fused_rollout(h, pol, n_steps, d_obs, d_rewards, d_done, d_actions, s);
        return rc == 1 ? LOB_EINVAL : rc;   // 1: not a configuration of the fused kernel
    }
    const size_t n = (size_t)h->cfg.n_envs, D = (size_t)h->D, A = (size_t)h->cfg.n_agents;
    for (int i = 0; i < n_steps; i++) {
        // the policy acts on the current observation (kept in the handle's buffer)
        int rc = policy_forward_internal(pol, h->d_obs, h->cfg.n_envs, precision, nullptr, nullptr, h->d_act, s);
        if (rc != LOB_OK) return rc;
        if (d_actions && cudaMemcpyAsync(d_actions + (size_t)i * n * A, h->d_act, n * A * 4,
                                         cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return LOB_ECUDA;
        rc = launch_steps(h, h->msgs, step_offsets(h), h->stride, h->cursor, 1, h->d_act, 0, h->d_obs, h->d_rew,
                          h->d_done, s, false, h->msg16);
        if (rc != LOB_OK) return rc;
        h->cursor++;
        h->t++;
        if (d_obs && cudaMemcpyAsync(d_obs + (size_t)i * n * A * D, h->d_obs, n * A * D * 4,
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return LOB_ECUDA;
        if (d_rewards && cudaMemcpyAsync(d_rewards + (size_t)i * n * A, h->d_rew, n * A * 8,
                                         cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return LOB_ECUDA;
        if (d_done && cudaMemcpyAsync(d_done + (size_t)i * n, h->d_done, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return LOB_ECUDA;
    }
    return LOB_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: a 64-byte header, then books, EnvState, counters,
// seeds, obs, rewards, done -- each region copied as one block.
namespace {
struct CkptHeader {
    uint64_t magic;
    int64_t n_envs, book_bytes, obs_bytes;
    int32_t t, cursor, n_agents, D;
    int32_t cap_sig, pad[3];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header");
constexpr uint64_t CKPT_MAGIC = 0x4C4F42434B505431ull;

int cap_signature(const lob_handle *h) {
    unsigned x = 2166136261u;
    for (int c : h->caps) x = (x ^ (unsigned)c) * 16777619u;
    return (int)x;
}

struct Region { void *dev; size_t bytes; };
std::vector<Region> ckpt_regions(lob_handle *h) {
    const size_t n = (size_t)h->cfg.n_envs, A = (size_t)h->cfg.n_agents, D = (size_t)h->D;
    std::vector<Region> r = {{h->d_books, (size_t)h->book_bytes}, {h->d_state, n * sizeof(EnvState)},
                             {h->d_counters, n * 8 * LOB_NCOUNTERS}, {h->d_seeds, n * 8}, {h->d_obs, n * A * D * 4},
                             {h->d_rew, n * A * 8}, {h->d_done, n}};
    if (h->d_agents) r.push_back({h->d_agents, n * A * sizeof(AgentState)});
    return r;
}
}  // namespace

extern "C" int64_t lob_checkpoint_bytes(const lob_handle *h) {
    if (!h) return 0;
    size_t b = sizeof(CkptHeader);
    for (const Region &r : ckpt_regions(const_cast<lob_handle *>(h))) b += r.bytes;
    return (int64_t)b;
}

extern "C" int lob_save(lob_handle *h, void *dst, void *stream) {
    if (!h || !dst) return LOB_EINVAL;
    if (!h->reset_done) return LOB_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = CKPT_MAGIC;
    hd.n_envs = h->cfg.n_envs;
    hd.book_bytes = h->book_bytes;
    hd.obs_bytes = (int64_t)h->cfg.n_envs * h->cfg.n_agents * h->D * 4;
    hd.t = h->t;
    hd.cursor = h->cursor;
    hd.n_agents = h->cfg.n_agents;
    hd.D = h->D;
    hd.cap_sig = cap_signature(h);
    hd.pad[0] = h->ep_mode ? 1 : 0;
    char *out = static_cast<char *>(dst);
    if (cudaMemcpyAsync(out, &hd, sizeof(hd), cudaMemcpyDefault, s) != cudaSuccess) return LOB_ECUDA;
    size_t off = sizeof(hd);
    for (const Region &r : ckpt_regions(h)) {
        if (cudaMemcpyAsync(out + off, r.dev, r.bytes, cudaMemcpyDefault, s) != cudaSuccess) return LOB_ECUDA;
        off += r.bytes;
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? LOB_OK : LOB_ECUDA;   // the header lives on this stack
}

extern "C" int lob_load(lob_handle *h, const void *src, void *stream) {
    if (!h || !src) return LOB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CkptHeader hd;
    if (cudaMemcpyAsync(&hd, src, sizeof(hd), cudaMemcpyDefault, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LOB_ECUDA;
    if (hd.magic != CKPT_MAGIC || hd.n_envs != h->cfg.n_envs || hd.book_bytes != h->book_bytes ||
        hd.n_agents != h->cfg.n_agents || hd.D != h->D || hd.cap_sig != cap_signature(h) || hd.t < 0 ||
        hd.pad[0] != (h->ep_mode ? 1 : 0) || (!h->ep_mode && hd.t > h->cfg.episode_len))
        return LOB_EINVAL;
    const char *in = static_cast<const char *>(src);
    size_t off = sizeof(hd);
    for (const Region &r : ckpt_regions(h)) {
        if (cudaMemcpyAsync(r.dev, in + off, r.bytes, cudaMemcpyDefault, s) != cudaSuccess) return LOB_ECUDA;
        off += r.bytes;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LOB_ECUDA;
    if (h->ep_mode) {
        // every env's episode must lie inside the data this handle now indexes
        std::vector<EnvState> st((size_t)h->cfg.n_envs);
        if (cudaMemcpy(st.data(), h->d_state, st.size() * sizeof(EnvState), cudaMemcpyDeviceToHost) != cudaSuccess)
            return LOB_ECUDA;
        for (const EnvState &x : st)
            if (x.ep_start < 0 || (int64_t)x.ep_start + h->cfg.episode_len > h->n_data_steps) {
                h->reset_done = false;
                return LOB_EINVAL;
            }
    }
    h->t = hd.t;
    h->cursor = hd.cursor;
    h->reset_done = true;
    return LOB_OK;
}
