// mbogen_gpu.cu -- the message model of mbogen.c drawn on the GPU, chunk by
// chunk, for streams too long to generate up front or to hold in memory (the
// 65,536-env stress mix over 256 steps is 16.8 G messages, 537 GB).
//
// Part of the input module: it writes message bytes and nothing else.  One
// thread per env runs exactly the per-env loop of mbogen.c's gen_env -- the
// same SplitMix64 stream, the same integer draws against the same threshold
// tables (built on the host by mbogen_tables), the same pool of issued ids
// with swap-removal -- so an env's messages are byte-identical to the host
// generator's, whatever the chunking.  The per-env state (random state,
// latent mid, next id, clock and the id pool) lives in device memory between
// chunks; a pool that would outgrow its capacity sets the status word (the
// chunk is then unusable) instead of growing.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t TAG_MSGS = 0x4D424F4D53475331ULL;

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm_next(uint64_t &s) {
    s += SM_GAMMA;
    return sm_mix(s);
}
__device__ __forceinline__ uint32_t lemire32(uint64_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)(uint32_t)(u >> 32) * (uint64_t)n) >> 32);
}
// First index with u < thr[i] (n if none), as mbogen.c's cdf_sample.
__device__ __forceinline__ int32_t cdf_index(const uint64_t *thr, int32_t n, uint64_t u) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (u < __ldg(thr + mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

struct Msg {
    int64_t ts, oid;
    int32_t px, qty;
    int16_t type, side;
    int32_t pad;
};
static_assert(sizeof(Msg) == 32, "message record");

struct EnvGen {              // per-env generator state between chunks
    uint64_t s;
    int64_t next_oid, clock;
    int32_t mid, pool_n;
};
struct PoolEntry {           // an issued, not yet fully cancelled order
    int64_t oid;
    int32_t px;
    int32_t q_side;          // quantity in bits 0..30, bit 31 set for a sell
};

struct GenParams {
    uint64_t thr_move, thr_add, thr_partial, thr_delete, thr_burst;
    const uint64_t *geom;
    int32_t geom_n;
    const uint64_t *size;
    int32_t size_n, size_base, size_plus1;   // size_plus1: 1 + Geom0 sizes
    EnvGen *st;
    PoolEntry *pool;
    int32_t pool_cap;
    int64_t n_envs;
    int32_t n_steps;                          // steps in this chunk
    const int32_t *counts;                    // [n_envs][n_steps] messages per step
    const int64_t *offsets;                   // [n_envs][n_steps + 1] record index of each step in out
    Msg *out;
    int *status;
};

__global__ void k_gen_init(EnvGen *st, const uint64_t *seeds, int64_t n, int32_t start_mid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    EnvGen g;
    g.s = sm_mix(seeds[e] ^ TAG_MSGS);
    g.next_oid = 0;
    g.clock = 0;
    g.mid = start_mid;
    g.pool_n = 0;
    st[e] = g;
}

__global__ void k_gen_chunk(const GenParams p) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.n_envs) return;
    EnvGen g = p.st[e];
    PoolEntry *pool = p.pool + e * (int64_t)p.pool_cap;
    uint64_t s = g.s;
    int32_t mid = g.mid, pool_n = g.pool_n;
    int64_t next_oid = g.next_oid, clock = g.clock;
    for (int32_t t = 0; t < p.n_steps; t++) {
        const int32_t m = p.counts[e * (int64_t)p.n_steps + t];
        Msg *o = p.out + p.offsets[e * (int64_t)(p.n_steps + 1) + t];
        int32_t n_burst = 0;
        if (p.thr_burst) {
            const uint64_t u = sm_next(s);
            if (u < p.thr_burst) {
                const int32_t b = pool_n / 2;
                n_burst = b < m ? b : m;
            }
        }
        for (int32_t i = 0; i < m; i++) {
            Msg r;
            r.ts = 0; r.oid = 0; r.px = 0; r.qty = 0; r.type = 0; r.side = 0; r.pad = 0;
            uint64_t u = sm_next(s);
            if (u < p.thr_move) mid += (sm_next(s) >> 63) ? 1 : -1;
            int type;
            if (i < n_burst) {
                type = 3;
            } else {
                u = sm_next(s);
                type = u < p.thr_add ? 1 : u < p.thr_partial ? 2 : u < p.thr_delete ? 3 : 4;
            }
            if ((type == 2 || type == 3) && pool_n == 0) type = 1;
            r.ts = clock++;
            r.type = (int16_t)type;
            if (type == 1 || type == 4) {
                const int16_t side = (sm_next(s) >> 63) ? -1 : 1;
                int32_t qty = p.size_base + cdf_index(p.size, p.size_n, sm_next(s));
                if (p.size_plus1) qty += 1;
                r.side = side;
                r.qty = qty;
                r.oid = next_oid++;
                if (type == 1) {
                    const int32_t gap = cdf_index(p.geom, p.geom_n, sm_next(s));
                    r.px = side == 1 ? mid - gap : mid + gap;
                    if (pool_n == p.pool_cap) {
                        atomicOr(p.status, 1);   // the pool is full: this chunk is unusable
                    } else {
                        PoolEntry pe;
                        pe.oid = r.oid;
                        pe.px = r.px;
                        pe.q_side = (qty & 0x7fffffff) | (side < 0 ? (int32_t)0x80000000 : 0);
                        pool[pool_n++] = pe;
                    }
                }
            } else {
                const uint32_t k = lemire32(sm_next(s), (uint32_t)pool_n);
                PoolEntry pe = pool[k];
                const int32_t q = pe.q_side & 0x7fffffff;
                r.oid = pe.oid;
                r.px = pe.px;
                r.side = pe.q_side < 0 ? -1 : 1;
                bool remove;
                int32_t left = q;
                if (type == 2) {
                    const int32_t span = q - 1 > 1 ? q - 1 : 1;
                    const int32_t amt = 1 + (int32_t)lemire32(sm_next(s), (uint32_t)span);
                    r.qty = amt;
                    left = q - amt;
                    remove = left <= 0;
                } else {
                    r.qty = q;
                    remove = true;
                }
                if (remove) {
                    pool[k] = pool[--pool_n];
                } else {
                    pe.q_side = (pe.q_side & (int32_t)0x80000000) | (left & 0x7fffffff);
                    pool[k] = pe;
                }
            }
            o[i] = r;
        }
    }
    g.s = s;
    g.mid = mid;
    g.pool_n = pool_n;
    g.next_oid = next_oid;
    g.clock = clock;
    p.st[e] = g;
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

struct mbogen_gpu {
    GenParams p;
    uint64_t *d_tables = nullptr;
    int *d_status = nullptr;
};

// Device generator of n_envs streams (host seeds, as mbogen_env_seed gives),
// at the start of every stream.  scal / geom / size: mbogen_tables' output.
int mbogen_gpu_create(int64_t n_envs, const uint64_t *h_seeds, int32_t start_mid, const uint64_t *scal,
                      const uint64_t *geom, int32_t geom_n, const uint64_t *size, int32_t size_n, int32_t size_base,
                      int32_t size_plus1, int32_t pool_cap, mbogen_gpu **out) {
    if (!out || n_envs < 1 || pool_cap < 1 || geom_n < 1 || size_n < 1) return -1;
    mbogen_gpu *g = new mbogen_gpu();
    GenParams &p = g->p;
    p.thr_move = scal[0]; p.thr_add = scal[1]; p.thr_partial = scal[2]; p.thr_delete = scal[3]; p.thr_burst = scal[4];
    p.geom_n = geom_n; p.size_n = size_n; p.size_base = size_base; p.size_plus1 = size_plus1;
    p.pool_cap = pool_cap;
    p.n_envs = n_envs;
    uint64_t *d_seeds = nullptr;
    bool fail = cudaMalloc(&g->d_tables, sizeof(uint64_t) * (size_t)(geom_n + size_n)) != cudaSuccess;
    fail = fail || cudaMalloc(&p.st, sizeof(EnvGen) * (size_t)n_envs) != cudaSuccess;
    fail = fail || cudaMalloc(&p.pool, sizeof(PoolEntry) * (size_t)n_envs * (size_t)pool_cap) != cudaSuccess;
    fail = fail || cudaMalloc(&g->d_status, sizeof(int)) != cudaSuccess;
    fail = fail || cudaMalloc(&d_seeds, sizeof(uint64_t) * (size_t)n_envs) != cudaSuccess;
    if (!fail) {
        fail = cudaMemcpy(g->d_tables, geom, sizeof(uint64_t) * (size_t)geom_n, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(g->d_tables + geom_n, size, sizeof(uint64_t) * (size_t)size_n, cudaMemcpyHostToDevice) !=
                   cudaSuccess ||
               cudaMemcpy(d_seeds, h_seeds, sizeof(uint64_t) * (size_t)n_envs, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemset(g->d_status, 0, sizeof(int)) != cudaSuccess;
    }
    if (!fail) {
        k_gen_init<<<(unsigned)((n_envs + 255) / 256), 256>>>(p.st, d_seeds, n_envs, start_mid);
        fail = cudaDeviceSynchronize() != cudaSuccess;
    }
    if (d_seeds) cudaFree(d_seeds);
    p.geom = g->d_tables;
    p.size = g->d_tables + geom_n;
    p.status = g->d_status;
    if (fail) {
        cudaGetLastError();
        if (g->d_tables) cudaFree(g->d_tables);
        if (p.st) cudaFree(p.st);
        if (p.pool) cudaFree(p.pool);
        if (g->d_status) cudaFree(g->d_status);
        delete g;
        return -2;
    }
    *out = g;
    return 0;
}

// The next n_steps steps of every stream into d_out (device, 16-byte aligned),
// step t of env e at record d_offsets[e * (n_steps + 1) + t] with
// d_counts[e * n_steps + t] records; enqueued on `stream`.
int mbogen_gpu_chunk(mbogen_gpu *g, int32_t n_steps, const int32_t *d_counts, const int64_t *d_offsets, void *d_out,
                     void *stream) {
    if (!g || n_steps < 1 || !d_counts || !d_offsets || !d_out) return -1;
    GenParams p = g->p;
    p.n_steps = n_steps;
    p.counts = d_counts;
    p.offsets = d_offsets;
    p.out = static_cast<Msg *>(d_out);
    k_gen_chunk<<<(unsigned)((p.n_envs + 127) / 128), 128, 0, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Nonzero once a pool has run out of room (synchronises the device).
int mbogen_gpu_status(mbogen_gpu *g) {
    if (!g) return -1;
    int st = 0;
    if (cudaMemcpy(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -3;
    return st;
}

int mbogen_gpu_destroy(mbogen_gpu *g) {
    if (!g) return -1;
    cudaDeviceSynchronize();
    cudaFree(g->d_tables);
    cudaFree(g->p.st);
    cudaFree(g->p.pool);
    cudaFree(g->d_status);
    delete g;
    return 0;
}

}  // extern "C"
