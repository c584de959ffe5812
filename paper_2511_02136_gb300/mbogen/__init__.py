"""Seeded synthetic MBO message streams (the input module).

Both the CPU oracle and the CUDA engine consume the bytes this module writes;
it holds none of the environment step's arithmetic.  It stands in for the
contiguous historical message store with per-episode start indices of Sec. 4
(Design); the paper's LOBSTER AMZN 2024 data is not available, so the
message model documented in ``mbogen.c`` replaces it.

Workload presets mirror the five benchmark configurations (plain replay of one
env, 1,024 uniform envs, 8,192 uneven envs, the fused-policy rollout, and the
heavy-tailed stress mix).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbogen.c")
_LIB = os.path.join(_HERE, "libmbogen.so")
_lock = threading.Lock()
_lib = None

MSG_DTYPE = np.dtype(
    [("ts", "<i8"), ("oid", "<i8"), ("px", "<i4"), ("qty", "<i4"),
     ("type", "<i2"), ("side", "<i2"), ("pad", "<i4")]
)
assert MSG_DTYPE.itemsize == 32

ADD, PARTIAL, DELETE, MARKET = 1, 2, 3, 4
BUY, SELL = 1, -1


class _Params(ctypes.Structure):
    _fields_ = [
        ("start_mid", ctypes.c_int32), ("msgs_mode", ctypes.c_int32),
        ("msgs_fixed", ctypes.c_int32), ("size_model", ctypes.c_int32),
        ("size_cap", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("p_move", ctypes.c_double), ("mix_add", ctypes.c_double),
        ("mix_partial", ctypes.c_double), ("mix_delete", ctypes.c_double),
        ("mix_market", ctypes.c_double), ("price_p", ctypes.c_double),
        ("size_p", ctypes.c_double), ("pareto_alpha", ctypes.c_double),
        ("p_burst", ctypes.c_double), ("lam_lo", ctypes.c_double),
        ("lam_hi", ctypes.c_double),
    ]


@dataclass
class MessageModel:
    """Parameters of the synthetic message model (defaults: the base mix)."""
    start_mid: int = 10_000
    p_move: float = 0.1
    mix_add: float = 0.55
    mix_partial: float = 0.15
    mix_delete: float = 0.20
    mix_market: float = 0.10
    price_p: float = 0.3          # g ~ Geom0(0.3) ticks from mid on the passive side
    size_model: int = 0           # 0: 1 + Geom0(size_p); 1: min(cap, floor(Pareto(1, alpha)))
    size_p: float = 0.01
    pareto_alpha: float = 1.5
    size_cap: int = 10_000
    p_burst: float = 0.0          # per env-step probability of a delete burst
    msgs_per_step: int = 100      # fixed M (msgs_mode 0)
    poisson: bool = False         # M_t ~ Poisson(lambda_env), lambda log-uniform
    lam_lo: float = 10.0
    lam_hi: float = 500.0

    def _c(self) -> _Params:
        return _Params(
            start_mid=self.start_mid, msgs_mode=1 if self.poisson else 0,
            msgs_fixed=self.msgs_per_step, size_model=self.size_model,
            size_cap=self.size_cap, pad0=0, p_move=self.p_move,
            mix_add=self.mix_add, mix_partial=self.mix_partial,
            mix_delete=self.mix_delete, mix_market=self.mix_market,
            price_p=self.price_p, size_p=self.size_p,
            pareto_alpha=self.pareto_alpha, p_burst=self.p_burst,
            lam_lo=self.lam_lo, lam_hi=self.lam_hi,
        )


STRESS_MODEL = MessageModel(mix_add=0.35, mix_partial=0.15, mix_delete=0.20,
                            mix_market=0.30, size_model=1, pareto_alpha=1.5,
                            size_cap=10_000, p_burst=0.05, msgs_per_step=1000)


def build(force: bool = False) -> str:
    """Compile libmbogen.so in-tree with the host C compiler (portable flags)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.mbogen_env_seed.restype = ctypes.c_uint64
        lib.mbogen_env_seed.argtypes = [ctypes.c_uint64, ctypes.c_int64]
        lib.mbogen_counts.restype = ctypes.c_int
        lib.mbogen_counts.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        lib.mbogen_offsets.restype = ctypes.c_int64
        lib.mbogen_offsets.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        lib.mbogen_generate.restype = ctypes.c_int
        lib.mbogen_generate.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        lib.mbogen_env_caps.restype = None
        lib.mbogen_env_caps.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p]
        _lib = lib
    return _lib


def env_seeds(seed: int, n_envs: int, first_env: int = 0) -> np.ndarray:
    """Per-env seeds: one SplitMix64 output of (seed xor env)."""
    lib = _load()
    return np.array([lib.mbogen_env_seed(seed & (2**64 - 1), first_env + e) for e in range(n_envs)],
                    dtype=np.uint64)


def env_caps(seed: int, n_envs: int, choices=(50, 100, 200, 500)) -> np.ndarray:
    lib = _load()
    ch = np.ascontiguousarray(np.array(choices, dtype=np.int32))
    out = np.empty(n_envs, dtype=np.int32)
    lib.mbogen_env_caps(seed & (2**64 - 1), n_envs, ch.ctypes.data, len(ch), out.ctypes.data)
    return out


@dataclass
class Streams:
    """Messages of all envs in one contiguous env-major array plus start indices.

    ``offsets[e, t]`` is the index of env ``e``'s first message of step ``t``;
    step ``t`` covers ``msgs[offsets[e, t]:offsets[e, t + 1]]``.
    """
    msgs: np.ndarray        # MSG_DTYPE [total]
    offsets: np.ndarray     # int64 [n_envs, n_steps + 1]
    counts: np.ndarray      # int32 [n_envs, n_steps]
    lambdas: np.ndarray     # float64 [n_envs]
    seeds: np.ndarray       # uint64 [n_envs]
    mids: np.ndarray | None = None   # int32 [n_envs, n_steps + 1]: latent mid at each step boundary


def generate(model: MessageModel, seeds: np.ndarray, n_steps: int, n_threads: int | None = None) -> Streams:
    lib = _load()
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    n_envs = len(seeds)
    p = model._c()
    counts = np.empty((n_envs, n_steps), dtype=np.int32)
    lambdas = np.empty(n_envs, dtype=np.float64)
    if lib.mbogen_counts(ctypes.byref(p), n_envs, seeds.ctypes.data, n_steps,
                         counts.ctypes.data, lambdas.ctypes.data):
        raise RuntimeError("mbogen_counts failed")
    offsets = np.empty((n_envs, n_steps + 1), dtype=np.int64)
    total = lib.mbogen_offsets(n_envs, n_steps, counts.ctypes.data, offsets.ctypes.data)
    msgs = np.empty(max(total, 1), dtype=MSG_DTYPE)[:total]
    if n_threads is None:
        n_threads = min(os.cpu_count() or 1, 64)
    mids = np.full((n_envs, n_steps + 1), model.start_mid, dtype=np.int32)
    if total and lib.mbogen_generate(ctypes.byref(p), n_envs, seeds.ctypes.data, n_steps,
                                     counts.ctypes.data, offsets.ctypes.data,
                                     msgs.ctypes.data, n_threads, mids.ctypes.data):
        raise RuntimeError("mbogen_generate failed")
    return Streams(msgs=msgs, offsets=offsets, counts=counts, lambdas=lambdas, seeds=seeds, mids=mids)


START_DTYPE = np.dtype([("data_step", "<i4"), ("last_px", "<i4"), ("n_bid", "<i4"), ("n_ask", "<i4")])
MSG16_DTYPE = np.dtype([("px", "<i4"), ("qty", "<i4"), ("word", "<i8")])


def pack16(msgs: np.ndarray) -> np.ndarray:
    """The 16-byte compact encoding of 32-byte records: px, qty and
    word = id << 4 | (side is sell) << 3 | type, type 0 when the record's type
    or side is invalid.  Ids must lie in [-2^59, 2^59)."""
    oid = msgs["oid"].astype(np.int64)
    if len(oid) and (oid.min() < -(1 << 59) or oid.max() >= (1 << 59)):
        raise ValueError("order id outside the compact range")
    t = msgs["type"].astype(np.int64)
    sd = msgs["side"].astype(np.int64)
    valid = (t >= 1) & (t <= 4) & ((sd == 1) | (sd == -1))
    code = np.where(valid, t | np.where(sd == -1, 8, 0), 0)
    out = np.empty(len(msgs), MSG16_DTYPE)
    out["px"] = msgs["px"]
    out["qty"] = msgs["qty"]
    out["word"] = (oid << 4) | code
    return out


def start_books(seed: int, mids: np.ndarray, start_steps, levels_per_side: int, min_levels: int = 0,
                max_gap: int = 3, qty_max: int = 50):
    """Synthetic book snapshots at episode starts (the role of the data set's
    order-book file at the start of each episode).

    For start j at data step s = start_steps[j] around the stream's latent mid m
    = mids[s]: best bid m - U{0..2}, best ask m + 1 + U{0..2}, further levels
    each 1 + U{0..max_gap-1} ticks away, level counts U{min_levels..levels_per_side}
    per side, sizes U{1..qty_max}; last trade price m.  Returns
    (starts START_DTYPE[n], levels int32[n, 2, levels_per_side, 2]) with
    (price, quantity) pairs best-first (bids descending, asks ascending).
    """
    rng = np.random.default_rng(seed)
    steps = np.asarray(start_steps, dtype=np.int64)
    n = len(steps)
    starts = np.zeros(n, START_DTYPE)
    levels = np.zeros((n, 2, levels_per_side, 2), np.int32)
    for j, s in enumerate(steps):
        m = int(mids[s])
        nb = int(rng.integers(min_levels, levels_per_side + 1))
        na = int(rng.integers(min_levels, levels_per_side + 1))
        px = m - int(rng.integers(0, 3))
        for i in range(nb):
            levels[j, 0, i] = (px, int(rng.integers(1, qty_max + 1)))
            px -= 1 + int(rng.integers(0, max_gap))
        px = m + 1 + int(rng.integers(0, 3))
        for i in range(na):
            levels[j, 1, i] = (px, int(rng.integers(1, qty_max + 1)))
            px += 1 + int(rng.integers(0, max_gap))
        starts[j] = (int(s), m, nb, na)
    return starts, levels


# ---------------------------------------------------------------- device generator
_GPU_SRC = os.path.join(_HERE, "mbogen_gpu.cu")
_GPU_LIB = os.path.join(_HERE, "libmbogen_gpu.so")
_gpu_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile libmbogen_gpu.so (the device generator) in-tree for sm_103a."""
    with _lock:
        if (not force and os.path.exists(_GPU_LIB)
                and os.path.getmtime(_GPU_LIB) >= os.path.getmtime(_GPU_SRC)):
            return _GPU_LIB
        tmp = _GPU_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _GPU_SRC])
        os.replace(tmp, _GPU_LIB)
        return _GPU_LIB


def _load_gpu():
    global _gpu_lib
    if _gpu_lib is None:
        lib = ctypes.CDLL(build_gpu())
        P = ctypes.c_void_p
        lib.mbogen_gpu_create.restype = ctypes.c_int
        lib.mbogen_gpu_create.argtypes = [ctypes.c_int64, P, ctypes.c_int32, P, P, ctypes.c_int32, P, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(P)]
        lib.mbogen_gpu_chunk.restype = ctypes.c_int
        lib.mbogen_gpu_chunk.argtypes = [P, ctypes.c_int32, P, P, P, P]
        lib.mbogen_gpu_status.restype = ctypes.c_int
        lib.mbogen_gpu_status.argtypes = [P]
        lib.mbogen_gpu_destroy.restype = ctypes.c_int
        lib.mbogen_gpu_destroy.argtypes = [P]
        _gpu_lib = lib
    return _gpu_lib


def tables(model: MessageModel):
    """The model's draw thresholds (as the host generator builds them)."""
    lib = _load()
    lib.mbogen_tables.restype = ctypes.c_int
    lib.mbogen_tables.argtypes = [ctypes.POINTER(_Params)] + [ctypes.c_void_p] * 6
    scal = np.zeros(5, np.uint64)
    geom = np.zeros(4096, np.uint64)
    size = np.zeros(1 << 16, np.uint64)
    gn, sn, sb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    p = model._c()
    if lib.mbogen_tables(ctypes.byref(p), scal.ctypes.data, geom.ctypes.data, ctypes.byref(gn), size.ctypes.data,
                         ctypes.byref(sn), ctypes.byref(sb)):
        raise RuntimeError("mbogen_tables failed")
    return scal, geom[:gn.value].copy(), size[:sn.value].copy(), sb.value


class GpuStreams:
    """The streams of n envs drawn on the current CUDA device, chunk by chunk:
    chunk(k_steps, out) writes every env's next k_steps steps (fixed messages
    per step, env-major: env e's step j at records (e * k_steps + j) * M) into
    the device tensor out, on the given stream.  Byte-identical to generate()."""

    def __init__(self, model: MessageModel, seeds: np.ndarray, pool_cap: int = 32768):
        import torch
        if model.poisson:
            raise ValueError("the device generator draws fixed messages per step")
        self.torch = torch
        self.model = model
        self.n = len(seeds)
        self.M = model.msgs_per_step
        scal, geom, size, base = tables(model)
        seeds = np.ascontiguousarray(seeds, np.uint64)
        lib = _load_gpu()
        h = ctypes.c_void_p()
        rc = lib.mbogen_gpu_create(self.n, seeds.ctypes.data, model.start_mid, scal.ctypes.data, geom.ctypes.data,
                                   len(geom), size.ctypes.data, len(size), base, 1 if model.size_model == 0 else 0,
                                   pool_cap, ctypes.byref(h))
        if rc:
            raise RuntimeError(f"mbogen_gpu_create failed ({rc})")
        self.h = h
        self._shape = None

    def offsets(self, k_steps):
        """int64 [n][k_steps + 1] record offsets of one chunk (host)."""
        e = np.arange(self.n, dtype=np.int64)[:, None]
        j = np.arange(k_steps + 1, dtype=np.int64)[None, :]
        return (e * k_steps + j) * self.M

    def chunk(self, k_steps, out, stream=None):
        torch = self.torch
        if self._shape != k_steps:
            self._counts = torch.full((self.n, k_steps), self.M, dtype=torch.int32, device="cuda")
            self._offs = torch.from_numpy(self.offsets(k_steps)).cuda()
            self._shape = k_steps
        if out.numel() * out.element_size() < self.n * k_steps * self.M * 32:
            raise ValueError("output buffer too small")
        s = (stream or torch.cuda.current_stream()).cuda_stream
        rc = _load_gpu().mbogen_gpu_chunk(self.h, k_steps, self._counts.data_ptr(), self._offs.data_ptr(),
                                          out.data_ptr(), s)
        if rc:
            raise RuntimeError(f"mbogen_gpu_chunk failed ({rc})")

    def ok(self):
        return _load_gpu().mbogen_gpu_status(self.h) == 0

    def close(self):
        if self.h:
            _load_gpu().mbogen_gpu_destroy(self.h)
            self.h = None
