"""Thin Python binding of liblob.so (the C ABI in include/lob.h).

Argument marshalling only: every stage of the environment step runs in the
CUDA kernels of the library.  PyTorch supplies device memory and streams.
Importing works without a GPU; loading the library requires it to be built
(``build()``), and every call that touches the device requires CUDA.  There is
no CPU fallback: if the library is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INC = os.path.join(_ROOT, "include")
# LOB_CHECKED=1 in the environment selects the checked build (index bounds and
# book invariants verified on the device, reported as LOB_ECHECK), built and
# loaded as liblob_checked.so
CHECKED = os.environ.get("LOB_CHECKED") == "1"
LIB_PATH = os.path.join(_PKG, "liblob_checked.so" if CHECKED else "liblob.so")
_SOURCES = [os.path.join(_CSRC, n) for n in
            ["lob_api.cu", "policy_api.cu", "rollout_fused_k4.cu", "rollout_fused_k8.cu", "steps_multi.cu",
             "steps_split.cu"] +
            [f"steps_k{k}.cu" for k in (1, 2, 4, 8, 16, 32)] +
            [f"steps_ma_k{k}.cu" for k in (1, 2, 4, 8, 16, 32)]]
_DEPS = _SOURCES + [os.path.join(_CSRC, n) for n in ("lob_device.cuh", "lob_ladder.cuh", "policy.cuh", "tc05.cuh", "ppo.cuh",
                                                      "fused.cuh", "rollout_fused.cuh", "lob_split.cuh",
                                                      "policy_internal.h",
                                                      "lob_steps.h", "steps_inst.cuh", "steps_ma_inst.cuh")] + \
    [os.path.join(_INC, "lob.h")]
_OBJDIR = os.path.join(_PKG, "_build")
_lock = threading.Lock()
_lib = None
_lib_path = None

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]

LOB_OK, LOB_EINVAL, LOB_ENOMEM, LOB_ECUDA, LOB_ETIMEOUT, LOB_ECAPACITY, LOB_EBADMSG, LOB_ESTATE, LOB_ECHECK = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
LOB_ACT_HOST, LOB_ACT_RANDOM = 0, 1
LOB_NCOUNTERS = 16
LOB_MAX_CAP = 1024
FILL_BYTES = 32

# Every entry point include/lob.h declares (checked by the test suite).
EXPORTS = [
    "lob_obs_dim", "lob_create", "lob_destroy", "lob_load_messages", "lob_reset", "lob_step",
    "lob_observe", "lob_rollout", "lob_step_host", "lob_book_bytes", "lob_get_book",
    "lob_get_counters", "lob_get_agents", "lob_get_env_misc", "lob_get_actions", "lob_set_trace",
    "lob_sync", "lob_set_launch", "lob_debug_wait", "lob_kernel_launches", "lob_strerror", "lob_step_noalloc",
    "lob_policy_param_count", "lob_policy_create", "lob_policy_destroy", "lob_policy_forward",
    "lob_policy_sync", "lob_rollout_policy", "lob_set_env_costs",
    "lob_checkpoint_bytes", "lob_save", "lob_load", "lob_set_episodes", "lob_get_episode_starts",
    "lob_step_host_async", "lob_load_messages16", "lob_set_episodes16", "lob_pack_messages16",
    "lob_live_orders", "lob_policy_get_params", "lob_ppo_update", "lob_set_multi_split",
    "lob_set_threads_per_env", "lob_set_tile_records",
]
LOB_PREC_FP32, LOB_PREC_BF16, LOB_PREC_BF16_FUSED = 0, 1, 2
LOB_REWARD_PV, LOB_REWARD_BUYSELL, LOB_REWARD_SPOONER = 0, 1, 2
LOB_MM_SPREAD_SKEW, LOB_MM_FIXED_QUANT, LOB_MM_DIRECTIONAL = 0, 1, 2
LOB_PV_TOUCH, LOB_PV_MID = 0, 1
LOB_INIT_ID = 0x4000000000000000
START_DTYPE = np.dtype([("data_step", "<i4"), ("last_px", "<i4"), ("n_bid", "<i4"), ("n_ask", "<i4")])
MSG16_DTYPE = np.dtype([("px", "<i4"), ("qty", "<i4"), ("word", "<i8")])
LOB_MSG16_ID_MIN, LOB_MSG16_ID_MAX = -(1 << 59), (1 << 59) - 1
POLICY_HIDDEN = 128
LOB_NOALLOC_MAX_ENVS = 16384
LOB_MAX_PER_TYPE = 16


class LobError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _load().lob_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class lob_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_envs", "n_agents", "cap_per_side", "top_levels", "episode_len", "mm_lot",
        "exec_target", "exec_dir", "action_mode", "trace", "start_px", "warps_per_block",
        "reward_mode", "spooner_lambda_pct", "inv_penalty", "exec_penalty_milli", "mm_space", "pv_ref")] + \
        [("reserved", ctypes.c_int32 * 2)]


class lob_ppo_hparams(ctypes.Structure):
    """Hyperparameters of lob_ppo_update (see include/lob.h)."""
    _fields_ = [(n, ctypes.c_float) for n in ("gamma", "gae_lambda", "clip_eps", "vf_coef", "ent_coef", "lr",
                                                "beta1", "beta2", "adam_eps", "max_grad_norm", "reward_scale")] + \
        [("n_minibatches", ctypes.c_int32)]


class lob_ppo_batch(ctypes.Structure):
    """Rollout data of lob_ppo_update (device pointers, see include/lob.h)."""
    _fields_ = [("T", ctypes.c_int32), ("n_envs", ctypes.c_int32)] + \
        [(n, ctypes.c_void_p) for n in ("d_obs", "d_actions", "d_logp_old", "d_values", "d_rewards", "d_done",
                                        "d_perm", "d_grad_out")]


class lob_noalloc_args(ctypes.Structure):
    """Arguments of lob_step_noalloc (see include/lob.h): every buffer is the caller's."""
    _fields_ = [("cfg", ctypes.POINTER(lob_config)), ("d_books", ctypes.c_void_p),
                ("d_env_state", ctypes.c_void_p), ("d_counters", ctypes.c_void_p),
                ("d_env_seeds", ctypes.c_void_p), ("d_msgs", ctypes.c_void_p),
                ("d_offsets", ctypes.c_void_p), ("stride", ctypes.c_int64), ("k", ctypes.c_int32),
                ("t", ctypes.c_int32), ("d_actions", ctypes.c_void_p), ("d_obs", ctypes.c_void_p),
                ("d_rewards", ctypes.c_void_p), ("d_done", ctypes.c_void_p), ("d_status", ctypes.c_void_p)]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def nvcc_cmd(out_path, extra=(), src=None):
    """Compile command of one translation unit (all of them for the shared object when src is None)."""
    base = ["nvcc", "-O3", "-std=c++17", *ARCH_FLAGS, "-lineinfo", "-Xcompiler", "-fPIC", "-I", _INC] + \
        (["-DLOB_CHECKED"] if CHECKED else [])
    if src is None:
        return base + ["-shared", "-o", out_path] + list(extra) + _SOURCES
    return base + ["-c", "-o", out_path] + list(extra) + [src]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblob.so in-tree for sm_103a: one nvcc per translation unit in
    parallel, then one link (nvcc cross-compiles without a GPU)."""
    with _lock:
        if not force and not _stale(LIB_PATH, _DEPS):
            return LIB_PATH
        os.makedirs(_OBJDIR, exist_ok=True)
        extra = ["-Xptxas", "-v"] if verbose else []
        procs, objs = [], []
        for src in _SOURCES:
            obj = os.path.join(_OBJDIR, os.path.basename(src) + f".{os.getpid()}.o")
            objs.append(obj)
            procs.append(subprocess.Popen(nvcc_cmd(obj, extra, src)))
        failed = [p.wait() for p in procs]
        if any(failed):
            raise RuntimeError("nvcc failed while building liblob.so")
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["nvcc", *ARCH_FLAGS, "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs)
        for o in objs:
            os.remove(o)
        os.replace(tmp, LIB_PATH)
        return LIB_PATH


def _load():
    global _lib, _lib_path
    if _lib is not None:
        # one library per process: handles, streams and device state belong to it
        if os.path.abspath(LIB_PATH) != _lib_path:
            raise RuntimeError(f"liblob.so already loaded from {_lib_path}; "
                               f"LIB_PATH now names {LIB_PATH}: use one process per library")
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblob.so is not built ({LIB_PATH}); call paper_2511_02136_gb300.lob.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "lob_obs_dim": (I32, [ctypes.POINTER(lob_config)]),
        "lob_create": (ctypes.c_int, [ctypes.POINTER(lob_config), P, ctypes.POINTER(P)]),
        "lob_destroy": (ctypes.c_int, [P]),
        "lob_load_messages": (ctypes.c_int, [P, P, P, I32, I64]),
        "lob_reset": (ctypes.c_int, [P, P, P]),
        "lob_step": (ctypes.c_int, [P, P, P]),
        "lob_observe": (ctypes.c_int, [P, P, P, P, P]),
        "lob_rollout": (ctypes.c_int, [P, I32, P, P, P, P, P]),
        "lob_step_host": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
        "lob_step_host_async": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
        "lob_load_messages16": (ctypes.c_int, [P, P, P, I32, I64]),
        "lob_set_episodes16": (ctypes.c_int, [P, P, P, I64, P, P, I32, I64]),
        "lob_pack_messages16": (ctypes.c_int, [P, I64, P, P, P]),
        "lob_book_bytes": (I64, [P]),
        "lob_get_book": (ctypes.c_int, [P, P, P]),
        "lob_get_counters": (ctypes.c_int, [P, P, P]),
        "lob_get_agents": (ctypes.c_int, [P, P, P]),
        "lob_get_env_misc": (ctypes.c_int, [P, P, P]),
        "lob_get_actions": (ctypes.c_int, [P, P, P]),
        "lob_live_orders": (ctypes.c_int, [P, P, P]),
        "lob_set_multi_split": (ctypes.c_int, [P, P]),
        "lob_set_threads_per_env": (ctypes.c_int, [P, I32]),
        "lob_set_tile_records": (ctypes.c_int, [P, I32]),
        "lob_set_trace": (ctypes.c_int, [P, P, I32, P, P, I64, P]),
        "lob_sync": (ctypes.c_int, [P, P]),
        "lob_set_launch": (ctypes.c_int, [P, I32, I32]),
        "lob_debug_wait": (ctypes.c_int, [P, ctypes.c_int64, I32]),
        "lob_kernel_launches": (I64, [P]),
        "lob_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lob_step_noalloc": (ctypes.c_int, [ctypes.POINTER(lob_noalloc_args), P]),
        "lob_policy_param_count": (I64, [I32]),
        "lob_policy_create": (ctypes.c_int, [I32, I32, P, ctypes.POINTER(P)]),
        "lob_policy_destroy": (ctypes.c_int, [P]),
        "lob_policy_forward": (ctypes.c_int, [P, P, I32, I32, P, P, P, P]),
        "lob_policy_sync": (ctypes.c_int, [P, P]),
        "lob_rollout_policy": (ctypes.c_int, [P, P, I32, I32, P, P, P, P, P]),
        "lob_set_env_costs": (ctypes.c_int, [P, P]),
        "lob_checkpoint_bytes": (I64, [P]),
        "lob_save": (ctypes.c_int, [P, P, P]),
        "lob_load": (ctypes.c_int, [P, P, P]),
        "lob_set_episodes": (ctypes.c_int, [P, P, P, I64, P, P, I32, I64]),
        "lob_get_episode_starts": (ctypes.c_int, [P, P, P]),
        "lob_policy_get_params": (ctypes.c_int, [P, P, P]),
        "lob_ppo_update": (ctypes.c_int, [P, ctypes.POINTER(lob_ppo_batch), ctypes.POINTER(lob_ppo_hparams), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    _lib_path = os.path.abspath(LIB_PATH)
    return lib


def _check(rc, what):
    if rc != LOB_OK:
        raise LobError(rc, what)
    return rc


def _dp(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---------------------------------------------------------------- same-name wrappers
def lob_obs_dim(cfg: lob_config) -> int:
    return _load().lob_obs_dim(ctypes.byref(cfg))


def lob_create(cfg: lob_config, caps=None):
    h = ctypes.c_void_p()
    c = None if caps is None else np.ascontiguousarray(caps, dtype=np.int32)
    _check(_load().lob_create(ctypes.byref(cfg), None if c is None else c.ctypes.data, ctypes.byref(h)),
           "lob_create")
    return h


def lob_destroy(h):
    return _check(_load().lob_destroy(h), "lob_destroy")


def lob_load_messages(h, msgs, offsets, n_steps, stride):
    return _check(_load().lob_load_messages(h, _dp(msgs), _dp(offsets), n_steps, stride), "lob_load_messages")


def lob_reset(h, seeds, stream=None):
    return _check(_load().lob_reset(h, _dp(seeds), _stream(stream)), "lob_reset")


def lob_step(h, actions=None, stream=None):
    return _check(_load().lob_step(h, _dp(actions), _stream(stream)), "lob_step")


def lob_observe(h, obs=None, rewards=None, done=None, stream=None):
    return _check(_load().lob_observe(h, _dp(obs), _dp(rewards), _dp(done), _stream(stream)), "lob_observe")


def lob_rollout(h, n_steps, actions=None, obs=None, rewards=None, done=None, stream=None):
    return _check(_load().lob_rollout(h, n_steps, _dp(actions), _dp(obs), _dp(rewards), _dp(done),
                                      _stream(stream)), "lob_rollout")


def lob_step_host(h, msgs, offsets, actions, obs, rewards, done, stream=None):
    """Host numpy (ideally pinned) buffers in and out; synchronises."""
    def hp(a):
        return None if a is None else a.ctypes.data
    return _check(_load().lob_step_host(h, hp(msgs), hp(offsets), hp(actions), hp(obs), hp(rewards), hp(done),
                                        _stream(stream)), "lob_step_host")


def lob_step_host_async(h, msgs, offsets, actions, obs, rewards, done, stream=None):
    """Pipelined host step: buffers (pinned torch tensors or numpy arrays) must stay
    untouched, and outputs unread, until `stream` is synchronised."""
    def hp(a):
        return None if a is None else _anyp(a)
    return _check(_load().lob_step_host_async(h, hp(msgs), hp(offsets), hp(actions), hp(obs), hp(rewards),
                                              hp(done), _stream(stream)), "lob_step_host_async")


def lob_book_bytes(h) -> int:
    return _load().lob_book_bytes(h)


def lob_get_book(h, out, stream=None):
    return _check(_load().lob_get_book(h, _dp(out), _stream(stream)), "lob_get_book")


def lob_get_counters(h, out, stream=None):
    return _check(_load().lob_get_counters(h, _dp(out), _stream(stream)), "lob_get_counters")


def lob_get_agents(h, out, stream=None):
    return _check(_load().lob_get_agents(h, _dp(out), _stream(stream)), "lob_get_agents")


def lob_get_env_misc(h, out, stream=None):
    return _check(_load().lob_get_env_misc(h, _dp(out), _stream(stream)), "lob_get_env_misc")


def lob_get_actions(h, out, stream=None):
    return _check(_load().lob_get_actions(h, _dp(out), _stream(stream)), "lob_get_actions")


def lob_set_threads_per_env(h, threads):
    """32: one warp per env; 64: one warp per book side for the plain step (see include/lob.h)."""
    return _check(_load().lob_set_threads_per_env(h, threads), "lob_set_threads_per_env")


def lob_set_tile_records(h, records):
    """Records per staged message tile: 16, 32 (default) or 64."""
    return _check(_load().lob_set_tile_records(h, records), "lob_set_tile_records")


def lob_set_multi_split(h, warps_per_class):
    """One persistent kernel over the capacity classes, with this many warps of
    each class per block (LOB_NCLASSES entries; see include/lob.h)."""
    w = np.ascontiguousarray(warps_per_class, dtype=np.int32)
    if w.shape != (6,):
        raise ValueError("six classes")
    return _check(_load().lob_set_multi_split(h, w.ctypes.data), "lob_set_multi_split")


def lob_live_orders(h, acc, stream=None):
    """Adds the resting orders of every env (bids + asks) to the int64 device scalar acc."""
    return _check(_load().lob_live_orders(h, _dp(acc), _stream(stream)), "lob_live_orders")


def lob_set_trace(h, fills=None, fill_cap=0, fill_counts=None, snaps=None, snap_cap=0, snap_count=None):
    return _check(_load().lob_set_trace(h, _dp(fills), fill_cap, _dp(fill_counts), _dp(snaps), snap_cap,
                                        _dp(snap_count)), "lob_set_trace")


def lob_sync(h, stream=None):
    """Returns the device status code (0, or LOB_EBADMSG / LOB_EINVAL / LOB_ETIMEOUT)."""
    return _load().lob_sync(h, _stream(stream))


def lob_set_launch(h, warps_per_block, persistent):
    return _check(_load().lob_set_launch(h, warps_per_block, persistent), "lob_set_launch")


def lob_debug_wait(h, cycles, hold):
    """Failure-detection hook: wait bound in SM cycles (0 = default) and, with
    hold=1, the next launch's first message tile left unrequested."""
    return _check(_load().lob_debug_wait(h, cycles, hold), "lob_debug_wait")


def lob_set_env_costs(h, costs=None):
    c = None if costs is None else np.ascontiguousarray(costs, dtype=np.float32)
    return _check(_load().lob_set_env_costs(h, None if c is None else c.ctypes.data), "lob_set_env_costs")


def lob_checkpoint_bytes(h) -> int:
    return _load().lob_checkpoint_bytes(h)


def _anyp(buf):
    """Pointer of a torch tensor (host or device) or a numpy array."""
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    return buf.ctypes.data


def lob_save(h, dst, stream=None):
    return _check(_load().lob_save(h, _anyp(dst), _stream(stream)), "lob_save")


def lob_load(h, src, stream=None):
    return _check(_load().lob_load(h, _anyp(src), _stream(stream)), "lob_load")


def lob_set_episodes(h, msgs_dev, step_offsets_dev, starts, levels):
    """Episode mode over one shared stream.  msgs_dev / step_offsets_dev: device
    tensors (32-byte records; int64 [n_data_steps + 1]); starts START_DTYPE[n]
    and levels int32 [n, 2, levels_per_side, 2] on the host (copied)."""
    starts = np.ascontiguousarray(starts, dtype=START_DTYPE)
    levels = np.ascontiguousarray(levels, dtype=np.int32)
    n_data = step_offsets_dev.shape[0] - 1
    return _check(_load().lob_set_episodes(h, _dp(msgs_dev), _dp(step_offsets_dev), n_data,
                                           starts.ctypes.data, levels.ctypes.data, levels.shape[2],
                                           len(starts)), "lob_set_episodes")


def lob_load_messages16(h, msgs_dev, offsets_dev, n_steps, stride):
    return _check(_load().lob_load_messages16(h, _dp(msgs_dev), _dp(offsets_dev), n_steps, stride),
                  "lob_load_messages16")


def lob_set_episodes16(h, msgs_dev, step_offsets_dev, starts, levels):
    starts = np.ascontiguousarray(starts, dtype=START_DTYPE)
    levels = np.ascontiguousarray(levels, dtype=np.int32)
    n_data = step_offsets_dev.shape[0] - 1
    return _check(_load().lob_set_episodes16(h, _dp(msgs_dev), _dp(step_offsets_dev), n_data, starts.ctypes.data,
                                             levels.ctypes.data, levels.shape[2], len(starts)), "lob_set_episodes16")


def lob_pack_messages16(src_dev, n, dst_dev, status_dev=None, stream=None):
    """Device 32-byte records -> 16-byte compact records (status int32 set to LOB_EINVAL on an id out of range)."""
    return _check(_load().lob_pack_messages16(_dp(src_dev), n, _dp(dst_dev), _dp(status_dev), _stream(stream)),
                  "lob_pack_messages16")


def lob_get_episode_starts(h, out, stream=None):
    return _check(_load().lob_get_episode_starts(h, _dp(out), _stream(stream)), "lob_get_episode_starts")


def lob_kernel_launches(h) -> int:
    return _load().lob_kernel_launches(h)


def lob_step_noalloc(args: lob_noalloc_args, stream=None):
    """One env step on caller-owned buffers; allocates nothing (see include/lob.h)."""
    return _check(_load().lob_step_noalloc(ctypes.byref(args), _stream(stream)), "lob_step_noalloc")


def noalloc_book_block_bytes(cap: int) -> int:
    """Bytes of one env's book block for lob_step_noalloc (48*S rounded up to 256)."""
    S = 32
    while S < cap:
        S *= 2
    return ((48 * S + 255) // 256) * 256


def lob_policy_param_count(obs_dim: int) -> int:
    return _load().lob_policy_param_count(obs_dim)


def lob_policy_create(n_agents, obs_dim, params):
    """params: host float32 array [n_agents, lob_policy_param_count(obs_dim)]."""
    w = np.ascontiguousarray(params, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(_load().lob_policy_create(n_agents, obs_dim, w.ctypes.data, ctypes.byref(h)), "lob_policy_create")
    return h


def lob_policy_destroy(pol):
    return _check(_load().lob_policy_destroy(pol), "lob_policy_destroy")


def lob_policy_forward(pol, obs, n_envs, precision, logits=None, values=None, actions=None, stream=None):
    return _check(_load().lob_policy_forward(pol, _dp(obs), n_envs, precision, _dp(logits), _dp(values),
                                             _dp(actions), _stream(stream)), "lob_policy_forward")


def lob_policy_sync(pol, stream=None):
    return _load().lob_policy_sync(pol, _stream(stream))


def lob_rollout_policy(h, pol, n_steps, precision, obs=None, rewards=None, done=None, actions=None, stream=None):
    return _check(_load().lob_rollout_policy(h, pol, n_steps, precision, _dp(obs), _dp(rewards), _dp(done),
                                             _dp(actions), _stream(stream)), "lob_rollout_policy")


def lob_policy_get_params(pol, out, stream=None):
    """The FP32 parameter blocks of every agent into the device tensor out [n_agents, P]."""
    return _check(_load().lob_policy_get_params(pol, _dp(out), _stream(stream)), "lob_policy_get_params")


def lob_ppo_update(pol, T, n_envs, obs, actions, logp_old, values, rewards, done, perm, hp: lob_ppo_hparams,
                   grad_out=None, stream=None):
    """One IPPO epoch on the GPU from rollout tensors (see include/lob.h for the layouts)."""
    b = lob_ppo_batch(T=T, n_envs=n_envs, d_obs=_dp(obs), d_actions=_dp(actions), d_logp_old=_dp(logp_old),
                      d_values=_dp(values), d_rewards=_dp(rewards), d_done=_dp(done), d_perm=_dp(perm),
                      d_grad_out=_dp(grad_out))
    return _check(_load().lob_ppo_update(pol, ctypes.byref(b), ctypes.byref(hp), _stream(stream)), "lob_ppo_update")


def ppo_hparams(**kw) -> lob_ppo_hparams:
    """The update's hyperparameters with the defaults of the FP64 reference update."""
    d = dict(gamma=0.99, gae_lambda=0.95, clip_eps=0.2, vf_coef=0.5, ent_coef=0.01, lr=2.5e-4, beta1=0.9,
             beta2=0.999, adam_eps=1e-5, max_grad_norm=0.5, reward_scale=1e-2, n_minibatches=4)
    d.update(kw)
    return lob_ppo_hparams(**d)


def init_policy_params(seed: int, n_agents: int, obs_dim: int) -> np.ndarray:
    """Weights N(0, 1/fan_in), biases 0, per agent (float32, host)."""
    rng = np.random.default_rng(seed)
    H = POLICY_HIDDEN
    out = []
    for _ in range(n_agents):
        w1 = rng.standard_normal((H, obs_dim)) / np.sqrt(obs_dim)
        w2 = rng.standard_normal((H, H)) / np.sqrt(H)
        w3 = rng.standard_normal((13, H)) / np.sqrt(H)
        out.append(np.concatenate([w1.ravel(), np.zeros(H), w2.ravel(), np.zeros(H), w3.ravel(), np.zeros(13)]))
    return np.stack(out).astype(np.float32)


def lob_strerror(code) -> str:
    return _load().lob_strerror(code).decode()


def book_dtype(C):
    return np.dtype([("n", "<i4", (2,)), ("px", "<i4", (2, C)), ("qty", "<i4", (2, C)),
                     ("id", "<i8", (2, C)), ("ts", "<i8", (2, C))])


FILL_DTYPE = np.dtype([("maker_id", "<i8"), ("taker_id", "<i8"), ("px", "<i4"), ("qty", "<i4"),
                       ("msg_idx", "<i4"), ("taker_side", "<i4")])


class LobEnv:
    """Convenience owner of a handle plus torch output buffers (all on the current CUDA device)."""

    def __init__(self, n_envs, n_agents=2, cap=100, top_levels=10, episode_len=1000, mm_lot=1,
                 exec_target=500, exec_dir=-1, action_mode=LOB_ACT_RANDOM, start_px=10_000,
                 warps_per_block=0, caps=None, reward_mode=0, spooner_lambda_pct=0, inv_penalty=0,
                 exec_penalty_milli=0, mm_space=0, pv_ref=0):
        import torch
        self.torch = torch
        self.cfg = lob_config(n_envs, n_agents, cap, top_levels, episode_len, mm_lot, exec_target,
                              exec_dir, action_mode, 0, start_px, warps_per_block, reward_mode,
                              spooner_lambda_pct, inv_penalty, exec_penalty_milli, mm_space, pv_ref)
        self.caps = caps
        self.h = lob_create(self.cfg, caps)
        self.n_envs, self.n_agents = n_envs, n_agents
        self.D = lob_obs_dim(self.cfg)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        self.obs = torch.zeros((n_envs, n_agents, self.D), dtype=torch.float32, device=dev)
        self.rew = torch.zeros((n_envs, max(n_agents, 1)), dtype=torch.int64, device=dev)
        self.done = torch.zeros(n_envs, dtype=torch.uint8, device=dev)
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            lob_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_messages(self, msgs_dev, offsets_dev):
        """msgs_dev: uint8/int64 tensor of 32-byte records; offsets_dev int64 [n_envs, n_steps+1]."""
        self._keep = [msgs_dev, offsets_dev]
        lob_load_messages(self.h, msgs_dev, offsets_dev, offsets_dev.shape[1] - 1, offsets_dev.shape[1])

    def set_episodes(self, msgs_dev, step_offsets_dev, starts, levels, compact=False):
        self._keep = [msgs_dev, step_offsets_dev]
        (lob_set_episodes16 if compact else lob_set_episodes)(self.h, msgs_dev, step_offsets_dev, starts, levels)

    def load_messages16(self, msgs16_dev, offsets_dev):
        """msgs16_dev: uint8/int64 tensor of 16-byte compact records; offsets_dev int64 [n_envs, n_steps+1]."""
        self._keep = [msgs16_dev, offsets_dev]
        lob_load_messages16(self.h, msgs16_dev, offsets_dev, offsets_dev.shape[1] - 1, offsets_dev.shape[1])

    def episode_starts(self):
        out = self.torch.zeros(self.n_envs, dtype=self.torch.int32, device=self.dev)
        lob_get_episode_starts(self.h, out)
        return out

    def reset(self, seeds_dev, stream=None):
        self._seeds = seeds_dev
        lob_reset(self.h, seeds_dev, stream)

    def step(self, actions=None, stream=None):
        lob_step(self.h, actions, stream)

    def observe(self, stream=None):
        lob_observe(self.h, self.obs, self.rew if self.n_agents else None, self.done, stream)
        return self.obs, self.rew, self.done

    def counters(self):
        out = self.torch.zeros((self.n_envs, LOB_NCOUNTERS), dtype=self.torch.int64, device=self.dev)
        lob_get_counters(self.h, out)
        return out

    def agents(self):
        out = self.torch.zeros((self.n_envs, max(self.n_agents, 1), 4), dtype=self.torch.int64, device=self.dev)
        lob_get_agents(self.h, out)
        return out[:, :self.n_agents]

    def env_misc(self):
        out = self.torch.zeros((self.n_envs, 4), dtype=self.torch.int64, device=self.dev)
        lob_get_env_misc(self.h, out)
        return out

    def actions(self):
        out = self.torch.zeros((self.n_envs, max(self.n_agents, 2)), dtype=self.torch.int32, device=self.dev)
        lob_get_actions(self.h, out)
        return out[:, :self.n_agents]

    def books(self):
        """List of per-env canonical book records (numpy) in env order."""
        nb = lob_book_bytes(self.h)
        out = self.torch.zeros(nb, dtype=self.torch.uint8, device=self.dev)
        lob_get_book(self.h, out)
        raw = out.cpu().numpy()
        caps = (np.full(self.n_envs, self.cfg.cap_per_side, np.int32) if self.caps is None
                else np.asarray(self.caps, np.int32))
        recs, off = [], 0
        for e in range(self.n_envs):
            dt = book_dtype(int(caps[e]))
            recs.append(np.frombuffer(raw[off:off + dt.itemsize].tobytes(), dtype=dt)[0])
            off += dt.itemsize
        return recs

    def books_live(self):
        """Mean number of live orders per env (bids + asks), read on the device."""
        nb = lob_book_bytes(self.h)
        if getattr(self, "_bookbuf", None) is None or self._bookbuf.numel() != nb:
            self._bookbuf = self.torch.zeros(nb, dtype=self.torch.uint8, device=self.dev)
            caps = (np.full(self.n_envs, self.cfg.cap_per_side, np.int64) if self.caps is None
                    else np.asarray(self.caps, np.int64))
            rec = 8 + 48 * caps
            off = np.concatenate([[0], np.cumsum(rec)[:-1]]) // 4
            self._nidx = self.torch.from_numpy(np.stack([off, off + 1], 1).reshape(-1)).to(self.dev)
        lob_get_book(self.h, self._bookbuf)
        n = self._bookbuf.view(self.torch.int32)[self._nidx]
        return n.double().sum().item() / self.n_envs

    def sync(self):
        return lob_sync(self.h)
