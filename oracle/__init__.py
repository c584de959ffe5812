"""CPU oracle of the batched LOB environment step -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it and shares no code with it.

``oracle.cpp`` is the plain C++ restatement of the environment step of
JaxMARL-HFT Sec. 4 ("Design"), one env at a time, with textbook std::map price
levels.  The tests pin it with hand-worked examples, invariants and an even
simpler pure-Python sorted-list book (``tests/brute_lob.py``) on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NCOUNTERS = 16
COUNTER_NAMES = [
    "msgs", "agent_msgs", "fills", "fill_vol", "add_vol", "mkt_vol", "mkt_discard_vol",
    "cancel_vol", "cancel_miss", "drop_vol", "drop_cnt", "evict_vol", "evict_cnt",
    "bad_msgs", "bg_cash", "bg_inv",
]
FILL_DTYPE = np.dtype([("maker_id", "<i8"), ("taker_id", "<i8"), ("px", "<i4"),
                       ("qty", "<i4"), ("msg_idx", "<i4"), ("taker_side", "<i4")])
TAG_SHUFFLE = 0x5348554646000001
TAG_POLICY = 0x504F4C4943590002
TAG_EPISODE = 0x4550495344450003
INIT_ID = 0x4000000000000000
START_DTYPE = np.dtype([("data_step", "<i4"), ("last_px", "<i4"), ("n_bid", "<i4"), ("n_ask", "<i4")])


class OrcConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_envs", "n_agents", "cap", "top_levels", "episode_len", "mm_lot", "exec_target",
        "exec_dir", "action_mode", "trace", "start_px", "n_threads", "reward_mode",
        "spooner_lambda_pct", "inv_penalty", "exec_penalty_milli", "mm_space", "pv_ref")]


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree (portable flags, no fast-math, no FMA contraction)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.POINTER(OrcConfig), P]
        lib.orc_destroy.argtypes = [P]
        lib.orc_reset.argtypes = [P, P]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_step.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int32]
        lib.orc_observe.argtypes = [P, P, P, P]
        lib.orc_set_episodes.argtypes = [P, P, P, ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_int64]
        lib.orc_step_episodes.restype = ctypes.c_int
        lib.orc_step_episodes.argtypes = [P, P]
        lib.orc_get_episode.argtypes = [P, P]
        lib.orc_obs_dim.restype = ctypes.c_int32
        lib.orc_obs_dim.argtypes = [P]
        lib.orc_get_book.argtypes = [P, ctypes.c_int64, P, P, P, P, P]
        lib.orc_get_counters.argtypes = [P, P]
        lib.orc_get_agents.argtypes = [P, P]
        lib.orc_get_env_misc.argtypes = [P, P]
        lib.orc_get_actions.argtypes = [P, P]
        lib.orc_get_fills.restype = ctypes.c_int64
        lib.orc_get_fills.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64]
        lib.orc_get_snapshots.restype = ctypes.c_int64
        lib.orc_get_snapshots.argtypes = [P, P, ctypes.c_int64]
        lib.orc_draw.restype = ctypes.c_uint64
        lib.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64]
        lib.orc_lemire.restype = ctypes.c_uint32
        lib.orc_lemire.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_splitmix.restype = ctypes.c_uint64
        lib.orc_splitmix.argtypes = [ctypes.c_uint64, ctypes.c_int64]
        _lib = lib
    return _lib


def draw(env_seed: int, t: int, tag: int, i: int) -> int:
    return _load().orc_draw(env_seed & (2**64 - 1), t, tag, i)


def splitmix(state: int, i: int) -> int:
    return _load().orc_splitmix(state & (2**64 - 1), i)


def lemire(x: int, n: int) -> int:
    return _load().orc_lemire(x & (2**64 - 1), n)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """One oracle instance: n_envs independent books plus agent state."""

    def __init__(self, n_envs, n_agents=2, cap=100, top_levels=10, episode_len=1000,
                 mm_lot=1, exec_target=500, exec_dir=-1, action_mode=1, trace=0,
                 start_px=10_000, n_threads=1, caps=None, reward_mode=0, spooner_lambda_pct=0,
                 inv_penalty=0, exec_penalty_milli=0, mm_space=0, pv_ref=0):
        self.lib = _load()
        self.cfg = OrcConfig(n_envs, n_agents, cap, top_levels, episode_len, mm_lot,
                             exec_target, exec_dir, action_mode, trace, start_px, n_threads,
                             reward_mode, spooner_lambda_pct, inv_penalty, exec_penalty_milli, mm_space, pv_ref)
        self.caps = None if caps is None else np.ascontiguousarray(caps, dtype=np.int32)
        self.h = self.lib.orc_create(ctypes.byref(self.cfg), _ptr(self.caps))
        if not self.h:
            raise ValueError("invalid oracle configuration")
        self.n_envs, self.n_agents = n_envs, n_agents
        self.obs_dim = self.lib.orc_obs_dim(self.h)
        self._msgs = self._offsets = None
        self._ep = None

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def cap_of(self, env):
        return int(self.caps[env]) if self.caps is not None else self.cfg.cap

    def reset(self, env_seeds):
        self._seeds = np.ascontiguousarray(env_seeds, dtype=np.uint64)
        self.lib.orc_reset(self.h, self._seeds.ctypes.data)

    def load_messages(self, msgs, offsets):
        self._msgs = np.ascontiguousarray(msgs)
        self._offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self._k = 0

    def set_episodes(self, msgs, step_offsets, starts, levels):
        """Episode mode over one shared stream: msgs MSG_DTYPE[N], step_offsets
        int64[n_data_steps + 1], starts START_DTYPE[n_starts], levels
        int32[n_starts, 2, levels_per_side, 2] (price, quantity), best first."""
        msgs = np.ascontiguousarray(msgs)
        off = np.ascontiguousarray(step_offsets, dtype=np.int64)
        starts = np.ascontiguousarray(starts, dtype=START_DTYPE)
        levels = np.ascontiguousarray(levels, dtype=np.int32)
        self._ep = (msgs, off, starts, levels)   # msgs must outlive the handle's use
        self.lib.orc_set_episodes(self.h, msgs.ctypes.data if len(msgs) else None, off.ctypes.data,
                                  len(off) - 1, starts.ctypes.data, levels.ctypes.data,
                                  levels.shape[2], len(starts))

    def episode_starts(self):
        out = np.zeros(self.n_envs, np.int64)
        self.lib.orc_get_episode(self.h, out.ctypes.data)
        return out

    def step(self, actions=None):
        acts = None if actions is None else np.ascontiguousarray(actions, dtype=np.int32)
        if self._ep is not None:
            return self.lib.orc_step_episodes(self.h, _ptr(acts))
        rc = self.lib.orc_step(self.h, _ptr(acts), self._msgs.ctypes.data,
                               self._offsets.ctypes.data, self._offsets.shape[1], self._k)
        self._k += 1
        return rc

    def observe(self):
        A, D = self.n_agents, self.obs_dim
        obs = np.zeros((self.n_envs, A, D), dtype=np.float32)
        rew = np.zeros((self.n_envs, A), dtype=np.int64)
        done = np.zeros(self.n_envs, dtype=np.uint8)
        self.lib.orc_observe(self.h, obs.ctypes.data, rew.ctypes.data, done.ctypes.data)
        return obs, rew, done

    def book(self, env):
        C = self.cap_of(env)
        n2 = np.zeros(2, np.int32)
        px = np.zeros((2, C), np.int32)
        qty = np.zeros((2, C), np.int32)
        oid = np.zeros((2, C), np.int64)
        ts = np.zeros((2, C), np.int64)
        self.lib.orc_get_book(self.h, env, n2.ctypes.data, px.ctypes.data, qty.ctypes.data,
                              oid.ctypes.data, ts.ctypes.data)
        return n2, px, qty, oid, ts

    def counters(self):
        out = np.zeros((self.n_envs, NCOUNTERS), np.int64)
        self.lib.orc_get_counters(self.h, out.ctypes.data)
        return out

    def agents(self):
        out = np.zeros((self.n_envs, max(self.n_agents, 1), 4), np.int64)
        self.lib.orc_get_agents(self.h, out.ctypes.data)
        return out[:, :self.n_agents]

    def env_misc(self):
        out = np.zeros((self.n_envs, 4), np.int64)
        self.lib.orc_get_env_misc(self.h, out.ctypes.data)
        return out

    def actions(self):
        out = np.zeros((self.n_envs, max(self.n_agents, 1)), np.int32)
        self.lib.orc_get_actions(self.h, out.ctypes.data)
        return out[:, :self.n_agents]

    def fills(self, env):
        n = self.lib.orc_get_fills(self.h, env, None, 0)
        out = np.zeros(n, FILL_DTYPE)
        if n:
            self.lib.orc_get_fills(self.h, env, out.ctypes.data, n)
        return out

    def snapshots(self):
        C = self.cap_of(0)
        n = self.lib.orc_get_snapshots(self.h, None, 0)
        rec = snapshot_dtype(C)
        out = np.zeros(n, rec)
        if n:
            self.lib.orc_get_snapshots(self.h, out.ctypes.data, n)
        return out


def snapshot_dtype(C):
    """Canonical book record: counts, then px/qty/id/ts per side in priority order."""
    return np.dtype([("n", "<i4", (2,)), ("px", "<i4", (2, C)), ("qty", "<i4", (2, C)),
                     ("id", "<i8", (2, C)), ("ts", "<i8", (2, C))])
