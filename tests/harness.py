"""Shared drivers for the GPU-vs-oracle parity tests.

Both sides read the same generated message bytes; neither sees the other's
results.  Integers (books, fills, counters, cash, inventory, rewards) must be
bit-identical; observations must match within 1e-6 relative (each entry is one
correctly rounded int->float conversion or one IEEE divide on both sides, so
in practice they are identical as well).
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2511_02136_gb300 import lob, mbogen

OBS_RTOL = 1e-6


def to_dev(a):
    import torch
    if a.dtype.fields is not None:
        a = a.view(np.uint8)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()


class Pair:
    """A GPU env handle and an oracle fed identical inputs."""

    def __init__(self, n_envs, st, *, n_agents=2, cap=100, caps=None, top_levels=10, episode_len=None,
                 mm_lot=1, exec_target=500, exec_dir=-1, action_mode=lob.LOB_ACT_RANDOM, start_px=10_000,
                 fill_cap=0, snap_cap=0, warps_per_block=0, persistent=0, n_threads=1, rewards=None,
                 episodes=None, seeds=None, mm_space=0, compact=False, threads_per_env=32, tile_records=32):
        """episodes: (starts, levels) puts both sides in episode mode over the
        single shared stream st (env 0 of st); seeds then gives the env seeds."""
        import torch
        self.torch = torch
        T = st.offsets.shape[1] - 1 if episode_len is None else episode_len
        self.n_envs, self.n_agents, self.T = n_envs, n_agents, T
        self.st = st
        self.env = lob.LobEnv(n_envs, n_agents=n_agents, cap=cap, top_levels=top_levels, episode_len=T,
                              mm_lot=mm_lot, exec_target=exec_target, exec_dir=exec_dir,
                              action_mode=action_mode, start_px=start_px, warps_per_block=warps_per_block,
                              caps=caps, mm_space=mm_space, **(rewards or {}))
        if warps_per_block or persistent:
            lob.lob_set_launch(self.env.h, warps_per_block or 4, persistent)
        if threads_per_env != 32:
            lob.lob_set_threads_per_env(self.env.h, threads_per_env)
        if tile_records != 32:
            lob.lob_set_tile_records(self.env.h, tile_records)
        self.orc = oracle.Oracle(n_envs, n_agents=n_agents, cap=cap, top_levels=top_levels, episode_len=T,
                                 mm_lot=mm_lot, exec_target=exec_target, exec_dir=exec_dir,
                                 action_mode=action_mode, trace=(1 if fill_cap else 0) | (2 if snap_cap else 0),
                                 start_px=start_px, n_threads=n_threads, caps=caps, mm_space=mm_space,
                                 **(rewards or {}))
        # compact: the GPU reads the 16-byte encoding, the oracle the 32-byte records
        dev_msgs = mbogen.pack16(st.msgs) if compact else st.msgs
        self.msgs_d = to_dev(dev_msgs) if len(dev_msgs) else torch.zeros(32, dtype=torch.uint8, device="cuda")
        self.off_d = to_dev(st.offsets)
        if episodes is None:
            (self.env.load_messages16 if compact else self.env.load_messages)(self.msgs_d, self.off_d)
            self.orc.load_messages(st.msgs, st.offsets)
        else:
            self.env.set_episodes(self.msgs_d, self.off_d[0], *episodes, compact=compact)
            self.orc.set_episodes(st.msgs, st.offsets[0], *episodes)
        seeds = st.seeds if seeds is None else np.ascontiguousarray(seeds, np.uint64)
        self.seeds_d = to_dev(seeds)
        self.env.reset(self.seeds_d)
        self.orc.reset(seeds)
        self.fill_cap, self.snap_cap = fill_cap, snap_cap
        if fill_cap or snap_cap:
            C = cap if caps is None else int(caps[0])
            self.fills_d = torch.zeros((n_envs, max(fill_cap, 1), 32), dtype=torch.uint8, device="cuda")
            self.fcnt_d = torch.zeros(n_envs, dtype=torch.int32, device="cuda")
            self.snap_dt = lob.book_dtype(C)
            self.snaps_d = torch.zeros((max(snap_cap, 1), self.snap_dt.itemsize), dtype=torch.uint8, device="cuda")
            self.scnt_d = torch.zeros(1, dtype=torch.int64, device="cuda")
            lob.lob_set_trace(self.env.h, self.fills_d if fill_cap else None, fill_cap,
                              self.fcnt_d if fill_cap else None, self.snaps_d if snap_cap else None, snap_cap,
                              self.scnt_d if snap_cap else None)

    def step(self, actions=None):
        a_d = None if actions is None else self.torch.from_numpy(np.ascontiguousarray(actions, np.int32)).cuda()
        self.env.step(a_d)
        rc_o = self.orc.step(actions)
        return rc_o

    # ---------------------------------------------------------------- checks
    def check_outputs(self):
        obs, rew, done = self.env.observe()
        o_obs, o_rew, o_done = self.orc.observe()
        g_obs = obs.cpu().numpy()
        np.testing.assert_allclose(g_obs, o_obs, rtol=OBS_RTOL, atol=0)
        if self.n_agents:
            np.testing.assert_array_equal(rew.cpu().numpy(), o_rew)
            np.testing.assert_array_equal(self.env.actions().cpu().numpy(), self.orc.actions())
        np.testing.assert_array_equal(done.cpu().numpy(), o_done)
        if self.orc._ep is not None:
            np.testing.assert_array_equal(self.env.episode_starts().cpu().numpy(), self.orc.episode_starts())
        return g_obs, o_obs

    def check_state(self, envs=None):
        envs = range(self.n_envs) if envs is None else envs
        g_cnt = self.env.counters().cpu().numpy()
        o_cnt = self.orc.counters()
        np.testing.assert_array_equal(g_cnt[list(envs)], o_cnt[list(envs)])
        if self.n_agents:
            np.testing.assert_array_equal(self.env.agents().cpu().numpy()[list(envs)], self.orc.agents()[list(envs)])
        g_misc = self.env.env_misc().cpu().numpy()
        o_misc = self.orc.env_misc()
        np.testing.assert_array_equal(g_misc[list(envs), :3], o_misc[list(envs), :3])
        assert np.all(g_misc[:, 3] == o_misc[0, 3])
        books = self.env.books()
        for e in envs:
            n2, px, qty, oid, ts = self.orc.book(e)
            b = books[e]
            assert b["n"].tolist() == n2.tolist(), f"env {e}: counts"
            for s in range(2):
                n = n2[s]
                np.testing.assert_array_equal(b["px"][s][:n], px[s][:n], err_msg=f"env {e} side {s} px")
                np.testing.assert_array_equal(b["qty"][s][:n], qty[s][:n], err_msg=f"env {e} side {s} qty")
                np.testing.assert_array_equal(b["id"][s][:n], oid[s][:n], err_msg=f"env {e} side {s} id")
                np.testing.assert_array_equal(b["ts"][s][:n], ts[s][:n], err_msg=f"env {e} side {s} ts")

    def check_fills(self):
        cnt = self.fcnt_d.cpu().numpy()
        raw = self.fills_d.cpu().numpy()
        for e in range(self.n_envs):
            want = self.orc.fills(e)
            assert cnt[e] == len(want), f"env {e}: fill count {cnt[e]} vs {len(want)}"
            k = min(len(want), self.fill_cap)
            got = np.frombuffer(raw[e, :k].tobytes(), dtype=lob.FILL_DTYPE)
            np.testing.assert_array_equal(got, want[:k].view(lob.FILL_DTYPE))

    def check_snapshots(self):
        n = int(self.scnt_d.cpu().item())
        want = self.orc.snapshots()
        assert n == len(want)
        k = min(n, self.snap_cap)
        got = np.frombuffer(self.snaps_d[:k].cpu().numpy().tobytes(), dtype=self.snap_dt)
        np.testing.assert_array_equal(got.view(np.uint8), want[:k].view(np.uint8))

    def close(self):
        if lob.CHECKED:   # checked build: no index bound or book invariant may have failed
            assert self.env.sync() != lob.LOB_ECHECK, "checked build: device invariant failed"
        self.env.close()
