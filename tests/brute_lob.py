"""Brute-force environment step: one Python list per side, re-sorted after every change.

A second, deliberately naive restatement of the env step (JaxMARL-HFT Sec. 4)
used only to pin the C++ oracle on tiny inputs.  It keeps each side as a flat
list of orders and recomputes priority order by sorting, so it has no price
level structure, no iterators and no special cases to share mistakes with.
"""
from __future__ import annotations

from fractions import Fraction

BUY, SELL = 1, -1
ADD, PARTIAL, DELETE, MARKET = 1, 2, 3, 4
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
TAG_SHUFFLE = 0x5348554646000001
TAG_POLICY = 0x504F4C4943590002
TAG_EPISODE = 0x4550495344450003
TAG_TASKDIR = 0x5441534B44495204
INIT_ID = 1 << 62


def _mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix_outputs(state, n):
    out = []
    for _ in range(n):
        state = (state + GAMMA) & M64
        out.append(_mix(state))
    return out


def keyed_draws(env_seed, t, tag, n):
    key = _mix(((_mix(env_seed ^ tag)) + GAMMA * (t + 1)) & M64)
    return splitmix_outputs(key, n)


def bounded(x, n):
    return ((x >> 32) * n) >> 32


def wrap(v):
    v &= M64
    return v - (1 << 64) if v >> 63 else v


class BruteEnv:
    def __init__(self, cap, n_agents=0, top_levels=2, episode_len=10, mm_lot=1,
                 exec_target=10, exec_dir=SELL, start_px=10_000, seed=0, action_mode=0,
                 reward_mode=0, spooner_lambda_pct=0, inv_penalty=0, exec_penalty_milli=0, mm_space=0,
                 pv_ref=0):
        self.cap, self.A, self.L, self.T = cap, n_agents, top_levels, episode_len
        self.mm_lot, self.exec_target = mm_lot, exec_target
        self.exec_dir_cfg = exec_dir              # 0: the side is drawn per episode
        self.action_mode, self.seed = action_mode, seed
        self.exec_dir = self._task_dir(0)
        self.reward_mode, self.lam_pct = reward_mode, spooner_lambda_pct
        self.inv_penalty, self.exec_penalty_milli = inv_penalty, exec_penalty_milli
        self.mm_space = mm_space
        self.pv_ref = pv_ref     # 0 liquidation touch, 1 mid (PV in half ticks)
        self.orders = {BUY: [], SELL: []}   # dicts: px, qty, id, ts
        self.ts_next = 0
        self.seq_next = 0
        self.last_px = start_px
        self.t = 0
        self.inv = [0] * n_agents
        self.cash = [0] * n_agents
        self.pv_prev = [0] * n_agents
        self.P = n_agents // 2            # agents per type: 0..P-1 execute, P..2P-1 make markets
        self.exec_done = [0] * n_agents
        self.bg_cash = 0
        self.bg_inv = 0
        self.c = dict(msgs=0, agent_msgs=0, fills=0, fill_vol=0, add_vol=0, mkt_vol=0,
                      mkt_discard_vol=0, cancel_vol=0, cancel_miss=0, drop_vol=0, drop_cnt=0,
                      evict_vol=0, evict_cnt=0, bad_msgs=0)
        self.fills = []
        D = 4 * top_levels + 5
        self.obs = [[0.0] * D for _ in range(n_agents)]
        for a in range(n_agents):
            self.obs[a][4 * top_levels + 2] = 1.0
            if a < n_agents // 2:
                signed = exec_dir == 0 and self.exec_dir == SELL
                self.obs[a][4 * top_levels + 3] = float(-exec_target if signed else exec_target)
        self.rew = [0] * n_agents
        self.done = 0
        self.acts = [0] * n_agents

    def _task_dir(self, k):
        if self.exec_dir_cfg != 0:
            return self.exec_dir_cfg
        return SELL if keyed_draws(self.seed, k, TAG_TASKDIR, 1)[0] >> 63 else BUY

    # -- episodes over one shared stream ----------------------------------------
    def set_episodes(self, msgs, step_offsets, starts, levels):
        self.ep = (msgs, step_offsets, starts, levels)

    def begin_episode(self, k):
        msgs, off, starts, levels = self.ep
        j = bounded(keyed_draws(self.seed, k, TAG_EPISODE, 1)[0], len(starts))
        st = starts[j]
        self.orders = {BUY: [], SELL: []}
        self.ts_next = 0
        self.seq_next = 0
        self.inv = [0] * self.A
        self.cash = [0] * self.A
        self.pv_prev = [0] * self.A
        self.exec_done = [0] * self.A
        self.last_px = int(st["last_px"])
        self.ep_start = int(st["data_step"])
        self.exec_dir = self._task_dir(k)
        idx = 0
        for s, side in enumerate((BUY, SELL)):
            for i in range(int(st["n_bid"] if s == 0 else st["n_ask"])):
                px, q = (int(v) for v in levels[j, s, i])
                self.orders[side].append(dict(px=px, qty=q, id=INIT_ID + idx, ts=self.ts_next))
                self.ts_next += 1
                idx += 1

    def reset_obs(self):
        """Observation at an episode start: the starting book, flat agents, full time and target."""
        self._write_obs(1.0)

    def step_episode(self, actions=None):
        msgs, off, starts, levels = self.ep
        te = self.t % self.T
        d = self.ep_start + te
        self.step(msgs[off[d]:off[d + 1]], actions, te=te)
        if te + 1 == self.T:
            self.begin_episode(self.t // self.T)
            if self.A:
                self.reset_obs()

    # -- book helpers -------------------------------------------------------
    def ranked(self, side):
        """Orders of one side sorted best-first: price priority, then arrival."""
        sgn = -1 if side == BUY else 1
        return sorted(self.orders[side], key=lambda o: (sgn * o["px"], o["ts"]))

    def owner(self, oid):
        if oid >= 0 or self.A == 0:
            return self.A
        return (-oid - 1) % self.A

    def touch(self, side):
        r = self.ranked(side)
        return r[0]["px"] if r else self.last_px

    def _credit(self, who, dcash, dinv):
        if who == self.A:
            self.bg_cash += dcash
            self.bg_inv += dinv
        else:
            self.cash[who] += dcash
            self.inv[who] += dinv

    def _fill(self, maker, taker_id, taker_side, f):
        om, ot = self.owner(maker["id"]), self.owner(taker_id)
        buyer, seller = (ot, om) if taker_side == BUY else (om, ot)
        self._credit(buyer, -maker["px"] * f, f)
        self._credit(seller, maker["px"] * f, -f)
        self.step_fills.append((buyer, seller, maker["px"], f))
        task_owner = seller if self.exec_dir == SELL else buyer
        if self.A and task_owner < self.P:
            self.exec_done[task_owner] += f
        self.last_px = maker["px"]
        self.c["fills"] += 1
        self.c["fill_vol"] += f
        self.fills.append((maker["id"], taker_id, maker["px"], f, self.msg_idx, taker_side))

    def _take(self, side, limit, q, taker_id):
        opp = -side
        while q > 0:
            r = self.ranked(opp)
            if not r:
                break
            best = r[0]
            if limit is not None and ((side == BUY and best["px"] > limit) or
                                      (side == SELL and best["px"] < limit)):
                break
            f = min(q, best["qty"])
            self._fill(best, taker_id, side, f)
            best["qty"] -= f
            q -= f
            if best["qty"] == 0:
                self.orders[opp].remove(best)
        return q

    def _rest(self, side, px, q, oid):
        mine = self.orders[side]
        if len(mine) >= self.cap:
            worst = self.ranked(side)[-1]   # worst price, latest arrival
            strictly_better = px > worst["px"] if side == BUY else px < worst["px"]
            if not strictly_better:
                self.c["drop_vol"] += q
                self.c["drop_cnt"] += 1
                return
            mine.remove(worst)
            self.c["evict_vol"] += worst["qty"]
            self.c["evict_cnt"] += 1
        mine.append(dict(px=px, qty=q, id=oid, ts=self.ts_next))
        self.ts_next += 1

    def process(self, typ, side, px, qty, oid, agent=False):
        self.c["msgs"] += 1
        if agent:
            self.c["agent_msgs"] += 1
        ok = typ in (ADD, PARTIAL, DELETE, MARKET) and side in (BUY, SELL)
        if ok and typ != DELETE and qty <= 0:
            ok = False
        if not ok:
            self.c["bad_msgs"] += 1
        elif typ == ADD:
            self.c["add_vol"] += qty
            left = self._take(side, px, qty, oid)
            if left:
                self._rest(side, px, left, oid)
        elif typ == MARKET:
            self.c["mkt_vol"] += qty
            self.c["mkt_discard_vol"] += self._take(side, None, qty, oid)
        else:
            hit = [o for o in self.orders[side] if o["id"] == oid and o["px"] == px]
            if not hit:
                self.c["cancel_miss"] += 1
            else:
                o = hit[0]
                c = min(qty, o["qty"]) if typ == PARTIAL else o["qty"]
                o["qty"] -= c
                self.c["cancel_vol"] += c
                if o["qty"] == 0:
                    self.orders[side].remove(o)
        self.msg_idx += 1

    # -- one env step ---------------------------------------------------------
    def step(self, msgs, actions=None, te=None):
        """One env step; te is the step within the episode (the global step when None)."""
        te = self.t if te is None else te
        self.fills = []
        self.step_fills = []   # (buyer, seller, price, qty) of this step
        self.msg_idx = 0
        mid_before = (self.touch(BUY) + self.touch(SELL)) / 2
        if self.A:
            P = self.P
            n_mm = (12, 8, 3)[self.mm_space]
            if self.action_mode == 1:
                draws = keyed_draws(self.seed, self.t, TAG_POLICY, self.A)
                self.acts = [bounded(draws[a], 12 if a < P else n_mm) for a in range(self.A)]
            else:
                self.acts = list(actions)
            bb, ba = self.touch(BUY), self.touch(SELL)
            want = []   # (agent, side, px, qty)
            for ag in range(P):
                remaining = self.exec_target - self.exec_done[ag]
                if remaining <= 0:
                    continue
                a = self.acts[ag]
                mult = (1, 2, 5)[a % 3]
                q0 = max(1, -(-self.exec_target // self.T))
                qty = min(mult * q0, remaining)
                if self.exec_dir == SELL:
                    prices = (bb, -((-(bb + ba)) // 2), ba, ba + 2)
                else:
                    prices = (ba, (bb + ba) // 2, bb, bb - 2)
                want.append((ag, self.exec_dir, prices[a // 3], qty))
            for ag in range(P, self.A):
                a = self.acts[ag]
                if self.mm_space == 0:
                    if 1 <= a <= 9:
                        quotes = (bb - (a - 1) // 3, ba + (a - 1) % 3)
                    else:
                        quotes = {10: (bb + 1, ba), 11: (bb, ba - 1)}.get(a, (None, None))
                elif self.mm_space == 1:
                    quotes = {1: (bb - 2, ba + 2), 2: (bb - 4, ba + 4), 3: (bb + 1, ba - 1), 4: (bb - 2, None),
                              5: (None, ba + 2), 6: (bb - 5, ba - 1), 7: (bb + 1, ba + 5)}.get(a, (None, None))
                else:
                    quotes = {1: (bb, None), 2: (None, ba)}.get(a, (None, None))
                if quotes[0] is not None:
                    want.append((ag, BUY, quotes[0], self.mm_lot))
                if quotes[1] is not None:
                    want.append((ag, SELL, quotes[1], self.mm_lot))
            kept = [0] * len(want)
            cancels = []
            for ag in range(self.A):
                for side in (BUY, SELL):
                    for o in self.ranked(side):
                        if o["id"] >= 0 or self.owner(o["id"]) != ag:
                            continue
                        m = [i for i, w in enumerate(want) if w[0] == ag and w[1] == side and w[2] == o["px"]]
                        if m:
                            kept[m[-1]] += o["qty"]
                        else:
                            cancels.append((side, o["px"], o["id"]))
            send = [(w[0], w[1], w[2], w[3] - k) for w, k in zip(want, kept) if w[3] - k > 0]
            n = len(send)
            draws = keyed_draws(self.seed, self.t, TAG_SHUFFLE, max(n - 1, 0))
            for d, i in enumerate(range(n - 1, 0, -1)):
                j = bounded(draws[d], i + 1)
                send[i], send[j] = send[j], send[i]
            for side, px, oid in cancels:
                self.process(DELETE, side, px, 0, oid, agent=True)
            for ag, side, px, q in send:
                oid = -(1 + ag + self.A * self.seq_next)
                self.seq_next += 1
                self.process(ADD, side, px, q, oid, agent=True)
        for m in msgs:
            self.process(int(m["type"]), int(m["side"]), int(m["px"]), int(m["qty"]), int(m["oid"]))
        if self.A:
            bb, ba = self.touch(BUY), self.touch(SELL)
            self._write_obs((self.T - (te + 1)) / self.T)
            for a in range(self.A):
                pref = bb if self.inv[a] > 0 else ba if self.inv[a] < 0 else 0
                pv = wrap(self.inv[a] * pref + self.cash[a])
                if self.pv_ref == 1:   # mid reference, in half ticks: twice the exact PV
                    pv = wrap(int(2 * (self.inv[a] * Fraction(bb + ba, 2) + self.cash[a])))
                self.rew[a] = wrap(pv - self.pv_prev[a])
                self.pv_prev[a] = pv
                if a >= self.P and self.reward_mode:
                    self.rew[a] = self._mm_reward(a, mid_before, (bb + ba) / 2)
                if a >= self.P:
                    self.rew[a] -= self.inv_penalty * self.inv[a] ** 2
                if a < self.P and te + 1 == self.T:
                    unfilled = max(0, self.exec_target - self.exec_done[a])
                    unit = 2 if self.pv_ref == 1 else 1
                    self.rew[a] = self.rew[a] - unit * self.exec_penalty_milli * unfilled / Fraction(1000)
                    self.rew[a] = self.rew[a].numerator // self.rew[a].denominator
        self.done = int(te + 1 == self.T)
        self.t += 1

    def _write_obs(self, time_left):
        bb, ba = self.touch(BUY), self.touch(SELL)
        anchor = (bb + ba) // 2
        D = 4 * self.L + 5
        self.obs = [[0.0] * D for _ in range(self.A)]
        levels = {}
        for s, side in enumerate((BUY, SELL)):
            lv = []
            for o in self.ranked(side):
                if lv and lv[-1][0] == o["px"]:
                    lv[-1][1] += o["qty"]
                else:
                    lv.append([o["px"], o["qty"]])
            levels[s] = lv
        rest = [0] * self.A
        for side in (BUY, SELL):
            for o in self.orders[side]:
                if o["id"] < 0:
                    rest[self.owner(o["id"])] += o["qty"]
        for a in range(self.A):
            ob = self.obs[a]
            for s in range(2):
                for i, (p, q) in enumerate(levels[s][: self.L]):
                    ob[s * 2 * self.L + 2 * i] = float(p - anchor)
                    ob[s * 2 * self.L + 2 * i + 1] = float(q)
            ob[4 * self.L] = float(self.inv[a])
            ob[4 * self.L + 1] = float(self.cash[a])
            ob[4 * self.L + 2] = time_left
            rem = self.exec_target - self.exec_done[a]
            if self.exec_dir_cfg == 0 and self.exec_dir == SELL:
                rem = -rem
            ob[4 * self.L + 3] = float(rem) if a < self.P else 0.0
            ob[4 * self.L + 4] = float(rest[a])

    def _mm_reward(self, a, mid_before, mid_after):
        """Eqs. 3-4 for agent a from the fill list, with exact fractions, returned in quarter ticks."""
        Fr = Fraction
        mbar = (Fr(mid_before) + Fr(mid_after)) / 2
        psi_b = sum(((mbar - p) * q for b, s, p, q in self.step_fills if b == a), Fr(0))
        psi_s = sum(((p - mbar) * q for b, s, p, q in self.step_fills if s == a), Fr(0))
        r = psi_b + psi_s
        if self.reward_mode == 2:
            psi_inv = self.inv[a] * (Fr(mid_after) - Fr(mid_before))
            r += psi_inv - Fr(100 - self.lam_pct, 100) * max(Fr(0), psi_inv)
        r4 = 4 * r
        return r4.numerator // r4.denominator   # floor: only the lambda damping can be fractional

    def book_arrays(self):
        out = []
        for side in (BUY, SELL):
            out.append([(o["px"], o["qty"], o["id"], o["ts"]) for o in self.ranked(side)])
        return out
