"""Benchmark of the batched limit-order-book environment step on GB300.

Workload (the 1,024-env configuration): 1,024 independent envs, book capacity
100 per side, 100 synthetic market-by-order messages per env-step, 1,000-step
episodes, two agents per env (execution + market making) acting from the
seeded uniform random policy, top-10-level observations.  One bench step is
one lob_step over all envs: load the books, convert actions (with carry-over
cancels), shuffle, match the agents' and the background messages, compute
observations / rewards / done, write the books back.

Timing: every timed step is bracketed by CUDA events on the launching stream;
a 256 MiB buffer is written between timed steps so the books and messages
come from HBM, not L2 (the flush is outside the events).  The metric is MBO
messages processed per second (background plus agent messages) and
env-steps per second on one GPU.  ``--impl reference`` times the CPU oracle
on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ENVS, CAP, M, T, L = 1024, 100, 100, 1000, 10
EXEC_TARGET = 500
METRIC = "MBO messages/sec and env-steps/sec on 1 GB300 (bit-exact vs oracle); % HBM roofline"
WORKLOAD = "1024 envs x cap 100/side x 100 msgs/step, 1000-step episodes, 2 agents (exec 500-lot sell + MM), random policy, top-10 obs"


def set_envs(n):
    """The same workload at another env count (the 16,384-env secondary line)."""
    global N_ENVS, WORKLOAD
    WORKLOAD = WORKLOAD.replace(f"{N_ENVS} envs", f"{n} envs", 1)
    N_ENVS = n


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def aggregate_over_ranks(total_s, msgs, device="cpu"):
    """Whole-job figures across ranks: the slowest rank's time and every rank's messages.
    Each rank runs its own replica (independent envs), so nothing but these two numbers
    crosses ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_s, msgs
    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    m = torch.tensor([float(msgs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return t.item(), m.item()


def replica_seed(base, rank):
    """Each rank replays its own synthetic episode (weak scaling)."""
    return base + rank


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class _NvmlPci(ctypes.Structure):
    """nvmlPciInfo_t (nvml.h)."""
    _fields_ = [("busIdLegacy", ctypes.c_char * 16), ("domain", ctypes.c_uint), ("bus", ctypes.c_uint),
                ("device", ctypes.c_uint), ("pciDeviceId", ctypes.c_uint), ("pciSubSystemId", ctypes.c_uint),
                ("busId", ctypes.c_char * 32)]


# NVML clock-event reason bits (nvml.h) reported by name
_REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region.

    NVML (read-only queries through ctypes) is polled about every 0.5 ms from a
    thread, so even a timed region of a millisecond or two gets samples; the
    device is matched to the CUDA device by PCI address.  Without NVML it falls
    back to nvidia-smi at 200 ms (which sees nothing of a short region)."""

    def __init__(self, gpu_index):
        import threading
        self.rows, self.p, self.nv, self.t_in = [], None, None, None
        try:
            import torch
            pr = torch.cuda.get_device_properties(gpu_index)
            want = (int(pr.pci_domain_id), int(pr.pci_bus_id), int(pr.pci_device_id))
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            cnt = ctypes.c_uint(0)
            nv.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
            self.dev = None
            for i in range(cnt.value):
                d = ctypes.c_void_p()
                info = _NvmlPci()
                if nv.nvmlDeviceGetHandleByIndex_v2(i, ctypes.byref(d)) == 0 and \
                        nv.nvmlDeviceGetPciInfo_v3(d, ctypes.byref(info)) == 0 and \
                        (info.domain, info.bus, info.device) == want:
                    self.dev = d
            if self.dev is None:
                raise OSError("no NVML device at the CUDA device's PCI address")
            self.nv = nv
            mx = ctypes.c_uint(0)
            nv.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx))   # 1 = NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            self.stop_flag = threading.Event()
            self.first = threading.Event()
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
            self.first.wait(2.0)
        except Exception:
            self.nv = None
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            try:
                self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "200"],
                                          stdout=self.f, stderr=subprocess.DEVNULL)
            except OSError:
                self.p = None

    def _poll(self):
        mhz, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self.stop_flag.is_set():
            ok = self.nv.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(mhz)) == 0
            if self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.dev, ctypes.byref(rs)) != 0:
                self.nv.nvmlDeviceGetCurrentClocksThrottleReasons(self.dev, ctypes.byref(rs))
            if ok:
                self.rows.append((time.perf_counter(), float(mhz.value), int(rs.value)))
            self.first.set()
            time.sleep(0.0005)

    def enter(self):
        """Marks the start of the timed region."""
        self.t_in = time.perf_counter()

    def stop(self):
        if self.nv is not None:
            t_out = time.perf_counter()
            self.stop_flag.set()
            self.th.join(timeout=5)
            t_in = self.t_in if self.t_in is not None else 0.0
            inside = [r for r in self.rows if t_in <= r[0] <= t_out]
            where = "inside the timed region"
            if not inside and self.rows:   # a region shorter than one poll: the samples bracketing it
                before = [r for r in self.rows if r[0] < t_in][-1:]
                after = [r for r in self.rows if r[0] > t_out][:1]
                inside, where = before + after, "the polls bracketing the timed region"
            if not inside:
                return None
            reasons = sorted({nm for _, _, m in inside for b, nm in _REASON_BITS.items() if m & b})
            return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(inside), "source": f"NVML, {where}"}
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        text = self.f.read()
        os.unlink(self.f.name)
        return parse_clock_rows(text)


def parse_clock_rows(text):
    """Median SM clock, max clock and active slowdown reasons from nvidia-smi
    CSV rows (index, clocks.sm, clocks.max.sm, power, active mask, then the
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown and sw_power_cap
    flags); None without a valid sample."""
    rows = [r.split(",") for r in text.strip().splitlines() if r.strip()]
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        if len(r) < 9:
            continue
        try:
            sm.append(float(r[1]))
            mx = float(r[2])
        except ValueError:
            continue
        for nm, v in zip(names, r[5:9]):
            if v.strip().lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


# the sources of the measured step kernel and of its launch (the traffic record
# is void once any of them changes)
TRAFFIC_SOURCES = ["include/lob.h"] + [f"paper_2511_02136_gb300/csrc/{n}" for n in (
    "lob_api.cu", "lob_device.cuh", "lob_ladder.cuh", "fused.cuh", "tc05.cuh", "lob_steps.h", "steps_inst.cuh",
    "steps_k4.cu")]


def traffic_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for src in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, src), "rb") as g:
            h.update(g.read())
    return h.hexdigest()


def _traffic_record():
    """ncu DRAM bytes per launch of the step kernel, if taken on the current source."""
    p = os.path.join(ROOT, "profiles", "k_env_steps_1024env_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("source_sha256") != traffic_sources_sha256():
        return None
    return float(rec["dram_bytes_per_launch"])


def bench_config(world):
    """The workload description both arms print (the GPU arm and the oracle arm)."""
    return {"workload": WORKLOAD, "n_envs": N_ENVS, "cap_per_side": CAP, "msgs_per_step": M,
            "episode_len": T, "top_levels": L, "global_batch": N_ENVS * world,
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "256 MiB buffer written between timed steps (outside the events)",
            "timing": "CUDA events per step on the launching stream, summed"}


def alg_bytes_per_env_step(live_orders, D):
    """Algorithmic bytes of one env-step: the step's messages, the book's live
    orders loaded and stored (24 bytes each way), the env state and counters
    read and written, seed and offsets read, observations and rewards of both
    agents and the done flag written.  live_orders = resting orders at the
    load plus those at the store (both sides)."""
    return M * 32 + 24 * live_orders + 2 * 128 + 2 * 16 * 8 + 8 + 16 + 2 * (4 * D + 8) + 1


def make_inputs(seed, gen_steps=T):
    from paper_2511_02136_gb300 import mbogen
    seeds = mbogen.env_seeds(seed, N_ENVS)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=M), seeds, gen_steps)
    return seeds, st


def run_gpu(args):
    import torch
    from paper_2511_02136_gb300 import lob

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lob.build()
    gen = min(T, args.gen_steps)
    seeds, st = make_inputs(replica_seed(1, rank), gen)
    dev = torch.device("cuda", local)
    msgs_d = torch.from_numpy(st.msgs.view(np.uint8)).to(dev)
    off_d = torch.from_numpy(st.offsets).to(dev)
    seeds_d = torch.from_numpy(seeds.view(np.int64).copy()).to(dev)
    env = lob.LobEnv(N_ENVS, cap=CAP, top_levels=L, episode_len=T, exec_target=EXEC_TARGET,
                     action_mode=lob.LOB_ACT_RANDOM, warps_per_block=args.wpb)
    lob.lob_set_threads_per_env(env.h, args.threads_per_env)
    env.load_messages(msgs_d, off_d)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    state = {"t": gen}

    def next_step():
        if state["t"] >= gen:                       # new episode: reset + rebind (untimed)
            env.reset(seeds_d)
            env.load_messages(msgs_d, off_d)
            state["t"] = 0
        env.step()
        state["t"] += 1

    for _ in range(args.warmup):
        next_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]

    def msgs_so_far():
        return int(env.counters()[:, 0].sum().item())

    msgs_total = -msgs_so_far()           # counters restart at every reset
    # resting orders at every timed step's load and store, summed on the
    # device (one small kernel after each step, outside the events), read once
    live_acc = torch.zeros(1, dtype=torch.int64, device=dev)
    lob.lob_live_orders(env.h, live_acc)       # the first timed step's load
    launches = 0
    clk = Clocks(local)
    clk.enter()
    t_wall0 = time.perf_counter()
    for i in range(K):
        if state["t"] >= gen:             # end of the generated window: bank its messages, reset (untimed)
            msgs_total += msgs_so_far()
            env.reset(seeds_d)
            env.load_messages(msgs_d, off_d)
            state["t"] = 0
        flush.fill_(i)
        l0 = lob.lob_kernel_launches(env.h)
        ev[i][0].record(stream)
        env.step()
        ev[i][1].record(stream)
        launches += lob.lob_kernel_launches(env.h) - l0
        state["t"] += 1
        # this step's store and (unless it is the last) the next step's load
        lob.lob_live_orders(env.h, live_acc)
        if i + 1 < K:
            lob.lob_live_orders(env.h, live_acc)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    msgs_total += msgs_so_far()
    live_sum = int(live_acc.item())       # sum over the K steps of (orders at load + orders at store)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    rc = env.sync()
    if rc != 0:
        raise RuntimeError(f"device status {lob.lob_strerror(rc)}")
    total_s = sum(step_ms) / 1e3
    total_s, msgs_total = aggregate_over_ranks(total_s, msgs_total, dev)
    env_steps = K * N_ENVS * world
    value = msgs_total / total_s
    # algorithmic bytes per launch (one launch per step), with the live
    # orders averaged over every timed step's load and store
    D = env.D
    live_ls = live_sum / (K * N_ENVS)      # per env-step: orders loaded + orders stored
    alg_bytes = alg_bytes_per_env_step(live_ls, D) * N_ENVS
    peak, peak_kind = _peaks()
    mean_step_s = total_s / K
    achieved = alg_bytes / mean_step_s / 1e9
    traffic = _traffic_record() if N_ENVS == 1024 else None   # the record is of the 1,024-env launch

    e2e = run_e2e(args, env, st, seeds_d) if rank == 0 else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(seeds, st, budget_s=args.cpu_seconds)
    env.close()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "msgs/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * mean_step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "env_steps_per_s": env_steps / total_s,
            "config": bench_config(world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                         "kernel": ("k_env_steps_split<4> (plain; one warp per book side)" if args.threads_per_env == 64
                                    else "k_env_steps<4> (plain; " + ("wide register budget, one wave)" if N_ENVS <= 1024
                                                                      else "default register budget, several waves)")),
                         "alg_bytes_per_launch": alg_bytes,
                         "mean_live_orders_per_env": live_ls / 2,
                         "live_orders_from": f"every timed step's load and store ({K} steps)"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu,
            "wall_s": t_wall,
        }
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(args, env, st, seeds_d):
    """Same metric through the host-buffer step: pinned host messages in, obs / rewards / done
    out, every step; the timed region ends when the last step's outputs are on the host."""
    import torch
    from paper_2511_02136_gb300 import lob
    K = min(args.e2e_steps, st.offsets.shape[1] - 1)
    env.reset(seeds_d)
    # per-step host slices: messages of every env for step t, packed, plus offsets
    packs = []
    for t in range(K):
        lo = st.offsets[:, t]
        hi = st.offsets[:, t + 1]
        idx = np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)])
        pm = torch.from_numpy(st.msgs[idx].view(np.uint8)).pin_memory()
        off = np.zeros(N_ENVS + 1, np.int64)
        off[1:] = np.cumsum(hi - lo)
        packs.append((pm, off))
    D = env.D
    obs = torch.zeros((N_ENVS, 2, D), dtype=torch.float32).pin_memory()
    rew = torch.zeros((N_ENVS, 2), dtype=torch.int64).pin_memory()
    done = torch.zeros(N_ENVS, dtype=torch.uint8).pin_memory()
    h = env.h
    lib = lob._load()
    s = torch.cuda.current_stream().cuda_stream

    def timed(fn):
        # untimed warm-up steps (the call's first-use buffers and events), then a fresh episode
        for t in range(min(3, K)):
            pm, off = packs[t]
            rc = fn(h, pm.data_ptr(), off.ctypes.data, None, obs.data_ptr(), rew.data_ptr(), done.data_ptr(), s)
            if rc:
                raise RuntimeError(lob.lob_strerror(rc))
        torch.cuda.synchronize()
        env.reset(seeds_d)
        msgs_before = int(env.counters()[:, 0].sum().item())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(K):
            pm, off = packs[t]
            rc = fn(h, pm.data_ptr(), off.ctypes.data, None, obs.data_ptr(), rew.data_ptr(), done.data_ptr(), s)
            if rc:
                raise RuntimeError(lob.lob_strerror(rc))
        torch.cuda.synchronize()   # the last step's outputs are in host memory
        el = time.perf_counter() - t0
        return (env.counters()[:, 0].sum().item() - msgs_before) / el, el

    # the pipelined call (next step's uploads overlap this step), then the synchronous one
    v_async, el = timed(lib.lob_step_host_async)
    v_sync, _ = timed(lib.lob_step_host)
    bi = int(np.mean([p[0].numel() + p[1].nbytes for p in packs]))
    bo = obs.numel() * 4 + rew.numel() * 8 + done.numel()
    return {"value": v_async, "unit": "msgs/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "steps": K, "env_steps_per_s": K * N_ENVS / el, "api": "lob_step_host_async",
            "synchronous_api_value": v_sync}


def cpu_baseline(seeds, st, budget_s=15.0, n_threads=None):
    """The oracle as it stands on the host cores: whole env steps of all envs until ~budget_s."""
    import oracle
    n_threads = n_threads or os.cpu_count() or 1
    o = oracle.Oracle(N_ENVS, cap=CAP, top_levels=L, episode_len=T, exec_target=EXEC_TARGET,
                      action_mode=1, n_threads=n_threads)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    t0 = time.perf_counter()
    steps = 0
    while steps < st.offsets.shape[1] - 1 and time.perf_counter() - t0 < budget_s:
        o.step()
        steps += 1
    el = time.perf_counter() - t0
    msgs = int(o.counters()[:, 0].sum())
    return {"value": msgs / el, "unit": "msgs/s", "cores": n_threads, "kind": "oracle",
            "sample": f"all {N_ENVS} envs, first {steps} steps of the same episode",
            "env_steps_per_s": steps * N_ENVS / el}


def run_reference(args):
    """The CPU oracle as the reference arm, on the same workload and metric."""
    rank, world = _dist()
    if rank != 0:
        return
    seeds, st = make_inputs(1)
    import oracle
    n_threads = os.cpu_count() or 1
    o = oracle.Oracle(N_ENVS, cap=CAP, top_levels=L, episode_len=T, exec_target=EXEC_TARGET,
                      action_mode=1, n_threads=n_threads)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    t = 0
    for _ in range(args.warmup):
        o.step()
        t += 1
    before = int(o.counters()[:, 0].sum())
    K = min(args.steps, T - t)
    t0 = time.perf_counter()
    for _ in range(K):
        o.step()
    el = time.perf_counter() - t0
    msgs = int(o.counters()[:, 0].sum()) - before
    value = msgs / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "msgs/s", "n_gpus": world,
           "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * el / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "env_steps_per_s": K * N_ENVS / el,
           "config": bench_config(world),
           "cpu_baseline": {"value": value, "unit": "msgs/s", "cores": n_threads, "kind": "oracle",
                            "sample": f"all {N_ENVS} envs, steps {t}..{t + K - 1} of one episode"},
           "e2e": {"value": value, "unit": "msgs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- other workloads
def _flush_and_time(run, reps, dev):
    """Time `run()` `reps` times with CUDA events, writing 256 MiB between runs."""
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    out = []
    for i in range(reps):
        flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b) / 1e3)
    return out


def run_workload(args):
    """Secondary lines: the uneven 8,192-env batch, the fused-policy rollout and
    the capacity-1,000 stress window (one JSON line each)."""
    import torch
    from paper_2511_02136_gb300 import autotune, lob, mbogen
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lob.build()
    wl = args.workload

    def upload(st, seeds):
        return (torch.from_numpy(st.msgs.view(np.uint8)).to(dev), torch.from_numpy(st.offsets).to(dev),
                torch.from_numpy(seeds.view(np.int64).copy()).to(dev))

    if wl == "uneven8192":
        n, T = 8192, 500
        seeds = mbogen.env_seeds(2, n)
        caps = mbogen.env_caps(2, n)
        st = mbogen.generate(mbogen.MessageModel(poisson=True), seeds, T)
        md, od, sd = upload(st, seeds)
        env = lob.LobEnv(n, cap=500, episode_len=T, exec_target=500, action_mode=lob.LOB_ACT_RANDOM, caps=caps)
        slots = np.array([max(32, 1 << int(np.ceil(np.log2(c)))) for c in caps], np.float64)
        costs = (st.lambdas * (1.0 + slots / 128.0)).astype(np.float32)
        D = env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device=dev)
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device=dev)
        T_tune = 25

        def tune_run():
            env.load_messages(md, od)
            env.reset(sd)
            lob.lob_rollout(env.h, T_tune, None, obs[:T_tune], rew[:T_tune], None)

        tried = []
        choice = autotune.tune(env.h, tune_run, costs=costs, repeats=1,
                               candidates=autotune.DEFAULT_CANDIDATES + autotune.MULTI_CANDIDATES +
                               autotune.SPLIT_CANDIDATES, timed=tried, tiles=autotune.TILE_CANDIDATES)
        stream = torch.cuda.Stream()
        env.load_messages(md, od)
        env.reset(sd, stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            lob.lob_rollout(env.h, T, None, obs, rew, None, stream=stream)

        # the reset before each replay is outside the timed region
        times = []
        for i in range(args.reps):
            env.load_messages(md, od)
            env.reset(sd)
            torch.cuda.synchronize()
            times += _flush_and_time(g.replay, 1, dev)
        msgs = float(env.counters()[:, 0].sum().item())
        t = min(times)
        line = {"workload": "uneven8192", "metric": METRIC, "value": msgs / t, "unit": "msgs/s",
                "env_steps_per_s": n * T / t, "seconds_per_rollout": t, "steps": T, "n_gpus": 1,
                "config": {"workload": "8192 envs, caps uniform {50,100,200,500}, M_t ~ Poisson(lambda), "
                                       "lambda log-uniform [10,500], 500 steps, random policy, one graph-captured "
                                       "lob_rollout in the autotuned launch shape",
                           "autotuned": choice.__dict__, "messages": msgs,
                           "tuning_window_ms": [{"warps_per_block": c.warps_per_block, "persistent": c.persistent,
                                                 "longest_first": c.longest_first, "threads_per_env": c.threads_per_env,
                                                 "tile_records": c.tile_records, "ms": c.ms} for c in tried]},
                "dtype": "int64", "data": "synthetic"}
        env.close()
        if args.per_class:
            # each capacity class alone on the whole GPU (its envs' streams, its best
            # of a few shapes): the time each class needs by itself
            per = {}
            for cls in sorted(set(int(x) for x in caps)):
                idx = np.nonzero(caps == cls)[0]
                parts = [st.msgs[st.offsets[e, 0]:st.offsets[e, -1]] for e in idx]
                base = np.concatenate([[0], np.cumsum([len(q) for q in parts])[:-1]]).astype(np.int64)
                off2 = (st.offsets[idx] - st.offsets[idx, :1] + base[:, None]).astype(np.int64)
                cmd, cod = (torch.from_numpy(np.concatenate(parts).view(np.uint8).copy()).to(dev),
                            torch.from_numpy(off2).to(dev))
                csd = torch.from_numpy(seeds[idx].view(np.int64).copy()).to(dev)
                cenv = lob.LobEnv(len(idx), cap=cls, episode_len=T, exec_target=500, action_mode=lob.LOB_ACT_RANDOM)
                best = None
                for wpb, pers, lf in ((1, 1, True), (2, 1, True), (4, 1, True), (4, 0, False)):
                    lob.lob_set_launch(cenv.h, wpb, pers)
                    lob.lob_set_env_costs(cenv.h, costs[idx] if lf else None)
                    cenv.load_messages(cmd, cod)
                    cenv.reset(csd)
                    torch.cuda.synchronize()
                    tt = _flush_and_time(lambda: lob.lob_rollout(cenv.h, T, None, None, None, None), 1, dev)[0]
                    cm = float(cenv.counters()[:, 0].sum().item())
                    if best is None or tt < best[0]:
                        best = (tt, wpb, pers, lf, cm)
                per[cls] = {"envs": int(len(idx)), "seconds": best[0], "messages": best[4],
                            "msgs_per_s": best[4] / best[0], "shape": {"warps_per_block": best[1],
                                                                        "persistent": best[2],
                                                                        "longest_first": best[3]},
                            "max_lambda": float(st.lambdas[idx].max())}
                cenv.close()
            line["per_class_alone"] = per
    elif wl == "policy4096":
        n, T = args.policy_envs, args.policy_steps
        seeds = mbogen.env_seeds(3, n)
        st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), seeds, T)
        md, od, sd = upload(st, seeds)
        env = lob.LobEnv(n, cap=200, episode_len=T, exec_target=512, action_mode=lob.LOB_ACT_HOST)
        params = lob.init_policy_params(5, 2, env.D)
        pol = lob.lob_policy_create(2, env.D, params)
        acts = torch.zeros((T, n, 2), dtype=torch.int32, device=dev)
        res = {}
        for prec, name in ((lob.LOB_PREC_BF16_FUSED, "bf16_fused"), (lob.LOB_PREC_BF16, "bf16"),
                           (lob.LOB_PREC_FP32, "fp32")):
            stream = torch.cuda.Stream()
            env.load_messages(md, od)
            env.reset(sd)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                lob.lob_rollout_policy(env.h, pol, T, prec, None, None, None, acts, stream=stream)
            times = []
            for i in range(args.reps):
                env.load_messages(md, od)
                env.reset(sd)
                torch.cuda.synchronize()
                times += _flush_and_time(g.replay, 1, dev)
            msgs = float(env.counters()[:, 0].sum().item())
            t = min(times)
            res[name] = {"msgs_per_s": msgs / t, "env_steps_per_s": n * T / t, "seconds_per_rollout": t}
            if prec == lob.LOB_PREC_BF16_FUSED:
                continue   # its forward runs inside the step kernel
            # policy forward alone on the final observations
            ob = torch.zeros((n, 2, env.D), dtype=torch.float32, device=dev)
            lob.lob_observe(env.h, ob)
            pt = _flush_and_time(lambda: lob.lob_policy_forward(pol, ob, n, prec, None, None, acts[0]), 20, dev)
            res[name]["policy_forward_us"] = 1e6 * float(np.median(pt))
        lob.lob_policy_destroy(pol)
        env.close()
        # the same rollout without a network: the seeded random policy inside the step kernel
        env = lob.LobEnv(n, cap=200, episode_len=T, exec_target=512, action_mode=lob.LOB_ACT_RANDOM)
        times = []
        for i in range(args.reps):
            env.load_messages(md, od)
            env.reset(sd)
            torch.cuda.synchronize()
            times += _flush_and_time(lambda: lob.lob_rollout(env.h, T, None, None, None, None), 1, dev)
        msgs = float(env.counters()[:, 0].sum().item())
        t = min(times)
        res["no_policy"] = {"msgs_per_s": msgs / t, "env_steps_per_s": n * T / t, "seconds_per_rollout": t,
                            "what": "lob_rollout with the seeded random policy (no network)"}
        env.close()
        head = res["bf16_fused"]
        head["step_time_vs_no_policy"] = head["seconds_per_rollout"] / t
        line = {"workload": "policy4096" if (n, T) == (4096, 128) else f"policy{n}x{T}", "metric": METRIC, "value": head["msgs_per_s"], "unit": "msgs/s",
                "env_steps_per_s": head["env_steps_per_s"], "bf16_fused": head, "bf16": res["bf16"],
                "fp32": res["fp32"], "no_policy": res["no_policy"],
                "config": {"workload": f"{n} envs x cap 200 x 100 msgs x {T} steps, per-agent MLP 45-128-128-13 "
                                       "(tanh) in the loop, one graph-captured lob_rollout_policy; value: the "
                                       "forward inside the step kernel (one launch per rollout); bf16: batched "
                                       "tcgen05 forward between step launches; fp32: register-tiled CUDA-core "
                                       "forward between step launches"},
                "dtype": "int64 book / bf16 policy", "data": "synthetic", "n_gpus": 1, "steps": T}
    elif wl == "ppo4096":
        # one IPPO epoch (4 minibatches per agent) on a policy-in-the-loop rollout
        # of the 4,096-env, capacity-200, 128-step configuration
        n, T, A, nmb = args.policy_envs, args.policy_steps, 2, 4
        seeds = mbogen.env_seeds(31, n)
        st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), seeds, T)
        md, od, sd = upload(st, seeds)
        env = lob.LobEnv(n, cap=200, episode_len=T, exec_target=512, action_mode=lob.LOB_ACT_HOST)
        env.load_messages(md, od)
        env.reset(sd)
        D = env.D
        params = lob.init_policy_params(5, A, D)
        pol = lob.lob_policy_create(A, D, params)
        obs0 = env.observe()[0].clone()
        obs = torch.zeros((T, n, A, D), dtype=torch.float32, device=dev)
        rew = torch.zeros((T, n, A), dtype=torch.int64, device=dev)
        done = torch.zeros((T, n), dtype=torch.uint8, device=dev)
        acts = torch.zeros((T, n, A), dtype=torch.int32, device=dev)
        lob.lob_rollout_policy(env.h, pol, T, lob.LOB_PREC_BF16_FUSED, obs, rew, done, acts)
        before = torch.cat([obs0[None], obs[:T - 1]], 0).contiguous()
        logits = torch.zeros((T + 1, n, A, 12), dtype=torch.float32, device=dev)
        values = torch.zeros((T + 1, n, A), dtype=torch.float32, device=dev)
        for t in range(T + 1):
            lob.lob_policy_forward(pol, (before[t] if t < T else obs[T - 1]).contiguous(), n, lob.LOB_PREC_BF16,
                                   logits[t], values[t])
        logp = torch.log_softmax(logits[:T], -1).gather(-1, acts.long()[..., None])[..., 0].contiguous()
        perm = torch.stack([torch.randperm(T * n, generator=torch.Generator().manual_seed(32 + a))
                            for a in range(A)]).to(torch.int32).to(dev)
        hp = lob.ppo_hparams(n_minibatches=nmb)
        upd = lambda: lob.lob_ppo_update(pol, T, n, before, acts, logp, values, rew, done, perm, hp)
        upd()   # first call: optimiser state and packed weights (untimed)
        torch.cuda.synchronize()
        times = _flush_and_time(upd, args.reps + 2, dev)
        if env.sync() != 0 or lob.lob_policy_sync(pol) != 0:
            raise RuntimeError("device status after the update")
        t = min(times)
        lob.lob_policy_destroy(pol)
        env.close()
        samples = T * n * A
        # per sample: the forward, 2 (D H + H H + H 13); the backward, the weight
        # gradients of all three layers (as many products again) and the input
        # gradients of layers 3 and 2, 2 (H 13 + H H)
        H = 128
        fwd = 2 * (D * H + H * H + H * 13)
        flops = samples * (2 * fwd + 2 * (H * 13 + H * H))
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        line = {"workload": "ppo4096" if (n, T) == (4096, 128) else f"ppo{n}x{T}",
                "metric": "IPPO samples/sec (one epoch: GAE, 4 minibatches of clipped-PPO gradient, clip, Adam)",
                "value": samples / t, "unit": "samples/s", "seconds_per_epoch": t, "samples": samples,
                "roofline": {"bound": "tensor", "achieved": flops / t / 1e12, "peak": peaks["bf16_tflops"],
                             "unit": "TFLOP/s", "frac": flops / t / 1e12 / peaks["bf16_tflops"],
                             "flops_per_epoch": flops, "what": "whole update (all its kernels) against the bf16 burst peak"},
                "config": {"workload": f"{n} envs x cap 200 x 100 msgs x {T} steps rollout (fused BF16 policy), "
                                       "2 agents, 4 minibatches, BF16 operands with FP32 accumulation"},
                "dtype": "bf16 / fp32", "data": "synthetic", "n_gpus": 1}
    elif wl == "episodes4096":
        # Table 2's training setup on one shared stream: 64-step episodes
        # starting every 64 data steps from book snapshots (top 10 levels),
        # 100 msgs/step, capacity 100, order size 10, execution task 600,
        # Fixed Quantity market maker with the Spooner reward and the
        # quadratic inventory penalty (rho 50), unfilled-task penalty 0.1;
        # 256 steps = 4 episodes per env in one lob_rollout launch
        n, T, EP = 4096, 256, 64
        n_data = 64 * 130
        dseed = mbogen.env_seeds(6, 1)
        st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), dseed, n_data)
        starts, levels = mbogen.start_books(6, st.mids[0], np.arange(0, n_data - EP + 1, EP), 10, min_levels=5)
        seeds = mbogen.env_seeds(7, n)
        env = lob.LobEnv(n, cap=100, episode_len=EP, mm_lot=10, exec_target=600, action_mode=lob.LOB_ACT_RANDOM,
                         reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=50, inv_penalty=50,
                         exec_penalty_milli=100, mm_space=lob.LOB_MM_FIXED_QUANT)
        md = torch.from_numpy(st.msgs.view(np.uint8)).to(dev)
        od = torch.from_numpy(st.offsets[0].copy()).to(dev)
        sd = torch.from_numpy(seeds.view(np.int64).copy()).to(dev)
        env.set_episodes(md, od, starts, levels)
        D = env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device=dev)
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device=dev)
        done = torch.zeros((T, n), dtype=torch.uint8, device=dev)
        times, msgs = [], 0.0
        for i in range(args.reps):
            env.reset(sd)
            torch.cuda.synchronize()
            times += _flush_and_time(lambda: lob.lob_rollout(env.h, T, None, obs, rew, done), 1, dev)
            msgs = float(env.counters()[:, 0].sum().item())
        assert env.sync() == 0
        assert int(done.sum().item()) == n * (T // EP)
        env.close()
        t = min(times)
        line = {"workload": "episodes4096", "metric": METRIC, "value": msgs / t, "unit": "msgs/s",
                "env_steps_per_s": n * T / t, "seconds_per_rollout": t, "steps": T, "n_gpus": 1,
                "config": {"workload": "4096 envs, one shared stream of 8,320 data steps x 100 msgs, 64-step "
                                       "episodes from 130 snapshot starts (every 64 data steps, top-10 levels), "
                                       "auto-reset in the kernel, cap 100, lot 10, exec task 600, Fixed Quantity "
                                       "MM, Spooner reward (lambda 0.5) + rho 50 + unfilled penalty 0.1, random "
                                       "policy, 256 steps in one lob_rollout", "messages": msgs},
                "dtype": "int64", "data": "synthetic"}
    elif wl == "table1":
        # Table 1's speed benchmark: 4,000 envs x 50 steps, two agent types
        # with 1, 5 or 10 agents each, 1 or 100 data messages per step, random
        # policy; book capacity 100 and order size 10 (Table 2).  The paper's
        # env-steps/s (JaxMARL-HFT on one L40S) is context for vs_baseline.
        paper = {(100, 1): 21969, (1, 1): 351119, (100, 5): 14801, (1, 5): 89062, (100, 10): 10724, (1, 10): 48312}
        n, T = 4000, 50
        rows = []
        for (m, per_type), ref in paper.items():
            seeds = mbogen.env_seeds(10 + m + per_type, n)
            st = mbogen.generate(mbogen.MessageModel(msgs_per_step=m), seeds, T)
            md, od, sd = upload(st, seeds)
            env = lob.LobEnv(n, n_agents=2 * per_type, cap=100, episode_len=T, mm_lot=10, exec_target=600,
                             action_mode=lob.LOB_ACT_RANDOM)
            A = 2 * per_type
            # every step's observations, rewards and done flags are written, as the RL loop needs them
            obs = torch.zeros((T, n, A, env.D), dtype=torch.float32, device=dev)
            rew = torch.zeros((T, n, A), dtype=torch.int64, device=dev)
            done = torch.zeros((T, n), dtype=torch.uint8, device=dev)
            times = []
            for i in range(args.reps):
                env.load_messages(md, od)
                env.reset(sd)
                torch.cuda.synchronize()
                times += _flush_and_time(lambda: lob.lob_rollout(env.h, T, None, obs, rew, done), 1, dev)
            assert env.sync() == 0
            msgs = float(env.counters()[:, 0].sum().item())
            env.close()
            t = min(times)
            rows.append({"data_msgs_per_step": m, "agents_per_type": per_type, "seconds": t,
                         "env_steps_per_s": n * T / t, "msgs_per_s": msgs / t,
                         "paper_env_steps_per_s_l40s": ref, "vs_paper": n * T / t / ref})
            del md, od, sd, obs, rew, done
        line = {"workload": "table1", "metric": "env-steps/sec (Table 1 speed benchmark)",
                "value": rows[0]["env_steps_per_s"], "unit": "env-steps/s", "higher_is_better": True,
                "vs_baseline": rows[0]["vs_paper"], "rows": rows, "n_gpus": 1, "steps": T,
                "config": {"workload": "4000 envs x 50 steps, 1 / 100 data msgs per step, 1 / 5 / 10 agents per "
                                       "type (execution + market making), random policy, cap 100, lot 10, task "
                                       "600; one lob_rollout launch per run writing every step's obs, rewards "
                                       "and done flags, inputs resident, 256 MiB written before each run", "value_row": "100 msgs/step, 1 agent per type"},
                "dtype": "int64", "data": "synthetic"}
    elif wl == "compact1024":
        # the benchmark workload stored as 16-byte compact records beside the
        # 32-byte ones: one 200-step lob_rollout each, inputs resident
        n, Tr = N_ENVS, 200
        seeds, st = make_inputs(1, Tr)
        packed = mbogen.pack16(st.msgs)
        od = torch.from_numpy(st.offsets).to(dev)
        sd = torch.from_numpy(seeds.view(np.int64).copy()).to(dev)
        res = {}
        for name, arr in (("msg32", st.msgs), ("msg16", packed)):
            md = torch.from_numpy(arr.view(np.uint8)).to(dev)
            env = lob.LobEnv(n, cap=CAP, top_levels=L, episode_len=Tr, exec_target=EXEC_TARGET,
                             action_mode=lob.LOB_ACT_RANDOM)
            bind = env.load_messages16 if name == "msg16" else env.load_messages
            times = []
            for i in range(args.reps):
                env.reset(sd)
                bind(md, od)
                torch.cuda.synchronize()
                times += _flush_and_time(lambda: lob.lob_rollout(env.h, Tr, None, None, None, None), 1, dev)
            assert env.sync() == 0
            msgs = float(env.counters()[:, 0].sum().item())
            env.close()
            t = min(times)
            res[name] = {"msgs_per_s": msgs / t, "seconds": t, "stream_bytes": int(arr.nbytes)}
            del md
        line = {"workload": "compact1024", "metric": METRIC, "value": res["msg16"]["msgs_per_s"], "unit": "msgs/s",
                "msg16": res["msg16"], "msg32": res["msg32"], "n_gpus": 1, "steps": Tr,
                "config": {"workload": "1024 envs x cap 100 x 100 msgs/step x 200 steps, random policy, one "
                                       "lob_rollout; the same stream as 16-byte compact and 32-byte records"},
                "dtype": "int64", "data": "synthetic"}
    elif wl == "stress65536":
        # the stress configuration at its stated length: 65,536 envs x capacity
        # 1,000 x 1,000 messages of the heavy-tailed mix x 256 steps (16.8 G
        # messages, 537 GB: more than HBM), top-20 observations, the BF16
        # policy in the loop.  The device generator draws the stream 8 steps
        # at a time into a double-buffered ring on its own stream while the
        # rollout consumes the other buffer; generation is timed apart.
        n, T, C = 65536, args.stress_steps, 8
        seeds = mbogen.env_seeds(4, n)
        gen = mbogen.GpuStreams(mbogen.STRESS_MODEL, seeds)
        M = mbogen.STRESS_MODEL.msgs_per_step
        ring = [torch.empty(n * C * M * 32, dtype=torch.uint8, device=dev) for _ in range(2)]
        off = torch.from_numpy(gen.offsets(C)).to(dev)
        env = lob.LobEnv(n, cap=1000, top_levels=20, episode_len=T, exec_target=2000, action_mode=lob.LOB_ACT_HOST)
        params = lob.init_policy_params(7, 2, env.D)
        pol = lob.lob_policy_create(2, env.D, params)
        lob.lob_set_launch(env.h, 4, 1)
        env.reset(torch.from_numpy(seeds.view(np.int64).copy()).to(dev))
        gs, ms = torch.cuda.Stream(), torch.cuda.current_stream()
        ev_gen = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        gen_ev, roll_ev = [], []
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        w0.record(ms)
        gs.wait_stream(ms)

        def gen_chunk(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if k >= 2:
                gs.wait_event(ev_free[k % 2])
            a.record(gs)
            gen.chunk(C, ring[k % 2], gs)
            b.record(gs)
            ev_gen[k % 2].record(gs)
            gen_ev.append((a, b))

        gen_chunk(0)
        for k in range(T // C):
            if k + 1 < T // C:
                gen_chunk(k + 1)
            ms.wait_event(ev_gen[k % 2])
            env.load_messages(ring[k % 2], off)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ms)
            lob.lob_rollout_policy(env.h, pol, C, lob.LOB_PREC_BF16, stream=ms)
            b.record(ms)
            ev_free[k % 2].record(ms)
            roll_ev.append((a, b))
        w1.record(ms)
        torch.cuda.synchronize()
        assert gen.ok(), "a generator pool ran out of room"
        assert env.sync() == 0 and lob.lob_policy_sync(pol) == 0
        msgs = float(env.counters()[:, 0].sum().item())
        t_roll = sum(x.elapsed_time(y) for x, y in roll_ev) / 1e3
        t_gen = sum(x.elapsed_time(y) for x, y in gen_ev) / 1e3
        t_wall = w0.elapsed_time(w1) / 1e3
        lob.lob_policy_destroy(pol)
        env.close()
        gen.close()
        line = {"workload": "stress65536", "metric": METRIC, "value": msgs / t_roll, "unit": "msgs/s",
                "env_steps_per_s": n * T / t_roll, "seconds_rollout": t_roll, "steps": T, "n_gpus": 1,
                "generation": {"seconds": t_gen, "msgs_per_s": msgs / t_gen, "where": "device generator, own stream"},
                "overlapped": {"seconds": t_wall, "msgs_per_s": msgs / t_wall},
                "config": {"workload": f"65536 envs x cap 1000 x 1000 msgs (30% aggressive, Pareto(1.5) sizes "
                                       f"capped at 1e4, delete bursts) x {T} steps, top-20 obs, BF16 policy in the "
                                       f"loop; {C}-step chunks generated on the device into a double-buffered ring",
                           "messages": msgs},
                "dtype": "int64 book / bf16 policy", "data": "synthetic"}
    else:
        raise SystemExit(f"unknown workload {wl}")
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--wpb", type=int, default=0, help="warps per block (0 = library default)")
    ap.add_argument("--threads-per-env", type=int, default=32, choices=[32, 64],
                    help="64: one warp per book side (the plain step)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="envs1024",
                    choices=["envs1024", "envs16384", "uneven8192", "policy4096", "ppo4096", "episodes4096",
                             "table1", "compact1024", "stress65536"],
                    help="envs1024 is the benchmark line; the others print secondary lines")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--per-class", action="store_true", help="uneven8192: also time each capacity class alone")
    ap.add_argument("--stress-steps", type=int, default=256)
    ap.add_argument("--policy-envs", type=int, default=4096, help="policy4096: envs (a smaller case for profiling)")
    ap.add_argument("--policy-steps", type=int, default=128, help="policy4096: rollout steps")
    ap.add_argument("--gen-steps", type=int, default=T,
                    help="steps of messages generated (the episode wraps there; default: the full episode)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "envs16384":
        set_envs(16384)   # the step kernel over several waves: its own roofline line
    if args.impl == "reference":
        run_reference(args)
    elif args.workload not in ("envs1024", "envs16384"):
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
