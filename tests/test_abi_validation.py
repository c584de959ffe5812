"""Argument validation of the C ABI that happens before any CUDA call, so it
runs without a GPU: each bad configuration or argument gets its documented
code (include/lob.h)."""
import numpy as np
import pytest

from paper_2511_02136_gb300 import lob


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()


def _cfg(**kw):
    c = lob.lob_config(8, 2, 100, 10, 10, 1, 10, -1, 1, 0, 10000, 0)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("field,val,code", [
    ("n_envs", 0, lob.LOB_EINVAL), ("n_agents", 3, lob.LOB_EINVAL),
    ("n_agents", 2 * lob.LOB_MAX_PER_TYPE + 2, lob.LOB_EINVAL),
    ("cap_per_side", 0, lob.LOB_EINVAL), ("cap_per_side", lob.LOB_MAX_CAP + 1, lob.LOB_ECAPACITY),
    ("top_levels", 0, lob.LOB_EINVAL), ("top_levels", 65, lob.LOB_EINVAL),
    ("episode_len", 0, lob.LOB_EINVAL), ("mm_lot", 0, lob.LOB_EINVAL), ("exec_target", -1, lob.LOB_EINVAL),
    ("exec_dir", 2, lob.LOB_EINVAL), ("action_mode", 7, lob.LOB_EINVAL), ("trace", 4, lob.LOB_EINVAL),
    ("warps_per_block", 9, lob.LOB_EINVAL), ("reward_mode", 3, lob.LOB_EINVAL),
    ("spooner_lambda_pct", 101, lob.LOB_EINVAL), ("inv_penalty", -1, lob.LOB_EINVAL),
    ("exec_penalty_milli", -5, lob.LOB_EINVAL), ("mm_space", 3, lob.LOB_EINVAL), ("pv_ref", 2, lob.LOB_EINVAL),
])
def test_create_rejects_before_touching_the_device(field, val, code):
    with pytest.raises(lob.LobError) as ei:
        lob.lob_create(_cfg(**{field: val}))
    assert ei.value.code == code


def test_per_env_capacities_checked():
    with pytest.raises(lob.LobError) as ei:
        lob.lob_create(_cfg(), caps=np.array([100] * 7 + [lob.LOB_MAX_CAP + 1], np.int32))
    assert ei.value.code == lob.LOB_ECAPACITY
    with pytest.raises(lob.LobError) as ei:
        lob.lob_create(_cfg(), caps=np.array([100] * 7 + [0], np.int32))
    assert ei.value.code == lob.LOB_EINVAL


def test_null_handles_and_bad_hooks():
    for call in (lambda: lob.lob_set_launch(None, 4, 0), lambda: lob.lob_debug_wait(None, 0, 0)):
        with pytest.raises(lob.LobError) as ei:
            call()
        assert ei.value.code == lob.LOB_EINVAL


def test_policy_create_validates_shapes():
    n = lob.lob_policy_param_count(45)
    for agents, dim, code in ((0, 45, lob.LOB_EINVAL), (2 * lob.LOB_MAX_PER_TYPE + 1, 45, lob.LOB_EINVAL),
                              (2, 46, lob.LOB_EINVAL), (2, 133, lob.LOB_ECAPACITY)):
        with pytest.raises(lob.LobError) as ei:
            lob.lob_policy_create(agents, dim, np.zeros((max(agents, 1), max(n, 1)), np.float32))
        assert ei.value.code == code


class _DefaultStream:
    """The legacy default stream, named without asking torch (no GPU here)."""
    cuda_stream = None


def _noalloc_args(cfg, **ptrs):
    """Arguments of lob_step_noalloc with fake, suitably aligned device
    addresses: every case below is refused before any CUDA call."""
    base = dict(d_books=0x100000, d_env_state=0x200000, d_counters=0x300000, d_env_seeds=0x400000,
                d_msgs=0x500000, d_offsets=0x600000, d_status=0x700000)
    base.update(ptrs)
    return lob.lob_noalloc_args(cfg=lob.ctypes.pointer(cfg), stride=5, k=0, t=0, d_actions=None, d_obs=None,
                                d_rewards=None, d_done=None, **base)


@pytest.mark.parametrize("field,val", [
    ("reward_mode", lob.LOB_REWARD_SPOONER), ("inv_penalty", 1), ("exec_penalty_milli", 10),
    ("mm_space", lob.LOB_MM_DIRECTIONAL), ("pv_ref", lob.LOB_PV_MID), ("exec_dir", 0), ("n_agents", 4)])
def test_noalloc_rejects_extended_options(field, val):
    """The allocation-free step runs the plain kernel only: every extended
    option is refused, not ignored."""
    cfg = _cfg()
    setattr(cfg, field, val)
    with pytest.raises(lob.LobError) as ei:
        lob.lob_step_noalloc(_noalloc_args(cfg), _DefaultStream)
    assert ei.value.code == lob.LOB_EINVAL, field


@pytest.mark.parametrize("ptr,addr", [
    ("d_msgs", 0x500008), ("d_env_state", 0x200008), ("d_books", 0x100010), ("d_books", 0x100080)])
def test_noalloc_rejects_misaligned_buffers(ptr, addr):
    """Messages and env state must sit on 16-byte boundaries and book blocks on
    256-byte ones (bulk copies and vector accesses): a misaligned pointer is an
    argument error on the host, never a launch."""
    with pytest.raises(lob.LobError) as ei:
        lob.lob_step_noalloc(_noalloc_args(_cfg(), **{ptr: addr}), _DefaultStream)
    assert ei.value.code == lob.LOB_EINVAL


def test_noalloc_rejects_oversize_on_the_host():
    with pytest.raises(lob.LobError) as ei:
        lob.lob_step_noalloc(_noalloc_args(_cfg(n_envs=lob.LOB_NOALLOC_MAX_ENVS + 1)), _DefaultStream)
    assert ei.value.code == lob.LOB_ECAPACITY


@pytest.mark.gpu
def test_multi_split_validated_on_the_host():
    """The one-launch mode's split: 1..8 warps, classes up to 512 slots, every
    class with envs covered by a warp of its class or a larger one."""
    h = lob.lob_create(_cfg(cap_per_side=100))   # one class (128 slots, index 2)
    for split, code in (((0, 0, 0, 0, 0, 0), lob.LOB_EINVAL), ((0, 0, 0, 0, 0, 1), lob.LOB_EINVAL),
                        ((0, 1, 0, 0, 0, 0), lob.LOB_EINVAL), ((3, 3, 3, 0, 0, 0), lob.LOB_EINVAL)):
        with pytest.raises(lob.LobError) as ei:
            lob.lob_set_multi_split(h, np.array(split, np.int32))
        assert ei.value.code == code, split
    lob.lob_set_multi_split(h, np.array((0, 0, 2, 2, 0, 0), np.int32))
