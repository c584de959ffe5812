"""Failure detection on the GPU without a GPU fault: a bounded device wait
that runs out (a message tile that is never requested) is reported as
LOB_ETIMEOUT and leaves the context usable; a device allocation that cannot
be satisfied is reported as LOB_ENOMEM."""
import numpy as np
import pytest

from harness import Pair
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"


@pytest.mark.parametrize("persistent,rollout", [(0, False), (1, False), (0, True)])
def test_held_tile_times_out_then_context_recovers(persistent, rollout):
    n, T = 40, 8
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(150, n), T)
    pr = Pair(n, st, cap=100, exec_target=60)
    if persistent:
        lob.lob_set_launch(pr.env.h, 4, 1)
    for _ in range(2):
        pr.step()
        pr.check_outputs()
    assert lob.lob_sync(pr.env.h) == 0
    # a wait bound of 20,000 SM cycles and the next launch's first tile held back
    lob.lob_debug_wait(pr.env.h, 20_000, 1)
    if rollout:
        lob.lob_rollout(pr.env.h, 3, None, None, None, None)
    else:
        pr.env.step()
    assert lob.lob_sync(pr.env.h) == lob.LOB_ETIMEOUT
    assert lob.lob_sync(pr.env.h) == 0                    # reported once, then cleared
    # the context still works: reset both sides and replay from the start
    lob.lob_debug_wait(pr.env.h, 0, 0)
    pr.env.reset(pr.seeds_d)
    pr.env.load_messages(pr.msgs_d, pr.off_d)
    pr.orc.reset(st.seeds)
    pr.orc.load_messages(st.msgs, st.offsets)
    for _ in range(4):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    assert lob.lob_sync(pr.env.h) == 0
    pr.close()


def test_wait_hook_rejects_bad_arguments():
    cfg = lob.lob_config(4, 2, 100, 10, 10, 1, 10, -1, 1, 0, 10000, 0)
    h = lob.lob_create(cfg)
    for cycles, hold in ((-1, 0), (10, 2)):
        with pytest.raises(lob.LobError) as ei:
            lob.lob_debug_wait(h, cycles, hold)
        assert ei.value.code == lob.LOB_EINVAL
    lob.lob_destroy(h)


def test_device_allocation_failure_reported():
    """Ten million envs at the largest capacity need ~490 GB of books, more
    than the device has: lob_create frees what it took and returns ENOMEM."""
    import torch
    free0, _ = torch.cuda.mem_get_info()
    cfg = lob.lob_config(10_000_000, 2, lob.LOB_MAX_CAP, 10, 10, 1, 10, -1, 1, 0, 10000, 0)
    with pytest.raises(lob.LobError) as ei:
        lob.lob_create(cfg)
    assert ei.value.code == lob.LOB_ENOMEM
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20                 # nothing left allocated
    # and the device still serves a normal handle
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=30), mbogen.env_seeds(151, 8), 3)
    pr = Pair(8, st, cap=50, exec_target=20)
    for _ in range(3):
        pr.step()
        pr.check_outputs()
    pr.close()
