"""The device generator (mbogen_gpu.cu) against the host generator: byte-
identical streams whatever the chunking, for the base mix and the
heavy-tailed stress mix with its delete bursts."""
import numpy as np
import pytest

from paper_2511_02136_gb300 import mbogen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,n,chunks", [
    (mbogen.MessageModel(msgs_per_step=100), 77, (3, 1, 4)),
    (mbogen.STRESS_MODEL, 40, (2, 5, 1)),
])
def test_device_generator_matches_host(model, n, chunks):
    import torch
    seeds = mbogen.env_seeds(555, n)
    T = sum(chunks)
    host = mbogen.generate(model, seeds, T)
    g = mbogen.GpuStreams(model, seeds)
    M = model.msgs_per_step
    t0 = 0
    for k in chunks:
        out = torch.zeros(n * k * M * 32, dtype=torch.uint8, device="cuda")
        g.chunk(k, out)
        got = out.cpu().numpy().view(mbogen.MSG_DTYPE).reshape(n, k, M)
        for e in range(n):
            want = host.msgs[host.offsets[e, t0]:host.offsets[e, t0 + k]].reshape(k, M)
            assert np.array_equal(got[e].view(np.uint8), want.view(np.uint8)), (e, t0)
        t0 += k
    assert g.ok()
    g.close()
