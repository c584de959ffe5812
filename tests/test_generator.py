"""The seeded input generator: determinism, layout and the message model's moments."""
import numpy as np
import pytest

from paper_2511_02136_gb300 import mbogen as g


def test_deterministic_per_seed_and_env():
    a = g.generate(g.MessageModel(), g.env_seeds(0, 3), 20)
    b = g.generate(g.MessageModel(), g.env_seeds(0, 3), 20, n_threads=1)
    assert a.msgs.tobytes() == b.msgs.tobytes()
    c = g.generate(g.MessageModel(), g.env_seeds(1, 3), 20)
    assert a.msgs.tobytes() != c.msgs.tobytes()
    # env e's stream depends only on its own seed
    d = g.generate(g.MessageModel(), g.env_seeds(0, 3)[1:2], 20)
    assert d.msgs.tobytes() == a.msgs[a.offsets[1, 0]:a.offsets[1, -1]].tobytes()


def test_layout_and_offsets():
    st = g.generate(g.MessageModel(msgs_per_step=7), g.env_seeds(2, 4), 5)
    assert st.offsets.shape == (4, 6)
    assert np.all(np.diff(st.offsets, axis=1) == 7)
    assert st.offsets[0, 0] == 0 and st.offsets[-1, -1] == len(st.msgs)
    assert np.all(st.offsets[1:, 0] == st.offsets[:-1, -1])


def test_base_mix_moments():
    st = g.generate(g.MessageModel(), g.env_seeds(3, 8), 500)
    m = st.msgs
    n = len(m)
    frac = {k: np.mean(m["type"] == k) for k in (1, 2, 3, 4)}
    # partial cancels / deletes fall back to adds only while the pool is empty
    assert abs(frac[1] - 0.55) < 0.01 and abs(frac[2] - 0.15) < 0.01
    assert abs(frac[3] - 0.20) < 0.01 and abs(frac[4] - 0.10) < 0.01
    sz = m["qty"][(m["type"] == 1) | (m["type"] == 4)]
    assert sz.min() >= 1 and abs(sz.mean() - 100.0) < 2.0      # 1 + Geom0(0.01): mean 100
    assert np.all(np.isin(m["side"], [1, -1]))
    assert np.all(m["ts"][st.offsets[0, 0]:st.offsets[0, -1]] == np.arange(st.offsets[0, -1]))
    assert n == 8 * 500 * 100


def test_price_offsets_geometric():
    """Reconstruct g = distance from the latent mid via adds right after a mid move is impossible;
    instead check the one-sided spread of add prices around a running median."""
    st = g.generate(g.MessageModel(p_move=0.0), g.env_seeds(4, 4), 200)
    m = st.msgs[st.msgs["type"] == 1]
    gap = np.where(m["side"] == 1, 10_000 - m["px"], m["px"] - 10_000)
    assert gap.min() == 0
    p0 = np.mean(gap == 0)
    assert abs(p0 - 0.3) < 0.01                                  # P(g = 0) = p
    assert abs(gap.mean() - 0.7 / 0.3) < 0.05                    # E g = (1-p)/p


def test_cancels_target_issued_ids():
    st = g.generate(g.MessageModel(), g.env_seeds(5, 2), 50)
    for e in range(2):
        m = st.msgs[st.offsets[e, 0]:st.offsets[e, -1]]
        issued = {}
        for r in m:
            if r["type"] == 1:
                issued[int(r["oid"])] = (int(r["px"]), int(r["side"]))
            elif r["type"] in (2, 3):
                assert issued[int(r["oid"])] == (int(r["px"]), int(r["side"]))
                assert r["qty"] >= 1


def test_poisson_counts():
    st = g.generate(g.MessageModel(poisson=True), g.env_seeds(6, 64), 400)
    assert np.all((st.lambdas >= 10) & (st.lambdas <= 500))
    means = st.counts.mean(axis=1)
    assert np.all(np.abs(means - st.lambdas) < 5 * np.sqrt(st.lambdas / 400) + 0.5)
    v = st.counts.var(axis=1)
    assert np.median(v / st.lambdas) > 0.85 and np.median(v / st.lambdas) < 1.15


def test_stress_mix_pareto_sizes_and_bursts():
    st = g.generate(g.STRESS_MODEL, g.env_seeds(7, 4), 60)
    m = st.msgs
    sz = m["qty"][(m["type"] == 1) | (m["type"] == 4)]
    assert sz.min() >= 1 and sz.max() <= 10_000
    for k in (2, 4, 10):
        assert abs(np.mean(sz >= k) - k ** -1.5) < 0.01           # P(floor X >= k) = k^-alpha
    assert abs(np.mean(m["type"] == 4) - 0.30) < 0.03


def test_env_caps_choices():
    caps = g.env_caps(9, 4000)
    vals, cnt = np.unique(caps, return_counts=True)
    assert vals.tolist() == [50, 100, 200, 500]
    assert np.all(np.abs(cnt / 4000 - 0.25) < 0.03)


def test_pack16_round_trip_and_malformed():
    """The compact encoding keeps price, size, id, type and side of every valid
    record; an invalid type or side becomes type 0; ids beyond 60 bits are refused."""
    st = g.generate(g.MessageModel(msgs_per_step=50), g.env_seeds(3, 4), 5)
    msgs = st.msgs.copy()
    msgs["type"][7] = 9
    msgs["side"][11] = 0
    msgs["oid"][13] = (1 << 59) - 1
    p = g.pack16(msgs)
    assert p.dtype.itemsize == 16
    w = p["word"].astype(np.int64)
    typ, sell, oid = w & 7, (w >> 3) & 1, w >> 4
    ok = np.ones(len(msgs), bool)
    ok[[7, 11]] = False
    np.testing.assert_array_equal(p["px"], msgs["px"])
    np.testing.assert_array_equal(p["qty"], msgs["qty"])
    np.testing.assert_array_equal(oid, msgs["oid"])
    np.testing.assert_array_equal(typ[ok], msgs["type"][ok])
    np.testing.assert_array_equal(np.where(sell[ok] == 1, -1, 1), msgs["side"][ok])
    assert typ[7] == 0 and typ[11] == 0
    bad = msgs[:2].copy()
    bad["oid"][0] = 1 << 59
    with pytest.raises(ValueError):
        g.pack16(bad)
