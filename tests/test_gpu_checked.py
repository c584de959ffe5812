"""The checked build (LOB_CHECKED=1: every slot number and position taken
from the priority index bounds-checked, and both books' invariants verified
on the device after every step) on a selection of the parity tests, each
also asserting that no check failed (LOB_ECHECK).  It stands in for a memory
checker, which this setup does not offer."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SELECTION = [
    "tests/test_gpu_parity.py::test_tiny_capacities_every_branch",
    "tests/test_gpu_parity.py::test_two_agents_random_policy_ragged",
    "tests/test_gpu_parity.py::test_host_actions_and_buy_task",
    "tests/test_gpu_parity.py::test_pool_boundary_capacities_filled",
    "tests/test_gpu_parity.py::test_uneven_caps_and_poisson_counts",
    "tests/test_gpu_parity.py::test_stress_mix_cap1000_top20",
    "tests/test_gpu_parity.py::test_rollout_matches_stepwise_oracle",
    "tests/test_gpu_episodes.py::test_episodes_random_policy_each_capacity_class",
    "tests/test_gpu_agents.py::test_agents_per_type_each_capacity_class",
    "tests/test_gpu_agents.py::test_most_agents_smallest_books",
    "tests/test_gpu_task_side.py",
]


def test_checked_build_parity_selection():
    env = dict(os.environ, LOB_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider", *SELECTION],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
