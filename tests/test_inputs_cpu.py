"""The seeded synthetic workloads (paper_1909_13263_gb300/inputs.py) have the shapes and distributions their
docstrings state: node grids of both boundary kinds, the batch mix (log-uniform sides, two Hamiltonians, random
phase, t_final in [0.1, 0.5]/pi^2) and Poisson request arrivals.  No GPU needed."""
import math

import numpy as np
import pytest

from paper_1909_13263_gb300 import inputs


def test_axes_of_both_boundary_kinds():
    x, dx = inputs.axis(8, -2.0, 2.0, "periodic")         # N nodes on [a, b): the right end is the left's image
    assert dx == 0.5 and x[0] == -2.0 and x[-1] == pytest.approx(1.5)
    x, dx = inputs.axis(9, -1.0, 1.0, "linextrap")        # N nodes on [a, b] including both ends
    assert dx == 0.25 and x[0] == -1.0 and x[-1] == pytest.approx(1.0)
    with pytest.raises(ValueError):
        inputs.axis(1, 0.0, 1.0, "linextrap")


def test_batch_mix_is_seeded_and_has_the_stated_distribution():
    a = inputs.batch_instances(512, 64, 1024)
    assert a == inputs.batch_instances(512, 64, 1024)      # same seed, same workload
    assert a != inputs.batch_instances(512, 64, 1024, seed=inputs.SEED + 1)
    n = np.array([i.n for i in a], dtype=float)
    assert n.min() >= 64 and n.max() <= 1024
    # log-uniform sides: mean of log n at the midpoint, E[n^2] = (hi^2 - lo^2) / (2 ln(hi/lo)) ~ 1.88e5
    assert np.mean(np.log(n)) == pytest.approx(0.5 * (math.log(64) + math.log(1024)), abs=0.12)
    assert np.mean(n**2) == pytest.approx((1024**2 - 64**2) / (2 * math.log(16)), rel=0.15)
    hams = [i.ham for i in a]
    assert set(hams) == {"burgers2d", "negcos2d"} and abs(hams.count("burgers2d") - 256) < 48
    tf = np.array([i.t_final for i in a]) * math.pi**2
    assert tf.min() >= 0.1 and tf.max() <= 0.5
    th = np.array([i.theta for i in a])
    assert th.min() >= 0.0 and th.max() < 2 * math.pi


def test_instance_initial_data_is_the_phase_shifted_example_3_profile():
    inst = inputs.Instance(40, "negcos2d", 0.7, 0.02)
    phi0, dx = inputs.instance_phi0(inst)
    x, _ = inputs.axis(40, -2.0, 2.0, "periodic")
    assert phi0.shape == (40, 40) and dx == pytest.approx(0.1)
    assert phi0[3, 5] == pytest.approx(-math.cos(math.pi * (x[5] + x[3]) / 2 + 0.7))
    # periodic on [-2, 2): the profile has period 4 in x and y
    assert -math.cos(math.pi * ((x[5] + 4.0) + x[3]) / 2 + 0.7) == pytest.approx(phi0[3, 5])


def test_request_stream_is_poisson_with_the_batch_mix():
    reqs = inputs.request_stream(200.0, 400, 128, 2048)
    t = np.array([a for a, _ in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 200.0, rel=0.15)     # exponential gaps of mean 1/rate
    assert gaps.std() == pytest.approx(gaps.mean(), rel=0.2)       # coefficient of variation 1
    sides = [i.n for _, i in reqs]
    assert min(sides) >= 128 and max(sides) <= 2048
    assert reqs == inputs.request_stream(200.0, 400, 128, 2048)
