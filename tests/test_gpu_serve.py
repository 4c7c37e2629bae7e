"""Continuous-batching server: requests submitted while others are resident join
the running batch, and each result equals the single solve of that request."""
import math
import time

import numpy as np
import pytest

from paper_1909_13263_gb300 import inputs, native
from test_gpu_batch import MIXED_SOLVE_TOL, oracle_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


def _single(inst):
    phi0, _ = inputs.instance_phi0(inst)
    with native.Solver(dim=2, nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham,
                       precision="mixed") as s:
        s.set_phi0(phi0)
        steps = s.step_to(inst.t_final)
        return s.get_phi(), steps


@pytest.mark.parametrize("round_tiles", [None, 0, 60])
def test_served_results_equal_single_solves(round_tiles):
    # None: the default tile limit; 0: every resident instance in every round; 60: instances
    # above 32 tiles (here up to 520^2 = 9 x 17 tiles) wait for their turn behind older ones
    insts = [inputs.Instance(i.n, i.ham, i.theta, i.t_final * 0.3)
             for i in inputs.batch_instances(18, 24, 520, seed=77)]
    with native.Server(hbm_budget_bytes=1 << 30, max_slots=6, max_side=520) as srv:
        srv.set_round_steps(2)
        if round_tiles is not None:
            srv.set_round_tiles(round_tiles)
        ids = []
        for k, inst in enumerate(insts):
            phi0, _ = inputs.instance_phi0(inst)
            ids.append(srv.submit(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham,
                                  phi0=phi0, t_final=inst.t_final))
            if k % 5 == 4:
                time.sleep(0.01)   # later requests arrive while earlier ones are resident
        results = {}
        for rid in ids:
            done, info, out = srv.poll(rid, timeout=120.0)
            assert done and info["status"] == 0 and info["latency_s"] > 0
            results[rid] = (out, info)
        st = srv.stats()
        assert st["completed"] == len(insts) and st["queued"] == 0
        assert st["free_rows"] == st["arena_rows"]
    for rid, inst in zip(ids, insts):
        ref, steps = _single(inst)
        out, info = results[rid]
        assert info["steps"] == steps
        assert np.array_equal(out, ref)


def test_server_limits():
    with native.Server(hbm_budget_bytes=256 << 20, max_slots=2, max_side=128) as srv:
        with pytest.raises(native.AlwError) as e:
            srv.submit(nx=200, ny=200, xlo=0, xhi=1, ylo=0, yhi=1, ham="burgers2d", phi0=np.zeros(40000),
                       t_final=0.01)
        assert e.value.status == native.EBUDGET
    with pytest.raises(native.AlwError) as e:
        native.Server(hbm_budget_bytes=1 << 20, max_slots=2, max_side=1024)
    assert e.value.status == native.EBUDGET


def test_served_results_match_oracle():
    # requests of uneven size and both Hamiltonians, submitted while others are resident: each
    # result against the oracle's solve of that request alone
    insts = [inputs.Instance(i.n, i.ham, i.theta, i.t_final * 0.3)
             for i in inputs.batch_instances(8, 24, 200, seed=91)]
    insts.append(inputs.Instance(65, "burgers2d" if insts[0].ham == "negcos2d" else "negcos2d", 1.3,
                                 0.1 / math.pi**2))
    assert {i.ham for i in insts} == {"burgers2d", "negcos2d"}
    with native.Server(hbm_budget_bytes=1 << 30, max_slots=4, max_side=256) as srv:
        srv.set_round_steps(2)
        ids = []
        for k, inst in enumerate(insts):
            phi0, _ = inputs.instance_phi0(inst)
            ids.append(srv.submit(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham,
                                  phi0=phi0, t_final=inst.t_final))
            if k % 3 == 2:
                time.sleep(0.005)
        results = [srv.poll(rid, timeout=120.0) for rid in ids]
    for inst, (done, info, out) in zip(insts, results):
        assert done and info["status"] == 0
        ref, _ = oracle_solve(inst, "arclength")
        err = float(np.max(np.abs(out - ref)))
        assert err <= MIXED_SOLVE_TOL, (inst, err)
