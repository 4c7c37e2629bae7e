"""Batched multi-instance solves: every instance gives exactly the result of a
single solve with the same scheme, whatever else is in the batch."""
import math

import numpy as np
import pytest

from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


def _mix(count, lo, hi, seed, tscale=0.25):
    insts = inputs.batch_instances(count, lo, hi, seed=seed)
    # shorter end times keep the test quick; sizes, Hamiltonians and phases are the batch mix
    return [inputs.Instance(i.n, i.ham, i.theta, i.t_final * tscale) for i in insts]


def _single(inst, precision, weights):
    phi0, dx = inputs.instance_phi0(inst)
    with native.Solver(dim=2, nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham,
                       precision=precision, weights=weights) as s:
        s.set_phi0(phi0)
        steps = s.step_to(inst.t_final)
        return s.get_phi(), steps


@pytest.mark.parametrize("precision,weights,uniform", [("mixed", "arclength", False), ("fp32", "jp", False),
                                                       ("mixed", "jp", False), ("mixed", "arclength", True)])
def test_batch_equals_single_solves(precision, weights, uniform):
    # uniform: every instance has the same Hamiltonian, so the batch runs that Hamiltonian's kernel
    insts = _mix(10, 24, 200, seed=11)
    insts.append(inputs.Instance(65, "negcos2d", 1.0, 0.3 / math.pi**2 * 0.25))   # ragged tiles
    if uniform:
        insts = [inputs.Instance(i.n, "negcos2d", i.theta, i.t_final) for i in insts]
    with native.Batch(precision=precision, weights=weights) as b:
        for inst in insts:
            phi0, _ = inputs.instance_phi0(inst)
            b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                  t_final=inst.t_final)
        b.run()
        for k, inst in enumerate(insts):
            ref, steps = _single(inst, precision, weights)
            got = b.get_phi(k)
            st = b.get_state(k)
            assert st.t == inst.t_final and st.steps == steps
            assert np.array_equal(got, ref), (k, inst, float(np.max(np.abs(got - ref))))


@pytest.mark.parametrize("run", [1, 4, 0])
def test_batch_fixed_tuning_orders_agree(run):
    # every order, runs of 1 and 4 entries per CTA and one stretch per CTA, and a CTA count below
    # the occupancy cap (so that many CTAs hold runs over several instances) give identical results
    insts = _mix(6, 32, 160, seed=5)
    outs = []
    for order, ctas in (("instance", 0), ("largest_first", 0), ("interleaved", 0), ("instance", 7)):
        with native.Batch() as b:
            for inst in insts:
                phi0, _ = inputs.instance_phi0(inst)
                b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                      t_final=inst.t_final)
            b.set_tuning(order=order, steps_per_graph=3, grid_ctas=ctas, run=run)
            b.run()
            tun = b.tuning()
            assert tun["order"] == order and tun["run"] == run and tun["grid_ctas"] == ctas
            outs.append([b.get_phi(k) for k in range(len(insts))])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_batch_errors_and_isolation():
    with pytest.raises(native.AlwError) as e:
        native.Batch(precision="fp64")
    assert e.value.status == native.EINVAL
    insts = _mix(4, 32, 96, seed=3)
    with native.Batch() as b:
        for k, inst in enumerate(insts):
            phi0, _ = inputs.instance_phi0(inst)
            if k == 1:
                phi0 = phi0.copy()
                phi0[3, 4] = np.nan
            b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                  t_final=inst.t_final)
        with pytest.raises(native.AlwError) as e:
            b.run()
        assert e.value.status == native.ENONFINITE
        # the other instances still reach their end time with the single-solve result
        for k in (0, 2, 3):
            ref, _ = _single(insts[k], "mixed", "arclength")
            assert np.array_equal(b.get_phi(k), ref)
        with pytest.raises(native.AlwError) as e:
            b.add(nx=8, ny=8, xlo=0, xhi=1, ylo=0, yhi=1, ham="burgers2d", phi0=np.zeros(64), t_final=0.1)
        assert e.value.status == native.EBUSY
