"""Batched multi-instance solves: every instance gives exactly the result of a
single solve with the same scheme, whatever else is in the batch."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu

# Float paths against the FP64 oracle: max |phi - phi_oracle| of a whole MIXED solve, the bound of
# the single-solve test test_mixed_solve_error_vs_fp64_oracle_is_bounded (phi of order one).
MIXED_SOLVE_TOL = 2e-6


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
    # uniform: every instance has the same Hamiltonian, so the batch runs that Hamiltonian's kernel.
    # With the single solver's 64 x 32 tiles the batch runs the same kernel on the same segments,
    # so its results are bitwise those of the single solves.
    insts = _mix(10, 24, 200, seed=11)
    insts.append(inputs.Instance(65, "negcos2d", 1.0, 0.3 / math.pi**2 * 0.25))   # ragged tiles
    if uniform:
        insts = [inputs.Instance(i.n, "negcos2d", i.theta, i.t_final) for i in insts]
    with native.Batch(precision=precision, weights=weights) as b:
        for inst in insts:
            phi0, _ = inputs.instance_phi0(inst)
            b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                  t_final=inst.t_final)
        b.set_tuning(order="largest_first", steps_per_graph=4, run=4, tile_w=64)
        b.run()
        for k, inst in enumerate(insts):
            ref, steps = _single(inst, precision, weights)
            got = b.get_phi(k)
            st = b.get_state(k)
            assert st.t == inst.t_final and st.steps == steps
            assert np.array_equal(got, ref), (k, inst, float(np.max(np.abs(got - ref))))


@pytest.mark.parametrize("precision,weights", [("mixed", "arclength"), ("fp32", "jp")])
def test_batch_narrow_tiles_match_wide_tiles_and_autotuner_reports_its_choice(precision, weights):
    # 32 x 32 tiles: another kernel instantiation over the same segments, so results agree with
    # the 64 x 32 tiling to rounding (bound: the mixed-solve bound against the oracle)
    insts = _mix(9, 24, 200, seed=31)
    insts.append(inputs.Instance(97, "negcos2d", 0.4, 0.2 / math.pi**2 * 0.25))   # 4 narrow tiles across
    outs = {}
    for w in (64, 32, None):
        with native.Batch(precision=precision, weights=weights) as b:
            for inst in insts:
                phi0, _ = inputs.instance_phi0(inst)
                b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                      t_final=inst.t_final)
            if w is not None:
                b.set_tuning(order="instance", steps_per_graph=3, run=4, tile_w=w)
            b.run()
            tun = b.tuning()
            assert tun["tile"] in ("64x32", "32x32")
            if w is not None:
                assert tun["tile"] == f"{w}x32"
            outs[w] = [b.get_phi(k) for k in range(len(insts))]
    for a, c, d in zip(outs[64], outs[32], outs[None]):
        assert np.max(np.abs(a - c)) <= MIXED_SOLVE_TOL
        assert np.max(np.abs(a - d)) <= MIXED_SOLVE_TOL


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



def oracle_solve(inst, weights):
    """The FP64 oracle's solve of one batch instance (Example 3 or 4 mix, lagged grid-wide alpha)."""
    phi0, dx = inputs.instance_phi0(inst)
    cfg = oracle.make_cfg(dim=2, nx=inst.n, ny=inst.n, dx=dx, ham=inst.ham, weights=weights,
                          alpha_mode="global_lagged", xlo=-2.0, ylo=-2.0)
    ref, steps, t, _, st = oracle.solve(cfg, phi0, inst.t_final)
    assert st == 0 and t == inst.t_final
    return ref, steps


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_batch_instances_match_oracle(weights):
    # every instance of a mixed-precision batch -- uneven sizes, ragged tiles, both Hamiltonians of
    # the batched workload -- against the oracle's solve of that instance alone
    insts = _mix(9, 24, 180, seed=23)
    insts += [inputs.Instance(65, "negcos2d", 0.7, 0.2 / math.pi**2), inputs.Instance(97, "burgers2d", 2.1,
                                                                                    0.15 / math.pi**2)]
    assert {i.ham for i in insts} == {"burgers2d", "negcos2d"}
    with native.Batch(precision="mixed", weights=weights) as b:
        for inst in insts:
            phi0, _ = inputs.instance_phi0(inst)
            b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                  t_final=inst.t_final)
        b.run()
        outs = [(b.get_phi(k), b.get_state(k)) for k in range(len(insts))]
    for k, (inst, (got, st)) in enumerate(zip(insts, outs)):
        ref, steps = oracle_solve(inst, weights)
        assert st.t == inst.t_final
        err = float(np.max(np.abs(got - ref)))
        assert err <= MIXED_SOLVE_TOL, (k, inst, err)


@pytest.mark.parametrize("tile_w", [64, 32])
def test_batch_one_launch_per_stage_matches_per_hamiltonian_launches(tile_w):
    # both Hamiltonians of the batched workload in one launch per RK stage (the kernel choosing each
    # tile's Hamiltonian) against one launch per Hamiltonian: another kernel instantiation over the
    # same segments, so the results agree to rounding (the mixed-solve bound against the oracle)
    insts = _mix(10, 24, 200, seed=47)
    assert {i.ham for i in insts} == {"burgers2d", "negcos2d"}
    outs = {}
    for one in (False, True):
        with native.Batch(precision="mixed") as b:
            for inst in insts:
                phi0, _ = inputs.instance_phi0(inst)
                b.add(nx=inst.n, ny=inst.n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham=inst.ham, phi0=phi0,
                      t_final=inst.t_final)
            b.set_tuning(order="interleaved", steps_per_graph=3, run=4, tile_w=tile_w, one_launch=one)
            b.run()
            assert b.tuning()["launches_per_stage"] == ("one" if one else "one per Hamiltonian")
            outs[one] = [(b.get_phi(k), b.get_state(k)) for k in range(len(insts))]
    for inst, (a, sa), (c, sc) in zip(insts, outs[False], outs[True]):
        assert sa.t == sc.t == inst.t_final
        assert np.max(np.abs(a - c)) <= MIXED_SOLVE_TOL
