"""Peak-temperature snapshots of the synchronized marching (Sec. II-A loop;
Sec. IV-A takes the static mechanical solves at peak-temperature snapshots)
on the CUDA path against the FP64 oracle's coupled loop.

A current source drives three z-edges inside a copper block for the first 12
of 40 coupled steps; the block's copper has a small heat capacity
(rho c_p = 100 J/m^3K) so that the heat spreads within the 40 steps: the
hottest node heats while the source is on and cools after, so the peak lies
inside the march. The peak step is an argmax decided in each side's own
arithmetic, so the test compares what is unique (the peak value, and the
oracle's field at the step the GPU chose) and checks that the GPU's step is
a valid argmax of the oracle's per-step maxima."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, hetero_problem, rel_l2
from workloads import constraints as BC

pytestmark = pytest.mark.gpu

STEPS, ON = 40, 12


def problem():
    p = hetero_problem(23, 14, 9, seed=31, em_bc=(0,) * 6, cpml=0, uniform_x=True)
    cu = dataclasses.replace(W.COPPER, rho_cp=100.0)
    mat = p.mat.copy()
    mat[2:7, 4:10, 6:16] = 1  # a copper block around the source edges
    return dataclasses.replace(p, materials=[W.DIELECTRIC, cu, W.SILICON, W.UNDERFILL], mat=mat)


def sources():
    edges = np.array([[10, 7, 3], [11, 7, 3], [10, 8, 3]], np.int32)
    amp = np.zeros(STEPS)
    amp[:ON] = 3e12
    return [(2, edges, amp)]


@pytest.fixture(scope="module")
def ref():
    p = problem()
    o = oracle.OracleSim(p)
    o.set_sources(sources())
    thetas = []
    for _ in range(STEPS):
        o.coupled_steps(1)
        thetas.append(o.theta.copy())
    return p, o.dt, thetas


_solves = {}


def oracle_solve(p, step, th):
    """the oracle's clamped-bottom solve with the field of `step` (cached: the
    FP64 and FP32 runs choose the same peak step)"""
    if step not in _solves:
        o = oracle.OracleSim(p)
        o.theta = th.copy()
        _solves[step] = o.stress_solve(BC.clamped_bottom(p), 300.0, rtol=1e-13)
    return _solves[step]


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (FP32, 1e-4)])
@pytest.mark.parametrize("every", [1, 4])
def test_peak_snapshot_and_stress_solve(ref, precision, tol, every, fused):
    p, dt, thetas = ref
    checks = [s for s in range(1, STEPS + 1) if s % every == 0 or s == STEPS]
    maxima = {s: float(thetas[s - 1].max()) for s in checks}
    best = max(maxima.values())
    assert 1 < max(maxima, key=maxima.get) < STEPS  # the peak lies inside the march

    ctx = context(p, precision, dt)
    ctx.set_sources(sources())
    rep = ctx.coupled_march(STEPS, check_every=every, fused=fused)
    assert rep["step"] in maxima and rep["peaks"] >= 1
    assert abs((rep["T_max"] - p.T_init) / best - 1) < tol
    # a valid argmax: the oracle's maximum at the chosen step is the peak
    assert maxima[rep["step"]] >= best * (1 - 10 * tol)
    snap = ctx.read(api.COSIM_F_T_PEAK) - p.T_init
    th = thetas[rep["step"] - 1]
    assert rel_l2(snap, th) < tol
    # the snapshot is not the final field: the block cooled after the peak
    assert np.abs(ctx.read(api.COSIM_F_DT) - snap).max() > 1.0

    # the static solve takes its load from the snapshot
    want = oracle_solve(p, rep["step"], th)
    got = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-9, refine=True,
                           temperature=api.COSIM_STRESS_T_PEAK)
    u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)], 1).reshape(-1)
    assert got["relres"] <= 1e-9
    assert rel_l2(u, want["u"]) < (1e-7 if precision == FP64 else 10 * tol)
    assert rel_l2(ctx.read(api.COSIM_F_VM), want["vm"]) < (1e-7 if precision == FP64 else 10 * tol)
    ctx.close()


def test_peak_march_rejects_bad_arguments_and_solve_without_snapshot():
    p = problem()
    ctx = context(p, FP64)
    with pytest.raises(api.CosimError) as e:
        ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, temperature=api.COSIM_STRESS_T_PEAK)
    assert e.value.status == api.COSIM_ERR_INVALID
    with pytest.raises(api.CosimError):
        ctx.coupled_march(4, check_every=0)
    ctx.close()
