"""CUDA EM step (fused H/E/Joule kernel) vs the FP64 oracle, element by element.

Tolerances: FP64 kernels agree with the oracle to rounding-order differences
(1e-11 relative L2 after tens of steps); FP32 kernels to 2e-5 after 20 steps
of random fields (single-precision rounding, ~6e-8 per operation, grows
roughly linearly with the step count here)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, hetero_problem, random_fields, read_eh, rel_l2, seed_both

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, ny, nz, em_bc, cpml): ragged over the 31 x 7 node tiles, every wall type
    (37, 11, 9, (2, 2, 1, 0, 0, 1), 4),
    (33, 16, 12, (0, 1, 2, 2, 2, 2), 4),
    (62, 15, 10, (2, 2, 2, 2, 0, 2), 4),
    (20, 1, 6, (1, 0, 1, 1, 0, 1), 0),
    (7, 30, 1, (0, 0, 2, 2, 1, 1), 8),
    # wide enough for interior tile pairs (two nodes per thread) between the
    # border tiles; nx even and odd, a z slab through most planes
    (150, 40, 6, (2, 2, 2, 2, 0, 2), 4),
    (141, 23, 7, (1, 0, 0, 2, 1, 2), 4),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-11), (FP32, 2e-5)])
def test_em_random_fields_mixed_walls(case, precision, tol):
    nx, ny, nz, bc, L = CASES[case]
    p = hetero_problem(nx, ny, nz, seed=case, em_bc=bc, cpml=L)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    E, H = random_fields(p, seed=100 + case)
    seed_both(o, ctx, E, H)
    steps = 20
    o.em_steps(steps)
    ctx.em_steps(steps)
    Eg, Hg = read_eh(ctx)
    for a in range(3):
        assert rel_l2(Eg[a], o.E[a]) < tol, ("E", a)
        assert rel_l2(Hg[a], o.H[a]) < tol, ("H", a)
    Qg = ctx.read(api.COSIM_F_Q)
    assert rel_l2(Qg, o.Q) < tol * 5
    assert ctx.query(api.COSIM_Q_STEP) == steps
    ctx.close()


def test_cfl_step_matches_oracle():
    p = W.tiny_package()
    ctx = context(p, FP64)
    assert abs(ctx.dt / oracle.cfl_dt(p) - 1) < 1e-15
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-11), (FP32, 1e-4)])
def test_tiny_package_source_burst(precision, tol):
    """the 32x32x16 package: PEC ground, 8-cell CPML on five faces, lumped
    Gaussian-derivative port, Joule accumulation over 400 steps"""
    p = W.tiny_package()
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    steps = 400
    tables = p.source_tables(o.dt, steps)
    # make the early part of the pulse visible: the amplitude is linear in J
    tables = [(a, e, v * 50.0) for a, e, v in tables]
    o.set_sources(tables)
    ctx.set_sources(tables)
    o.em_steps(steps)
    ctx.em_steps(steps)
    Eg, Hg = read_eh(ctx)
    for a in range(3):
        assert rel_l2(Eg[a], o.E[a]) < tol
        assert rel_l2(Hg[a], o.H[a]) < tol
    assert rel_l2(ctx.read(api.COSIM_F_Q), o.Q) < tol
    tot = ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
    assert abs(tot / o.Q.sum() - 1) < tol
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-11), (FP32, 1e-4)])
def test_average_power_with_pending_joule_window(precision, tol):
    """FINALIZE_AVG_POWER straight after 70 accumulating steps (two full
    32-step windows and a partial one, nothing read in between): the power
    adds the pending window on the fly, and the energy read afterwards is
    complete"""
    p = W.tiny_package()
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    steps = 70
    tables = [(a, e, v * 50.0) for a, e, v in p.source_tables(o.dt, steps)]
    o.set_sources(tables)
    ctx.set_sources(tables)
    o.em_steps(steps)
    ctx.em_steps(steps)
    ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER, want_total=False)
    o.joule_finalize_avg_power()
    assert np.abs(o.P).max() > 0
    assert rel_l2(ctx.read(api.COSIM_F_P), o.P) < tol
    assert rel_l2(ctx.read(api.COSIM_F_Q), o.Q) < tol
    ctx.close()


def test_em_steps_deterministic_bitwise():
    p = hetero_problem(37, 11, 9, seed=3, em_bc=(2, 2, 2, 2, 0, 2), cpml=4)
    outs = []
    for _ in range(2):
        ctx = context(p, FP32, 1e-16)
        E, H = random_fields(p, seed=9)
        for a in range(3):
            ctx.write(api.COSIM_F_EX + a, E[a].astype(np.float32))
        ctx.em_steps(15)
        outs.append([ctx.read(api.COSIM_F_EX + a, np.float32) for a in range(3)] + [ctx.read(api.COSIM_F_Q)])
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_write_fields_zeroes_non_unknowns():
    p = hetero_problem(12, 5, 4, seed=1, em_bc=(0, 1, 0, 0, 1, 0), cpml=0)
    ctx = context(p, FP64)
    ones = np.ones(p.n_nodes)
    ctx.write(api.COSIM_F_EX, ones)
    got = ctx.read(api.COSIM_F_EX).reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    assert np.all(got[:, :, p.nx] == 0)          # beyond the last cell
    assert np.all(got[:, 0, :p.nx] == 0)         # tangential on the PEC y- wall
    assert np.all(got[0, 1:p.ny, :p.nx] == 1)    # PMC z- wall leaves it free
    ctx.close()
