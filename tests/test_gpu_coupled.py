"""Synchronized electro-thermal marching (Sec. II-A) on the CUDA path vs the
FP64 oracle's og_coupled_step: sigma(T^n) per voxel at each edge's
temperature inside the EM step, the step's Joule power, and a thermal step
with the EM dt. Large random fields (Joule heating of ~0.1 K over the test)
and a 0-1 K temperature spread (0.4 % conductivity spread in copper, far
above the field tolerances) make both the heating and the conductivity
feedback visible."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, field_rel_l2, hetero_problem, random_fields, read_eh, rel_l2

pytestmark = pytest.mark.gpu


def _seed(o, ctx, p, seed):
    E, H = random_fields(p, seed, e_scale=1e7, h_scale=2e4)
    for a in range(3):
        o.E[a][:] = E[a]
        o.H[a][:] = H[a]
        ctx.write(api.COSIM_F_EX + a, E[a])
        ctx.write(api.COSIM_F_HX + a, H[a])
    T = p.T_init + 1.0 * np.random.default_rng(seed + 1).random(p.n_nodes)
    o.T = T
    ctx.write(api.COSIM_F_T, T)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-11), (FP32, 2e-5)])
@pytest.mark.parametrize("case", [0, 1])
def test_coupled_steps_random_state(precision, tol, case, fused):
    bc, L = [((0,) * 6, 0), ((2, 2, 0, 2, 0, 2), 3)][case]
    p = hetero_problem(23, 14, 9, seed=30 + case, em_bc=bc, cpml=L)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    _seed(o, ctx, p, 40 + case)
    th0 = o.theta.copy()
    steps = 12
    o.coupled_steps(steps)
    ctx.em_steps(steps, coupled=True, fused=fused)
    Eg, Hg = read_eh(ctx)
    assert field_rel_l2(Eg, o.E)[0] < tol
    assert field_rel_l2(Hg, o.H)[0] < tol
    dT_g = ctx.read(api.COSIM_F_T) - p.T_init - th0
    dT_o = o.theta - th0
    assert np.abs(dT_o).max() > 1e-3  # the steps heated the conductors measurably
    # FP32 stores the rise T - T_init: the 1 K spread resolves the ~1e-3 K
    # heating to ~1e-4 of itself, rounding of the state included
    assert rel_l2(dT_g, dT_o) < (5e-10 if precision == FP64 else 1e-3)
    assert rel_l2(ctx.read(api.COSIM_F_P), o.P) < 10 * tol
    assert rel_l2(ctx.read(api.COSIM_F_Q), o.Q) < 10 * tol
    ctx.close()


def test_coupled_feedback_changes_the_fields():
    """The same start with alpha = 0 gives different fields: the coupled path
    really uses sigma(T) (and the oracle agrees on both)."""
    p = hetero_problem(17, 11, 7, seed=50, em_bc=(0,) * 6, cpml=0)
    o = oracle.OracleSim(p)
    ctx = context(p, FP64, o.dt)
    _seed(o, ctx, p, 51)
    ctx.em_steps(6, coupled=True)
    Ec, _ = read_eh(ctx)
    ctx2 = context(p, FP64, o.dt)
    _seed(oracle.OracleSim(p), ctx2, p, 51)
    ctx2.em_steps(6)
    Eu, _ = read_eh(ctx2)
    assert field_rel_l2(Ec, Eu)[0] > 1e-6
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("precision", [FP64, FP32])
def test_coupled_graph_replay_equals_plain(precision, fused):
    p = W.tiny_package()
    s = torch.cuda.Stream()
    a = api.Context(p, precision=precision, stream=s)
    b = api.Context(p, precision=precision, stream=s, dt_em=a.dt)
    tables = p.source_tables(a.dt, 200)
    for c in (a, b):
        c.set_sources(tables)
        c.write(api.COSIM_F_T, p.T_init + 30.0 * np.random.default_rng(3).random(p.n_nodes))
    a.em_steps(128, coupled=True, fused=fused)
    b.em_graph_capture(64, coupled=True, fused=fused)
    b.em_graph_launch(2)
    for f in (api.COSIM_F_EZ, api.COSIM_F_HX, api.COSIM_F_T, api.COSIM_F_P, api.COSIM_F_Q):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def test_tiny_package_coupled_burst_fp64():
    """The 32x32x16 package with its port and copper traces: 300 coupled steps."""
    p = W.tiny_package()
    o = oracle.OracleSim(p)
    ctx = context(p, FP64, o.dt)
    tables = p.source_tables(o.dt, 300)
    o.set_sources(tables)
    ctx.set_sources(tables)
    o.coupled_steps(300)
    ctx.em_steps(300, coupled=True)
    Eg, Hg = read_eh(ctx)
    assert field_rel_l2(Eg, o.E)[0] < 1e-10
    assert field_rel_l2(Hg, o.H)[0] < 1e-10
    # the rises are tiny (~1e-25 K): compare the stored rise itself (COSIM_F_DT)
    dT = ctx.read(api.COSIM_F_DT)
    assert np.abs(o.theta).max() > 0
    assert rel_l2(dT, o.theta) < 1e-10
    assert rel_l2(ctx.read(api.COSIM_F_Q), o.Q) < 1e-10
    ctx.close()
