"""CUDA thermal step, Joule hand-off, HEX8 matvec and stress solve vs the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import (FP32, FP64, context, hetero_problem, interleaved_to_soa, oracle_mask_from_bits,
                               rel_l2, soa_to_interleaved)
from workloads import constraints as BC

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-12), (FP32, 1e-6)])
def test_thermal_steps_random_state(precision, tol):
    p = hetero_problem(37, 11, 9, seed=4, em_bc=(0,) * 6, cpml=0)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    rng = np.random.default_rng(2)
    T0 = 300 + 20 * rng.random(p.n_nodes)
    Pn = 1e-4 * rng.random(p.n_nodes)
    o.T, o.P = T0.copy(), Pn.copy()
    ctx.write(api.COSIM_F_T, T0)
    ctx.write(api.COSIM_F_P, Pn)
    lim_g = ctx.query(api.COSIM_Q_DT_TH_LIMIT)
    assert abs(lim_g / o.thermal_dt_limit() - 1) < (1e-13 if precision == FP64 else 1e-6)
    dt = 0.9 * o.thermal_dt_limit()
    o.thermal_steps(30, dt=dt)
    ctx.thermal_steps(30, dt)
    assert rel_l2(ctx.read(api.COSIM_F_T) - 300, o.T - 300) < tol * 100
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-12), (FP32, 2e-6)])
def test_joule_finalize_power_and_energy(precision, tol):
    p = hetero_problem(20, 9, 7, seed=5, em_bc=(0,) * 6, cpml=0)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    Q = 1e-9 * np.random.default_rng(3).random(p.n_nodes)
    ctx.write(api.COSIM_F_Q, Q)
    o.Q = Q.copy()
    o.n_acc = 0
    ctx.joule(api.COSIM_JOULE_RESET)
    assert np.all(ctx.read(api.COSIM_F_Q) == 0)
    ctx.write(api.COSIM_F_Q, Q)
    # the accumulated step count sets the averaging window: run 0 EM steps -> use energy mode
    tot = ctx.joule(api.COSIM_JOULE_FINALIZE_ENERGY)
    assert abs(tot / Q.sum() - 1) < 1e-13
    o.joule_finalize_energy()
    assert rel_l2(ctx.read(api.COSIM_F_T) - 300, o.T - 300) < tol
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-12), (FP32, 3e-6)])
@pytest.mark.parametrize("shape", [(37, 11, 9), (31, 7, 3), (5, 40, 2)])
def test_hex8_matvec_random(precision, tol, shape):
    nx, ny, nz = shape
    p = hetero_problem(nx, ny, nz, seed=sum(shape), em_bc=(0,) * 6, cpml=0)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    rng = np.random.default_rng(7)
    bits = (rng.random(p.n_nodes) < 0.15).astype(np.uint8) * rng.integers(1, 8, p.n_nodes).astype(np.uint8)
    u = rng.standard_normal((3, p.n_nodes)) * 1e-7
    dt = np.float64 if precision == FP64 else np.float32
    y = ctx.stress_apply(u.astype(dt), bc=api.COSIM_MECH_MASK, node_mask=bits)
    yo = interleaved_to_soa(o.matvec(oracle_mask_from_bits(bits), soa_to_interleaved(u)))
    assert rel_l2(y, yo) < tol
    ctx.close()


def _thermal_load_problem(precision, bc):
    p = hetero_problem(23, 13, 8, seed=11, em_bc=(0,) * 6, cpml=0, uniform_x=True)
    o = oracle.OracleSim(p)
    ctx = context(p, precision, o.dt)
    rng = np.random.default_rng(5)
    T = 300 + 40 * rng.random(p.n_nodes)
    o.T = T.copy()
    ctx.write(api.COSIM_F_T, T)
    if bc == api.COSIM_MECH_CLAMPED_BOTTOM:
        fixed = BC.clamped_bottom(p)
    else:
        fixed = BC.kinematic_mount(p)
    return p, o, ctx, fixed


@pytest.mark.parametrize("bc", [api.COSIM_MECH_CLAMPED_BOTTOM, api.COSIM_MECH_KINEMATIC_MOUNT])
def test_stress_solve_fp64(bc):
    """GPU Jacobi-PCG to 1e-12 vs the oracle's to 1e-13: displacement, thermal
    load and von Mises within 1e-8; with the default 1e-9 residual, 1e-6."""
    p, o, ctx, fixed = _thermal_load_problem(FP64, bc)
    ref = o.stress_solve(fixed, 300.0, rtol=1e-13)
    for rtol, tol in [(1e-12, 1e-8), (1e-9, 1e-6)]:
        rep = ctx.stress_solve(bc=bc, T_ref=300.0, rtol=rtol, check_every=8)
        assert rep["relres"] <= rtol
        f = np.stack([ctx.read(api.COSIM_F_FX + c) for c in range(3)])
        assert rel_l2(f, interleaved_to_soa(ref["f"])) < 1e-12
        u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)])
        assert rel_l2(u, interleaved_to_soa(ref["u"])) < tol
        assert rel_l2(ctx.read(api.COSIM_F_VM), ref["vm"]) < tol
        assert rel_l2(ctx.read(api.COSIM_F_UMAG), ref["umag"]) < tol
    ctx.close()


def test_stress_solve_fp32_converges():
    """FP32 vectors, FP64 dots: the recursively updated residual reaches 1e-6
    and the displacement is within 1e-4 of the FP64 oracle solution."""
    p, o, ctx, fixed = _thermal_load_problem(FP32, api.COSIM_MECH_CLAMPED_BOTTOM)
    ref = o.stress_solve(fixed, 300.0, rtol=1e-13)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-6, check_every=8)
    assert rep["relres"] <= 1e-6
    u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)])
    assert rel_l2(u, interleaved_to_soa(ref["u"])) < 1e-4
    ctx.close()


@pytest.mark.parametrize("bc", [api.COSIM_MECH_CLAMPED_BOTTOM, api.COSIM_MECH_KINEMATIC_MOUNT])
def test_stress_solve_fp32_in_fp64_refinement(bc):
    """FP32 vectors and matvecs inside FP64 iterative refinement: the true FP64
    residual reaches 1e-9 and displacement / von Mises match the oracle to 1e-6."""
    p, o, ctx, fixed = _thermal_load_problem(FP32, bc)
    ref = o.stress_solve(fixed, 300.0, rtol=1e-13)
    rep = ctx.stress_solve(bc=bc, T_ref=300.0, rtol=1e-9, refine=True, inner_rtol=1e-4, check_every=8)
    assert rep["relres"] <= 1e-9 and rep["refine_steps"] >= 2
    u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)])
    assert rel_l2(u, interleaved_to_soa(ref["u"])) < 1e-6
    assert rel_l2(ctx.read(api.COSIM_F_VM), ref["vm"]) < 1e-6
    ctx.close()


def test_stress_not_converged_status():
    p, o, ctx, fixed = _thermal_load_problem(FP64, api.COSIM_MECH_CLAMPED_BOTTOM)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-12, maxit=3, check_every=1,
                           allow_not_converged=True)
    assert rep["status"] == api.COSIM_ERR_NOT_CONVERGED and rep["iters"] == 3
    ctx.close()


@pytest.mark.parametrize("dT_scale", [1e-9, 1e-12])
def test_stress_solve_fp32_tiny_loads(dT_scale):
    """A temperature rise of nano- or pico-kelvins (a short EM burst) gives
    loads of 1e-14 N and displacements of 1e-19 m on this grid: near the
    tolerance the FP32 products r D^-1 r and p K p fall below FP32's normal
    range. The solver's power-of-two right-hand-side scaling keeps the
    iteration in range, so the FP32 solve still converges to the FP64
    oracle's displacement."""
    p = hetero_problem(23, 13, 8, seed=11, em_bc=(0,) * 6, cpml=0, uniform_x=True)
    o = oracle.OracleSim(p)
    ctx = context(p, FP32, o.dt)
    rng = np.random.default_rng(5)
    T = 300 + dT_scale * rng.random(p.n_nodes)
    o.T = T.copy()
    ctx.write(api.COSIM_F_T, T)
    fixed = BC.clamped_bottom(p)
    ref = o.stress_solve(fixed, 300.0, rtol=1e-13)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-6, check_every=8)
    assert rep["relres"] <= 1e-6
    u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)])
    assert np.all(np.isfinite(u))
    # (the device holds the rise over the initial temperature, so a nano-kelvin
    # rise is represented to FP32 relative precision)
    assert rel_l2(u, interleaved_to_soa(ref["u"])) < 1e-4
    ctx.close()


def test_async_reads_match_sync_reads():
    """cosim_read_fields_async: the copy holds the field as of the call (a
    later write does not reach it), overlaps a stress solve, and a second
    asynchronous read reuses the staging buffer after the first has landed."""
    import torch
    p, o, ctx, fixed = _thermal_load_problem(FP32, api.COSIM_MECH_CLAMPED_BOTTOM)
    T_ref = ctx.read(api.COSIM_F_T)
    T_host = torch.empty(p.n_nodes, dtype=torch.float32).pin_memory().numpy()
    T_dev = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    api.cosim_read_fields_async(ctx.h, api.COSIM_F_T, T_host)
    api.cosim_read_fields_async(ctx.h, api.COSIM_F_T, T_dev)
    ctx.write(api.COSIM_F_T, np.full(p.n_nodes, 400.0))  # after the reads were enqueued
    ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-6, check_every=8)
    VM_host = torch.empty(p.n_cells, dtype=torch.float32).pin_memory().numpy()
    api.cosim_read_fields_async(ctx.h, api.COSIM_F_VM, VM_host)
    api.cosim_wait_reads(ctx.h)
    api.cosim_wait_reads(ctx.h)  # nothing pending: returns at once
    assert np.array_equal(T_host, T_ref.astype(np.float32))
    assert np.array_equal(T_dev.cpu().numpy(), T_ref)
    assert np.array_equal(VM_host, ctx.read(api.COSIM_F_VM).astype(np.float32))
    assert np.all(ctx.read(api.COSIM_F_T) == 400.0)
    with pytest.raises(api.CosimError):
        api.cosim_read_fields_async(ctx.h, api.COSIM_F_T, np.empty(3, np.float32))
    ctx.close()
