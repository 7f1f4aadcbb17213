"""Pins of the oracle's two-way electro-thermal coupling (Sec. II-A): the
synchronized step with sigma(T) = sigma0 / (1 + alpha (T - T0)).

- alpha = 0 everywhere: the coupled step is exactly the uncoupled H, E, Joule
  and thermal routines run in sequence (no new arithmetic sneaks in);
- a uniformly heated conductor under a uniform field dissipates
  P = E^2 Vol / rho(T) with the linear resistivity law
  rho(T) = rho0 (1 + alpha (T - T0)) (closed form, any cell sizes);
- adiabatic heat balance: sum_i C_i (T_i' - T_i) = dt sum_i P_i, because the
  conduction terms cancel pairwise;
- temperature feedback is local: only the heated half's conductivity drops."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W


def _box(nx, ny, nz, seed, mats, mat=None, h_conv=(0.0,) * 6, T_init=300.0):
    rng = np.random.default_rng(seed)
    if mat is None:
        mat = rng.integers(0, len(mats), (nz, ny, nx)).astype(np.uint8)
    return W.Problem(name="box", nx=nx, ny=ny, nz=nz, dx=rng.uniform(3e-6, 8e-6, nx),
                     dy=rng.uniform(3e-6, 8e-6, ny), dz=rng.uniform(1e-6, 4e-6, nz), mat=mat, materials=mats,
                     em_bc=(0,) * 6, cpml_cells=0, h_conv=h_conv, T_amb=T_init, T_init=T_init)


def _random_state(o, seed, dtheta=40.0):
    rng = np.random.default_rng(seed)
    n = o.g.n_nodes
    for a in range(3):
        o.E[a][:] = rng.standard_normal(n) * 1e3
        o.H[a][:] = rng.standard_normal(n) * 3.0
    o.theta = dtheta * rng.random(n)


def test_alpha_zero_coupled_step_equals_the_uncoupled_routines():
    mats = [dataclasses.replace(m, tcr=0.0) for m in (W.DIELECTRIC, W.COPPER, W.SILICON, W.UNDERFILL)]
    p = _box(9, 8, 7, 1, mats, h_conv=(0.0, 2e4, 0.0, 0.0, 0.0, 1e4))
    a, b = oracle.OracleSim(p), oracle.OracleSim(p)
    _random_state(a, 2)
    _random_state(b, 2)
    a.coupled_steps(1)
    b.h_half_step()
    Eold = [e.copy() for e in b.E]
    b.e_step(accumulate_joule=False)
    b.P = b.joule_of(Eold, b.E) / b.dt  # energy of the step -> power
    b.thermal_steps(1, dt=b.dt)
    for q in range(3):
        assert np.array_equal(a.E[q], b.E[q]) and np.array_equal(a.H[q], b.H[q])
    assert np.allclose(a.P, b.P, rtol=1e-14, atol=0)
    assert np.abs(a.theta - b.theta).max() <= 1e-12 * np.abs(b.theta).max()


@pytest.mark.parametrize("T_init,dT", [(300.0, 0.0), (300.0, 75.0), (320.0, 35.0), (350.0, -40.0)])
def test_uniformly_heated_conductor_follows_linear_resistivity(T_init, dT):
    mat = np.full((5, 6, 7), 0, np.uint8)
    p = _box(7, 6, 5, 3, [W.COPPER], mat=mat, T_init=T_init)
    o = oracle.OracleSim(p)
    E0 = 250.0  # uniform field along x [V/m], unchanged over the step
    Ex = np.zeros(o.g.n_nodes)
    i, j, k = np.meshgrid(np.arange(p.nx + 1), np.arange(p.ny + 1), np.arange(p.nz + 1), indexing="ij")
    Ex[o.g.nid(i[i < p.nx], j[i < p.nx], k[i < p.nx])] = E0
    Eb = [Ex, np.zeros_like(Ex), np.zeros_like(Ex)]
    P = o.joule_power_T(Eb, Eb, theta=np.full(o.g.n_nodes, dT))
    vol = p.dx.sum() * p.dy.sum() * p.dz.sum()
    rho0 = 1.0 / W.COPPER.sigma0
    rho_T = rho0 * (1.0 + W.COPPER.tcr * (T_init + dT - W.COPPER.T0))
    assert P.sum() == pytest.approx(E0 ** 2 * vol / rho_T, rel=1e-13)


def test_coupled_step_heat_balance_is_exact():
    p = _box(8, 7, 6, 5, [W.DIELECTRIC, W.COPPER, W.SILICON, W.UNDERFILL])
    o = oracle.OracleSim(p)
    _random_state(o, 6, dtheta=80.0)
    C = o.capacity()
    th0 = o.theta.copy()
    o.coupled_steps(1)
    assert o.P.sum() > 0
    gained = np.sum(C * (o.theta - th0))
    assert gained == pytest.approx(o.dt * o.P.sum(), rel=1e-10)


def test_feedback_is_local_to_the_heated_region():
    mat = np.full((4, 5, 10), 1, np.uint8)  # copper everywhere (material 1)
    p = _box(10, 5, 4, 7, [W.DIELECTRIC, W.COPPER], mat=mat)
    o = oracle.OracleSim(p)
    rng = np.random.default_rng(8)
    Eb = [rng.standard_normal(o.g.n_nodes) * 1e2 for _ in range(3)]
    cold = o.joule_power_T(Eb, Eb, theta=np.zeros(o.g.n_nodes))
    th = np.zeros(o.g.n_nodes)
    i = np.arange(o.g.n_nodes) % (p.nx + 1)
    th[i >= 6] = 100.0  # the x >= 6 part is 100 K hotter
    hot = o.joule_power_T(Eb, Eb, theta=th)
    assert np.array_equal(hot[i <= 4], cold[i <= 4])  # nodes whose edges all stay cold
    ratio = 1.0 / (1.0 + W.COPPER.tcr * 100.0)
    deep = i >= 7  # all incident edges hot
    assert np.allclose(hot[deep], ratio * cold[deep], rtol=1e-13, atol=0)


def test_edge_temperature_is_the_mean_of_its_end_nodes():
    """Only the x-edges from i = 5 to i = 6 carry field; i >= 6 is 100 K hotter,
    so those edges sit at the mean, 50 K above the cold side."""
    mat = np.full((4, 5, 10), 1, np.uint8)
    p = _box(10, 5, 4, 9, [W.DIELECTRIC, W.COPPER], mat=mat)
    o = oracle.OracleSim(p)
    i = np.arange(o.g.n_nodes) % (p.nx + 1)
    Ex = np.where(i == 5, 300.0, 0.0)
    Eb = [Ex, np.zeros_like(Ex), np.zeros_like(Ex)]
    th = np.where(i >= 6, 100.0, 0.0)
    cold = o.joule_power_T(Eb, Eb, theta=np.zeros(o.g.n_nodes))
    hot = o.joule_power_T(Eb, Eb, theta=th)
    ends = (i == 5) | (i == 6)
    assert np.all(cold[ends] > 0) and np.all(cold[~ends] == 0)
    assert np.allclose(hot[ends], cold[ends] / (1.0 + W.COPPER.tcr * 50.0), rtol=1e-14, atol=0)
