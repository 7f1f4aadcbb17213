"""Pins of the oracle's thermal step (Sec. II-A, Eqs. 4-5)."""
import math

import numpy as np
from scipy.special import erfc

import oracle
import workloads as W
from tests.fit_metric import Metric


def hetero(seed, nx=6, ny=5, nz=4, h_conv=(0.0,) * 6):
    rng = np.random.default_rng(seed)
    mats = [W.Material(f"m{q}", 1, 1, 0, 0, 300, float(rng.uniform(0.2, 400)),
                       float(rng.uniform(1e6, 4e6)), 1e9, 0.3, 1e-6) for q in range(3)]
    return W.Problem(name="th", nx=nx, ny=ny, nz=nz, dx=rng.uniform(1e-6, 4e-6, nx),
                     dy=rng.uniform(1e-6, 4e-6, ny), dz=rng.uniform(1e-6, 4e-6, nz),
                     mat=rng.integers(0, 3, (nz, ny, nx)).astype(np.uint8), materials=mats,
                     em_bc=(0,) * 6, cpml_cells=0, h_conv=h_conv, T_amb=300.0, T_init=300.0)


def test_uniform_temperature_is_stationary():
    p = hetero(1)
    o = oracle.OracleSim(p)
    o.T = np.full(o.g.n_nodes, 412.5)
    o.thermal_steps(20, source=False)
    assert np.all(o.T == 412.5)


def test_heat_balance_adiabatic_with_source():
    """sum_i C_i T_i grows by exactly dt * sum_i P_i per step (adiabatic walls,
    conservative edge fluxes), with C_i the node's dual-volume heat capacity."""
    p = hetero(2)
    o = oracle.OracleSim(p)
    rng = np.random.default_rng(3)
    o.T = 300 + 50 * rng.random(o.g.n_nodes)
    o.P = 1e-3 * rng.random(o.g.n_nodes)
    C = Metric(p).node_capacity()
    e0 = (C * o.T).sum()
    dt = o.thermal_steps(7)
    e1 = (C * o.T).sum()
    assert abs((e1 - e0) - 7 * dt * o.P.sum()) < 1e-11 * e0


def test_convective_face_loss():
    """Uniform T, film coefficient on the top face only: the heat lost in one
    step is dt * h * (whole top area) * (T - T_amb)."""
    p = hetero(4, h_conv=(0, 0, 0, 0, 0, 2.5e4))
    o = oracle.OracleSim(p)
    o.T = np.full(o.g.n_nodes, 350.0)
    C = Metric(p).node_capacity()
    dt = o.thermal_steps(1, source=False)
    lost = (C * (50.0 - o.theta)).sum()  # the oracle's state is the rise over T_init = 300 K
    area = p.dx.sum() * p.dy.sum()
    assert abs(lost / (dt * 2.5e4 * area * 50.0) - 1) < 1e-12


def test_dt_limit_matches_textbook_ftcs():
    """uniform adiabatic grid: min C/sum G = rho c / (2 k (1/dx^2 + 1/dy^2 + 1/dz^2))"""
    p = W.uniform_box(5, 4, 3, h=(2e-6, 3e-6, 1.5e-6), material=W.COPPER)
    o = oracle.OracleSim(p)
    ref = W.COPPER.rho_cp / (2 * W.COPPER.k * (1 / 4e-12 + 1 / 9e-12 + 1 / 2.25e-12))
    assert abs(o.thermal_dt_limit() / ref - 1) < 1e-13


def _erfc_error(nx):
    """1-D bar (one cell in y and z), step initial condition at the middle;
    max error against T_lo + (T_hi - T_lo)/2 erfc((x - x_m)/(2 sqrt(kappa t)))
    at a fixed time before the diffusion front reaches the ends."""
    Lb = 1e-3
    h = Lb / nx
    p = W.uniform_box(nx, 1, 1, h=(h, 1e-2, 1e-2), material=W.COPPER)
    o = oracle.OracleSim(p)
    x = np.arange(nx + 1) * h
    xm = Lb / 2
    T0 = np.where(x < xm, 400.0, 300.0)
    T0[np.isclose(x, xm)] = 350.0
    o.T = np.tile(T0, 4).astype(np.float64)
    kappa = W.COPPER.k / W.COPPER.rho_cp
    t_end = 2.5e-9 / kappa
    nsteps = int(math.ceil(t_end / (0.45 * o.thermal_dt_limit())))
    dt = t_end / nsteps
    o.thermal_steps(nsteps, dt=dt, source=False)
    exact = 300.0 + 50.0 * erfc((x - xm) / (2 * math.sqrt(kappa * t_end)))
    return np.max(np.abs(o.T.reshape(2, 2, nx + 1)[0, 0] - exact))


def test_erfc_second_order_convergence():
    e1, e2 = _erfc_error(100), _erfc_error(200)
    assert e1 < 0.5
    assert 3.0 < e1 / e2 < 5.0
