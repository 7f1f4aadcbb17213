"""Closed-form pins of the oracle's heterogeneous thermal conductance (Sec.
II-A, Eq. 4: M_kk = V0a^T D_k V0a, one conductance k_e A*_e / l_e per edge) and
of its Gauss-point thermal load (Sec. II-B, Eq. 8 right-hand side).

Every expected value here is computed by hand from the continuum problem:

* parallel conduction: a bar along x whose cross-section holds several
  materials side by side, each running the bar's full length, with a
  temperature linear in x (slope a) and adiabatic walls. The linear profile
  is the exact steady state, so one explicit step leaves every interior node
  unchanged, and the heat that enters through an end face is a * sum_m k_m A_m
  (the materials conduct in parallel). A rule other than the area-weighted
  arithmetic mean of k over an edge's voxels (a harmonic or an unweighted
  mean) changes the end-face heat;
* series conduction: layers perpendicular to x with a piecewise-linear
  temperature that carries the same flux density q through every layer; the
  bar then conducts with the harmonic effective conductance
  A / sum_l (h_l / k_l), and an x-edge that takes its conductivity from any
  cell but the one it crosses breaks the steady state;
* thermal load: with a bilinear virtual displacement v_d = x_d x_e (d != e),
  which the trilinear element reproduces exactly, f . v equals
  sum_cells (3 lambda + 2 mu) alpha_L int x_e dT dV, and for a trilinear dT the
  integral is a sum of 1-D moments of the linear shape functions. A thermal
  strain taken at the element centroid, or from one node, misses it whenever
  dT varies along x_e.

Each pin is also run against copies of the oracle with the named mistake
planted (tests/oracle_mutants.py) and must fail there.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.fit_metric import Metric, coords
from tests.oracle_mutants import mutant


def _mat(k, rho_cp=2.0e6, E=1e9, nu=0.3, alpha=1e-6):
    return W.Material("m", 1.0, 1.0, 0.0, 0.0, 300.0, float(k), float(rho_cp), float(E), float(nu), float(alpha))


def _problem(nx, ny, nz, dx, dy, dz, mat, mats):
    return W.Problem(name="pin", nx=nx, ny=ny, nz=nz, dx=np.asarray(dx, float), dy=np.asarray(dy, float),
                     dz=np.asarray(dz, float), mat=np.ascontiguousarray(mat, np.uint8), materials=mats,
                     em_bc=(0,) * 6, cpml_cells=0, h_conv=(0.0,) * 6, T_amb=300.0, T_init=300.0)


# ---------------------------------------------------------------- conduction

def parallel_bar(seed=11):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 5, 4, 3
    ks = [0.3, 150.0, 400.0]
    mats = [_mat(k, rho_cp=float(rng.uniform(1.5e6, 3.5e6))) for k in ks]
    cross = rng.integers(0, 3, (nz, ny))
    cross[0, 0], cross[1, 1], cross[2, 2] = 0, 1, 2  # every material present
    mat = np.broadcast_to(cross[:, :, None], (nz, ny, nx))
    p = _problem(nx, ny, nz, rng.uniform(1e-6, 4e-6, nx), rng.uniform(1e-6, 4e-6, ny),
                 rng.uniform(1e-6, 4e-6, nz), mat, mats)
    # sum_m k_m A_m over the cross-section, by hand
    kA = sum(ks[cross[k, j]] * p.dy[j] * p.dz[k] for k in range(nz) for j in range(ny))
    return p, kA


def conduct_one_step(p, rise):
    """one explicit step from the temperature T_init + rise (no source);
    returns (change of each node, heat gained by each node per second,
    C_i dT_i / dt). The change is taken on the stored rise over T_init, so
    it keeps FP64 resolution on small changes."""
    o = oracle.OracleSim(p)
    o.theta = np.ascontiguousarray(rise, np.float64)
    dt = o.thermal_steps(1, source=False, safety=0.5)
    dT = o.theta - rise
    C = Metric(p).node_capacity()
    return dT, C * dT / dt


def parallel_errors(seed=11):
    """(interior change / end-face change, relative error of the end-face heat)"""
    p, kA = parallel_bar(seed)
    a = 2.0e6  # K/m
    x = coords(p.dx)
    rise = np.broadcast_to(a * x, (p.nz + 1, p.ny + 1, p.nx + 1)).reshape(-1)
    dT, gain = conduct_one_step(p, rise)
    dT = dT.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    gain = gain.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    interior = np.max(np.abs(dT[:, :, 1:-1])) / np.max(np.abs(dT[:, :, 0]))
    g0 = gain[:, :, 0].sum()     # the x = 0 face gains heat (T rises with x)
    g1 = -gain[:, :, -1].sum()   # the x = L face loses the same heat
    return interior, max(abs(g0 / (a * kA) - 1), abs(g1 / (a * kA) - 1))


def series_stack(seed=12):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 6, 3, 2
    ks = [0.3, 150.0, 400.0]
    mats = [_mat(k, rho_cp=float(rng.uniform(1.5e6, 3.5e6))) for k in ks]
    layers = np.array([0, 2, 1, 0, 1, 2])
    mat = np.broadcast_to(layers[None, None, :], (nz, ny, nx))
    p = _problem(nx, ny, nz, rng.uniform(1e-6, 4e-6, nx), rng.uniform(1e-6, 4e-6, ny),
                 rng.uniform(1e-6, 4e-6, nz), mat, mats)
    return p, np.array([ks[m] for m in layers])


def series_errors(seed=12):
    """(interior change / end-face change, relative error of the end-face heat
    against the harmonic effective conductance)"""
    p, k = series_stack(seed)
    q = 5.0e6  # W/m^2 toward -x
    drop = q * p.dx / k                         # per layer
    Tx = np.concatenate([[0.0], np.cumsum(drop)])  # rise over T_init
    dT, gain = conduct_one_step(p, np.broadcast_to(Tx, (p.nz + 1, p.ny + 1, p.nx + 1)).reshape(-1))
    dT = dT.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    gain = gain.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    interior = np.max(np.abs(dT[:, :, 1:-1])) / np.max(np.abs(dT[:, :, 0]))
    A = p.dy.sum() * p.dz.sum()
    G_eff = A / np.sum(p.dx / k)                # harmonic: layers in series
    expect = G_eff * (Tx[-1] - Tx[0])
    g0 = gain[:, :, 0].sum()
    g1 = -gain[:, :, -1].sum()
    return interior, max(abs(g0 / expect - 1), abs(g1 / expect - 1))


def test_parallel_materials_conduct_area_weighted():
    interior, face = parallel_errors()
    assert interior < 1e-11
    assert face < 1e-12


def test_series_layers_conduct_harmonic():
    interior, face = series_errors()
    assert interior < 1e-11
    # the x = L face changes by ~1e-6 of its stored rise in one step, so the
    # rounding of that rise (~1e-16 relative) shows at ~1e-12 here
    assert face < 1e-11


@pytest.mark.parametrize("name", ["harmonic_conductance", "unweighted_conductance"])
def test_parallel_pin_catches_wrong_averaging(name):
    with mutant(name):
        interior, face = parallel_errors()
    assert face > 1e-3


def test_series_pin_catches_wrong_edge_cell():
    with mutant("edge_cell_off_by_one"):
        interior, face = series_errors()
    assert interior > 1e-3 or face > 1e-3


# ---------------------------------------------------------------- thermal load

def load_problem(seed=21):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 3, 2, 2
    mats = [_mat(1.0, E=float(rng.uniform(5e9, 130e9)), nu=float(rng.uniform(0.2, 0.4)),
                 alpha=float(rng.uniform(2e-6, 50e-6))) for _ in range(3)]
    mat = rng.integers(0, 3, (nz, ny, nx))
    return _problem(nx, ny, nz, rng.uniform(1e-6, 4e-6, nx), rng.uniform(1e-6, 4e-6, ny),
                    rng.uniform(1e-6, 4e-6, nz), mat, mats)


def moment_integral(p, rise, e):
    """sum over cells of (3 lambda + 2 mu) alpha_L * int x_e dT dV, with dT the
    trilinear interpolant of the nodal rises, written out by hand:
    int N_a x_e dV = prod_{b != e} h_b / 2 * (x0_e h_e / 2 + h_e^2 (1/3 if a_e
    is the upper node else 1/6)); 3 lambda + 2 mu = E / (1 - 2 nu)."""
    h = [np.asarray(p.dx), np.asarray(p.dy), np.asarray(p.dz)]
    x0 = [coords(h[0]), coords(h[1]), coords(h[2])]
    r = rise.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    total = 0.0
    for k in range(p.nz):
        for j in range(p.ny):
            for i in range(p.nx):
                m = p.materials[int(p.mat[k, j, i])]
                beta = m.E / (1 - 2 * m.nu) * m.alpha_L
                c = (i, j, k)
                s = 0.0
                for az in (0, 1):
                    for ay in (0, 1):
                        for ax in (0, 1):
                            av = (ax, ay, az)
                            w = 1.0
                            for b in range(3):
                                hb = h[b][c[b]]
                                if b == e:
                                    w *= x0[b][c[b]] * hb / 2 + hb * hb * (1 / 3 if av[b] else 1 / 6)
                                else:
                                    w *= hb / 2
                            s += w * r[k + az, j + ay, i + ax]
                total += beta * s
    return total


def load_errors(seed=21):
    """max over (d, e), d != e, of |f . v - expected| / |expected| for v_d = x_d x_e"""
    p = load_problem(seed)
    o = oracle.OracleSim(p)
    rng = np.random.default_rng(seed + 1)
    rise = 40.0 * rng.standard_normal(o.g.n_nodes)
    free = np.zeros(3 * o.g.n_nodes, np.uint8)
    f = o.thermal_load(free, 300.0, 300.0 + rise).reshape(-1, 3)
    X = [np.broadcast_to(c, (p.nz + 1, p.ny + 1, p.nx + 1)).reshape(-1)
         for c in (coords(p.dx)[None, None, :], coords(p.dy)[None, :, None], coords(p.dz)[:, None, None])]
    worst = 0.0
    for d in range(3):
        for e in range(3):
            if d == e:
                continue
            fv = float(f[:, d] @ (X[d] * X[e]))
            ref = moment_integral(p, rise, e)
            worst = max(worst, abs(fv / ref - 1))
    return worst


def test_thermal_load_bilinear_virtual_work():
    assert load_errors() < 1e-12


@pytest.mark.parametrize("name", ["centroid_rise", "nodal_lump_rise"])
def test_thermal_load_pin_catches_wrong_interpolation(name):
    with mutant(name):
        err = load_errors()
    assert err > 1e-3
