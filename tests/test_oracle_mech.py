"""Pins of the oracle's thermoelastic HEX8 solve (Sec. II-B, Eqs. 7-9)."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import constraints as BC
from tests.fit_metric import coords

CU = W.COPPER


def tensor_element(hx, hy, hz, lam, mu):
    """K_e of a brick from exact 1-D integrals of linear shape functions:
    int dN_a/dx_p dN_b/dx_q dV factors into 1-D mass (h/6 [2 1; 1 2]),
    stiffness (1/h [1 -1; -1 1]) and first-moment ([-1/2 -1/2; 1/2 1/2])
    matrices; K_{ai,bj} = lam I_ij + mu (delta_ij sum_d I_dd + I_ji)."""
    hs = (hx, hy, hz)
    M = [h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]]) for h in hs]
    S = [1 / h * np.array([[1.0, -1.0], [-1.0, 1.0]]) for h in hs]
    D = np.array([[-0.5, -0.5], [0.5, 0.5]])

    def I(p, q):
        F = []
        for d in range(3):
            if p == q == d:
                F.append(S[d])
            elif d == p:
                F.append(D)
            elif d == q:
                F.append(D.T)
            else:
                F.append(M[d])
        return np.kron(F[2], np.kron(F[1], F[0]))  # node a = ax + 2 ay + 4 az

    K = np.zeros((24, 24))
    lap = I(0, 0) + I(1, 1) + I(2, 2)
    for i in range(3):
        for j in range(3):
            blk = lam * I(i, j) + mu * I(j, i) + (mu * lap if i == j else 0)
            K[i::3, j::3] = blk
    return K


def test_element_gauss_equals_exact_tensor_product():
    for hh in [(1.0, 1.0, 1.0), (2e-6, 3e-6, 0.7e-6)]:
        Kl, Km = oracle.hex8_element(*hh)
        for lam, mu in [(1.0, 0.0), (0.0, 1.0), (7.3e10, 4.1e10)]:
            ref = tensor_element(*hh, lam, mu)
            got = lam * Kl + mu * Km
            assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_element_cube_diagonal_and_rank():
    """unit cube: K_aa(x,x) = (lam + 4 mu)/9; six rigid modes span the null space"""
    Kl, Km = oracle.hex8_element(1.0, 1.0, 1.0)
    lam, mu = 2.0, 3.0
    K = lam * Kl + mu * Km
    assert np.allclose(np.diag(K), (lam + 4 * mu) / 9, rtol=1e-14)
    w = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == 6 and w.min() > -1e-10 * w.max()


def hetero(seed, nx=5, ny=4, nz=3, nmat=3):
    rng = np.random.default_rng(seed)
    mats = [W.Material(f"m{q}", 1, 1, 0, 0, 300, 1, 1e6, float(rng.uniform(5e9, 130e9)),
                       float(rng.uniform(0.2, 0.4)), float(rng.uniform(2e-6, 50e-6)))
            for q in range(nmat)]
    return W.Problem(name="mech", nx=nx, ny=ny, nz=nz, dx=rng.uniform(1e-6, 4e-6, nx),
                     dy=rng.uniform(1e-6, 4e-6, ny), dz=rng.uniform(1e-6, 4e-6, nz),
                     mat=rng.integers(0, nmat, (nz, ny, nx)).astype(np.uint8), materials=mats,
                     em_bc=(0,) * 6, cpml_cells=0)


def node_xyz(p):
    x, y, z = coords(p.dx), coords(p.dy), coords(p.dz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def test_rigid_modes_in_null_space():
    p = hetero(1)
    o = oracle.OracleSim(p)
    free = np.zeros(3 * o.g.n_nodes, np.uint8)
    X, Y, Z = node_xyz(p)
    one, zero = np.ones_like(X), np.zeros_like(X)
    modes = [(one, zero, zero), (zero, one, zero), (zero, zero, one),
             (-Y, X, zero), (zero, -Z, Y), (Z, zero, -X)]
    Kdiag = o.diag(free).max()
    for mx, my, mz in modes:
        u = np.stack([mx, my, mz], 1).reshape(-1)
        y = o.matvec(free, u)
        assert np.max(np.abs(y)) < 1e-12 * Kdiag * np.max(np.abs(u))


def test_patch_linear_field_interior_equilibrium():
    p = hetero(2, nmat=1)
    o = oracle.OracleSim(p)
    free = np.zeros(3 * o.g.n_nodes, np.uint8)
    X, Y, Z = node_xyz(p)
    A = np.random.default_rng(0).standard_normal((3, 3))
    u = (A @ np.stack([X, Y, Z])).T.reshape(-1)
    y = o.matvec(free, u).reshape(p.nz + 1, p.ny + 1, p.nx + 1, 3)
    inner = y[1:-1, 1:-1, 1:-1]
    assert np.max(np.abs(inner)) < 1e-12 * o.diag(free).max() * np.max(np.abs(u))
    assert np.max(np.abs(y)) > 1e-3 * o.diag(free).max() * np.max(np.abs(u))


def test_constrained_operator_symmetric_identity_rows():
    p = hetero(3)
    o = oracle.OracleSim(p)
    rng = np.random.default_rng(1)
    fixed = (rng.random(3 * o.g.n_nodes) < 0.2).astype(np.uint8)
    u, v = rng.standard_normal((2, 3 * o.g.n_nodes))
    Ku, Kv = o.matvec(fixed, u), o.matvec(fixed, v)
    assert abs(u @ Kv - v @ Ku) < 1e-12 * abs(u @ Kv)
    assert np.array_equal(Ku[fixed == 1], u[fixed == 1])


def test_free_bar_uniform_heating_zero_stress():
    """Kinematic mount (Sec. III-B), uniform dT: u = alpha dT (x - x_c), sigma = 0."""
    rng = np.random.default_rng(5)
    nx, ny, nz = 6, 4, 3
    p = W.uniform_box(nx, ny, nz, material=CU)
    p.dx[:] = rng.uniform(1e-6, 3e-6, nx)
    p.dy[:] = rng.uniform(1e-6, 3e-6, ny)
    p.dz[:] = rng.uniform(1e-6, 3e-6, nz)
    o = oracle.OracleSim(p)
    fixed = BC.kinematic_mount(p)
    dT = 25.0
    T = np.full(o.g.n_nodes, 300.0 + dT)
    f = o.thermal_load(fixed, 300.0, T)
    u, it, rr = o.pcg(fixed, f, rtol=1e-14)
    X, Y, Z = node_xyz(p)
    xc = coords(p.dx)[nx // 2]
    yc = coords(p.dy)[ny // 2]
    ue = (CU.alpha_L * dT * np.stack([X - xc, Y - yc, Z])).T.reshape(-1)
    assert np.max(np.abs(u - ue)) < 1e-9 * np.max(np.abs(ue))
    vm, um = o.von_mises(u, 300.0, T)
    assert np.max(vm) < 1e-6 * CU.E * CU.alpha_L * dT
    assert np.allclose(um, np.linalg.norm(ue.reshape(-1, 3), axis=1), rtol=0, atol=1e-9 * np.max(np.abs(ue)))


def test_roller_bar_uniaxial_stress():
    """u_x = 0 on both x-end faces, laterally free: sigma_xx = -E alpha dT,
    sigma_VM = E alpha dT in every element; u_y = (1+nu) alpha dT y."""
    rng = np.random.default_rng(6)
    nx, ny, nz = 5, 4, 3
    p = W.uniform_box(nx, ny, nz, material=CU)
    p.dx[:] = rng.uniform(1e-6, 3e-6, nx)
    p.dy[:] = rng.uniform(1e-6, 3e-6, ny)
    p.dz[:] = rng.uniform(1e-6, 3e-6, nz)
    o = oracle.OracleSim(p)
    fixed = np.zeros((nz + 1, ny + 1, nx + 1, 3), np.uint8)
    fixed[:, :, 0, 0] = fixed[:, :, nx, 0] = 1
    fixed[0, 0, 0, 1] = fixed[0, 0, 0, 2] = 1
    fixed[0, ny, 0, 2] = 1
    fixed = fixed.reshape(-1)
    dT = -40.0
    T = np.full(o.g.n_nodes, 300.0 + dT)
    f = o.thermal_load(fixed, 300.0, T)
    u, it, rr = o.pcg(fixed, f, rtol=1e-14)
    X, Y, Z = node_xyz(p)
    s = (1 + CU.nu) * CU.alpha_L * dT
    ue = np.stack([0 * X, s * Y, s * Z]).T.reshape(-1)
    assert np.max(np.abs(u - ue)) < 1e-9 * np.max(np.abs(ue))
    vm, _ = o.von_mises(u, 300.0, T)
    assert np.allclose(vm, CU.E * CU.alpha_L * abs(dT), rtol=1e-8)


def test_pcg_residual_heterogeneous():
    p = hetero(7, 6, 5, 4)
    o = oracle.OracleSim(p)
    fixed = BC.clamped_bottom(p)
    T = 300 + 30 * np.random.default_rng(2).random(o.g.n_nodes)
    f = o.thermal_load(fixed, 300.0, T)
    u, it, rr = o.pcg(fixed, f, rtol=1e-12)
    r = f - o.matvec(fixed, u)
    assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(f)
    assert rr <= 1e-12 and it > 5
