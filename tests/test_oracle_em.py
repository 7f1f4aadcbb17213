"""Pins of the oracle's EM step (Sec. II-A, Eqs. 1-3) and Joule heat against
closed forms and exact discrete invariants, independent of the oracle's code."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from tests.fit_metric import EPS0, MU0, Metric, coords, dual

VAC = W.Material("vacuum", 1.0, 1.0, 0.0, 0.0, 300.0, 1.0, 1e6, 1e9, 0.3, 1e-6)


def mixed_problem(seed, nx=7, ny=6, nz=5, bc=(0, 1, 0, 1, 1, 0), lossy=False):
    """small non-uniform grid, heterogeneous eps/mu (and sigma), PEC/PMC walls"""
    rng = np.random.default_rng(seed)
    mats = [W.Material(f"m{q}", float(rng.uniform(1, 6)), float(rng.uniform(1, 3)),
                       float(rng.uniform(0, 5e5)) if lossy else 0.0,
                       0.0, 300.0, 1.0, 1e6, 1e9, 0.3, 1e-6) for q in range(3)]
    p = W.Problem(name="mixed", nx=nx, ny=ny, nz=nz,
                  dx=rng.uniform(0.5e-4, 2e-4, nx), dy=rng.uniform(0.5e-4, 2e-4, ny),
                  dz=rng.uniform(0.5e-4, 2e-4, nz),
                  mat=rng.integers(0, 3, (nz, ny, nx)).astype(np.uint8), materials=mats,
                  em_bc=bc, cpml_cells=0, h_conv=(0.0,) * 6)
    return p


def seed_fields(o, p, rng, h_scale=2e-3):
    """random E on the free edges and random H on the faces; every other slot 0"""
    m = Metric(p)
    for a in range(3):
        o.E[a][:] = 0.0
        o.H[a][:] = 0.0
        for n in m.edges(a):
            o.E[a][m.nid(n)] = rng.standard_normal()
        for n in m.faces(a):
            o.H[a][m.nid(n)] = rng.standard_normal() * h_scale


def test_dof_counts_match_paper(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_dof_counts.json")))
    nx, ny, nz = g["grid_cells"]
    p = W.uniform_box(nx, ny, nz, em_bc=(W.BC_PMC,) * 6)
    assert oracle.count_dofs(p) == (g["em_dofs"], g["thermal_dofs"], g["mechanical_dofs"])


def _te101(ncell, steps=40):
    """PEC cavity a x b x d (x, y, z); seed E_y = sin(pi x/a) sin(pi z/d)."""
    a_len, d_len = 10e-3, 8e-3
    nx, nz = ncell, int(round(ncell * 0.8))
    h = a_len / nx
    p = W.uniform_box(nx, 3, nz, h=(h, 1.3 * h, h), material=VAC, em_bc=(W.BC_PEC,) * 6)
    o = oracle.OracleSim(p)
    g = o.g
    x = coords(p.dx)
    z = coords(p.dz)
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(p.ny + 1), np.arange(nx + 1), indexing="ij")
    mode = np.sin(np.pi * x[I] / a_len) * np.sin(np.pi * z[K] / d_len)
    mode[:, p.ny, :] = 0.0  # no E_y edge beyond the last cell in y
    mode[:, :, [0, nx]] = 0.0  # PEC walls
    mode[[0, nz], :, :] = 0.0
    o.E[1][:] = mode.reshape(-1)
    hist = []
    for _ in range(steps):
        hist.append(o.E[1].copy())
        o.em_step(accumulate_joule=False)
    hist.append(o.E[1].copy())
    lam = (4 / MU0) * (math.sin(math.pi * h / (2 * a_len)) ** 2 / h ** 2
                       + math.sin(math.pi * h / (2 * d_len)) ** 2 / h ** 2)
    cos_th = 1 - o.dt ** 2 * lam / (2 * EPS0)
    return o, hist, cos_th, (a_len, d_len)


def test_te101_discrete_dispersion():
    """Eliminating H gives e^{n+1} + e^{n-1} = (2 - dt^2 lambda/eps) e^n with the
    discrete curl-curl eigenvalue lambda of the sampled TE101 mode."""
    o, hist, cos_th, _ = _te101(10)
    for n in range(2, len(hist) - 1):
        en = hist[n]
        sel = np.abs(en) > 0.5 * np.abs(en).max()
        meas = (hist[n + 1][sel] + hist[n - 1][sel]) / (2 * en[sel])
        assert np.max(np.abs(meas - cos_th)) < 1e-11


def test_te101_continuous_frequency_second_order():
    """f -> (c/2) sqrt(1/a^2 + 1/d^2) with O(h^2) error."""
    errs = []
    for ncell in (10, 20):
        o, hist, cos_th, (a_len, d_len) = _te101(ncell, steps=4)
        f_disc = math.acos(cos_th) / (2 * math.pi * o.dt)
        f_cont = 0.5 / math.sqrt(EPS0 * MU0) * math.sqrt(1 / a_len ** 2 + 1 / d_len ** 2)
        errs.append(abs(f_disc / f_cont - 1))
    assert errs[0] < 1e-2
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_lossless_energy_conserved_nonuniform_pec_pmc():
    """sigma = 0, no source: W^n = 1/2 E^T M_eps E + 1/2 H^{n-1/2} M_mu H^{n+1/2}
    is an exact invariant of the leapfrog for the FIT metric (edge integrals of
    eps, series-mean mu on faces, half dual cells at walls)."""
    p = mixed_problem(3)
    o = oracle.OracleSim(p, cfl=0.9)
    m = Metric(p)
    seed_fields(o, p, np.random.default_rng(5))
    energies = []
    for _ in range(30):
        E_n = [e.copy() for e in o.E]
        H_old = [h.copy() for h in o.H]
        o.h_half_step()
        energies.append(m.em_energy(E_n, H_old, o.H))
        o.e_step(accumulate_joule=False)
    energies = np.array(energies)
    assert np.max(np.abs(energies / energies[0] - 1)) < 1e-12


def test_poynting_balance_joule_and_source_work():
    """With sigma > 0 and a source: W^0 - W^N - sum_n dt sum_e V_e J_e ebar_e
    = sum of the Joule heat deposited on nodes (exact discrete identity with
    the time-centred ebar)."""
    p = mixed_problem(11, lossy=True)
    o = oracle.OracleSim(p, cfl=0.9)
    m = Metric(p)
    rng = np.random.default_rng(7)
    src_edges = np.array([[2, 3, 1], [2, 3, 2], [4, 1, 2]], np.int32)
    nsteps = 40
    amp = rng.standard_normal(nsteps) * 1e3
    o.set_sources([(2, src_edges, amp)])
    seed_fields(o, p, rng, h_scale=0.0)
    o.em_step(accumulate_joule=False)
    o.joule_reset()
    work = 0.0
    W0 = None
    for n in range(1, nsteps - 1):
        E_n = [e.copy() for e in o.E]
        H_old = [h.copy() for h in o.H]
        o.h_half_step()
        Wn = m.em_energy(E_n, H_old, o.H)
        if W0 is None:
            W0 = Wn
        else:
            Wlast = Wn
        if n == nsteps - 2:
            break
        o.e_step(accumulate_joule=True)
        for e in src_edges:
            ebar = 0.5 * (E_n[2][m.nid(e)] + o.E[2][m.nid(e)])
            work += o.dt * m.edge_volume(2, tuple(e)) * amp[n] * ebar
    joule = o.Q.sum()
    assert joule > 0
    lhs = W0 - Wlast - work
    assert abs(lhs - joule) < 1e-10 * max(abs(W0), joule)


def test_joule_dc_bar_is_V2_over_R():
    """A uniform field V/L along a conductor bar dissipates V^2/R, R = L/(sigma A),
    including bar-surface edges that see the conductor in only 1-2 voxels."""
    rng = np.random.default_rng(2)
    nx, ny, nz = 9, 8, 7
    cu = W.COPPER
    p = W.Problem(name="bar", nx=nx, ny=ny, nz=nz, dx=rng.uniform(1e-6, 3e-6, nx),
                  dy=rng.uniform(1e-6, 3e-6, ny), dz=rng.uniform(1e-6, 3e-6, nz),
                  mat=np.zeros((nz, ny, nx), np.uint8), materials=[W.DIELECTRIC, cu],
                  em_bc=(W.BC_PEC,) * 6, cpml_cells=0)
    i0, i1, j0, j1, k0, k1 = 2, 7, 3, 6, 1, 4
    p.mat[k0:k1, j0:j1, i0:i1] = 1
    o = oracle.OracleSim(p)
    L = p.dx[i0:i1].sum()
    A = p.dy[j0:j1].sum() * p.dz[k0:k1].sum()
    V = 1.7e-3
    Ex = np.full(o.g.n_nodes, V / L)
    E = [Ex, np.zeros_like(Ex), np.zeros_like(Ex)]
    Q = o.joule_of(E, E)
    P = cu.sigma0 * A * V * V / L
    assert abs(Q.sum() / (o.dt * P) - 1) < 1e-13
    # the energy lands on nodes of the bar only, half from each edge end
    Qn = Q.reshape(o.g.node_shape)
    assert Qn[:, :, :i0].sum() == 0 and Qn[:, :, i1 + 1:].sum() == 0


def test_yee_matches_second_order_update_eq2():
    """The leapfrog reproduces Eq. 2-3: (D_eps + dt/2 D_sig) e^{n+1} =
    (2 D_eps - dt^2 S) e^n - (D_eps - dt/2 D_sig) e^{n-1} - dt^2 (dJ/dt)^n,
    with S = curl mu^-1 curl applied by numpy differences (uniform grid,
    interior edges, heterogeneous eps/sigma/mu, a driven source)."""
    rng = np.random.default_rng(4)
    nx, ny, nz, h = 8, 7, 6, 1e-4
    p = mixed_problem(21, nx, ny, nz, bc=(0,) * 6, lossy=True)
    p.dx[:] = h
    p.dy[:] = h
    p.dz[:] = h
    o = oracle.OracleSim(p, cfl=0.9)
    nsteps = 12
    amp = rng.standard_normal(nsteps) * 1e4
    src = np.array([[3, 3, 2], [4, 3, 2]], np.int32)
    o.set_sources([(0, src, amp)])
    seed_fields(o, p, rng, h_scale=0.0)
    o.em_step(False)
    hist = [[e.copy() for e in o.E]]
    for _ in range(3):
        o.em_step(False)
        hist.append([e.copy() for e in o.E])
    n = 2  # check e^{n+1} from e^n, e^{n-1}; o.step was n at the e^n -> e^{n+1} update
    tab = p.material_table()
    mat = p.mat.astype(int)
    eps_c = EPS0 * tab[mat, 0]
    sig_c = tab[mat, 2]
    imu_c = 1.0 / (MU0 * tab[mat, 1])
    shp = o.g.node_shape

    def edge_mean(cell, a):
        # mean over the four voxels around interior edges of axis a (uniform grid)
        c = np.pad(cell, 1)  # (nz+2, ny+2, nx+2), voxel (i,j,k) at [k+1, j+1, i+1]
        out = np.zeros(shp)
        for d1 in (0, 1):
            for d2 in (0, 1):
                if a == 0:
                    out[:, :, :nx] += c[d1:d1 + nz + 1, d2:d2 + ny + 1, 1:nx + 1] / 4
                elif a == 1:
                    out[:, :ny, :] += c[d1:d1 + nz + 1, 1:ny + 1, d2:d2 + nx + 1] / 4
                else:
                    out[:nz, :, :] += c[1:nz + 1, d1:d1 + ny + 1, d2:d2 + nx + 1] / 4
        return out

    def face_mu_inv(a):
        c = np.pad(imu_c, 1)
        out = np.zeros(shp)
        for d in (0, 1):
            if a == 0:
                out[:nz, :ny, :] += c[1:nz + 1, 1:ny + 1, d:d + nx + 1] / 2
            elif a == 1:
                out[:nz, :, :nx] += c[1:nz + 1, d:d + ny + 1, 1:nx + 1] / 2
            else:
                out[:, :ny, :nx] += c[d:d + nz + 1, 1:ny + 1, 1:nx + 1] / 2
        return out

    def curl_e(E):
        Ex, Ey, Ez = [e.reshape(shp) for e in E]
        Hx = np.zeros(shp); Hy = np.zeros(shp); Hz = np.zeros(shp)
        Hx[:nz, :ny, :] = (Ez[:nz, 1:, :] - Ez[:nz, :ny, :] - Ey[1:, :ny, :] + Ey[:nz, :ny, :]) / h
        Hy[:nz, :, :nx] = (Ex[1:, :, :nx] - Ex[:nz, :, :nx] - Ez[:nz, :, 1:] + Ez[:nz, :, :nx]) / h
        Hz[:, :ny, :nx] = (Ey[:, :ny, 1:] - Ey[:, :ny, :nx] - Ex[:, 1:, :nx] + Ex[:, :ny, :nx]) / h
        return Hx, Hy, Hz

    def curl_h_interior(H):
        Hx, Hy, Hz = H
        C = [np.zeros(shp) for _ in range(3)]
        C[0][1:-1, 1:-1, :nx] = (Hz[1:-1, 1:-1, :nx] - Hz[1:-1, :-2, :nx]
                                 - Hy[1:-1, 1:-1, :nx] + Hy[:-2, 1:-1, :nx]) / h
        C[1][1:-1, :ny, 1:-1] = (Hx[1:-1, :ny, 1:-1] - Hx[:-2, :ny, 1:-1]
                                 - Hz[1:-1, :ny, 1:-1] + Hz[1:-1, :ny, :-2]) / h
        C[2][:nz, 1:-1, 1:-1] = (Hy[:nz, 1:-1, 1:-1] - Hy[:nz, 1:-1, :-2]
                                 - Hx[:nz, 1:-1, 1:-1] + Hx[:nz, :-2, 1:-1]) / h
        return C

    Hc = curl_e(hist[n])
    Se = curl_h_interior([face_mu_inv(a) * Hc[a] for a in range(3)])
    dt = o.dt
    J = [np.zeros(shp) for _ in range(3)]
    for e in src:
        J[0][e[2], e[1], e[0]] += amp[n + 1] - amp[n]  # J^{n+1/2} - J^{n-1/2} of that update
    for a in range(3):
        D_eps, D_sig = edge_mean(eps_c, a), edge_mean(sig_c, a)
        lhs = (D_eps + dt / 2 * D_sig) * hist[n + 1][a].reshape(shp)
        rhs = ((2 * D_eps) * hist[n][a].reshape(shp) - dt * dt * Se[a]
               - (D_eps - dt / 2 * D_sig) * hist[n - 1][a].reshape(shp) - dt * J[a])
        sl = [slice(1, -1)] * 3
        sl[2 - a] = slice(0, shp[2 - a] - 1)
        sl = tuple(sl)
        scale = np.abs(D_eps[sl] * hist[n][a].reshape(shp)[sl]).max()
        assert np.max(np.abs(lhs[sl] - rhs[sl])) < 1e-11 * scale


def _line(axis, ncells, src_at, probe_at, steps, h=0.5e-3, cpml=8):
    """quasi-1D TEM line along `axis`: E along b=(axis+1)%3, H along c;
    PEC walls normal to b, PMC walls normal to c, CPML at both ends."""
    b, c = (axis + 1) % 3, (axis + 2) % 3
    n = [1, 1, 1]
    n[axis] = ncells
    bc = [0] * 6
    bc[2 * axis] = bc[2 * axis + 1] = W.BC_CPML
    bc[2 * b] = bc[2 * b + 1] = W.BC_PEC
    bc[2 * c] = bc[2 * c + 1] = W.BC_PMC
    p = W.uniform_box(*n, h=(h, h, h), material=VAC, em_bc=tuple(bc), cpml_cells=cpml)
    o = oracle.OracleSim(p)
    edges = []
    for q in (0, 1):
        e = [0, 0, 0]
        e[axis] = src_at
        e[c] = q
        edges.append(e)
    wf = W.GaussianDerivative(j0=1e3, sigma_t=10e-12)
    amp = wf((np.arange(steps) + 0.5) * o.dt)
    o.set_sources([(b, np.array(edges, np.int32), amp)])
    pr = [0, 0, 0]
    pr[axis] = probe_at
    pid = o.g.nid(*pr)
    rec = []
    for _ in range(steps):
        o.em_step(False)
        rec.append(o.E[b][pid])
    return np.array(rec)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cpml_reflection_below_minus_40dB(axis):
    steps = 700
    short = _line(axis, 160, 40, 80, steps)
    ref = _line(axis, 1400, 640, 680, steps)
    refl = np.max(np.abs(short - ref)) / np.max(np.abs(ref))
    assert 20 * math.log10(refl) < -40.0


def test_cpml_profile_shape():
    """sigma grows as depth^3 into the layer; b in (0, 1), c = b - 1; untouched
    outside the layers."""
    p = W.uniform_box(40, 4, 4, h=(1e-4, 1e-4, 1e-4), material=VAC,
                      em_bc=(2, 2, 0, 0, 0, 0), cpml_cells=8)
    g = oracle.Grid(p)
    import ctypes as C
    b = np.zeros(41)
    c = np.zeros(41)
    dt = oracle.cfl_dt(p)
    oracle.lib().og_cpml_table(g.ref, 0, 0, dt, b.ctypes.data_as(C.POINTER(C.c_double)),
                               c.ctypes.data_as(C.POINTER(C.c_double)))
    assert np.all(b[8:33] == 1.0) and np.all(c[8:33] == 0.0)
    assert np.all((b[:8] > 0) & (b[:8] < 1)) and np.allclose(c, b - 1)
    sig = -np.log(b[:8]) * EPS0 / dt
    depth = (8 - np.arange(8)) / 8
    smax = 0.8 * 4 / (math.sqrt(MU0 / EPS0) * 1e-4)
    assert np.allclose(sig, smax * depth ** 3, rtol=1e-12)
    assert np.allclose(b[:8], b[40:32:-1], rtol=0, atol=1e-15)


def test_cfl_dt_tiny_package():
    p = W.tiny_package()
    dt = oracle.cfl_dt(p, 0.99)
    c0 = 1 / math.sqrt(EPS0 * MU0)
    ref = 0.99 / (c0 * math.sqrt(2 / 25e-12 + 1 / 4e-12))
    assert abs(dt / ref - 1) < 1e-14
