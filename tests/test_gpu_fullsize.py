"""The full-scale 1024 x 1024 x 128 package in the launch configuration the
benchmark times (FP32, sources on, Joule accumulation), checked against the
FP64 oracle on sampled windows.

After s steps a node's value depends only on nodes within s cells, so the
oracle runs on a window (domain faces keep their walls, cut faces are PEC) and
the comparison skips a margin of s + 2 cells next to every cut face. Windows:
the x-/y- CPML corner, a signal line's port, and the top CPML over a chiplet
edge (bumps, underfill, Si). Tolerance: FP32 rounding over a few steps
(2e-5 relative L2 of each field on the compared region)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, context, rel_l2, unknown_masks
from workloads import constraints as BC

pytestmark = pytest.mark.gpu

STEPS = 3


@pytest.fixture(scope="module")
def full():
    p = W.full_package()
    ctx = context(p, FP32)
    ctx.set_sources(p.source_tables(ctx.dt, 64))
    rng = np.random.default_rng(11)
    em, hm = unknown_masks(p)
    E0 = [np.where(em[a], rng.standard_normal(p.n_nodes, dtype=np.float32), 0).astype(np.float32) for a in range(3)]
    H0 = [np.where(hm[a], 2e-3 * rng.standard_normal(p.n_nodes, dtype=np.float32), 0).astype(np.float32)
          for a in range(3)]
    for a in range(3):
        ctx.write(api.COSIM_F_EX + a, E0[a])
        ctx.write(api.COSIM_F_HX + a, H0[a])
    ctx.em_steps(STEPS)
    E = [ctx.read(api.COSIM_F_EX + a, np.float32) for a in range(3)]
    H = [ctx.read(api.COSIM_F_HX + a, np.float32) for a in range(3)]
    Q = ctx.read(api.COSIM_F_Q)
    yield dict(p=p, ctx=ctx, dt=ctx.dt, E0=E0, H0=H0, E=E, H=H, Q=Q)
    ctx.close()


def windows(p):
    """[lo, hi) cell boxes; a box that would cut through a CPML slab is widened
    to the domain face (a cut face inside a slab would drop its psi terms)."""
    s0 = p.sources[0]
    e = s0.edges[0]
    z = int(e[2])
    n = (p.nx, p.ny, p.nz)
    L = p.cpml_cells
    raw = [((0, 0, 0), (48, 48, p.nz)),                                      # CPML corner, PEC ground
           ((int(e[0]) - 20, int(e[1]) - 20, z - 10), (int(e[0]) + 20, int(e[1]) + 20, z + 10)),  # a port
           ((n[0] // 2 - 20, (190 * n[1]) // 1024, 90), (n[0] // 2 + 20, (230 * n[1]) // 1024, p.nz))]  # top
    out = []
    for lo, hi in raw:
        lo, hi = list(lo), list(hi)
        for a in range(3):
            low_slab = L if p.em_bc[2 * a] == W.BC_CPML else 0
            high_slab = L if p.em_bc[2 * a + 1] == W.BC_CPML else 0
            if lo[a] <= low_slab + STEPS + 2:
                lo[a] = 0
            if hi[a] >= n[a] - high_slab - STEPS - 2:
                hi[a] = n[a]
        out.append((tuple(lo), tuple(hi)))
    return out


def _sub(arr, p, lo, hi):
    a = arr.reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    return np.ascontiguousarray(a[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1], dtype=np.float64).reshape(-1)


def _interior(p, wp, lo, hi, m):
    """node mask of the window, minus m cells next to each cut face"""
    K, J, I = np.meshgrid(np.arange(wp.nz + 1), np.arange(wp.ny + 1), np.arange(wp.nx + 1), indexing="ij")
    ok = np.ones(K.shape, bool)
    for P, a, b, n in ((I, lo[0], hi[0], p.nx), (J, lo[1], hi[1], p.ny), (K, lo[2], hi[2], p.nz)):
        w = b - a
        if a != 0:
            ok &= P >= m
        if b != n:
            ok &= P <= w - m
    return ok.reshape(-1)


@pytest.mark.parametrize("w", range(3))
def test_full_package_em_windows(full, w):
    p = full["p"]
    lo, hi = windows(p)[w]
    wp = W.crop(p, lo, hi)
    o = oracle.OracleSim(wp, dt=full["dt"])
    o.set_sources(wp.source_tables(full["dt"], 64))
    for a in range(3):
        o.E[a][:] = _sub(full["E0"][a], p, lo, hi)
        o.H[a][:] = _sub(full["H0"][a], p, lo, hi)
    o.em_steps(STEPS)
    keep = _interior(p, wp, lo, hi, STEPS + 2)
    for a in range(3):
        assert rel_l2(_sub(full["E"][a], p, lo, hi)[keep], o.E[a][keep]) < 2e-5, ("E", a)
        assert rel_l2(_sub(full["H"][a], p, lo, hi)[keep], o.H[a][keep]) < 2e-5, ("H", a)
    assert rel_l2(_sub(full["Q"], p, lo, hi)[keep], o.Q[keep]) < 1e-4


def test_full_package_thermal_and_matvec_windows(full):
    p, ctx = full["p"], full["ctx"]
    rng = np.random.default_rng(12)
    T0 = (300 + 30 * rng.random(p.n_nodes, dtype=np.float32)).astype(np.float32)
    P0 = (1e-6 * rng.random(p.n_nodes, dtype=np.float32)).astype(np.float32)
    ctx.write(api.COSIM_F_T, T0)
    ctx.write(api.COSIM_F_P, P0)
    dt_th = 0.9 * ctx.query(api.COSIM_Q_DT_TH_LIMIT)
    ctx.thermal_steps(2, dt_th)
    T = ctx.read(api.COSIM_F_T, np.float32)
    u = (1e-7 * rng.standard_normal((3, p.n_nodes))).astype(np.float32)
    y = ctx.stress_apply(u, bc=api.COSIM_MECH_CLAMPED_BOTTOM)
    for lo, hi in windows(p):
        wp = W.crop(p, lo, hi)
        o = oracle.OracleSim(wp)
        o.T = _sub(T0, p, lo, hi)
        o.P = _sub(P0, p, lo, hi)
        o.thermal_steps(2, dt=dt_th)
        keep = _interior(p, wp, lo, hi, 3)
        assert rel_l2(_sub(T, p, lo, hi)[keep] - 300, o.T[keep] - 300) < 1e-5
        fixed = BC.clamped_bottom(wp) if lo[2] == 0 else np.zeros(3 * wp.n_nodes, np.uint8)
        uw = np.stack([_sub(u[c], p, lo, hi) for c in range(3)], 1).reshape(-1)
        yo = o.matvec(fixed, uw).reshape(-1, 3)
        keepm = _interior(p, wp, lo, hi, 1)
        for c in range(3):
            assert rel_l2(_sub(y[c], p, lo, hi)[keepm], yo[keepm, c]) < 1e-5, ("Ku", c)
