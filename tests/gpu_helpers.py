"""Shared pieces of the GPU parity tests (CUDA path vs the FP64 oracle)."""
from __future__ import annotations

import numpy as np

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from paper_2603_07038_b300.build import build

FP64, FP32 = api.COSIM_FP64, api.COSIM_FP32


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def field_rel_l2(got3, ref3):
    """relative L2 of a vector field (all three components together) and the
    per-component error norms measured against that same field norm"""
    ref = np.concatenate([np.asarray(r, np.float64) for r in ref3])
    n = np.linalg.norm(ref)
    n = n if n > 0 else 1.0
    per = [np.linalg.norm(np.asarray(g, np.float64) - np.asarray(r, np.float64)) / n for g, r in zip(got3, ref3)]
    return float(np.sqrt(sum(e * e for e in per))), per


def context(p, precision, dt=0.0):
    build()
    return api.Context(p, precision=precision, dt_em=dt)


def unknown_masks(p):
    """boolean node-shaped masks of the E and H unknowns (edges inside the grid
    not held by a PEC wall; faces inside the grid)."""
    n = (p.nx, p.ny, p.nz)
    K, J, I = np.ogrid[0:p.nz + 1, 0:p.ny + 1, 0:p.nx + 1]
    P = (I, J, K)
    shape = (p.nz + 1, p.ny + 1, p.nx + 1)
    em, hm = [], []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        ok = np.broadcast_to(P[a] < n[a], shape).copy()
        for d in (b, c):
            if p.em_bc[2 * d] != W.BC_PMC:
                ok &= P[d] != 0
            if p.em_bc[2 * d + 1] != W.BC_PMC:
                ok &= P[d] != n[d]
        em.append(ok.reshape(-1))
        hm.append(np.broadcast_to((P[b] < n[b]) & (P[c] < n[c]), shape).reshape(-1))
    return em, hm


def random_fields(p, seed, e_scale=1.0, h_scale=2e-3):
    rng = np.random.default_rng(seed)
    em, hm = unknown_masks(p)
    nn = p.n_nodes
    E = [np.where(em[a], rng.standard_normal(nn) * e_scale, 0.0) for a in range(3)]
    H = [np.where(hm[a], rng.standard_normal(nn) * h_scale, 0.0) for a in range(3)]
    return E, H


def seed_both(o, ctx, E, H):
    for a in range(3):
        o.E[a][:] = E[a]
        o.H[a][:] = H[a]
        ctx.write(api.COSIM_F_EX + a, E[a])
        ctx.write(api.COSIM_F_HX + a, H[a])


def read_eh(ctx):
    return ([ctx.read(api.COSIM_F_EX + a) for a in range(3)], [ctx.read(api.COSIM_F_HX + a) for a in range(3)])


def hetero_problem(nx, ny, nz, seed, em_bc, cpml=4, conductor=True, uniform_x=False):
    """odd-sized non-uniform grid, four materials including a good conductor.
    uniform_x keeps the y and z spacings random but makes x uniform, so the
    oracle's element-matrix cache (keyed on the cell shape) hits along x rows."""
    rng = np.random.default_rng(seed)
    mats = [W.DIELECTRIC, W.COPPER if conductor else W.UNDERFILL, W.SILICON, W.UNDERFILL]
    mat = rng.integers(0, 4, (nz, ny, nx)).astype(np.uint8)
    dx = rng.uniform(3e-6, 8e-6, nx)
    if uniform_x:
        dx[:] = 5e-6
    return W.Problem(name=f"hetero{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
                     dx=dx, dy=rng.uniform(3e-6, 8e-6, ny),
                     dz=rng.uniform(1e-6, 4e-6, nz), mat=mat, materials=mats, em_bc=tuple(em_bc),
                     cpml_cells=cpml, cpml_eps_r=3.5, h_conv=(0.0, 2e4, 0.0, 0.0, 0.0, 1e4),
                     T_amb=300.0, T_init=300.0)


def oracle_mask_from_bits(bits):
    return np.stack([(bits >> c) & 1 for c in range(3)], 1).astype(np.uint8).reshape(-1)


def soa_to_interleaved(u3):
    return np.stack(u3, 1).reshape(-1)


def interleaved_to_soa(u):
    return u.reshape(-1, 3).T.copy()
