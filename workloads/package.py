"""Seeded synthetic voxelised packages.

The paper's package (a 26-layer stack: organic substrate, silicon interposer,
micro-bump arrays, logic and HBM dies; Sec. III-A) is proprietary, so these
generators stand in for it with layered stacks of the same kinds of features
(routing layers, TSVs, micro-bumps, chiplets), at the sizes of the solver's
workloads. Everything here is input description: materials per voxel, cell
sizes per axis, boundary choices and source edges.

Layout conventions (shared by every consumer):
  * cells (i, j, k), 0 <= i < nx etc.; ``mat`` has shape (nz, ny, nx), x fastest;
  * ``dx[i]``, ``dy[j]``, ``dz[k]`` are cell sizes in metres (non-uniform allowed);
  * an edge is named by its lower node (i, j, k) and its axis (0=x, 1=y, 2=z);
  * faces are ordered x-, x+, y-, y+, z-, z+.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Callable

import numpy as np

BC_PEC, BC_PMC, BC_CPML = 0, 1, 2


@dataclass(frozen=True)
class Material:
    """Per-voxel constants (SI units). sigma0 is the conductivity at T0 and
    tcr the temperature coefficient of resistance (Eq. 6)."""
    name: str
    eps_r: float
    mu_r: float
    sigma0: float
    tcr: float
    T0: float
    k: float        # thermal conductivity [W/(m K)]
    rho_cp: float   # volumetric heat capacity [J/(m^3 K)]
    E: float        # Young's modulus [Pa]
    nu: float       # Poisson ratio
    alpha_L: float  # linear CTE [1/K]

    def as_row(self):
        return [self.eps_r, self.mu_r, self.sigma0, self.tcr, self.T0,
                self.k, self.rho_cp, self.E, self.nu, self.alpha_L]


# Material table of the synthetic packages. Values the paper prints (Sec. III-A)
# are Cu alpha=17 ppm, Si E=130 GPa alpha=2.6 ppm; the rest are standard
# packaging constants chosen for these workloads.
DIELECTRIC = Material("dielectric", 3.5, 1.0, 0.0, 0.0, 300.0, 0.3, 1.55e6, 5e9, 0.35, 50e-6)
COPPER = Material("copper", 1.0, 1.0, 5.8e7, 3.93e-3, 300.0, 400.0, 3.45e6, 110e9, 0.34, 17e-6)
SILICON = Material("silicon", 11.7, 1.0, 10.0, 0.0, 300.0, 150.0, 1.63e6, 130e9, 0.28, 2.6e-6)
UNDERFILL = Material("underfill", 3.2, 1.0, 0.0, 0.0, 300.0, 0.5, 1.7e6, 8e9, 0.35, 30e-6)

M_DIEL, M_CU, M_SI, M_UF = 0, 1, 2, 3


@dataclass
class Source:
    """Soft current-density source on a set of edges of one axis.

    ``edges`` is an (n, 3) int32 array of lower-node indices (i, j, k).
    ``waveform(t)`` returns J [A/m^2]; the solvers use it at t = (n + 1/2) dt.
    """
    axis: int
    edges: np.ndarray
    waveform: Callable

    def amp_table(self, dt: float, nsteps: int, t0: float = 0.0) -> np.ndarray:
        """J at t0 + (n + 1/2) dt, n < nsteps (t0: start of the simulated window)."""
        if hasattr(self.waveform, "table"):
            if t0 != 0.0:
                raise ValueError("a sampled waveform has no time offset")
            return self.waveform.table(dt, nsteps)
        t = t0 + (np.arange(nsteps, dtype=np.float64) + 0.5) * dt
        return np.asarray(self.waveform(t), dtype=np.float64)


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    mat: np.ndarray                     # (nz, ny, nx) uint8
    materials: list
    em_bc: tuple = (BC_CPML,) * 4 + (BC_PEC, BC_CPML)
    cpml_cells: int = 8
    cpml_order: float = 3.0
    cpml_eps_r: float = 1.0
    h_conv: tuple = (0.0,) * 5 + (1e4,)
    T_amb: float = 300.0
    T_init: float = 300.0
    sources: list = field(default_factory=list)
    em_steps: int = 0                   # steps of the workload's EM burst
    thermal_steps: int = 0

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    def material_table(self) -> np.ndarray:
        return np.array([m.as_row() for m in self.materials], dtype=np.float64)

    def source_tables(self, dt: float, nsteps: int, t0: float = 0.0):
        """[(axis, edges int32 (n,3), amp float64 (nsteps,)), ...]; t0 shifts
        the sampled window of every waveform (a burst window that starts
        later than t = 0)."""
        return [(s.axis, np.ascontiguousarray(s.edges, dtype=np.int32),
                 s.amp_table(dt, nsteps, t0)) for s in self.sources]


def _check(p: Problem) -> Problem:
    assert p.mat.shape == (p.nz, p.ny, p.nx) and p.mat.dtype == np.uint8
    assert len(p.dx) == p.nx and len(p.dy) == p.ny and len(p.dz) == p.nz
    assert int(p.mat.max(initial=0)) < len(p.materials)
    return p


def uniform_box(nx, ny, nz, h=(1e-5, 1e-5, 1e-5), material=DIELECTRIC,
                em_bc=(BC_PEC,) * 6, h_conv=(0.0,) * 6, **kw) -> Problem:
    """A single-material box (used by closed-form checks)."""
    hx, hy, hz = h
    p = Problem(
        name=f"box{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
        dx=np.full(nx, hx), dy=np.full(ny, hy), dz=np.full(nz, hz),
        mat=np.zeros((nz, ny, nx), np.uint8), materials=[material],
        em_bc=tuple(em_bc), h_conv=tuple(h_conv), **kw)
    return _check(p)


def tiny_package(seed: int = 1) -> Problem:
    """32x32x16 voxels (dx=dy=5 um, dz=2 um), Si base, dielectric above, four
    2-voxel-wide Cu traces along x in routing layers z=3 and z=6, a lumped
    z-directed port from the ground plane up to trace 0, PEC bottom and an
    8-cell CPML on the other five faces, convective top."""
    nx, ny, nz = 32, 32, 16
    rng = np.random.default_rng(seed)
    mat = np.full((nz, ny, nx), M_DIEL, np.uint8)
    mat[0:2] = M_SI
    traces = []
    for z in (3, 6):
        # two non-overlapping 2-wide traces with start rows in the 16x16 interior
        while True:
            a, b = sorted(rng.choice(np.arange(8, 23), size=2, replace=False))
            if b - a >= 3:
                break
        for j0 in (a, b):
            mat[z, j0:j0 + 2, :] = M_CU
            traces.append((z, int(j0)))
    z0, j0 = traces[0]
    dx = dy = 5e-6
    # lumped port: z-edges from node z=0 (PEC ground) to node z=z0 (trace bottom),
    # at the first interior x node, centred on the trace's width
    i_port, j_port = 8, j0 + 1
    edges = np.array([[i_port, j_port, k] for k in range(z0)], np.int32)
    j_peak = 10e-3 / (dx * dy)        # 10 mA through one node's dual face
    src = Source(axis=2, edges=edges,
                 waveform=GaussianDerivativeJ(j_peak * np.exp(0.5), 20e-12))
    p = Problem(
        name="tiny_package", nx=nx, ny=ny, nz=nz,
        dx=np.full(nx, dx), dy=np.full(ny, dy), dz=np.full(nz, 2e-6),
        mat=mat, materials=[DIELECTRIC, COPPER, SILICON],
        em_bc=(BC_CPML, BC_CPML, BC_CPML, BC_CPML, BC_PEC, BC_CPML),
        cpml_cells=8, cpml_eps_r=3.5, h_conv=(0.0,) * 5 + (1e4,),
        T_amb=300.0, T_init=300.0, sources=[src], em_steps=1000, thermal_steps=100)
    return _check(p)


def GaussianDerivativeJ(j0, sigma_t):
    from .waveforms import GaussianDerivative
    return GaussianDerivative(j0=j0, sigma_t=sigma_t)


# --- full-scale layered package -------------------------------------------------

# z stack (cell indices) of the 128-cell package
Z_SUB = (0, 64)        # organic substrate with 8 routing layers
Z_INT = (64, 96)       # Si interposer with Cu TSVs
Z_BUMP = (96, 104)     # underfill with Cu micro-bumps
Z_DIE = (104, 128)     # chiplets (Si) in underfill
ROUTING_Z = tuple(8 * r + 4 for r in range(8))


def _stack(nz: int = 128):
    """z ranges (substrate, interposer, bumps, dies) and routing-layer planes
    of an nz-cell stack: the 128-cell stack's proportions (1/2, 1/4, 1/16,
    3/16), eight routing layers spread through the substrate. nz = 128 gives
    the constants above."""
    f = lambda z: (z * nz) // 128  # noqa: E731
    return ((0, f(Z_SUB[1])), (f(Z_INT[0]), f(Z_INT[1])), (f(Z_BUMP[0]), f(Z_BUMP[1])), (f(Z_DIE[0]), nz),
            tuple(f(z) for z in ROUTING_Z))


def _dz_profile(nz: int = 128) -> np.ndarray:
    _, z_int, z_bump, _, routing = _stack(nz)
    thin = set(routing) | set(range(*z_bump)) | {z_int[0], z_int[1] - 1}
    return np.array([2e-6 if k in thin else 5e-6 for k in range(nz)], np.float64)


def layered_package(nx: int = 1024, ny: int = 1024, seed: int = 2, n_lines: int = 32,
                    tsv_pitch: int = 5, bump_pitch: int = 4, chiplet: int | None = None,
                    em_steps: int | None = None, nz: int = 128) -> Problem:
    """Layered package on an nx x ny x 128 voxel grid (10 um lateral, 2-5 um z).

    z 0-63: dielectric substrate with 8 Manhattan routing layers (one Cu cell
    thick, alternating x/y preferred direction, 1-2 voxel wide segmented
    tracks at 5-voxel pitch, about 30 % fill); z 64-95: Si interposer with
    1x1-voxel Cu TSVs at ``tsv_pitch``; z 96-103: underfill with 2x2-voxel Cu
    micro-bumps at ``bump_pitch`` under the chiplets; z 104-127: four Si
    chiplets (``chiplet`` voxels square, 2x2 arrangement) in underfill.
    ``n_lines`` routing segments carry PRBS7 10 Gb/s ports. ``nz`` other than
    128 scales the stack's regions in proportion (``_stack``).
    """
    if nz < 64:
        raise ValueError("the layered stack needs nz >= 64")
    z_sub, z_int, z_bump, z_die, routing = _stack(nz)
    rng = np.random.default_rng(seed)
    mat = np.empty((nz, ny, nx), np.uint8)
    mat[z_sub[0]:z_sub[1]] = M_DIEL
    mat[z_int[0]:z_int[1]] = M_SI
    mat[z_bump[0]:z_die[1]] = M_UF
    segments = []  # (z, axis, along0, along1, across0, width)
    for r, z in enumerate(routing):
        axis = r % 2               # 0: tracks run along x, 1: along y
        n_along, n_across = (nx, ny) if axis == 0 else (ny, nx)
        for c0 in range(1, n_across - 2, 5):
            w = int(rng.integers(1, 3))
            pos = int(rng.integers(0, 40))
            # segment lengths 48-320 voxels; axes shorter than 256 voxels
            # (small designs) draw proportionally shorter segments
            seg_lo, seg_hi = (48, 320) if n_along >= 256 else (max(8, n_along // 6), max(16, n_along // 2))
            while pos < n_along:
                seg = int(rng.integers(seg_lo, seg_hi))
                a0, a1 = pos, min(n_along, pos + seg)
                if axis == 0:
                    mat[z, c0:c0 + w, a0:a1] = M_CU
                else:
                    mat[z, a0:a1, c0:c0 + w] = M_CU
                segments.append((z, axis, a0, a1, c0, w))
                pos = a1 + int(rng.integers(2, 7))
    # TSVs
    ii = (np.arange(nx) % tsv_pitch) == tsv_pitch // 2
    jj = (np.arange(ny) % tsv_pitch) == tsv_pitch // 2
    tsv = np.logical_and.outer(jj, ii)
    mat[z_int[0]:z_int[1]][:, tsv] = M_CU
    # chiplets and bumps
    if chiplet is None:
        chiplet = max(2, (300 * min(nx, ny)) // 1024)
    gap = max(2, (24 * min(nx, ny)) // 1024)
    mx = (nx - 2 * chiplet - gap) // 2
    my = (ny - 2 * chiplet - gap) // 2
    foot = np.zeros((ny, nx), bool)
    for cx in (mx, mx + chiplet + gap):
        for cy in (my, my + chiplet + gap):
            foot[cy:cy + chiplet, cx:cx + chiplet] = True
    mat[z_die[0]:z_die[1]][:, foot] = M_SI
    bi = np.isin(np.arange(nx) % bump_pitch, (1, 2))
    bj = np.isin(np.arange(ny) % bump_pitch, (1, 2))
    bump = np.logical_and.outer(bj, bi) & foot
    mat[z_bump[0]:z_bump[1]][:, bump] = M_CU
    dx = np.full(nx, 10e-6)
    dy = np.full(ny, 10e-6)
    dz = _dz_profile(nz)
    # signal lines: long segments away from the CPML, ports at their start
    L = 8
    min_len = min(64, min(nx, ny) // 3)  # small grids: shorter port segments
    cand = [s for s in segments
            if s[3] - s[2] >= min_len and s[2] > L and s[4] > L
            and s[4] + s[5] < (ny if s[1] == 0 else nx) - L
            and s[3] < (nx if s[1] == 0 else ny) - L]
    pick = rng.choice(len(cand), size=min(n_lines, len(cand)), replace=False)
    sources = []
    from .waveforms import PRBSBurst
    for n, q in enumerate(sorted(int(x) for x in pick)):
        z, axis, a0, a1, c0, w = cand[q]
        edges = []
        for c in range(c0, c0 + w + 1):
            for k in (z, z + 1):
                edges.append((a0, c, k) if axis == 0 else (c, a0, k))
        area = w * (dy[0] if axis == 0 else dx[0]) * dz[z]
        sources.append(Source(axis=axis, edges=np.array(edges, np.int32),
                              waveform=PRBSBurst(j0=10e-3 / area, seed=seed * 1000 + n)))
    p = Problem(
        name=f"layered_package_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
        mat=mat, materials=[DIELECTRIC, COPPER, SILICON, UNDERFILL],
        em_bc=(BC_CPML, BC_CPML, BC_CPML, BC_CPML, BC_PEC, BC_CPML),
        cpml_cells=L, cpml_eps_r=3.5, h_conv=(0.0,) * 5 + (1e4,),
        T_amb=300.0, T_init=300.0, sources=sources,
        em_steps=em_steps if em_steps is not None else 0, thermal_steps=10_000)
    return _check(p)


def full_package(seed: int = 2) -> Problem:
    """The full-scale single-package workload: 1024 x 1024 x 128 voxels."""
    return layered_package(1024, 1024, seed=seed)


def crop(p: Problem, lo, hi) -> Problem:
    """Sub-window [lo, hi) (cell indices per axis) of a problem.

    Faces of the window that are faces of the original domain keep their
    boundary choice; cut faces become PEC with no convection. Source edges
    inside the window are kept, shifted to window coordinates."""
    (i0, j0, k0), (i1, j1, k1) = lo, hi
    bc = list(p.em_bc)
    h = list(p.h_conv)
    for f, (a, b, n) in enumerate([(i0, i1, p.nx), (j0, j1, p.ny), (k0, k1, p.nz)]):
        if a != 0:
            bc[2 * f], h[2 * f] = BC_PEC, 0.0
        if b != n:
            bc[2 * f + 1], h[2 * f + 1] = BC_PEC, 0.0
    srcs = []
    for s in p.sources:
        e = np.asarray(s.edges, np.int64) - np.array([i0, j0, k0])
        hi_e = np.array([i1 - i0, j1 - j0, k1 - k0])
        inside = np.all(e >= 0, axis=1) & np.all(e <= hi_e, axis=1) & (e[:, s.axis] < hi_e[s.axis])
        if inside.any():
            srcs.append(Source(axis=s.axis, edges=e[inside].astype(np.int32), waveform=s.waveform))
    return _check(replace(
        p, name=p.name + f"[{i0}:{i1},{j0}:{j1},{k0}:{k1}]",
        nx=i1 - i0, ny=j1 - j0, nz=k1 - k0,
        dx=p.dx[i0:i1].copy(), dy=p.dy[j0:j1].copy(), dz=p.dz[k0:k1].copy(),
        mat=np.ascontiguousarray(p.mat[k0:k1, j0:j1, i0:i1]),
        em_bc=tuple(bc), h_conv=tuple(h), sources=srcs))


def paper_setup_package(nx: int = 192, ny: int = 192, nz: int = 64, seed: int = 7, n_pairs: int = 8,
                        n_gsg: int = 8, port_current: float = 10e-3) -> Problem:
    """The paper's boundary and excitation scheme (Sec. III-B) on the layered
    synthetic stack (``layered_package`` geometry):

    * EM walls: PMC on the four sides and the top, PEC ground plane at z = 0;
      thermal: adiabatic on every face (no film); no CPML;
    * substrate: ``n_pairs`` differential port pairs, x-oriented, on adjacent
      x-running tracks of the top x-routing layer, polarity alternating along
      y, driven by the Ricker trigger (t0 = 40 ps);
    * bump arrays: ``n_gsg`` ground-signal-ground triples along x under the
      "logic" chiplets (the two with the lower y) carrying the 5 GHz sine,
      and as many under the "HBM" chiplets carrying the 40 GHz 3-bit data
      burst; within a triple the signal bump carries +J and each ground bump
      -J/2 (x-directed edges), so the feed sinks its own current;
    * every port has its own seeded jitter (+-20 % amplitude, +-10 % width,
      +-10 ps timing); the two halves of a differential pair are jittered
      independently, so they do not cancel exactly.
    The observation window is 300 ps."""
    from .waveforms import GaussianPulseTrain, Jitter, Ricker, Scaled, Sine
    base = layered_package(nx, ny, seed=seed, nz=nz, n_lines=0)
    mat = base.mat
    z_sub, z_int, z_bump, z_die, routing = _stack(nz)
    rng = np.random.default_rng(seed + 101)
    dx, dy, dz = base.dx, base.dy, base.dz
    sources = []
    port = 0
    # differential pairs: rows j, j + 5 of the top x-running routing layer
    zr = [z for r, z in enumerate(routing) if r % 2 == 0][-1]
    layer = mat[zr] == M_CU
    cand = []
    for j in range(6, ny - 12, 5):
        for i in range(nx // 8, nx - nx // 8):
            if layer[j, i] and layer[j + 5, i]:
                cand.append((i, j))
                break
    pick = rng.choice(len(cand), size=min(n_pairs, len(cand)), replace=False) if cand else []
    for q in sorted(int(x) for x in pick):
        i, j = cand[q]
        for n_side, jj in enumerate((j, j + 5)):
            sign = 1.0 if (n_side + q) % 2 == 0 else -1.0  # alternating polarity along y
            edges = [(i, jj + dj, k) for dj in (0, 1) for k in (zr, zr + 1)]
            j0 = port_current / (dy[jj] * dz[zr])
            sources.append(Source(axis=0, edges=np.array(edges, np.int32),
                                  waveform=Scaled(Ricker(j0, jitter=Jitter.seeded(seed * 7919 + port)), sign)))
            port += 1
    # G-S-G triples on the bump layer, x-directed, 2x2-voxel bumps at 4-voxel pitch
    kb = (z_bump[0] + z_bump[1]) // 2
    bumps = mat[kb] == M_CU
    # bump corners (voxel (i, j) with bump voxels at i, i+1 and j, j+1)
    corners = [(i, j) for j in range(1, ny - 2) for i in range(1, nx - 10)
               if bumps[j, i] and bumps[j + 1, i + 1] and not bumps[j, i - 1] and not bumps[j - 1, i]]
    trip = [(i, j) for (i, j) in corners if bumps[j, i + 4] and bumps[j, i + 8]]
    logic = [t for t in trip if t[1] < ny // 2]
    hbm = [t for t in trip if t[1] >= ny // 2]
    for group, kind in ((logic, "sine"), (hbm, "burst")):
        if not group:
            continue
        sel = rng.choice(len(group), size=min(n_gsg, len(group)), replace=False)
        for q in sorted(int(x) for x in sel):
            i, j = group[q]
            jit = Jitter.seeded(seed * 7919 + port)
            j0 = port_current / (2 * dy[j] * dz[kb])
            if kind == "sine":
                w = Sine(j0, jitter=jit)
            else:
                bits = tuple(int(b) for b in rng.integers(0, 2, 3))
                w = GaussianPulseTrain(j0, bits=bits if any(bits) else (1, 0, 1), jitter=jit)
            for di, share in ((0, -0.5), (4, 1.0), (8, -0.5)):  # ground, signal, ground
                edges = [(i + di + ex, j + ey, kb) for ex in (0, 1) for ey in (0, 1, 2)]
                sources.append(Source(axis=0, edges=np.array(edges, np.int32), waveform=Scaled(w, share)))
            port += 1
    p = replace(base, name=f"paper_setup_{nx}x{ny}x{nz}",
                em_bc=(BC_PMC, BC_PMC, BC_PMC, BC_PMC, BC_PEC, BC_PMC), cpml_cells=0,
                h_conv=(0.0,) * 6, sources=sources, em_steps=0)
    return _check(p)
