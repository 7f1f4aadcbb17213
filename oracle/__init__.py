"""FP64 CPU oracle of the coupled EM-thermal-mechanical package solver.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The
product path (``paper_2603_07038_b300``) never imports it, and it shares no
code with the CUDA sources: the arithmetic lives in plain C loops in
``cosim_oracle.c`` (built with ``-ffp-contract=off``), this module only owns
the numpy state and orders the steps the way the paper does:

  EM (Sec. II-A, Eqs. 1-3): H half-step, then E step with sigma, eps and the
  source current J, then (optionally) Joule heat P = D_sigma e^2 of the step;
  thermal (Eqs. 4-5): forward-Euler nodal steps driven by the Joule source;
  mechanics (Sec. II-B, Eqs. 7-9): HEX8 thermal load, Jacobi-PCG, von Mises.

Parity status of each function is recorded with the pins in tests/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cosim_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_cosim_oracle.so")
_lib = None

PEC, PMC, CPML = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OgGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.POINTER(C.c_double) * 3),
                ("mat", C.POINTER(C.c_uint8)), ("nmat", C.c_int), ("tab", C.POINTER(C.c_double)),
                ("em_bc", C.c_int * 6), ("cpml_cells", C.c_int), ("cpml_order", C.c_double),
                ("cpml_eps_r", C.c_double), ("h_conv", C.c_double * 6), ("T_amb", C.c_double)]


_P = np.ctypeslib.ndpointer


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        G = C.POINTER(OgGrid)
        d = C.c_double
        dp = C.POINTER(C.c_double)
        pp3 = dp * 3
        u8 = C.POINTER(C.c_uint8)
        L.og_cfl_dt.argtypes = [G, d]
        L.og_cfl_dt.restype = d
        L.og_cpml_table.argtypes = [G, C.c_int, C.c_int, d, dp, dp]
        L.og_h_update.argtypes = [G, d, pp3, pp3, dp]
        L.og_e_update.argtypes = [G, d, pp3, pp3, dp, C.c_void_p]
        L.og_joule_accumulate.argtypes = [G, d, pp3, pp3, dp]
        L.og_count_dofs.argtypes = [G, C.POINTER(C.c_int64)] + [C.POINTER(C.c_int64)] * 2
        L.og_thermal_dt_limit.argtypes = [G]
        L.og_thermal_dt_limit.restype = d
        L.og_thermal_step.argtypes = [G, d, dp, dp, dp]
        L.og_node_capacity.argtypes = [G, dp]
        L.og_hex8_element.argtypes = [dp, dp, dp]
        L.og_hex8_matvec.argtypes = [G, u8, dp, dp]
        L.og_hex8_diag.argtypes = [G, u8, dp]
        L.og_thermal_load.argtypes = [G, u8, dp, d, dp]
        L.og_pcg.argtypes = [G, u8, dp, dp, d, C.c_int64, C.POINTER(C.c_int64), dp]
        L.og_von_mises.argtypes = [G, dp, dp, d, dp, dp]
        L.og_joule_power_T.argtypes = [G, pp3, pp3, dp, d, dp]
        L.og_coupled_step.argtypes = [G, d, pp3, pp3, dp, C.c_void_p, dp, d, dp, dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _p3(arrs):
    return (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in arrs])


class Grid:
    """ctypes view of a workloads.Problem (keeps the numpy buffers alive)."""

    def __init__(self, p):
        self.p = p
        self.nx, self.ny, self.nz = p.nx, p.ny, p.nz
        self._h = [np.ascontiguousarray(p.dx, np.float64), np.ascontiguousarray(p.dy, np.float64),
                   np.ascontiguousarray(p.dz, np.float64)]
        self._mat = np.ascontiguousarray(p.mat, np.uint8)
        self._tab = np.ascontiguousarray(p.material_table(), np.float64)
        g = OgGrid()
        g.nx, g.ny, g.nz = p.nx, p.ny, p.nz
        for a in range(3):
            g.h[a] = _dp(self._h[a])
        g.mat = _u8(self._mat.reshape(-1))
        g.nmat = len(p.materials)
        g.tab = _dp(self._tab.reshape(-1))
        for f in range(6):
            g.em_bc[f] = int(p.em_bc[f])
            g.h_conv[f] = float(p.h_conv[f])
        g.cpml_cells = int(p.cpml_cells)
        g.cpml_order = float(p.cpml_order)
        g.cpml_eps_r = float(p.cpml_eps_r)
        # temperatures are handled as the rise over T_init (Eq. 5 is unchanged by
        # a constant shift of T and T_amb); this keeps FP64 resolution on rises
        # far below the absolute temperature
        g.T_amb = float(p.T_amb) - float(p.T_init)
        self.T0 = float(p.T_init)
        self.g = g
        self.ref = C.byref(g)

    @property
    def n_nodes(self):
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def node_shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    def nid(self, i, j, k):
        return (np.asarray(k) * (self.ny + 1) + np.asarray(j)) * (self.nx + 1) + np.asarray(i)


def cfl_dt(p, cfl: float = 0.99) -> float:
    g = Grid(p)
    return lib().og_cfl_dt(g.ref, cfl)


def count_dofs(p):
    g = Grid(p)
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    lib().og_count_dofs(g.ref, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def hex8_element(hx, hy, hz):
    """(Kl, Km) 24x24 with K_e = lambda*Kl + mu*Km; DOF = 3*local_node + comp,
    local node a = ax + 2 ay + 4 az."""
    hh = np.array([hx, hy, hz], np.float64)
    Kl = np.zeros(576)
    Km = np.zeros(576)
    lib().og_hex8_element(_dp(hh), _dp(Kl), _dp(Km))
    return Kl.reshape(24, 24), Km.reshape(24, 24)


class OracleSim:
    """State and step ordering of the co-simulation, FP64, host memory.

    E[a], H[a], Q (Joule energy per node, J), T and displacement are node-sized
    flat arrays (x fastest); see cosim_oracle.c for which entries are used.
    """

    def __init__(self, p, dt: float | None = None, cfl: float = 0.99):
        self.p = p
        self.g = Grid(p)
        L = lib()
        self.dt = L.og_cfl_dt(self.g.ref, cfl) if dt is None else float(dt)
        nn = self.g.n_nodes
        self.E = [np.zeros(nn) for _ in range(3)]
        self.H = [np.zeros(nn) for _ in range(3)]
        self.psi = np.zeros(12 * nn) if CPML in p.em_bc else None
        self.Q = np.zeros(nn)
        self.P = np.zeros(nn)
        self.theta = np.zeros(nn)  # T - T_init
        self.T0 = float(p.T_init)
        self.step = 0
        self.n_acc = 0
        self._src = []
        self._amp_len = 0

    # --- sources -----------------------------------------------------------
    def set_sources(self, tables):
        """tables: [(axis, edges (n,3) int32, amp float64[nsteps]), ...]"""
        self._src = [(int(a), np.asarray(e, np.int64).reshape(-1, 3), np.asarray(v, np.float64))
                     for a, e, v in tables]

    def _J(self, n):
        if not self._src:
            return None
        J = [np.zeros(self.g.n_nodes) for _ in range(3)]
        for axis, edges, amp in self._src:
            if n < len(amp):
                ids = self.g.nid(edges[:, 0], edges[:, 1], edges[:, 2])
                np.add.at(J[axis], ids, amp[n])
        return J

    # --- EM ------------------------------------------------------------------
    def h_half_step(self):
        """H^{n-1/2} -> H^{n+1/2} from E^n."""
        psi = _dp(self.psi) if self.psi is not None else None
        lib().og_h_update(self.g.ref, self.dt, _p3(self.E), _p3(self.H), psi)

    def e_step(self, accumulate_joule: bool = True):
        """E^n -> E^{n+1} from H^{n+1/2} and J^{n+1/2}; Joule heat of the step."""
        L = lib()
        psi = _dp(self.psi) if self.psi is not None else None
        Eold = [e.copy() for e in self.E] if accumulate_joule else None
        J = self._J(self.step)
        L.og_e_update(self.g.ref, self.dt, _p3(self.H), _p3(self.E), psi,
                      C.cast(_p3(J), C.c_void_p) if J is not None else None)
        if accumulate_joule:
            L.og_joule_accumulate(self.g.ref, self.dt, _p3(Eold), _p3(self.E), _dp(self.Q))
            self.n_acc += 1
        self.step += 1

    def em_step(self, accumulate_joule: bool = True):
        self.h_half_step()
        self.e_step(accumulate_joule)

    def joule_of(self, Eold, Enew) -> np.ndarray:
        """Joule energy per node of one step with the given old/new edge fields."""
        Q = np.zeros(self.g.n_nodes)
        lib().og_joule_accumulate(self.g.ref, self.dt, _p3([np.ascontiguousarray(e) for e in Eold]),
                                  _p3([np.ascontiguousarray(e) for e in Enew]), _dp(Q))
        return Q

    def em_steps(self, n: int, accumulate_joule: bool = True):
        for _ in range(n):
            self.em_step(accumulate_joule)

    # --- two-way electro-thermal coupling (Sec. II-A) ------------------------
    def joule_power_T(self, Eold, Enew, theta=None) -> np.ndarray:
        """Joule power per node [W] of one step with the conductivities at the
        temperature theta + T_init (theta defaults to the current rise)."""
        P = np.zeros(self.g.n_nodes)
        th = self.theta if theta is None else np.ascontiguousarray(theta, np.float64)
        lib().og_joule_power_T(self.g.ref, _p3([np.ascontiguousarray(e) for e in Eold]),
                               _p3([np.ascontiguousarray(e) for e in Enew]), _dp(th), self.T0, _dp(P))
        return P

    def coupled_steps(self, n: int, accumulate_joule: bool = True):
        """n synchronized steps: sigma(T^n), H and E, P^{n+1}, thermal step at
        the EM dt (og_coupled_step). self.P holds the last step's power."""
        L = lib()
        psi = _dp(self.psi) if self.psi is not None else None
        th = np.ascontiguousarray(self.theta, np.float64).copy()
        th2 = np.empty_like(th)
        for _ in range(n):
            J = self._J(self.step)
            L.og_coupled_step(self.g.ref, self.dt, _p3(self.E), _p3(self.H), psi,
                              C.cast(_p3(J), C.c_void_p) if J is not None else None,
                              _dp(th), self.T0, _dp(self.P), _dp(th2), _dp(self.Q) if accumulate_joule else None)
            th, th2 = th2, th
            self.step += 1
            if accumulate_joule:
                self.n_acc += 1
        self.theta = th

    def joule_reset(self):
        self.Q[:] = 0.0
        self.n_acc = 0

    def joule_finalize_avg_power(self) -> float:
        """Burst-averaged Joule power per node [W] becomes the thermal source."""
        if self.n_acc > 0:
            self.P = self.Q / (self.n_acc * self.dt)
        return float(self.Q.sum())

    def joule_finalize_energy(self) -> float:
        """Deposit the burst's Joule energy as an instantaneous temperature rise."""
        C_node = self.capacity()
        self.theta = self.theta + self.Q / C_node
        return float(self.Q.sum())

    @property
    def T(self):
        """absolute temperature [K] (a copy; assign to set)"""
        return self.theta + self.T0

    @T.setter
    def T(self, values):
        self.theta = np.asarray(values, np.float64) - self.T0

    # --- thermal -------------------------------------------------------------
    def capacity(self):
        c = np.zeros(self.g.n_nodes)
        lib().og_node_capacity(self.g.ref, _dp(c))
        return c

    def thermal_dt_limit(self) -> float:
        return lib().og_thermal_dt_limit(self.g.ref)

    def thermal_steps(self, n: int, dt: float | None = None, safety: float = 0.9, source=True):
        dt = safety * self.thermal_dt_limit() if not dt else float(dt)
        L = lib()
        th = np.ascontiguousarray(self.theta, np.float64).copy()
        T2 = np.empty_like(th)
        P = _dp(self.P) if source else None
        for _ in range(n):
            L.og_thermal_step(self.g.ref, dt, _dp(th), P, _dp(T2))
            th, T2 = T2, th
        self.theta = th
        return dt

    # --- mechanics -----------------------------------------------------------
    def matvec(self, fixed: np.ndarray, u: np.ndarray) -> np.ndarray:
        y = np.zeros(3 * self.g.n_nodes)
        lib().og_hex8_matvec(self.g.ref, _u8(fixed), _dp(np.ascontiguousarray(u, np.float64)), _dp(y))
        return y

    def diag(self, fixed):
        d = np.zeros(3 * self.g.n_nodes)
        lib().og_hex8_diag(self.g.ref, _u8(fixed), _dp(d))
        return d

    def _rise(self, T):
        return self.theta if T is None else np.ascontiguousarray(np.asarray(T, np.float64) - self.T0)

    def thermal_load(self, fixed, T_ref, T=None):
        f = np.zeros(3 * self.g.n_nodes)
        lib().og_thermal_load(self.g.ref, _u8(fixed), _dp(self._rise(T)), float(T_ref) - self.T0, _dp(f))
        return f

    def pcg(self, fixed, f, rtol=1e-13, maxit=100000):
        u = np.zeros(3 * self.g.n_nodes)
        it = C.c_int64()
        rr = C.c_double()
        lib().og_pcg(self.g.ref, _u8(fixed), _dp(np.ascontiguousarray(f)), _dp(u), float(rtol), int(maxit),
                     C.byref(it), C.byref(rr))
        return u, it.value, rr.value

    def von_mises(self, u, T_ref, T=None):
        vm = np.zeros(self.p.n_cells)
        um = np.zeros(self.g.n_nodes)
        lib().og_von_mises(self.g.ref, _dp(np.ascontiguousarray(u)), _dp(self._rise(T)), float(T_ref) - self.T0,
                           _dp(vm), _dp(um))
        return vm, um

    def stress_solve(self, fixed, T_ref, rtol=1e-13, maxit=100000):
        f = self.thermal_load(fixed, T_ref)
        u, it, rr = self.pcg(fixed, f, rtol, maxit)
        vm, um = self.von_mises(u, T_ref)
        return dict(u=u, iters=it, relres=rr, vm=vm, umag=um, f=f)
