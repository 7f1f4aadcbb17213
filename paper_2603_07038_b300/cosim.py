"""Python binding of libcosim: the C-ABI calls under the same names.

Only argument marshalling lives here (ctypes structures, numpy/torch buffer
pointers, the stream and allocator hand-off to PyTorch); every step of the
solver runs in the CUDA library. There is no fallback: if libcosim.so is
missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcosim.so")

# ---- constants (mirror include/cosim.h)
COSIM_OK, COSIM_ERR_INVALID, COSIM_ERR_OOM, COSIM_ERR_CUDA = 0, 1, 2, 3
COSIM_ERR_NOT_CONVERGED, COSIM_ERR_TIMEOUT, COSIM_ERR_NONFINITE = 4, 5, 6
COSIM_FP64, COSIM_FP32 = 0, 1
COSIM_BC_PEC, COSIM_BC_PMC, COSIM_BC_CPML = 0, 1, 2
COSIM_ACCUM_JOULE = 1
COSIM_COUPLED_THERMAL = 2
COSIM_COUPLED_FUSED = 4
COSIM_JOULE_RESET, COSIM_JOULE_FINALIZE_AVG_POWER, COSIM_JOULE_FINALIZE_ENERGY = 0, 1, 2
COSIM_MECH_CLAMPED_BOTTOM, COSIM_MECH_KINEMATIC_MOUNT, COSIM_MECH_MASK = 0, 1, 2
(COSIM_F_EX, COSIM_F_EY, COSIM_F_EZ, COSIM_F_HX, COSIM_F_HY, COSIM_F_HZ, COSIM_F_T, COSIM_F_Q, COSIM_F_P,
 COSIM_F_UX, COSIM_F_UY, COSIM_F_UZ, COSIM_F_VM, COSIM_F_UMAG, COSIM_F_FX, COSIM_F_FY, COSIM_F_FZ,
 COSIM_F_DT, COSIM_F_T_PEAK) = range(19)
COSIM_STRESS_T_CURRENT, COSIM_STRESS_T_PEAK = 0, 1
COSIM_OPT_WAIT_CYCLES = 0
(COSIM_Q_DT_EM, COSIM_Q_DT_TH_LIMIT, COSIM_Q_STEP, COSIM_Q_BYTES_RESIDENT, COSIM_Q_JOULE_STEPS,
 COSIM_Q_N_CELLS, COSIM_Q_N_NODES, COSIM_Q_PRECISION, COSIM_Q_LAUNCHES, COSIM_Q_EM_TILE_Y,
 COSIM_Q_TH_BLOCK_Y) = range(11)

STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT", 6: "NONFINITE"}

EXPORTED = ["cosim_create", "cosim_set_sources", "cosim_em_steps", "cosim_joule_accumulate",
            "cosim_thermal_steps", "cosim_stress_solve", "cosim_stress_apply", "cosim_read_fields",
            "cosim_write_fields", "cosim_query", "cosim_last_error", "cosim_destroy", "cosim_read_fields_async",
            "cosim_wait_reads", "cosim_coupled_march", "cosim_batch_create", "cosim_batch_em_steps",
            "cosim_batch_graph_capture", "cosim_batch_graph_launch", "cosim_batch_last_error", "cosim_batch_destroy",
            "cosim_set_option", "cosim_wait_selftest", "cosim_checkpoint_size", "cosim_checkpoint_save",
            "cosim_checkpoint_load"]


class CosimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cosim {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class cosim_material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eps_r", "mu_r", "sigma0", "tcr", "T0", "k", "rho_cp", "E", "nu",
                                           "alpha_L")]


class cosim_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.POINTER(C.c_double)), ("dy", C.POINTER(C.c_double)), ("dz", C.POINTER(C.c_double)),
                ("mat", C.POINTER(C.c_uint8)), ("nmat", C.c_int32), ("mats", C.POINTER(cosim_material)),
                ("em_bc", C.c_int32 * 6), ("cpml_cells", C.c_int32), ("cpml_order", C.c_double),
                ("cpml_eps_r", C.c_double), ("h_conv", C.c_double * 6), ("T_amb", C.c_double),
                ("T_init", C.c_double)]


class cosim_source(C.Structure):
    _fields_ = [("axis", C.c_int32), ("n_edges", C.c_int32), ("edge_ijk", C.POINTER(C.c_int32)),
                ("nsteps", C.c_int64), ("amp", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class cosim_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class cosim_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("cfl", C.c_double), ("dt_em", C.c_double),
                ("thermal_safety", C.c_double), ("stream", C.c_void_p),
                ("allocator", C.POINTER(cosim_allocator))]


class cosim_stress_opts(C.Structure):
    _fields_ = [("bc", C.c_int32), ("node_mask", C.POINTER(C.c_uint8)), ("T_ref", C.c_double),
                ("rtol", C.c_double), ("maxit", C.c_int64), ("check_every", C.c_int32),
                ("refine", C.c_int32), ("inner_rtol", C.c_double), ("max_refine", C.c_int32),
                ("temperature", C.c_int32)]


class cosim_peak_report(C.Structure):
    _fields_ = [("T_max", C.c_double), ("step", C.c_int64), ("peaks", C.c_int64)]


class cosim_stress_report(C.Structure):
    _fields_ = [("iters", C.c_int64), ("relres", C.c_double), ("seconds", C.c_double),
                ("refine_steps", C.c_int64)]


_lib = None


def load():
    """Load libcosim.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_07038_b300.build.build()")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    P = C.c_void_p
    L.cosim_create.argtypes = [C.POINTER(cosim_grid_desc), C.POINTER(cosim_options), C.POINTER(P)]
    L.cosim_create.restype = st
    L.cosim_set_sources.argtypes = [P, C.c_int32, C.POINTER(cosim_source)]
    L.cosim_set_sources.restype = st
    L.cosim_em_steps.argtypes = [P, C.c_int64, C.c_uint32]
    L.cosim_em_steps.restype = st
    L.cosim_coupled_march.argtypes = [P, C.c_int64, C.c_uint32, C.c_int64, C.c_int32, C.POINTER(cosim_peak_report)]
    L.cosim_coupled_march.restype = st
    L.cosim_em_graph_capture.argtypes = [P, C.c_int64, C.c_uint32]
    L.cosim_em_graph_capture.restype = st
    L.cosim_em_graph_launch.argtypes = [P, C.c_int64]
    L.cosim_em_graph_launch.restype = st
    L.cosim_autotune.argtypes = [P, C.c_uint32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.cosim_autotune.restype = st
    L.cosim_joule_accumulate.argtypes = [P, C.c_int32, C.POINTER(C.c_double)]
    L.cosim_joule_accumulate.restype = st
    L.cosim_thermal_steps.argtypes = [P, C.c_int64, C.c_double]
    L.cosim_thermal_steps.restype = st
    L.cosim_stress_solve.argtypes = [P, C.POINTER(cosim_stress_opts), C.POINTER(cosim_stress_report)]
    L.cosim_stress_solve.restype = st
    L.cosim_stress_apply.argtypes = [P, C.POINTER(cosim_stress_opts), P, P, C.c_int32]
    L.cosim_stress_apply.restype = st
    L.cosim_read_fields.argtypes = [P, C.c_int32, C.c_int32, P, C.c_size_t, C.c_int32]
    L.cosim_read_fields.restype = st
    L.cosim_write_fields.argtypes = [P, C.c_int32, C.c_int32, P, C.c_size_t, C.c_int32]
    L.cosim_write_fields.restype = st
    L.cosim_read_fields_async.argtypes = [P, C.c_int32, C.c_int32, P, C.c_size_t, C.c_int32]
    L.cosim_read_fields_async.restype = st
    L.cosim_wait_reads.argtypes = [P]
    L.cosim_wait_reads.restype = st
    L.cosim_query.argtypes = [P, C.c_int32, C.POINTER(C.c_double)]
    L.cosim_query.restype = st
    L.cosim_last_error.argtypes = [P]
    L.cosim_last_error.restype = C.c_char_p
    L.cosim_destroy.argtypes = [P]
    L.cosim_destroy.restype = None
    L.cosim_batch_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.POINTER(P)]
    L.cosim_batch_create.restype = st
    L.cosim_batch_em_steps.argtypes = [P, C.c_int64, C.c_uint32]
    L.cosim_batch_em_steps.restype = st
    L.cosim_batch_graph_capture.argtypes = [P, C.c_int64, C.c_uint32]
    L.cosim_batch_graph_capture.restype = st
    L.cosim_batch_graph_launch.argtypes = [P, C.c_int64]
    L.cosim_batch_graph_launch.restype = st
    L.cosim_batch_last_error.argtypes = [P]
    L.cosim_batch_last_error.restype = C.c_char_p
    L.cosim_batch_destroy.argtypes = [P]
    L.cosim_batch_destroy.restype = None
    L.cosim_set_option.argtypes = [P, C.c_int32, C.c_double]
    L.cosim_set_option.restype = st
    L.cosim_wait_selftest.argtypes = [P]
    L.cosim_wait_selftest.restype = st
    L.cosim_checkpoint_size.argtypes = [P, C.POINTER(C.c_size_t)]
    L.cosim_checkpoint_size.restype = st
    L.cosim_checkpoint_save.argtypes = [P, P, C.c_size_t, C.c_int32]
    L.cosim_checkpoint_save.restype = st
    L.cosim_checkpoint_load.argtypes = [P, P, C.c_size_t, C.c_int32]
    L.cosim_checkpoint_load.restype = st
    L.cosim_sum_f64_noalloc.argtypes = [P, C.c_int64, P, C.c_int32, P]
    L.cosim_sum_f64_noalloc.restype = st
    _lib = L
    return L


def _check(status, ctx=None):
    if status != COSIM_OK:
        msg = load().cosim_last_error(ctx)
        raise CosimError(status, msg.decode() if msg else "")


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- marshalling

class Desc:
    """cosim_grid_desc built from a problem description (keeps buffers alive)."""

    def __init__(self, problem):
        p = problem
        self._h = [np.ascontiguousarray(p.dx, np.float64), np.ascontiguousarray(p.dy, np.float64),
                   np.ascontiguousarray(p.dz, np.float64)]
        self._mat = np.ascontiguousarray(p.mat, np.uint8).reshape(-1)
        rows = [m.as_row() for m in p.materials]
        self._mats = (cosim_material * len(rows))(*[cosim_material(*r) for r in rows])
        d = cosim_grid_desc()
        d.nx, d.ny, d.nz = p.nx, p.ny, p.nz
        d.dx, d.dy, d.dz = (_dp(a) for a in self._h)
        d.mat = self._mat.ctypes.data_as(C.POINTER(C.c_uint8))
        d.nmat = len(rows)
        d.mats = self._mats
        for f in range(6):
            d.em_bc[f] = int(p.em_bc[f])
            d.h_conv[f] = float(p.h_conv[f])
        d.cpml_cells = int(p.cpml_cells)
        d.cpml_order = float(p.cpml_order)
        d.cpml_eps_r = float(p.cpml_eps_r)
        d.T_amb = float(p.T_amb)
        d.T_init = float(p.T_init)
        self.c = d


class TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)
        self.c = cosim_allocator(self._alloc, self._free, None)

    def _a(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _f(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


def cosim_create(problem, precision=COSIM_FP32, cfl=0.99, dt_em=0.0, thermal_safety=0.9, stream=None,
                 allocator=None):
    """-> (ctx handle, keep-alive tuple). stream: a torch.cuda.Stream, an int handle, or None."""
    L = load()
    desc = Desc(problem)
    o = cosim_options()
    o.precision = precision
    o.cfl = cfl
    o.dt_em = dt_em
    o.thermal_safety = thermal_safety
    if stream is not None:
        o.stream = stream if isinstance(stream, int) else stream.cuda_stream
    if allocator is not None:
        o.allocator = C.pointer(allocator.c)
    h = C.c_void_p()
    _check(L.cosim_create(C.byref(desc.c), C.byref(o), C.byref(h)), None)
    return h, (desc, allocator)


def cosim_set_sources(ctx, tables):
    """tables: [(axis, edges int32 (n,3), amp float64 (nsteps,)), ...]"""
    keep = []
    arr = (cosim_source * max(1, len(tables)))()
    for q, (axis, edges, amp) in enumerate(tables):
        e = np.ascontiguousarray(edges, np.int32).reshape(-1)
        a = np.ascontiguousarray(amp, np.float64)
        keep += [e, a]
        arr[q] = cosim_source(int(axis), len(e) // 3, e.ctypes.data_as(C.POINTER(C.c_int32)), len(a), _dp(a))
    _check(load().cosim_set_sources(ctx, len(tables), arr), ctx)


def cosim_em_steps(ctx, nsteps, flags=COSIM_ACCUM_JOULE):
    _check(load().cosim_em_steps(ctx, int(nsteps), int(flags)), ctx)


def cosim_em_graph_capture(ctx, nsteps, flags=COSIM_ACCUM_JOULE):
    _check(load().cosim_em_graph_capture(ctx, int(nsteps), int(flags)), ctx)


def cosim_em_graph_launch(ctx, count=1):
    _check(load().cosim_em_graph_launch(ctx, int(count)), ctx)


COSIM_TUNE_FORCE, COSIM_TUNE_FIXED = 1, 2


def cosim_autotune(ctx, force=False, fixed=None):
    """-> (EM tile height, thermal block height). fixed=(ty, by) sets them without timing."""
    ty, by = C.c_int32(fixed[0] if fixed else 0), C.c_int32(fixed[1] if fixed else 0)
    flags = (COSIM_TUNE_FORCE if force else 0) | (COSIM_TUNE_FIXED if fixed else 0)
    _check(load().cosim_autotune(ctx, flags, C.byref(ty), C.byref(by)), ctx)
    return ty.value, by.value


def cosim_joule_accumulate(ctx, op, want_total=True):
    t = C.c_double(0.0)
    _check(load().cosim_joule_accumulate(ctx, int(op), C.byref(t) if want_total else None), ctx)
    return t.value


def cosim_thermal_steps(ctx, nsteps, dt=0.0):
    _check(load().cosim_thermal_steps(ctx, int(nsteps), float(dt)), ctx)


def _stress_opts(bc, node_mask, T_ref, rtol, maxit, check_every):
    o = cosim_stress_opts()
    o.bc = bc
    o.T_ref = T_ref
    o.rtol = rtol
    o.maxit = maxit
    o.check_every = check_every
    keep = None
    if node_mask is not None:
        keep = np.ascontiguousarray(node_mask, np.uint8)
        o.node_mask = keep.ctypes.data_as(C.POINTER(C.c_uint8))
    return o, keep


def cosim_stress_solve(ctx, bc=COSIM_MECH_CLAMPED_BOTTOM, node_mask=None, T_ref=300.0, rtol=1e-9,
                       maxit=200000, check_every=32, allow_not_converged=False, refine=False, inner_rtol=0.0,
                       max_refine=0, temperature=COSIM_STRESS_T_CURRENT):
    """temperature: COSIM_STRESS_T_CURRENT (the current field) or
    COSIM_STRESS_T_PEAK (the peak snapshot of cosim_coupled_march)."""
    o, keep = _stress_opts(bc, node_mask, T_ref, rtol, maxit, check_every)
    o.temperature = temperature
    o.refine = 1 if refine else 0
    o.inner_rtol = inner_rtol
    o.max_refine = max_refine
    rep = cosim_stress_report()
    st = load().cosim_stress_solve(ctx, C.byref(o), C.byref(rep))
    if not (allow_not_converged and st == COSIM_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return dict(iters=rep.iters, relres=rep.relres, seconds=rep.seconds, status=st,
                refine_steps=rep.refine_steps)


def cosim_coupled_march(ctx, nsteps, check_every=1, accumulate_joule=True, reset=False, fused=False):
    """nsteps synchronized electro-thermal steps with peak-temperature
    snapshots every check_every steps; returns the peak report as a dict."""
    r = cosim_peak_report()
    flags = (COSIM_ACCUM_JOULE if accumulate_joule else 0) | (COSIM_COUPLED_FUSED if fused else 0)
    _check(load().cosim_coupled_march(ctx, int(nsteps), flags, int(check_every), 1 if reset else 0, C.byref(r)), ctx)
    return dict(T_max=r.T_max, step=r.step, peaks=r.peaks)


def cosim_set_option(ctx, what, value):
    _check(load().cosim_set_option(ctx, int(what), float(value)), ctx)


def cosim_wait_selftest(ctx):
    """the status of the bounded-wait health check (COSIM_ERR_TIMEOUT when the
    timeout path works)"""
    return load().cosim_wait_selftest(ctx)


def cosim_checkpoint_save(ctx, dst=None):
    """the checkpoint blob: into a new host uint8 array (dst None) or into a
    CUDA uint8 tensor of the right size"""
    n = C.c_size_t()
    _check(load().cosim_checkpoint_size(ctx, C.byref(n)), ctx)
    if dst is None:
        out = np.empty(n.value, np.uint8)
        _check(load().cosim_checkpoint_save(ctx, out.ctypes.data, n.value, 0), ctx)
        return out
    if dst.numel() != n.value or not dst.is_cuda or not dst.is_contiguous():
        raise ValueError(f"dst must be a contiguous CUDA tensor of {n.value} bytes")
    _check(load().cosim_checkpoint_save(ctx, dst.data_ptr(), n.value, 1), ctx)
    return dst


def cosim_checkpoint_load(ctx, blob):
    if isinstance(blob, np.ndarray):
        b = np.ascontiguousarray(blob, np.uint8)
        _check(load().cosim_checkpoint_load(ctx, b.ctypes.data, b.nbytes, 0), ctx)
    else:
        if not blob.is_cuda or not blob.is_contiguous():
            raise ValueError("blob must be a host array or a contiguous CUDA tensor")
        _check(load().cosim_checkpoint_load(ctx, blob.data_ptr(), blob.numel() * blob.element_size(), 1), ctx)


def cosim_stress_apply(ctx, u, bc=COSIM_MECH_CLAMPED_BOTTOM, node_mask=None):
    """u: (3, n_nodes) array of the context precision (numpy: host, torch CUDA: device) -> K u."""
    o, keep = _stress_opts(bc, node_mask, 300.0, 0.0, 0, 0)
    if isinstance(u, np.ndarray):
        uu = np.ascontiguousarray(u)
        y = np.empty_like(uu)
        _check(load().cosim_stress_apply(ctx, C.byref(o), uu.ctypes.data, y.ctypes.data, 0), ctx)
        return y
    y = u.new_empty(u.shape)
    _check(load().cosim_stress_apply(ctx, C.byref(o), u.contiguous().data_ptr(), y.data_ptr(), 1), ctx)
    return y


def cosim_read_fields(ctx, field, dst):
    """dst: numpy float64/float32 array (host) or a torch CUDA tensor (device)."""
    if isinstance(dst, np.ndarray):
        assert dst.flags.c_contiguous
        dt = COSIM_FP64 if dst.dtype == np.float64 else COSIM_FP32
        _check(load().cosim_read_fields(ctx, field, dt, dst.ctypes.data, dst.nbytes, 0), ctx)
    else:
        import torch
        assert dst.is_cuda and dst.is_contiguous()
        dt = COSIM_FP64 if dst.dtype == torch.float64 else COSIM_FP32
        _check(load().cosim_read_fields(ctx, field, dt, dst.data_ptr(), dst.numel() * dst.element_size(), 1), ctx)
    return dst


def cosim_read_fields_async(ctx, field, dst):
    """Start reading a field into dst (pinned numpy array or torch CUDA tensor);
    dst is filled once cosim_wait_reads(ctx) returns."""
    if isinstance(dst, np.ndarray):
        assert dst.flags.c_contiguous
        dt = COSIM_FP64 if dst.dtype == np.float64 else COSIM_FP32
        _check(load().cosim_read_fields_async(ctx, field, dt, dst.ctypes.data, dst.nbytes, 0), ctx)
    else:
        import torch
        assert dst.is_cuda and dst.is_contiguous()
        dt = COSIM_FP64 if dst.dtype == torch.float64 else COSIM_FP32
        _check(load().cosim_read_fields_async(ctx, field, dt, dst.data_ptr(), dst.numel() * dst.element_size(), 1),
               ctx)
    return dst


def cosim_wait_reads(ctx):
    _check(load().cosim_wait_reads(ctx), ctx)


def cosim_write_fields(ctx, field, src):
    if isinstance(src, np.ndarray):
        s = np.ascontiguousarray(src)
        dt = COSIM_FP64 if s.dtype == np.float64 else COSIM_FP32
        _check(load().cosim_write_fields(ctx, field, dt, s.ctypes.data, s.nbytes, 0), ctx)
    else:
        import torch
        s = src.contiguous()
        dt = COSIM_FP64 if s.dtype == torch.float64 else COSIM_FP32
        _check(load().cosim_write_fields(ctx, field, dt, s.data_ptr(), s.numel() * s.element_size(), 1), ctx)


def cosim_query(ctx, what):
    v = C.c_double()
    _check(load().cosim_query(ctx, what, C.byref(v)), ctx)
    return v.value


def cosim_last_error(ctx=None):
    m = load().cosim_last_error(ctx)
    return m.decode() if m else ""


def cosim_destroy(ctx):
    if ctx:
        load().cosim_destroy(ctx)


def cosim_sum_f64_noalloc(x, n=None, out=None, stream=None):
    """Sum of the first n elements of a CUDA float64 tensor without any device
    allocation by the library.

    x must be a contiguous float64 CUDA tensor and 0 <= n <= x.numel() (n
    defaults to x.numel()); out is None (the sum is returned as a Python float
    through host memory) or a float64 CUDA tensor on x's device that receives
    the sum in its first element. The call runs on x's device and is ordered on
    `stream`, by default the caller's current torch stream of that device, so
    it sees the work already queued there. Every check runs before the library
    is called: a tensor of another dtype, a strided view or an n beyond the
    tensor would make the kernel read outside the caller's buffer."""
    import torch

    if x.dtype != torch.float64:
        raise TypeError(f"cosim_sum_f64_noalloc: x must be float64, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError("cosim_sum_f64_noalloc: x must be contiguous")
    n = x.numel() if n is None else int(n)
    if not 0 <= n <= x.numel():
        raise ValueError(f"cosim_sum_f64_noalloc: n = {n} outside [0, {x.numel()}]")
    if not x.is_cuda:
        raise ValueError("cosim_sum_f64_noalloc: x must be a CUDA tensor")
    if out is not None:
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
            raise ValueError("cosim_sum_f64_noalloc: out must be a float64 CUDA tensor with at least one element")
        if out.device != x.device:
            raise ValueError("cosim_sum_f64_noalloc: out must be on x's device")
    with torch.cuda.device(x.device):
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        s = stream if isinstance(stream, int) else stream.cuda_stream
        if out is None:
            v = C.c_double()
            _check(load().cosim_sum_f64_noalloc(x.data_ptr(), n, C.addressof(v), 0, s), None)
            return v.value
        _check(load().cosim_sum_f64_noalloc(x.data_ptr(), n, out.data_ptr(), 1, s), None)
        return out


def _bcheck(status, b):
    if status != COSIM_OK:
        m = load().cosim_batch_last_error(b)
        raise CosimError(status, m.decode() if m else "")


class Batch:
    """A batch of contexts stepped together (cosim_batch_*): one launch per EM
    step over the tiles of every design. The contexts must share one stream
    and precision and have their sources set; they stay owned by the caller."""

    def __init__(self, contexts, persistent=True):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h for c in self.contexts])
        h = C.c_void_p()
        _bcheck(load().cosim_batch_create(arr, len(self.contexts), 1 if persistent else 0, C.byref(h)), None)
        self.h = h

    def em_steps(self, n, accumulate_joule=True):
        _bcheck(load().cosim_batch_em_steps(self.h, int(n), COSIM_ACCUM_JOULE if accumulate_joule else 0), self.h)

    def graph_capture(self, n, accumulate_joule=True):
        _bcheck(load().cosim_batch_graph_capture(self.h, int(n), COSIM_ACCUM_JOULE if accumulate_joule else 0),
                self.h)

    def graph_launch(self, count=1):
        _bcheck(load().cosim_batch_graph_launch(self.h, int(count)), self.h)

    def close(self):
        if self.h:
            load().cosim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience

class Context:
    """Owns one cosim context; methods are the C-ABI calls with the handle bound."""

    def __init__(self, problem, precision=COSIM_FP32, cfl=0.99, dt_em=0.0, thermal_safety=0.9, stream=None,
                 use_torch_allocator=False):
        self.problem = problem
        alloc = TorchAllocator(stream=stream) if use_torch_allocator else None
        self.h, self._keep = cosim_create(problem, precision, cfl, dt_em, thermal_safety, stream, alloc)
        self.precision = precision
        self.nx, self.ny, self.nz = problem.nx, problem.ny, problem.nz
        self.n_nodes = (self.nx + 1) * (self.ny + 1) * (self.nz + 1)
        self.n_cells = self.nx * self.ny * self.nz
        self.dt = cosim_query(self.h, COSIM_Q_DT_EM)

    @property
    def node_shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    def set_sources(self, tables):
        cosim_set_sources(self.h, tables)

    def em_steps(self, n, accumulate_joule=True, coupled=False, fused=False):
        """coupled: the synchronized electro-thermal marching (sigma(T), a
        thermal step with the EM dt after every EM step); fused: that thermal
        step inside the EM launch."""
        cosim_em_steps(self.h, n, (COSIM_ACCUM_JOULE if accumulate_joule else 0)
                       | (COSIM_COUPLED_THERMAL if coupled else 0) | (COSIM_COUPLED_FUSED if fused else 0))

    def coupled_march(self, n, check_every=1, accumulate_joule=True, reset=False, fused=False):
        return cosim_coupled_march(self.h, n, check_every, accumulate_joule, reset, fused)

    def em_graph_capture(self, n, accumulate_joule=True, coupled=False, fused=False):
        cosim_em_graph_capture(self.h, n, (COSIM_ACCUM_JOULE if accumulate_joule else 0)
                               | (COSIM_COUPLED_THERMAL if coupled else 0) | (COSIM_COUPLED_FUSED if fused else 0))

    def checkpoint(self, dst=None):
        return cosim_checkpoint_save(self.h, dst)

    def restore(self, blob):
        cosim_checkpoint_load(self.h, blob)

    def set_option(self, what, value):
        cosim_set_option(self.h, what, value)

    def em_graph_launch(self, count=1):
        cosim_em_graph_launch(self.h, count)

    def autotune(self, force=False, fixed=None):
        return cosim_autotune(self.h, force, fixed)

    def joule(self, op, want_total=True):
        return cosim_joule_accumulate(self.h, op, want_total)

    def thermal_steps(self, n, dt=0.0):
        cosim_thermal_steps(self.h, n, dt)

    def stress_solve(self, **kw):
        return cosim_stress_solve(self.h, **kw)

    def stress_apply(self, u, **kw):
        return cosim_stress_apply(self.h, u, **kw)

    def read(self, field, dtype=np.float64):
        n = self.n_cells if field == COSIM_F_VM else self.n_nodes
        return cosim_read_fields(self.h, field, np.empty(n, dtype))

    def write(self, field, values):
        cosim_write_fields(self.h, field, values)

    def query(self, what):
        return cosim_query(self.h, what)

    def close(self):
        if self.h:
            cosim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
