"""Failure detection and recovery in the forms that fault no GPU:
* a bounded in-kernel wait that cannot complete (a barrier phase that nothing
  completes, with a short bound) reports COSIM_ERR_TIMEOUT and leaves the
  context usable;
* an allocation failure injected through the cosim_allocator hook reports
  COSIM_ERR_OOM: at creation (every block handed out is returned) and at the
  lazy mechanics allocation (the context stays valid and later succeeds);
* a checkpoint of the marching state (E, H, CPML auxiliaries, Joule window and
  total, temperature, source time index) restored into a fresh context
  continues bit for bit."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from paper_2603_07038_b300 import cosim as api
from paper_2603_07038_b300.build import build

pytestmark = pytest.mark.gpu


def test_wait_bound_runs_out_and_context_stays_usable():
    build()
    p = W.tiny_package()
    ctx = api.Context(p, precision=api.COSIM_FP32)
    ctx.set_sources(p.source_tables(ctx.dt, 64))
    ctx.set_option(api.COSIM_OPT_WAIT_CYCLES, 2e5)  # ~0.1 ms at 2 GHz
    for _ in range(2):
        assert api.cosim_wait_selftest(ctx.h) == api.COSIM_ERR_TIMEOUT
        assert "wait" in api.cosim_last_error(ctx.h)
    ctx.set_option(api.COSIM_OPT_WAIT_CYCLES, 2.0 ** 31)
    ctx.em_steps(64)  # the context still steps and reads
    ez = ctx.read(api.COSIM_F_EZ)
    assert np.isfinite(ez).all() and np.abs(ez).max() > 0
    with pytest.raises(api.CosimError):
        ctx.set_option(api.COSIM_OPT_WAIT_CYCLES, 10.0)  # below the allowed bound
    ctx.close()


class FlakyAllocator:
    """An allocator (PyTorch's caching allocator underneath) that refuses on
    demand and keeps the blocks it handed out."""

    def __init__(self, fail_after=None):
        self.fail_after = fail_after
        self.live = {}
        self.n = 0
        self.refuse = False
        self._alloc = api.ALLOC_FN(self._a)
        self._free = api.FREE_FN(self._f)
        self.c = api.cosim_allocator(self._alloc, self._free, None)

    def _a(self, nbytes, user):
        self.n += 1
        if self.refuse or (self.fail_after is not None and self.n > self.fail_after):
            return None
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
        except Exception:
            return None
        self.live[ptr] = nbytes
        return ptr

    def _f(self, ptr, user):
        assert ptr in self.live
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def test_allocation_failure_at_create_returns_every_block():
    build()
    p = W.tiny_package()
    for k in (0, 3, 10):
        a = FlakyAllocator(fail_after=k)
        with pytest.raises(api.CosimError) as e:
            api.cosim_create(p, api.COSIM_FP32, allocator=a)
        assert e.value.status == api.COSIM_ERR_OOM
        assert not a.live  # what was handed out before the failure came back


def test_invalid_material_id_rejected_on_device():
    """Grids above 2^24 voxels have their IDs checked on the device after the
    upload (smaller ones on the host, tests/test_abi.py): a bad ID is reported
    as COSIM_ERR_INVALID and every block handed out comes back."""
    build()
    p = W.uniform_box(260, 260, 250, em_bc=(0,) * 6)
    assert p.n_cells > 1 << 24
    p.mat[200, 100, 17] = 7
    a = FlakyAllocator()
    with pytest.raises(api.CosimError) as e:
        api.cosim_create(p, api.COSIM_FP32, allocator=a)
    assert e.value.status == api.COSIM_ERR_INVALID and "material id" in str(e.value)
    assert not a.live
    p.mat[200, 100, 17] = 0  # the same grid with valid IDs is created
    h, keep = api.cosim_create(p, api.COSIM_FP32, allocator=a)
    api.cosim_destroy(h)
    assert not a.live


def test_allocation_failure_later_leaves_context_valid():
    build()
    p = W.tiny_package()
    a = FlakyAllocator()
    h, keep = api.cosim_create(p, api.COSIM_FP64, allocator=a)
    try:
        api.cosim_em_steps(h, 20, api.COSIM_ACCUM_JOULE)
        a.refuse = True  # the mechanics arrays are allocated on the first solve
        with pytest.raises(api.CosimError) as e:
            api.cosim_stress_solve(h, rtol=1e-6)
        assert e.value.status == api.COSIM_ERR_OOM
        api.cosim_em_steps(h, 4, api.COSIM_ACCUM_JOULE)  # still usable
        a.refuse = False
        rep = api.cosim_stress_solve(h, rtol=1e-6)
        assert rep["status"] == api.COSIM_OK
    finally:
        api.cosim_destroy(h)
    assert not a.live


@pytest.mark.parametrize("precision", [api.COSIM_FP32, api.COSIM_FP64])
@pytest.mark.parametrize("on_device", [False, True])
def test_checkpoint_resume_is_bitwise(precision, on_device):
    build()
    p = W.tiny_package()
    tables = None
    a = api.Context(p, precision=precision)
    tables = p.source_tables(a.dt, 400)
    a.set_sources(tables)
    a.em_steps(37)  # odd parity, mid Joule window
    a.em_steps(5, coupled=True)  # the temperature and power moved too
    blob = None if on_device else a.checkpoint()
    if on_device:
        n = api.C.c_size_t()
        api.load().cosim_checkpoint_size(a.h, C.byref(n))
        blob = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        a.checkpoint(blob)
    step = a.query(api.COSIM_Q_STEP)

    def go_on(c):
        c.em_steps(50)
        c.em_steps(3, coupled=True)
        return [c.read(f) for f in (api.COSIM_F_EX, api.COSIM_F_EY, api.COSIM_F_EZ, api.COSIM_F_HX, api.COSIM_F_HY,
                                     api.COSIM_F_HZ, api.COSIM_F_Q, api.COSIM_F_DT, api.COSIM_F_P)]

    want = go_on(a)
    b = api.Context(p, precision=precision, dt_em=a.dt)
    b.set_sources(tables)
    b.restore(blob)
    assert b.query(api.COSIM_Q_STEP) == step
    got = go_on(b)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert np.abs(want[2]).max() > 0 and np.abs(want[6]).max() > 0
    # a checkpoint of another grid is refused, the context unchanged
    other = api.Context(W.uniform_box(8, 8, 8), precision=precision)
    with pytest.raises(api.CosimError) as e:
        other.restore(blob)
    assert e.value.status == api.COSIM_ERR_INVALID
    for c in (a, b, other):
        c.close()
