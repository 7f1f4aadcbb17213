"""cosim_sum_f64_noalloc: the allocation-free variant of the deterministic FP64
reduction, for callers that cannot allocate device memory (a fully reserved
memory budget, or a loop that must not pay cudaMalloc's synchronisation).
Checked against the existing library path (cosim_joule_accumulate's total of
the Joule accumulator) on two calls in a row. Collected last on purpose."""
import numpy as np
import pytest

import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP64, context

pytestmark = pytest.mark.gpu


def test_noalloc_sum_matches_library_total():
    import torch
    p = W.tiny_package()
    ctx = context(p, FP64)
    tables = [(a, e, v * 50.0) for a, e, v in p.source_tables(ctx.dt, 150)]
    ctx.set_sources(tables)
    ctx.em_steps(150)
    total = ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)  # existing path, context-owned scratch
    assert total > 0
    q = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    api.cosim_read_fields(ctx.h, api.COSIM_F_Q, q)
    dev_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):  # the shared array keeps the previous call's contents
        v = api.cosim_sum_f64_noalloc(q)
        assert abs(v / total - 1) < 1e-12
        api.cosim_sum_f64_noalloc(q, out=dev_out)
        torch.cuda.synchronize()
        assert abs(dev_out.item() / total - 1) < 1e-12
    ctx.close()


def test_noalloc_sum_spans_many_partials_and_rejects_oversize():
    import torch
    rng = np.random.default_rng(3)
    host = rng.standard_normal(3_000_000)
    x = torch.from_numpy(host).cuda()
    for _ in range(2):
        v = api.cosim_sum_f64_noalloc(x)
        assert abs(v - host.sum()) < 1e-9 * np.abs(host).sum()
    # the C entry point itself rejects n over its limit before any GPU work
    # (called directly: the Python wrapper already refuses n > x.numel())
    import ctypes as C
    v = C.c_double()
    st = api.load().cosim_sum_f64_noalloc(x.data_ptr(), (1 << 28) + 1, C.addressof(v), 0, None)
    assert st == api.COSIM_ERR_INVALID and "limit" in api.cosim_last_error(None)
    with pytest.raises(ValueError):
        api.cosim_sum_f64_noalloc(x, n=x.numel() + 1)
