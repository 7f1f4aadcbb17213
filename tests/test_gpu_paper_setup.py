"""The paper's boundary and excitation scheme (Sec. III-B) through the CUDA
path: PMC walls with a PEC ground plane, adiabatic faces, differential
Ricker pairs in the substrate and G-S-G bump feeds (5 GHz sine, 40 GHz 3-bit
burst) with per-port jitter, marched with the synchronized electro-thermal
loop, against the FP64 oracle. The sources are sampled from t = 38 ps so the
window contains the Ricker trigger."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, field_rel_l2, read_eh, rel_l2

pytestmark = pytest.mark.gpu

STEPS = 150


@pytest.fixture(scope="module")
def ref():
    p = W.paper_setup_package(64, 64, 64, seed=7)
    o = oracle.OracleSim(p)
    tables = p.source_tables(o.dt, STEPS, t0=38e-12)
    o.set_sources(tables)
    o.coupled_steps(STEPS)
    return p, o, tables


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (FP32, 1e-4)])
def test_paper_setup_coupled_window(ref, precision, tol):
    p, o, tables = ref
    ctx = context(p, precision, o.dt)
    ctx.set_sources(tables)
    ctx.em_steps(STEPS, coupled=True)
    Eg, Hg = read_eh(ctx)
    assert max(np.abs(e).max() for e in o.E) > 1.0  # the feeds excited the package
    assert field_rel_l2(Eg, o.E)[0] < tol
    assert field_rel_l2(Hg, o.H)[0] < tol
    assert rel_l2(ctx.read(api.COSIM_F_Q), o.Q) < 10 * tol
    assert rel_l2(ctx.read(api.COSIM_F_P), o.P) < 10 * tol
    # temperature rises are ~1e-9 K in this short window: compare the stored
    # rise (COSIM_F_DT), which keeps its own precision, element by element
    assert np.abs(o.theta).max() > 0
    assert rel_l2(ctx.read(api.COSIM_F_DT), o.theta) < 10 * tol
    ctx.close()
