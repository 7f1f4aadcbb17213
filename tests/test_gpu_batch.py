"""Design batches (cosim_batch_*): several package designs of different
grids advanced by one launch per EM step (one CTA per tile, or a persistent
launch taking tiles from a device counter). Each design's fields and Joule
energy equal those of the same design stepped alone with cosim_em_steps: the
batch runs the same tiles with the same formulas, so FP64 agrees bit for bit
and FP32 to rounding (the batch kernel is compiled apart from the one-design
kernel, and the code generator may contract a packed FP32 product into the
following addition differently there). The two batch modes share one
compiled tile body and agree bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2603_07038_b300 import cosim as api
from paper_2603_07038_b300.build import build

pytestmark = pytest.mark.gpu

FIELDS = (api.COSIM_F_EX, api.COSIM_F_EY, api.COSIM_F_EZ, api.COSIM_F_HX, api.COSIM_F_HY, api.COSIM_F_HZ,
          api.COSIM_F_Q)


def designs():
    # uneven grids: a tiny package, two layered packages of different sizes
    # and depths, and one with a different TSV pitch and seed
    return [W.tiny_package(),
            W.layered_package(160, 96, seed=5, nz=64, n_lines=4),
            W.layered_package(96, 130, seed=6, nz=96, tsv_pitch=7, n_lines=3),
            W.layered_package(200, 70, seed=7, nz=64, n_lines=2)]


def run_alone(p, precision, nsteps, stream):
    c = api.Context(p, precision=precision, stream=stream)
    c.set_sources(p.source_tables(c.dt, nsteps))
    c.em_steps(nsteps)
    out = [c.read(f) for f in FIELDS]
    c.close()
    return out


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision", [api.COSIM_FP32, api.COSIM_FP64])
def test_batch_equals_each_design_alone(precision, persistent):
    build()
    s = torch.cuda.Stream()
    ps = designs()
    nsteps = 70  # two folds of the 32-step Joule window and a partial one
    ctxs = []
    for p in ps:
        c = api.Context(p, precision=precision, stream=s)
        c.set_sources(p.source_tables(c.dt, nsteps))
        ctxs.append(c)
    b = api.Batch(ctxs, persistent=persistent)
    b.em_steps(30)
    b.em_steps(40)
    for p, c in zip(ps, ctxs):
        want = run_alone(p, precision, nsteps, s)
        got = [c.read(f) for f in FIELDS]
        assert max(np.abs(w).max() for w in want[:3]) > 0  # the ports drove the package
        for f, g, w in zip(FIELDS, got, want):
            if precision == api.COSIM_FP64:
                assert np.array_equal(g, w), (p.name, f)
            else:  # a few FP32 roundings per node and step, over 70 steps
                assert np.linalg.norm(g - w) <= 1e-5 * np.linalg.norm(w), (p.name, f)
        assert c.query(api.COSIM_Q_STEP) == nsteps
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("precision", [api.COSIM_FP32, api.COSIM_FP64])
def test_batch_modes_agree_bitwise(precision):
    """the persistent and the one-CTA-per-tile launches run the same compiled
    tile body: identical bits"""
    build()
    s = torch.cuda.Stream()
    ps = designs()
    runs = []
    for persistent in (False, True):
        ctxs = []
        for p in ps:
            c = api.Context(p, precision=precision, stream=s)
            c.set_sources(p.source_tables(c.dt, 70))
            ctxs.append(c)
        b = api.Batch(ctxs, persistent=persistent)
        b.em_steps(70)
        runs.append([[c.read(f) for f in FIELDS] for c in ctxs])
        b.close()
        for c in ctxs:
            c.close()
    for a, g in zip(runs[0], runs[1]):
        for x, y in zip(a, g):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("persistent", [True, False])
def test_batch_graph_replay_equals_batch_steps(persistent):
    build()
    s = torch.cuda.Stream()
    ps = designs()
    runs = []
    for graph in (False, True):
        ctxs = []
        for p in ps:
            c = api.Context(p, precision=api.COSIM_FP32, stream=s)
            c.set_sources(p.source_tables(c.dt, 128))
            ctxs.append(c)
        b = api.Batch(ctxs, persistent=persistent)
        if graph:
            b.graph_capture(64)
            b.graph_launch(2)
        else:
            b.em_steps(128)
        runs.append([[c.read(f) for f in FIELDS] for c in ctxs])
        b.close()
        for c in ctxs:
            c.close()
    for a, g in zip(runs[0], runs[1]):
        for x, y in zip(a, g):
            assert np.array_equal(x, y)


def test_batch_rejects_mixed_states():
    build()
    s = torch.cuda.Stream()
    ps = designs()[:2]
    ctxs = [api.Context(p, precision=api.COSIM_FP32, stream=s) for p in ps]
    for p, c in zip(ps, ctxs):
        c.set_sources(p.source_tables(c.dt, 8))
    ctxs[0].em_steps(1)  # parities now differ
    b = api.Batch(ctxs)
    with pytest.raises(api.CosimError) as e:
        b.em_steps(2)
    assert e.value.status == api.COSIM_ERR_INVALID
    ctxs[1].em_steps(1)
    b.em_steps(2)
    ctxs[0].set_sources(ps[0].source_tables(ctxs[0].dt, 8))  # sources changed after creation
    with pytest.raises(api.CosimError):
        b.em_steps(2)
    b.close()
    other = api.Context(ps[0], precision=api.COSIM_FP32, stream=torch.cuda.Stream())
    with pytest.raises(api.CosimError):  # a second stream
        api.Batch([ctxs[0], other])
    for c in ctxs + [other]:
        c.close()
