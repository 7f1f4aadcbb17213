"""EM steps recorded once into a CUDA graph and replayed equal the same steps
launched one by one, bit for bit: the device-resident source time index
advances per replay, the Joule window folds in the same places and the E/H
parity returns to the captured one. Capture and launch preconditions are
enforced with COSIM_ERR_INVALID."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, build

pytestmark = pytest.mark.gpu

FIELDS = [api.COSIM_F_EX, api.COSIM_F_EY, api.COSIM_F_EZ, api.COSIM_F_HX, api.COSIM_F_HY, api.COSIM_F_HZ,
          api.COSIM_F_Q]


def _pair(precision, stream):
    build()
    p = W.tiny_package()
    a = api.Context(p, precision=precision, stream=stream)
    b = api.Context(p, precision=precision, stream=stream, dt_em=a.dt)
    tables = p.source_tables(a.dt, 400)
    a.set_sources(tables)
    b.set_sources(tables)
    return a, b


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_graph_replay_equals_plain_steps(precision):
    s = torch.cuda.Stream()
    a, b = _pair(precision, s)
    a.em_steps(3 * 64)
    b.em_graph_capture(64)
    assert b.query(api.COSIM_Q_STEP) == 0  # capturing runs nothing
    b.em_graph_launch(2)
    b.em_graph_launch(1)
    for f in FIELDS:
        x, y = a.read(f), b.read(f)
        assert np.array_equal(x, y), f
    assert np.any(a.read(api.COSIM_F_EZ) != 0)
    assert a.query(api.COSIM_Q_STEP) == b.query(api.COSIM_Q_STEP) == 192
    assert a.query(api.COSIM_Q_JOULE_STEPS) == b.query(api.COSIM_Q_JOULE_STEPS) == 192
    assert a.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER) == b.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
    # plain steps after replays continue from the same source time index
    a.em_steps(10)
    b.em_steps(10)
    assert np.array_equal(a.read(api.COSIM_F_EZ), b.read(api.COSIM_F_EZ))
    a.close()
    b.close()


def test_graph_preconditions():
    build()
    p = W.tiny_package()
    c = api.Context(p, precision=FP32)  # default stream: capture refused
    with pytest.raises(api.CosimError):
        c.em_graph_capture(64)
    c.close()
    s = torch.cuda.Stream()
    a, b = _pair(FP32, s)
    with pytest.raises(api.CosimError):
        a.em_graph_capture(48)  # not a multiple of 32
    with pytest.raises(api.CosimError):
        a.em_graph_launch(1)  # nothing captured
    a.em_steps(5)
    with pytest.raises(api.CosimError):
        a.em_graph_capture(64)  # Joule window not aligned
    a.joule(api.COSIM_JOULE_RESET)
    a.em_graph_capture(64, accumulate_joule=False)  # without accumulation only the parity matters
    a.em_graph_launch(1)  # parity of the capture (5 steps taken: odd) is the current one
    a.em_steps(1)
    with pytest.raises(api.CosimError):
        a.em_graph_launch(1)  # parity differs now
    a.set_sources(p.source_tables(a.dt, 10))
    a.em_steps(1)
    with pytest.raises(api.CosimError):
        a.em_graph_launch(1)  # new sources discard the graph
    torch.cuda.synchronize()
    a.close()
    b.close()
