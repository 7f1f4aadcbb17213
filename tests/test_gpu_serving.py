"""Designs served concurrently on one GPU: a design's outputs are the same,
bit for bit, whether it runs alone or beside other designs (contexts share
no device state, kernels are deterministic); the captured-graph EM path
equals plain steps; the admission estimate bounds the measured footprint."""
import numpy as np
import pytest

from paper_2603_07038_b300 import serving as S
from tests.gpu_helpers import build

pytestmark = pytest.mark.gpu


def _same(a, b):
    for k in ("T", "vm", "u"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("joule_J", "T_max", "vm_max", "cg_iters", "cg_relres"):
        assert a[k] == b[k], k


def test_alone_equals_mix_and_graph_equals_plain():
    build()
    specs = S.design_mix(4, seed=5, em_steps=96, thermal_steps=20, scale=0.25)
    runner = S.DesignRunner(specs, workers=4, keep_fields=True)
    alone = [runner.run(s, 0) for s in specs]
    rep = S.serve(specs, [0.0] * len(specs), runner.run, workers=4, footprint=S.footprint_bytes)
    for q, s in enumerate(specs):
        mixed = rep["records"][q].result
        _same(alone[q], mixed)
        assert S.footprint_bytes(s) >= mixed["bytes"]
        assert mixed["joule_J"] > 0 and mixed["T_max"] > 300.0
    plain = S.DesignRunner(specs[:1], workers=1, keep_fields=True, use_graph=False).run(specs[0], 0)
    _same(alone[0], plain)
    assert max(r.worker for r in rep["records"]) > 0  # more than one stream was used
