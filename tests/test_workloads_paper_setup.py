"""The paper's excitation scheme (Sec. III-B) as seeded inputs: waveform
shapes checked against their closed forms, jitter bounds, port structure of
the differential pairs and G-S-G triples, and the boundary choices."""
import numpy as np
import pytest

import workloads as W
from workloads.waveforms import GaussianPulseTrain, Jitter, PRBSBurst, Ricker, Scaled, Sine, prbs7_bits


def test_ricker_closed_form():
    r = Ricker(2.0)
    assert r(40e-12) == pytest.approx(2.0)                   # peak J0 at t0
    tz = 1.0 / (np.sqrt(2.0) * np.pi * 50e9)                 # (1 - 2a) = 0
    assert abs(r(40e-12 + tz)) < 1e-12 and abs(r(40e-12 - tz)) < 1e-12
    t = np.linspace(0, 80e-12, 200001)
    assert abs(np.trapezoid(r(t), t)) < 1e-6 * np.trapezoid(np.abs(r(t)), t)  # zero mean
    assert np.abs(r(np.array([15e-12, 65e-12]))).max() < 1e-3 * 2.0  # confined to ~20-60 ps


def test_prbs_burst_closed_form():
    """the NRZ PRBS7 burst: J0 sum_b (2 bit_b - 1) [Phi((t - t_b)/s) - Phi((t - t_{b+1})/s)],
    t_b = t_start + b t_bit, written out with math.erfc per sample; the
    plateaus sit at +-J0 between edges"""
    import math
    w = PRBSBurst(j0=2.5, seed=4)
    assert np.array_equal(w.bits, prbs7_bits(4, w.n_bits))
    t = np.linspace(0.0, 2.4e-9, 401)
    tb = 1.0 / w.bit_rate

    def phi(x):
        return 0.5 * math.erfc(-x / math.sqrt(2.0))

    want = np.array([w.j0 * sum((2.0 * float(bit) - 1.0) * (phi((x - (w.t_start + b * tb)) / w.edge_sigma)
                                                           - phi((x - (w.t_start + (b + 1) * tb)) / w.edge_sigma))
                                for b, bit in enumerate(w.bits)) for x in t])
    assert np.abs(w(t) - want).max() < 1e-12 * w.j0
    # bit centres lie 2.5 edge widths from both edges: each neighbouring
    # transition pulls the level by 2 Phi(-2.5) = 1.2 % of the swing
    mid = w.t_start + (np.arange(w.n_bits) + 0.5) * tb
    assert np.allclose(w(mid), w.j0 * (2.0 * w.bits - 1.0), rtol=0, atol=2.6e-2 * w.j0)


def test_sine_and_window():
    s = Sine(1.0)
    t = np.array([-1e-12, 0.0, 50e-12, 100e-12, 299e-12, 300e-12, 350e-12])
    v = s(t)
    assert v[0] == 0 and v[-1] == 0 and v[-2] == 0          # off outside [0, 300) ps
    assert v[2] == pytest.approx(1.0) and abs(v[3]) < 1e-12  # quarter and half of the 200 ps period


def test_pulse_train_bits_and_carrier():
    g = GaussianPulseTrain(1.0, bits=(1, 0, 1))
    slot = 50e-12
    centres = 80e-12 + (np.arange(3) + 0.5) * slot
    env = np.exp(-0.5 * ((centres[:, None] - centres[None, :]) / (slot / 6)) ** 2)
    # at the centre of the 0 bit only the neighbours' tails remain (e^-18)
    assert abs(g(centres[1])) < 1e-7
    # at a crest of the 40 GHz carrier (4.25 cycles: 106.25 ps) the value is the envelope
    tp = 4.25 / 40e9
    assert g(tp) == pytest.approx(np.exp(-0.5 * ((tp - centres[1 - 1]) / (slot / 6)) ** 2), rel=1e-12)
    assert env[0, 2] < 1e-30


@pytest.mark.parametrize("seed", range(20))
def test_jitter_bounds(seed):
    j = Jitter.seeded(seed)
    assert 0.8 <= j.amp <= 1.2 and 0.9 <= j.width <= 1.1 and abs(j.shift) <= 10e-12
    r = Ricker(1.0, jitter=j)
    assert r(40e-12 + j.shift) == pytest.approx(j.amp)


def test_paper_setup_structure():
    p = W.paper_setup_package(96, 96, 64, seed=7)
    assert p.em_bc == (W.BC_PMC,) * 4 + (W.BC_PEC, W.BC_PMC)
    assert p.h_conv == (0.0,) * 6 and p.cpml_cells == 0
    kinds = [type(s.waveform.waveform).__name__ for s in p.sources]
    assert kinds.count("Ricker") >= 2 and kinds.count("Sine") >= 3 and kinds.count("GaussianPulseTrain") >= 3
    t = np.linspace(0, 300e-12, 3001)
    # differential pairs: consecutive Ricker ports, opposite polarity
    ricker = [s for s in p.sources if isinstance(s.waveform.waveform, Ricker)]
    for a, b in zip(ricker[0::2], ricker[1::2]):
        assert a.waveform.sign == -b.waveform.sign
        assert a.axis == b.axis == 0
    # G-S-G: each triple shares one jittered waveform, shares -1/2, +1, -1/2 -> sinks its own current
    gsg = [s for s in p.sources if not isinstance(s.waveform.waveform, Ricker)]
    assert len(gsg) % 3 == 0
    for q in range(0, len(gsg), 3):
        tri = gsg[q:q + 3]
        assert tri[0].waveform.waveform is tri[1].waveform.waveform is tri[2].waveform.waveform
        assert [s.waveform.sign for s in tri] == [-0.5, 1.0, -0.5]
        total = sum(s.waveform(t) * len(s.edges) for s in tri)
        assert np.abs(total).max() < 1e-9 * np.abs(tri[1].waveform(t)).max() * len(tri[1].edges)
    # every source edge is an x edge inside the grid
    for s in p.sources:
        e = np.asarray(s.edges)
        assert np.all(e[:, 0] < p.nx) and np.all(e[:, 1] <= p.ny) and np.all(e[:, 2] <= p.nz)
