"""Current-density excitation waveforms J(t) [A/m^2].

The method takes J on a set of source edges as an input (the right-hand side
of the second-order Maxwell system, Eq. 1-2). These classes only evaluate the
prescribed excitation at given instants; the solvers sample it at the
half-steps t = (n + 1/2) * dt of the leapfrog.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import ndtr


@dataclass
class GaussianDerivative:
    """J(t) = -J0 * ((t - t0)/s) * exp(-(t - t0)^2 / (2 s^2)).

    The magnitude peaks at |t - t0| = s with value J0 * exp(-1/2).
    """
    j0: float
    sigma_t: float = 20e-12
    t0: float | None = None

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        t0 = 3.0 * self.sigma_t if self.t0 is None else self.t0
        x = (t - t0) / self.sigma_t
        return -self.j0 * x * np.exp(-0.5 * x * x)


def prbs7_bits(seed: int, n: int) -> np.ndarray:
    """n bits of the PRBS7 sequence (polynomial x^7 + x^6 + 1), seeded state."""
    s = (seed % 127) + 1  # any nonzero 7-bit state
    out = np.empty(n, dtype=np.int8)
    for b in range(n):
        new = ((s >> 6) ^ (s >> 5)) & 1
        s = ((s << 1) | new) & 0x7F
        out[b] = new
    return out


@dataclass
class PRBSBurst:
    """NRZ PRBS7 burst with Gaussian-smoothed edges.

    J(t) = J0 * sum_b level_b * [Phi((t - t_b)/s) - Phi((t - t_{b+1})/s)],
    level_b = 2*bit_b - 1, t_b = t_start + b * t_bit, Phi = standard normal CDF.
    """
    j0: float
    seed: int
    bit_rate: float = 10e9
    n_bits: int = 19
    edge_sigma: float = 20e-12
    t_start: float = 60e-12
    bits: np.ndarray = field(init=False)

    def __post_init__(self):
        self.bits = prbs7_bits(self.seed, self.n_bits)

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        tb = 1.0 / self.bit_rate
        nb = len(self.bits)
        # the CDF at every bit edge t_q = t_start + q t_bit, q = 0..n_bits, once
        # (bit b spans edges b and b+1), the bits' terms summed in order
        tq = (self.t_start + np.arange(nb + 1) * tb).reshape((nb + 1,) + (1,) * t.ndim)
        edges = ndtr((t - tq) / self.edge_sigma)  # edge q in edges[q]
        lvl = 2.0 * self.bits.astype(np.float64) - 1.0
        out = np.zeros_like(t)
        for b in range(nb):
            out += lvl[b] * (edges[b] - edges[b + 1])
        return self.j0 * out


@dataclass
class Sampled:
    """A waveform given directly as samples at t = (n + 1/2) dt."""
    values: np.ndarray

    def table(self, dt: float, nsteps: int) -> np.ndarray:
        v = np.zeros(nsteps, dtype=np.float64)
        m = min(nsteps, len(self.values))
        v[:m] = self.values[:m]
        return v


# ---- the paper's transient excitation scheme (Sec. III-B): a broadband
# trigger, background logic noise and a high-speed data burst, each with
# deterministic per-port jitter of amplitude, pulse width and timing.

@dataclass(frozen=True)
class Jitter:
    """Per-port variation: amplitude factor, width factor, time shift [s]."""
    amp: float = 1.0
    width: float = 1.0
    shift: float = 0.0

    @staticmethod
    def seeded(seed: int, amp=0.20, width=0.10, shift=10e-12) -> "Jitter":
        """Uniform in +-amp (relative), +-width (relative), +-shift (s)."""
        r = np.random.default_rng(seed).uniform(-1.0, 1.0, 3)
        return Jitter(1.0 + amp * r[0], 1.0 + width * r[1], shift * r[2])


@dataclass
class Ricker:
    """Ricker wavelet J(t) = J0 (1 - 2 a) exp(-a), a = (pi f (t - t0))^2.

    Peak J0 at t0; zero mean; its envelope exp(-a) falls to e^-9 at
    |t - t0| = 3 / (pi f), so f = 50 GHz confines it to t0 +- 19 ps (the
    paper's 20-60 ps trigger with t0 = 40 ps). Jitter scales J0, divides f by
    the width factor and shifts t0."""
    j0: float
    t0: float = 40e-12
    f: float = 50e9
    jitter: Jitter = Jitter()

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        f = self.f / self.jitter.width
        a = (np.pi * f * (t - (self.t0 + self.jitter.shift))) ** 2
        return self.j0 * self.jitter.amp * (1.0 - 2.0 * a) * np.exp(-a)


@dataclass
class Sine:
    """Continuous J0 sin(2 pi f (t - shift)) on [t_on, t_off) (the paper's
    5 GHz logic noise on 0-300 ps); width jitter scales the period."""
    j0: float
    f: float = 5e9
    t_on: float = 0.0
    t_off: float = 300e-12
    jitter: Jitter = Jitter()

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        f = self.f / self.jitter.width
        on = (t >= self.t_on) & (t < self.t_off)
        return np.where(on, self.j0 * self.jitter.amp * np.sin(2.0 * np.pi * f * (t - self.jitter.shift)), 0.0)


@dataclass
class GaussianPulseTrain:
    """A carrier J0 sin(2 pi f_c t) modulated by n_bits Gaussian pulses, one
    per bit slot of [t_on, t_off) (centred in the slot, sigma = slot/6, so a
    pulse has fallen to e^-4.5 at the slot edges) and present where the bit
    is 1 (the paper's 40 GHz data burst, 3 bits on 80-230 ps). Jitter scales
    J0 and the pulse width and shifts the whole train."""
    j0: float
    bits: tuple = (1, 0, 1)
    f_c: float = 40e9
    t_on: float = 80e-12
    t_off: float = 230e-12
    jitter: Jitter = Jitter()

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64) - self.jitter.shift
        slot = (self.t_off - self.t_on) / len(self.bits)
        s = slot / 6.0 * self.jitter.width
        env = np.zeros_like(t)
        for b, bit in enumerate(self.bits):
            if bit:
                c = self.t_on + (b + 0.5) * slot
                env += np.exp(-0.5 * ((t - c) / s) ** 2)
        return self.j0 * self.jitter.amp * env * np.sin(2.0 * np.pi * self.f_c * t)


@dataclass
class Scaled:
    """sign * waveform(t): a port's share of a differential or G-S-G feed."""
    waveform: object
    sign: float

    def __call__(self, t):
        return self.sign * self.waveform(t)
