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
        out = np.zeros_like(t)
        phi = ndtr
        for b, bit in enumerate(self.bits):
            lo = self.t_start + b * tb
            hi = lo + tb
            lvl = 2.0 * float(bit) - 1.0
            out += lvl * (phi((t - lo) / self.edge_sigma) - phi((t - hi) / self.edge_sigma))
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
