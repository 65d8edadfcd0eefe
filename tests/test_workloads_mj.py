"""The Maxwell-Juttner momentum loader of the input generator (used by the
numerical-heating workload, Sec. 4.1 of the paper) against what the
distribution fixes independently of the sampling algorithm:

* <gamma> = K1(1/theta) / K2(1/theta) + 3 theta (modified Bessel functions);
* <u^2 / gamma> = 3 theta (the pressure of the distribution is n theta m c^2);
* isotropy (zero mean, equal variances per component);
* the whole kinetic-energy distribution against the CDF integrated numerically
  from the density u^2 exp(-(gamma - 1) / theta) (Kolmogorov-Smirnov).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2607_13507_b300 import workloads as W

N = 400_000


def _sample(theta, seed=11):
    return W.maxwell_juttner(W.generator(seed), theta, N)


@pytest.mark.parametrize("theta", [1e-6, 1.0 / 511.0, 0.05, 1.0, 5.0, 3000.0])
def test_mean_gamma_and_pressure(theta):
    u = _sample(theta)
    gam = np.sqrt(1.0 + (u ** 2).sum(0))
    exact = special.kve(1, 1.0 / theta) / special.kve(2, 1.0 / theta) + 3.0 * theta
    se = gam.std() / math.sqrt(N)
    assert abs(gam.mean() - exact) < 5.0 * se + 1e-15
    p = (u ** 2).sum(0) / gam
    assert abs(p.mean() - 3.0 * theta) < 5.0 * p.std() / math.sqrt(N)


@pytest.mark.parametrize("theta", [1.0 / 511.0, 1.0])
def test_isotropy(theta):
    u = _sample(theta, seed=12)
    v = u.var(axis=1)
    for c in range(3):
        assert abs(u[c].mean()) < 5.0 * u[c].std() / math.sqrt(N)
        # variance of a sample variance ~ sqrt(2/N) relative for near-normal tails
        assert abs(v[c] / v.mean() - 1.0) < 0.02


@pytest.mark.parametrize("theta", [0.5, 2.0])      # both envelopes of the sampler
def test_energy_distribution_ks(theta):
    u = _sample(theta, seed=13)
    e = np.sort(np.sqrt(1.0 + (u ** 2).sum(0)) - 1.0)
    dens = lambda x: math.sqrt(x * (x + 2.0)) * (1.0 + x) * math.exp(-x / theta)
    norm = integrate.quad(dens, 0.0, np.inf)[0]
    grid = np.quantile(e, np.linspace(0.01, 0.99, 60))
    cdf = np.array([integrate.quad(dens, 0.0, x)[0] / norm for x in grid])
    emp = np.searchsorted(e, grid, side="right") / N
    assert np.max(np.abs(emp - cdf)) < 1.63 / math.sqrt(N) * 2.0


def test_nonrelativistic_limit_is_maxwellian():
    theta = 1e-5
    u = _sample(theta, seed=14)
    # each component ~ N(0, theta) up to O(theta) corrections
    for c in range(3):
        assert abs(u[c].var() / theta - 1.0) < 0.01
