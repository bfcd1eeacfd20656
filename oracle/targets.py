"""Tuning targets of Sec. 2.6 (test infrastructure, part of the oracle).

b_eff(z) = 0.183 [(1+z)/3.3]^3.47 and beta(z) = 1.76 [(1+z)/3.3]^-2.32 are
the power-law targets fitted to eBOSS DR16; b_eff = b (1 + 2 beta/3 +
beta^2/5)^(1/2) relates the effective bias to b and beta (Hamilton 1991
monopole); Fbar(z) = exp(-0.0028 (1+z)^3.45) is the paper's mean-flux
target, and exp(-0.0025 (1+z)^3.7) the mean-flux target of the tuning
comparison.
"""
import math


def b_eff_target(z):
    return 0.183 * ((1.0 + z) / 3.3) ** 3.47


def beta_target(z):
    return 1.76 * ((1.0 + z) / 3.3) ** -2.32


def b_from_b_eff(b_eff, beta):
    return b_eff / math.sqrt(1.0 + 2.0 * beta / 3.0 + beta * beta / 5.0)


def mean_flux_paper(z):
    return math.exp(-0.0028 * (1.0 + z) ** 3.45)


def mean_flux_tuning(z):
    return math.exp(-0.0025 * (1.0 + z) ** 3.7)
