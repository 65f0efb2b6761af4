"""Exact Stokes-flow results used to pin the discretised operator (test infrastructure).

Two equal rigid spheres of radius a, centres R apart, translating along their line of
centres in unbounded Stokes flow, each feel the drag F = 6 pi mu a U lambda, with lambda a
series in bispherical coordinates (cosh(alpha) = R / (2 a)):

* the same velocity U (Stimson & Jeffery 1926, Proc. R. Soc. Lond. A 111, 110-116):
  lambda -> 1 - 3a/(2R) + 9a^2/(4R^2) far apart, 0.6451 at contact;
* opposite velocities, approaching (Brenner 1961, Chem. Eng. Sci. 16, 242-251; Maude
  1961): lambda -> 1 + 3a/(2R) + 9a^2/(4R^2) far apart, and the lubrication divergence
  lambda ~ a / (2 h) as the gap h = R - 2a closes.

Rotating about their line of centres with angular velocities Omega and +-Omega (Jeffery
1915, Proc. Lond. Math. Soc. 14, 327-338), each needs the torque T = 8 pi mu a^3 Omega zeta,
zeta = sinh^3(alpha) * sum_n (+-1)^(n+1) csch^3(n alpha): the alternating sum for rotation in
the same sense (zeta -> 1 - (a/R)^3 far apart), the plain sum for opposite senses (1 + (a/R)^3).
"""
import numpy as np


def stimson_jeffery(R: float, a: float = 1.0, nmax: int = 5000) -> float:
    """Drag factor lambda of two equal spheres moving together along their line of centres."""
    al = float(np.arccosh(R / (2.0 * a)))
    sh1, sh2 = np.sinh(al), np.sinh(2.0 * al)
    total = 0.0
    for n in range(1, nmax + 1):
        x = (2 * n + 1) * al
        if x > 600.0:          # the remaining terms are below double precision
            break
        num = 2.0 * np.sinh(x) + (2 * n + 1) * sh2
        den = 4.0 * np.sinh(0.5 * x) ** 2 - (2 * n + 1) ** 2 * sh1 ** 2
        term = n * (n + 1) / ((2 * n - 1) * (2 * n + 3)) * (1.0 - den / num)
        total += term
        if abs(term) < 1e-18 * abs(total):
            break
    return 4.0 / 3.0 * sh1 * total


def brenner_approach(R: float, a: float = 1.0, nmax: int = 20000) -> float:
    """Drag factor lambda of two equal spheres approaching each other along their line of centres."""
    al = float(np.arccosh(R / (2.0 * a)))
    sh1, sh2 = np.sinh(al), np.sinh(2.0 * al)
    total = 0.0
    for n in range(1, nmax + 1):
        x = (2 * n + 1) * al
        if x > 600.0:
            break
        num = 4.0 * np.cosh(0.5 * x) ** 2 + (2 * n + 1) ** 2 * sh1 ** 2
        den = 2.0 * np.sinh(x) - (2 * n + 1) * sh2
        term = n * (n + 1) / ((2 * n - 1) * (2 * n + 3)) * (num / den - 1.0)
        total += term
        if abs(term) < 1e-18 * abs(total):
            break
    return 4.0 / 3.0 * sh1 * total


def jeffery_rotation(R: float, a: float = 1.0, same_sense: bool = True, nmax: int = 5000) -> float:
    """Torque factor zeta of two equal spheres rotating about their line of centres."""
    al = float(np.arccosh(R / (2.0 * a)))
    total = 0.0
    for n in range(1, nmax + 1):
        if n * al > 200.0:
            break
        term = 1.0 / np.sinh(n * al) ** 3
        total += (term if (n % 2 == 1 or not same_sense) else -term)
    return np.sinh(al) ** 3 * total
