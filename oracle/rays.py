"""Emitter ray sets on the CPU (float64, rounded to float32) -- TEST INFRASTRUCTURE ONLY.

Only `tests/` and `bench.py`'s CPU leg may import this module.

fibonacci(N): the spherical Fibonacci lattice, z_i = 1 - (2i + 1) / N, phi_i = i pi (3 - sqrt 5).

zonal(N): centre points of the recursive zonal equal-area partition of the unit sphere into N
regions (Leopardi, "A partition of the unit sphere into regions of equal area and small diameter",
2006), the paper's ray set (Sec. III-C).  Steps, for N > 2: two polar caps of one region's area
(colatitude theta_c = 2 arcsin(1 / sqrt N)); the ideal collar angle sqrt(4 pi / N); the number of
collars n = max(1, round((pi - 2 theta_c) / angle)); the fitting angle (pi - 2 theta_c) / n; the
ideal region count of each collar y_i (its area over the region area) rounded with the running
discrepancy carried to the next collar; the collar boundaries then placed so that the caps they
close hold exactly the cumulative region counts (theta(k) = 2 arcsin(sqrt(k / N))).  Each collar is
split into m_i equal longitude arcs; a region's centre is the midpoint of its colatitude and
longitude ranges.  Reading (the paper gives no rotation between collars): collar i's arcs start at
longitude offset_i, offset_1 = 0 and offset_{i+1} = offset_i + pi / m_{i+1} (half a region of the
next collar), reduced modulo 2 pi.  N = 1: the north pole; N = 2: both poles.
"""
from __future__ import annotations

import math

import numpy as np


def fibonacci(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], 1).astype(np.float32)


def zonal_collars(n: int):
    """(cumulative region counts at the zone boundaries from the north pole, region counts per zone).
    Zones: north cap, the collars, south cap."""
    if n == 1:
        return [0, 1], [1]
    if n == 2:
        return [0, 1, 2], [1, 1]
    area = 4.0 * math.pi / n
    theta_c = 2.0 * math.asin(math.sqrt(1.0 / n))
    ideal_angle = math.sqrt(area)
    n_collars = max(1, int(round((math.pi - 2.0 * theta_c) / ideal_angle)))
    fit = (math.pi - 2.0 * theta_c) / n_collars
    counts = [1]
    carry = 0.0
    for i in range(n_collars):
        t0, t1 = theta_c + i * fit, theta_c + (i + 1) * fit
        y = 2.0 * math.pi * (math.cos(t0) - math.cos(t1)) / area
        m = int(round(y + carry))
        carry += y - m
        counts.append(m)
    counts.append(1)
    cum = [0]
    for m in counts:
        cum.append(cum[-1] + m)
    assert cum[-1] == n
    return cum, counts


def zone_theta(k: int, n: int) -> float:
    """Colatitude of the cap holding k of the n regions."""
    return 2.0 * math.asin(math.sqrt(min(1.0, k / n)))


def zonal(n: int) -> np.ndarray:
    cum, counts = zonal_collars(n)
    out = np.zeros((n, 3), np.float64)
    if n == 1:
        out[0] = (0.0, 0.0, 1.0)
        return out.astype(np.float32)
    if n == 2:
        out[0] = (0.0, 0.0, 1.0)
        out[1] = (0.0, 0.0, -1.0)
        return out.astype(np.float32)
    out[0] = (0.0, 0.0, 1.0)
    out[n - 1] = (0.0, 0.0, -1.0)
    offset = 0.0
    for z in range(1, len(counts) - 1):
        m = counts[z]
        if z > 1:
            offset = math.fmod(offset + math.pi / m, 2.0 * math.pi)
        t0, t1 = zone_theta(cum[z], n), zone_theta(cum[z + 1], n)
        th = 0.5 * (t0 + t1)
        j = np.arange(m, dtype=np.float64)
        phi = offset + (j + 0.5) * (2.0 * math.pi / m)
        s = math.sin(th)
        out[cum[z]:cum[z + 1]] = np.stack([s * np.cos(phi), s * np.sin(phi), np.full(m, math.cos(th))], 1)
    return out.astype(np.float32)
