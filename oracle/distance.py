"""Spectral distances between graph descriptors (test infrastructure).

Sec. 4.2 compares snapshots by the distance between their descriptors; the
paper does not print the formula.  Reading: NetLSD distance is the Euclidean
norm over the time grid of the difference of heat (or complex wave) traces;
VNGE distance is the absolute difference of the entropies.
"""
from __future__ import annotations

import math

import numpy as np


def heat_distance(a, b) -> float:
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return math.sqrt(math.fsum((d * d).tolist()))


def wave_distance(a_re, a_im, b_re, b_im) -> float:
    dr = np.asarray(a_re, np.float64) - np.asarray(b_re, np.float64)
    di = np.asarray(a_im, np.float64) - np.asarray(b_im, np.float64)
    return math.sqrt(math.fsum((dr * dr).tolist() + (di * di).tolist()))


def vnge_distance(a: float, b: float) -> float:
    return abs(float(a) - float(b))
