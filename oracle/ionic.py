"""Aliev-Panfilov two-variable cell model (the ionic model I_ion, g of Eq. monodomain).

The paper runs the PCG model, whose equations are not reproduced in it; the
workloads here use the published Aliev-Panfilov model instead:

  I_ion(V, v) = k V (V - a)(V - 1) + V v
  g(V, v)     = eps(V, v) ( -v - k V (V - a - 1) ),   eps = eps0 + mu1 v / (V + mu2)

with V dimensionless (rest 0, peak ~1) and standard parameters k = 8,
a = 0.15, eps0 = 0.002, mu1 = 0.2, mu2 = 0.3.  One model time unit is
``time_scale`` ms (default 1), i.e. both right-hand sides are divided by it.
The denominator V + mu2 is clamped below at 1e-6.

The state update is the partitioned first-order exponential integrator of
Sec. 2.3 (the Rush-Larsen analogue): g is linear in v with rate -eps frozen at
the step start, so v <- v_inf + (v - v_inf) exp(-eps dt), v_inf = -k V (V - a - 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

EPS_DEN_MIN = 1e-6


def params(prob):
    k, a, eps0, mu1, mu2, ts = (list(prob.ionic_params) + [1.0] * 6)[:6]
    return k, a, eps0, mu1, mu2, ts


def i_ion(prob, V, v):
    if prob.ionic_model < 0:
        return np.zeros_like(V)
    k, a, eps0, mu1, mu2, ts = params(prob)
    return (k * V * (V - a) * (V - 1.0) + V * v) / ts


def eps(prob, V, v):
    k, a, eps0, mu1, mu2, ts = params(prob)
    den = np.maximum(V + mu2, EPS_DEN_MIN)
    return eps0 + mu1 * v / den


def v_inf(prob, V):
    k, a, eps0, mu1, mu2, ts = params(prob)
    return -k * V * (V - a - 1.0)


def g(prob, V, v):
    if prob.ionic_model < 0:
        return np.zeros_like(V)
    k, a, eps0, mu1, mu2, ts = params(prob)
    return eps(prob, V, v) * (-v + v_inf(prob, V)) / ts


def step_state(prob, V, v, dt, integrator):
    """One step of the internal variable from the values at the step start."""
    if prob.ionic_model < 0:
        return v.copy()
    if integrator == 0:
        return v + dt * g(prob, V, v)
    k, a, eps0, mu1, mu2, ts = params(prob)
    vi = v_inf(prob, V)
    return vi + (v - vi) * np.exp(-eps(prob, V, v) * dt / ts)
