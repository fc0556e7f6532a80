"""Pins of the oracle's conductivity tensor and of the physics it drives (CPU, -m "not gpu").

D = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m) (Eq. contGal, D = kappa / (chi C_m)) is
checked two ways that do not reuse its formula:

* against the spectral form: the rotation Q that carries e_1 to the fibre f gives
  D = Q diag(sigma_l, sigma_t, ...) Q^T / (chi C_m); for a fibre along a coordinate axis D is
  diagonal; n^T D n is the conductivity sigma_t + (sigma_l - sigma_t)(n.f)^2 over chi C_m;
* end to end, through the whole oracle step (SIPG operator, Aliev-Panfilov current, forward
  Euler, activation times of Sec. 3.3): with the recovery variable frozen (eps0 = mu1 = 0,
  so g = 0 and v stays 0) the monodomain equation along a thin strip reduces to the Nagumo
  (bistable reaction-diffusion) equation V_t = D_n V_xx - k V (V - a)(V - 1), whose planar
  front from V = 1 into V = 0 travels at the textbook closed-form speed
  c = sqrt(k D_n / 2) (1 - 2a),  D_n = n^T D n.
  The activation times measured on the strip must converge to 1/c at second order in h, along
  and across the fibre, and the ratio of the two speeds to sqrt(sigma_l / sigma_t).  A factor
  lost in chi C_m, a swap of sigma_l and sigma_t, a wrong cubic root or a wrong LAT time all
  move c by far more than the stated discretisation tolerances.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lts
from oracle.sipg import diffusion_tensor

CHI, CM = 1400.0, 1.0
SIG_L, SIG_T = 1.2, 0.4


def _prob(dim, fibre, sigma_l=SIG_L, sigma_t=SIG_T, chi=CHI, cm=CM):
    return W.Problem(dim=dim, fibre=tuple(fibre) + (0.0,) * (3 - len(fibre)), sigma_l=sigma_l,
                     sigma_t=sigma_t, chi=chi, cm=cm)


def _rotation_to(f):
    """Orthogonal Q whose first column is the unit vector f (Householder reflection of e_1)."""
    f = np.asarray(f, dtype=np.float64)
    f = f / np.linalg.norm(f)
    e1 = np.zeros_like(f)
    e1[0] = 1.0
    w = e1 - f
    if np.linalg.norm(w) < 1e-14:
        return np.eye(f.size)
    w = w / np.linalg.norm(w)
    return np.eye(f.size) - 2.0 * np.outer(w, w)


@pytest.mark.parametrize("dim", [2, 3])
def test_fibre_along_an_axis_gives_a_diagonal_tensor(dim):
    for axis in range(dim):
        f = [0.0] * dim
        f[axis] = 1.0
        D = diffusion_tensor(_prob(dim, f, chi=700.0, cm=2.0))
        want = np.full(dim, SIG_T)
        want[axis] = SIG_L
        assert np.array_equal(D, np.diag(want) / (700.0 * 2.0))


def test_rotated_fibre_2d_matches_rotation_of_the_principal_tensor():
    for theta in (0.0, 0.3, math.pi / 4, 1.1, math.pi / 2, 2.5):
        c, s = math.cos(theta), math.sin(theta)
        R = np.array([[c, -s], [s, c]])
        want = R @ np.diag([SIG_L, SIG_T]) @ R.T / (CHI * CM)
        D = diffusion_tensor(_prob(2, [c, s]))
        assert np.abs(D - want).max() < 1e-18


def test_rotated_fibre_3d_spectral_form_and_directional_conductivity():
    rng = np.random.default_rng(7)
    for _ in range(6):
        f = rng.standard_normal(3)
        Q = _rotation_to(f)
        want = Q @ np.diag([SIG_L, SIG_T, SIG_T]) @ Q.T / (CHI * CM)
        # the fibre is given unnormalised: the tensor must normalise it
        D = diffusion_tensor(_prob(3, list(3.0 * f)))
        assert np.abs(D - want).max() < 1e-18
        fu = f / np.linalg.norm(f)
        # eigenpairs: sigma_l along the fibre, sigma_t (twice) across it
        ev = np.sort(np.linalg.eigvalsh(D))
        assert np.allclose(ev, np.array([SIG_T, SIG_T, SIG_L]) / (CHI * CM), rtol=1e-13, atol=0)
        assert np.allclose(D @ fu, SIG_L / (CHI * CM) * fu, rtol=0, atol=1e-18)
        for _ in range(4):
            n = rng.standard_normal(3)
            n /= np.linalg.norm(n)
            dn = (SIG_T + (SIG_L - SIG_T) * float(n @ fu) ** 2) / (CHI * CM)
            assert abs(float(n @ D @ n) - dn) < 1e-18


# --------------------------------------------------------------------------
# Planar Nagumo front on a thin strip: the closed-form speed.
# --------------------------------------------------------------------------

K_AP, A_AP = 8.0, 0.15


def _strip_speed(nx, axis, length=0.4):
    """Front speed (cm/ms) from the activation times of a planar front on a strip of `nx`
    Q1 elements along `axis` (two across it), fibre along x, recovery frozen."""
    h = length / nx
    ext = (length, 2 * h, 1.0) if axis == 0 else (2 * h, length, 1.0)
    base = (nx, 2, 1) if axis == 0 else (2, nx, 1)
    hi = (0.04, 1.0, 1.0) if axis == 0 else (1.0, 0.04, 1.0)
    prob = W.Problem(dim=2, order=1, extent=ext, base=base, sigma_l=SIG_L, sigma_t=SIG_T,
                     fibre=(1.0, 0.0, 0.0), chi=CHI, cm=CM,
                     ionic_params=(K_AP, A_AP, 0.0, 0.0, 0.3, 1.0),
                     stimuli=[W.Stimulus((0, 0, 0), hi, 1.0, 0.0, 0.5)], dt_barrier=0.0,
                     state_integrator=W.STATE_FE)
    sim = lts.Sim(prob)
    d_n = (SIG_L if axis == 0 else SIG_T) / (CHI * CM)
    c_exact = math.sqrt(K_AP * d_n / 2.0) * (1.0 - 2.0 * A_AP)
    sim.step_to(0.9 * length / c_exact)
    assert not np.any(sim.v), "the recovery variable must stay frozen at 0"
    xs = sim.probe_x[:, axis]
    sel = (xs > 0.35 * length) & (xs < 0.8 * length)
    lat = sim.lat[sel]
    assert np.isfinite(lat).all(), "the front must cross the measuring window"
    A = np.stack([xs[sel], np.ones(sel.sum())], axis=1)
    coef, *_ = np.linalg.lstsq(A, lat, rcond=None)
    # a planar front: LAT is linear in the coordinate across the whole window
    assert np.abs(A @ coef - lat).max() < 0.01 * (lat.max() - lat.min())
    return 1.0 / coef[0], c_exact


def test_nagumo_front_speed_along_and_across_the_fibre():
    speeds = {}
    for axis in (0, 1):
        c20, ce = _strip_speed(20, axis)
        c40, _ = _strip_speed(40, axis)
        e20, e40 = abs(c20 - ce) / ce, abs(c40 - ce) / ce
        # second-order convergence of the front speed (h halves: error falls ~4x)
        assert e40 < e20 / 3.0, (axis, e20, e40)
        # discretisation tolerance at h = 0.01 cm: 1% along the fibre (front width ~0.015 cm),
        # 3% across it (front width ~0.009 cm); Richardson extrapolation within 1%
        assert e40 < (0.01 if axis == 0 else 0.03), (axis, c40, ce)
        c_rich = (4.0 * c40 - c20) / 3.0
        assert abs(c_rich - ce) / ce < 0.01, (axis, c_rich, ce)
        speeds[axis] = c_rich
    # speeds along and across the fibre stand in the ratio sqrt(sigma_l / sigma_t)
    assert abs(speeds[0] / speeds[1] - math.sqrt(SIG_L / SIG_T)) < 0.01 * math.sqrt(SIG_L / SIG_T)
