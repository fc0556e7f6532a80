"""Pins for the oracle's basis and cell model against textbook values and closed forms."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import basis, ionic


def test_gauss_legendre_textbook_values():
    x, w = basis.gauss_legendre(1)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = basis.gauss_legendre(2)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lagrange_reproduces_polynomials(p):
    nodes, _ = basis.gauss_legendre(p)
    x = np.linspace(-1.3, 1.3, 17)
    B, G = basis.basis_1d(nodes, x)
    for deg in range(p + 1):
        f = nodes ** deg
        assert np.allclose(B @ f, x ** deg, atol=1e-13)
        df = deg * x ** (deg - 1) if deg > 0 else 0 * x
        assert np.allclose(G @ f, df, atol=1e-12)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_tensor_basis_partition_of_unity_and_gradients(dim, p):
    rng = np.random.default_rng(1)
    xi = rng.uniform(-1, 1, size=(11, dim))
    phi, dphi = basis.eval_basis(dim, p, xi)
    assert np.allclose(phi.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(dphi.sum(axis=1), 0.0, atol=1e-12)
    nodes = basis.node_points(dim, p)
    # reproduces x_0 * x_{dim-1}: gradient check
    f = nodes[:, 0] * nodes[:, dim - 1]
    assert np.allclose(phi @ f, xi[:, 0] * xi[:, dim - 1], atol=1e-13)
    # weights integrate 1 over the reference cube
    assert abs(basis.node_weights(dim, p).sum() - 2.0 ** dim) < 1e-13


AP = W.Problem()


def test_ap_cubic_roots_and_sign():
    """I_ion(V, 0) = k V (V - a)(V - 1): zeros at 0, a, 1; negative between a and 1 (excitable)."""
    k, a = AP.ionic_params[0], AP.ionic_params[1]
    V = np.array([0.0, a, 1.0])
    assert np.allclose(ionic.i_ion(AP, V, np.zeros(3)), 0.0, atol=1e-15)
    assert ionic.i_ion(AP, np.array([0.5 * (a + 1)]), np.zeros(1))[0] < 0.0
    assert ionic.i_ion(AP, np.array([0.5 * a]), np.zeros(1))[0] > 0.0
    # the recovery term adds V v
    assert np.isclose(ionic.i_ion(AP, np.array([0.4]), np.array([0.3]))[0],
                      k * 0.4 * (0.4 - a) * (0.4 - 1) + 0.4 * 0.3)


def test_ap_recovery_nullcline_and_rate():
    k, a, eps0, mu1, mu2 = AP.ionic_params[:5]
    # g = 0 on v = -k V (V - a - 1): at V = 1 that is k a = 1.2
    assert np.isclose(ionic.v_inf(AP, np.array([1.0]))[0], k * a)
    assert np.allclose(ionic.g(AP, np.array([1.0]), np.array([k * a])), 0.0)
    # rest state is a fixed point
    assert ionic.g(AP, np.zeros(1), np.zeros(1))[0] == 0.0
    # eps at rest is eps0
    assert np.isclose(ionic.eps(AP, np.zeros(1), np.zeros(1))[0], eps0)


def test_exponential_step_converges_to_forward_euler_first_order():
    V = np.array([0.7, 0.2, 0.05])
    v = np.array([0.1, 0.5, 0.9])
    errs = []
    for dt in [0.04, 0.02, 0.01]:
        fe = ionic.step_state(AP, V, v, dt, 0)
        ex = ionic.step_state(AP, V, v, dt, 1)
        errs.append(np.abs(fe - ex).max())
    # both are first-order one-step maps of the same ODE: they differ by O(dt^2) per step
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_single_cell_action_potential_shape():
    """Qualitative: a suprathreshold kick fires an upstroke to ~1 and recovers to rest."""
    V = np.array([0.3]); v = np.array([0.0])
    dt = 0.01
    peak = 0.0
    for n in range(int(600 / dt)):
        Vn = V - dt * ionic.i_ion(AP, V, v)
        v = ionic.step_state(AP, V, v, dt, 1)
        V = Vn
        peak = max(peak, V[0])
    assert 0.95 < peak < 1.1
    assert abs(V[0]) < 0.05
