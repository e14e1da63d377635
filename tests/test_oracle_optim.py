"""Pins of the optimisation oracle (oracle/optim.py) against closed forms and
finite differences -- no GPU."""
import numpy as np

from oracle import optim as O


def test_first_step_is_signed_learning_rate():
    """t = 1: m_hat = g and v_hat = g^2, so the step is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    th, g = rng.normal(size=100), rng.normal(size=100) * 10.0 ** rng.uniform(-6, 3, 100)
    new, m, v, _ = O.adam_step(th, g, np.zeros(100), np.zeros(100), 1, 0.01)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_constant_gradient_moves_linearly():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step, so theta_t = theta_0 - t lr g / (|g| + eps)."""
    th0 = np.array([0.3, -2.0, 5.0])
    g = np.array([1e-3, -4.0, 0.25])
    th, m, v = th0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 51):
        th, m, v, _ = O.adam_step(th, g, m, v, t, 1e-3)
    assert np.allclose(th, th0 - 50 * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-14)


def test_sigmoid_chain_matches_finite_differences():
    """For the sigmoid group the raw gradient is dL/da * a (1 - a): compare
    with a central difference of L(sigmoid(theta)) at t = 1, where the step
    is -lr sign(dL/dtheta)."""
    rng = np.random.default_rng(1)
    th = rng.normal(size=20) * 3
    w = rng.normal(size=20)
    loss = lambda t: float((w * O.sigmoid(t) ** 2).sum())
    g_act = 2 * w * O.sigmoid(th)                      # dL/da
    h = 1e-6
    fd = np.array([(loss(th + h * e) - loss(th - h * e)) / (2 * h) for e in np.eye(20)])
    new, m, _, a = O.adam_step(th, g_act, np.zeros(20), np.zeros(20), 1, 0.1, O.SIGMOID, eps=0.0)
    assert np.allclose(m / 0.1, fd, rtol=1e-6, atol=1e-9)          # m_1 = (1 - b1) g_theta
    assert np.allclose(new, th - 0.1 * np.sign(fd))
    assert np.allclose(a, 1 / (1 + np.exp(-new)))


def test_clamp_projects_onto_nonnegative():
    th = np.array([0.001, 0.5, 2.0, 0.0])
    g = np.array([1.0, 1.0, -1.0, 1.0])
    new, _, _, a = O.adam_step(th, g, np.zeros(4), np.zeros(4), 1, 0.01, O.CLAMP0)
    assert np.allclose(new, np.maximum(th - 0.01 * np.sign(g), 0.0), atol=1e-9)
    assert (new >= 0).all() and np.array_equal(new, a)


def test_l1_loss_and_gradient():
    rng = np.random.default_rng(2)
    out, tgt = rng.normal(size=1000), rng.normal(size=1000)
    tgt[:10] = out[:10]   # ties: zero gradient
    L, d = O.loss_l1(out, tgt, 0.5)
    assert np.isclose(L, 0.5 * sum(abs(float(a) - float(b)) for a, b in zip(out, tgt)))
    h = 1e-7
    for i in (10, 500, 999):
        e = np.zeros(1000); e[i] = h
        fd = (O.loss_l1(out + e, tgt, 0.5)[0] - O.loss_l1(out - e, tgt, 0.5)[0]) / (2 * h)
        assert np.isclose(d[i], fd, rtol=1e-6)
    assert np.all(d[:10] == 0)


# --------------------------------------------------------------------------
# silhouette IoU loss (Eq. sil_loss)


def test_sil_iou_exact_and_disjoint():
    """Coverage equal to a binary mask: IoU 1, loss 0; coverage disjoint from
    it: IoU 0, loss 1; a two-pixel example by hand."""
    rng = np.random.default_rng(3)
    M = (rng.uniform(size=500) < 0.4).astype(np.float64)
    assert abs(O.loss_sil_iou(M, M)[0]) < 1e-15
    assert abs(O.loss_sil_iou(1.0 - M, M)[0] - 1.0) < 1e-15
    # A = (0.5, 1), M = (1, 0): I = 0.5, U = (0.5 + 1 - 0.5) + 1 = 2, loss 0.75
    loss, g = O.loss_sil_iou([0.5, 1.0], [1.0, 0.0], scale=2.0)
    assert abs(loss - 1.5) < 1e-15
    # dL/dA_0 = -2 (1 * 2 - 0.5 * 0) / 4 = -1;  dL/dA_1 = -2 (0 - 0.5 * 1) / 4 = 0.25
    np.testing.assert_allclose(g, [-1.0, 0.25], rtol=1e-15)


def test_sil_iou_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    A = rng.uniform(0, 1, 64)
    M = rng.uniform(0, 1, 64)
    loss, g = O.loss_sil_iou(A, M, scale=0.7)
    for i in rng.choice(64, 10, replace=False):
        h = 1e-6
        Ap, Am = A.copy(), A.copy()
        Ap[i] += h
        Am[i] -= h
        fd = (O.loss_sil_iou(Ap, M, 0.7)[0] - O.loss_sil_iou(Am, M, 0.7)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-8
