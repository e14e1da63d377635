"""FP64 oracle of the optimisation step -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference arm
of ``bench.py`` may import this module.  It shares no code with the CUDA path.

* ``adam_step``: Adam (Kingma & Ba 2014, Algorithm 1), which the paper's
  section "Training and Optimization" uses for all surfel parameters and the
  environment map.  The paper gives no Adam constants; the defaults here are
  Kingma & Ba's (beta1 0.9, beta2 0.999, eps 1e-8).  The renderer consumes
  activated values, so the step first chains dL/d(activated) to the raw
  parameter: identity for positions, quaternions and log-scales, the logistic
  sigmoid for albedo, roughness and metallic, and identity followed by the
  projection onto [0, inf) for the HDR environment texels (an HDR radiance
  cannot be negative).
* ``loss_l1``: the l1 term of Eq. photo_loss on linear values,
  scale * sum |out - target|, and its gradient scale * sign(out - target).
* ``loss_sil_iou``: the silhouette term of Eq. sil_loss, the soft
  intersection-over-union loss between the rendered coverage 1 - T_{K+1}
  and a mask, per image: 1 - I / U with I = sum A M and
  U = sum (A + M - A M), and its gradient with respect to A.
"""
from __future__ import annotations

import numpy as np

IDENTITY, SIGMOID, CLAMP0 = 0, 1, 2


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def activate(theta, activation):
    """Activated value the renderer reads."""
    theta = np.asarray(theta, np.float64)
    return sigmoid(theta) if activation == SIGMOID else theta.copy()


def adam_step(theta, grad_act, m, v, step, lr, activation=IDENTITY, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Algorithm 1 of Kingma & Ba) on raw parameters.

    grad_act is dL/d(activated value); step is t >= 1.  Returns the new
    (theta, m, v, activated value), all float64."""
    theta = np.asarray(theta, np.float64)
    g = np.asarray(grad_act, np.float64)
    m = np.asarray(m, np.float64)
    v = np.asarray(v, np.float64)
    if activation == SIGMOID:
        a = sigmoid(theta)
        g = g * a * (1.0 - a)          # d sigmoid / d theta
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    theta = theta - lr * m_hat / (np.sqrt(v_hat) + eps)
    if activation == CLAMP0:
        theta = np.maximum(theta, 0.0)
    return theta, m, v, activate(theta, activation)


def loss_l1(out, target, scale=1.0):
    """(loss, d loss / d out) of scale * sum |out - target|."""
    d = np.asarray(out, np.float64) - np.asarray(target, np.float64)
    return scale * float(np.abs(d).sum()), scale * np.sign(d)


def loss_sil_iou(coverage, mask, scale=1.0):
    """Soft IoU loss of one image (Eq. sil_loss): A = coverage, M = mask in
    [0, 1]; I = sum A M is the soft intersection, U = sum (A + M - A M) the
    soft union (the probabilistic 'or'); loss = scale (1 - I / U) and
    dloss/dA = -scale (M U - I (1 - M)) / U^2 (quotient rule, dI/dA = M,
    dU/dA = 1 - M).  Returns (loss, gradient)."""
    A = np.asarray(coverage, np.float64)
    M = np.asarray(mask, np.float64)
    inter = float((A * M).sum())
    union = float((A + M - A * M).sum())
    loss = scale * (1.0 - inter / union)
    grad = -scale * (M * union - inter * (1.0 - M)) / union ** 2
    return loss, grad
