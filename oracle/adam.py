"""FP64 oracle of the optimiser step (test infrastructure only).

RoGs Sec. 4.2 (implementation details): the parameters are optimised with
Adam, with per-parameter learning rates (alpha, scales and rotation 1e-4,
z 1.6e-4 x scene size decaying to 1.6e-6 x scene size, colour 0.008,
semantics 0.1, exposure 0.001).  The paper does not state beta1, beta2 or
epsilon; the reading here is Adam's usual 0.9, 0.999, 1e-8.  Adam itself
(Kingma and Ba, Algorithm 1): with gradient g at step t >= 1,
    m <- b1 m + (1 - b1) g,     v <- b2 v + (1 - b2) g^2,
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in FP64; returns (p, m, v) (new arrays)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def z_learning_rate(step, total_steps, scene_size, start=1.6e-4, end=1.6e-6):
    """Learning rate of z: proportional to the scene size, the ratio falling
    from 1.6e-4 to 1.6e-6 over training.  The paper does not give the shape
    of the decay; the reading here is log-linear (exponential) in the step."""
    f = min(max(step / max(total_steps, 1), 0.0), 1.0)
    return scene_size * start * (end / start) ** f
