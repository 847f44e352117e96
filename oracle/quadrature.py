"""Sinc quadrature of the Balakrishnan integral. Test infrastructure only.

L^{-beta} = sin(pi beta)/pi * int_0^inf s^{-beta} (L + s)^{-1} ds (Eq. 2).
With the coefficients of Eq. 4,
    c_const = pi / (2 k sin(pi beta)),  c_I^(l) = c_const e^{-2 beta y_l},
    c_L^(l) = c_I^(l) e^{2 y_l},        y_l = l k,
the approximation is L^{-beta} ~ sum_{l=-K^-}^{K^+} (c_I^(l) I + c_L^(l) L)^{-1}
with the limits of Sec. 4.1,
    K^- = ceil(pi^2 / (4 k^2 beta)),  K^+ = ceil(pi^2 / (4 k^2 (1 - beta))).
Equivalently (c_I I + c_L L)^{-1} = w_l (I + t_l L)^{-1} with t_l = e^{2 y_l}
and w_l = 1 / c_I^(l) = (2 k sin(pi beta) / pi) e^{2 beta y_l}.

Reading taken: the Eq. 4 form with the index range -K^- .. K^+ (Eq. 3 prints
a different substitution and a different lower index).
"""
from __future__ import annotations

import math

import numpy as np


def limits(beta: float, k: float) -> tuple[int, int]:
    if not (0.0 < beta < 1.0):
        raise ValueError("quadrature needs 0 < beta < 1")
    km = math.ceil(math.pi ** 2 / (4.0 * k * k * beta))
    kp = math.ceil(math.pi ** 2 / (4.0 * k * k * (1.0 - beta)))
    return km, kp


def coefficients(beta: float, k: float):
    """(c_I, c_L) per node, Eq. 4."""
    km, kp = limits(beta, k)
    y = np.arange(-km, kp + 1, dtype=np.float64) * k
    c_const = math.pi / (2.0 * k * math.sin(math.pi * beta))
    c_i = c_const * np.exp(-2.0 * beta * y)
    c_l = c_i * np.exp(2.0 * y)
    return c_i, c_l


def nodes(beta: float, k: float):
    """(t_l, w_l) per node: (c_I M + c_L K)^{-1} = w_l (M + t_l K)^{-1}."""
    c_i, c_l = coefficients(beta, k)
    return c_l / c_i, 1.0 / c_i


def scalar(lam, beta: float, k: float):
    """q(lambda) = sum_l w_l / (1 + t_l lambda), the quadrature's approximation
    of lambda^{-beta}."""
    t, w = nodes(beta, k)
    lam = np.asarray(lam, np.float64)
    return (w[None, :] / (1.0 + t[None, :] * lam.reshape(-1, 1))).sum(axis=1).reshape(lam.shape)
