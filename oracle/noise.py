"""Lumped-mass FEM white noise b = M_L^{1/2} xi (Eq. wh_def with the diagonal
factor of Sec. 2.5). Test infrastructure only (see package header).

xi ~ N(0, I): word x of the Philox stream becomes the uniform
u = (x + 1/2) 2^-32 in (0, 1); consecutive word pairs (x0, x1) and (x2, x3) of
one Philox block give two normals each by the Box-Muller transform
    r = sqrt(-2 ln u_a),  n_a = r cos(2 pi u_b),  n_b = r sin(2 pi u_b).
DOF j uses word j mod 4 of block j div 4 (counter layout in philox.noise_words).
"""
from __future__ import annotations

import numpy as np

from .philox import noise_words


def uniforms(words: np.ndarray) -> np.ndarray:
    return (words.astype(np.float64) + 0.5) * 2.0 ** -32


def box_muller(u: np.ndarray) -> np.ndarray:
    """u: [..., 4k] uniforms in (0,1). Returns normals of the same shape."""
    ua = u[..., 0::2]
    ub = u[..., 1::2]
    r = np.sqrt(-2.0 * np.log(ua))
    out = np.empty_like(u)
    out[..., 0::2] = r * np.cos(2.0 * np.pi * ub)
    out[..., 1::2] = r * np.sin(2.0 * np.pi * ub)
    return out


def standard_normals(seed: int, n_dofs: int, n_samples: int) -> np.ndarray:
    """xi, shape [n_samples, n_dofs]."""
    nq4 = ((n_dofs + 3) // 4) * 4
    w = noise_words(seed, nq4, n_samples)
    return box_muller(uniforms(w))[:, :n_dofs]


def white_noise(ml: np.ndarray, seed: int, n_samples: int) -> np.ndarray:
    """b = sqrt(M_L) xi, shape [n_samples, n_dofs]."""
    return np.sqrt(ml)[None, :] * standard_normals(seed, ml.shape[0], n_samples)
