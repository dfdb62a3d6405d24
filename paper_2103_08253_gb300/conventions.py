"""Conversions between the library's Mandel vectors and Voigt vectors.

The C ABI takes strains and stresses as Mandel vectors ordered (11, 22, 33, 23,
13, 12), shear entries times sqrt(2), so that Euclidean norms and dot products
are the tensor ones and tangents are symmetric 6x6 matrices.  FE codes mostly
use Voigt vectors: engineering shear strain gamma_ij = 2 eps_ij and plain shear
stress, often in another order (for example (11, 22, 33, 12, 13, 23)).  These
functions convert arrays of shape [..., 6] (vectors) and [..., 6, 6] (tangents,
d stress / d strain) with numpy or torch alike.

`order` is the Voigt ordering as component names; DMN_ORDER is the library's.
"""
from __future__ import annotations

import math

import numpy as np

DMN_ORDER = ("11", "22", "33", "23", "13", "12")
ABAQUS_ORDER = ("11", "22", "33", "12", "13", "23")
_R2 = math.sqrt(2.0)


def _perm(order):
    """Index into the library's ordering of each entry of `order`."""
    order = tuple(order)
    if sorted(order) != sorted(DMN_ORDER):
        raise ValueError("order must be a permutation of %s" % (DMN_ORDER,))
    return [DMN_ORDER.index(c) for c in order]


def _scale(x, w):
    """x times the weights w (broadcast over the leading axes), for numpy arrays and torch tensors."""
    return x * x.new_tensor(w) if hasattr(x, "new_tensor") else x * np.asarray(w)


def mandel_to_voigt_strain(e, order=DMN_ORDER):
    """Mandel strain -> Voigt strain with engineering shear (gamma = sqrt(2) x Mandel shear)."""
    return _scale(e, [1.0, 1.0, 1.0, _R2, _R2, _R2])[..., _perm(order)]


def voigt_to_mandel_strain(g, order=DMN_ORDER):
    """Voigt strain with engineering shear -> Mandel strain."""
    p = _perm(order)
    inv = [p.index(i) for i in range(6)]
    return _scale(g[..., inv], [1.0, 1.0, 1.0, 1.0 / _R2, 1.0 / _R2, 1.0 / _R2])


def mandel_to_voigt_stress(s, order=DMN_ORDER):
    """Mandel stress -> Voigt stress (plain shear = Mandel shear / sqrt(2))."""
    return _scale(s, [1.0, 1.0, 1.0, 1.0 / _R2, 1.0 / _R2, 1.0 / _R2])[..., _perm(order)]


def voigt_to_mandel_stress(s, order=DMN_ORDER):
    """Voigt stress -> Mandel stress."""
    p = _perm(order)
    inv = [p.index(i) for i in range(6)]
    return _scale(s[..., inv], [1.0, 1.0, 1.0, _R2, _R2, _R2])


def mandel_to_voigt_tangent(C, order=DMN_ORDER):
    """Mandel tangent -> the Voigt matrix mapping engineering strain to plain stress:
    C_v[I, J] = C_m[I, J] / (w_I w_J), w = (1, 1, 1, sqrt2, sqrt2, sqrt2)."""
    w = [1.0, 1.0, 1.0, 1.0 / _R2, 1.0 / _R2, 1.0 / _R2]
    p = _perm(order)
    ws = [[w[i] * w[j] for j in range(6)] for i in range(6)]
    return _scale(C, ws)[..., p, :][..., :, p]


def voigt_to_mandel_tangent(Cv, order=DMN_ORDER):
    """Inverse of mandel_to_voigt_tangent."""
    p = _perm(order)
    inv = [p.index(i) for i in range(6)]
    w = [1.0, 1.0, 1.0, _R2, _R2, _R2]
    ws = [[w[i] * w[j] for j in range(6)] for i in range(6)]
    return _scale(Cv[..., inv, :][..., :, inv], ws)
