"""Mandel <-> Voigt conversions of paper_2103_08253_gb300.conventions (host only).

Pinned by what the conversions must preserve: round trips are the identity;
the work sigma : eps is the plain dot product in both notations; a Mandel
tangent and its Voigt form map the same strain to the same stress; the
library's tensor_to_mandel generator agrees on a symmetric tensor; the
Abaqus ordering swaps the 12 and 23 entries.
"""
import numpy as np
import pytest
import torch

from paper_2103_08253_gb300 import conventions as cv, workloads as W


@pytest.mark.parametrize("order", [cv.DMN_ORDER, cv.ABAQUS_ORDER])
def test_round_trips_work_and_tangent(order):
    rng = np.random.default_rng(1)
    e = rng.standard_normal((5, 6))
    s = rng.standard_normal((5, 6))
    A = rng.standard_normal((5, 6, 6))
    C = A + np.swapaxes(A, 1, 2)
    np.testing.assert_allclose(cv.voigt_to_mandel_strain(cv.mandel_to_voigt_strain(e, order), order), e, atol=1e-15)
    np.testing.assert_allclose(cv.voigt_to_mandel_stress(cv.mandel_to_voigt_stress(s, order), order), s, atol=1e-15)
    np.testing.assert_allclose(cv.voigt_to_mandel_tangent(cv.mandel_to_voigt_tangent(C, order), order), C, atol=1e-14)
    ev, sv, Cv = cv.mandel_to_voigt_strain(e, order), cv.mandel_to_voigt_stress(s, order), cv.mandel_to_voigt_tangent(C, order)
    np.testing.assert_allclose((ev * sv).sum(1), (e * s).sum(1), rtol=1e-14)              # sigma : eps
    np.testing.assert_allclose(np.einsum("nij,nj->ni", Cv, ev),
                               cv.mandel_to_voigt_stress(np.einsum("nij,nj->ni", C, e), order), atol=1e-13)
    # torch tensors give the same numbers
    np.testing.assert_allclose(cv.mandel_to_voigt_tangent(torch.from_numpy(C), order).numpy(), Cv, atol=0)


def test_against_tensor_components_and_abaqus_order():
    T = np.array([[1.0, 6.0, 5.0], [6.0, 2.0, 4.0], [5.0, 4.0, 3.0]])       # eps_12 = 6, eps_13 = 5, eps_23 = 4
    m = W.tensor_to_mandel(T[None])[0]
    np.testing.assert_allclose(cv.mandel_to_voigt_strain(m), [1, 2, 3, 8, 10, 12], atol=1e-14)   # gamma = 2 eps
    np.testing.assert_allclose(cv.mandel_to_voigt_stress(m), [1, 2, 3, 4, 5, 6], atol=1e-14)
    np.testing.assert_allclose(cv.mandel_to_voigt_strain(m, cv.ABAQUS_ORDER), [1, 2, 3, 12, 10, 8], atol=1e-14)
    with pytest.raises(ValueError):
        cv.mandel_to_voigt_strain(m, ("11", "22", "33", "12", "12", "23"))
