"""Host-side parts of offline training: the learning-rate schedule (Sec. 4.4)
and the stiffness loss (Sec. 3.1) on CPU tensors.  The training itself, through
the GPU adjoint, is covered by test_gpu_training.py."""
import numpy as np
import torch

from paper_2103_08253_gb300 import training as T


def test_schedule_follows_the_formula():
    assert abs(T.lr_schedule(0) - 1.5e-2) < 1e-15
    assert abs(T.lr_schedule(50) - 0.999 ** 50 * 1.5e-3) < 1e-15
    assert abs(T.lr_schedule(100) - 0.999 ** 100 * 1.5e-2) < 1e-15


def test_stiffness_loss_matches_its_definition():
    rng = np.random.default_rng(1)
    C = torch.from_numpy(rng.standard_normal((5, 6, 6)))
    Ct = torch.from_numpy(rng.standard_normal((5, 6, 6)))
    w = np.array([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)])
    s = 1.0 / np.outer(w, w)
    e = np.abs((C.numpy() - Ct.numpy()) * s).reshape(5, -1).sum(1) / np.abs(Ct.numpy() * s).reshape(5, -1).sum(1)
    ref = (e ** 10).sum() ** 0.1 / 5
    assert abs(float(T.stiffness_loss(C, Ct)) - ref) < 1e-14 * ref
