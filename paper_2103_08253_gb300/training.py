"""Offline training of an interpolated DMN with the GPU adjoint (Sec. 3.1, 4.4).

The loss of Sec. 3.1: for a batch of N_b samples, the q-norm over the samples
of the relative p-norm errors of the effective stiffness, divided by N_b, plus
the penalty lambda (sum_i <v_i>_+ - 1)^2 on the leaf weights w = <v>_+.  The
paper takes p = 1 (the l1 norm of the Voigt components), q = 10 and
lambda = 1e3, AMSGrad with the learning rate

    alpha(m) = gamma^m (alpha_min + (alpha_max - alpha_min) (1 + cos(pi m / M)) / 2),

M = 50, gamma = 0.999, alpha_max = 1.5e-2, alpha_min = 1.5e-3, initial angle
coefficients uniform on [0, 2 pi] and weights uniform on [0, 1], rescaled to sum 1.

The paper's training data (FFT-computed stiffnesses of SAM microstructures) are
not available; the targets here come from a second, seeded DMN: effective
stiffnesses of elastic phases and, optionally, stresses of one elastoplastic
increment from the virgin state (relative Frobenius error), as in the
differentiation workload.  Every forward and backward pass runs through
dmn_update and dmn_grad.

Learning rates: the paper sets them by a learning-rate sweep and finds them
almost equal for p, q and v.  The weights here start at 1/2^K each, so one
AMSGrad step of the angle coefficients' size (about alpha) would move every
weight by several times its value; the weights' rate is scaled by
min(1, 8 / 2^K) (`lr_scale_v`), which bounds a step at about a tenth of a
weight.

The stiffness samples take, by default, the tangent of one update from the virgin
state at zero strain in the mixed form (its tangent is the FP64 final sweep's,
exact for elastic phases) and a tangent-seeded adjoint: one reverse pass through
the laminate recursion per sample (`stiffness_method="tangent"`).  The previous
route, six stresses at the Mandel unit strains and six stress adjoints per
sample, remains as `stiffness_method="stress"` (needed with an FP32 tangent).
The plastic samples' forward solves use the mixed form with an FP32 tangent
(`plastic_precision`): the Newton iteration stops on the same FP64 residual
criterion, so the stresses the loss reads are the FP64 solution's (to about
1e-11), and the adjoint recomputes in FP64 at the converged jumps.  The plastic
solves are latency-bound (few points, many line-search steps), and the FP32
condensation has shorter dependency chains.

A weight that reaches zero stays there (the Macaulay bracket has no gradient
below zero), and the tree is compressed (Sec. 3.1): with `compress` (default)
the weights are w = <v>_+ exactly, and whenever the set of zero weights changes
the DMN handles are rebuilt on the newly compressed tree, so that later epochs
condense fewer laminates.  Without it, w is floored at `w_floor` and the tree
stays whole.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import autograd as ag
from . import dmn
from . import workloads as W


def lr_schedule(m, alpha_min=1.5e-3, alpha_max=1.5e-2, M=50, gamma=0.999):
    """Learning rate of epoch m (Sec. 4.4)."""
    return gamma ** m * (alpha_min + 0.5 * (alpha_max - alpha_min) * (1.0 + math.cos(math.pi * m / M)))


def voigt_scale(device):
    """Factors turning a Mandel stiffness into its Voigt (engineering shear strain) form:
    C_voigt[I, J] = C_mandel[I, J] / (w_I w_J) with w = (1, 1, 1, sqrt2, sqrt2, sqrt2)."""
    import torch
    w = torch.tensor([1.0, 1.0, 1.0, math.sqrt(2.0), math.sqrt(2.0), math.sqrt(2.0)], dtype=torch.float64,
                     device=device)
    return 1.0 / (w[:, None] * w[None, :])


def stiffness_loss(C, C_t, p_norm=1, q_norm=10):
    """(1/N_b) (sum_s (||C_s - C_t,s||_p / ||C_t,s||_p)^q)^(1/q), norms over the Voigt components."""
    import torch
    vs = voigt_scale(C.device)
    d = ((C - C_t) * vs).reshape(C.shape[0], -1)
    t = (C_t * vs).reshape(C.shape[0], -1)
    e = torch.linalg.vector_norm(d, ord=p_norm, dim=1) / torch.linalg.vector_norm(t, ord=p_norm, dim=1)
    return torch.linalg.vector_norm(e, ord=q_norm) / C.shape[0]


def sample_errors(C, C_t):
    """Sample-wise errors e_s = ||C_s - C_t,s||_1 / ||C_t,s||_1 (Voigt components)."""
    import torch
    vs = voigt_scale(C.device)
    d = ((C - C_t) * vs).reshape(C.shape[0], -1)
    t = (C_t * vs).reshape(C.shape[0], -1)
    return torch.linalg.vector_norm(d, ord=1, dim=1) / torch.linalg.vector_norm(t, ord=1, dim=1)


class Trainer:
    """AMSGrad on (p, q, v) of a depth-K DMN with linear shape functions.

    target: TreeParams of the reference DMN; elastic phases (fiber, elastic matrix) for the
    stiffness samples; `plastic` (a J2 phase) adds stress samples of one increment."""

    def __init__(self, K, target, n_stiff, seed, elastic_matrix, plastic=None, n_plastic=0, lam_pen=1e3,
                 w_floor=1e-9, alpha_max=1.5e-2, alpha_min=1.5e-3, lr_scale_v=None, compress=True,
                 plastic_precision="mixed-f32-tangent", elastic_precision="mixed", stiffness_method=None):
        import torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        rng = np.random.default_rng(seed)
        N, L, M = (1 << K) - 1, 1 << K, 3
        self.K, self.lam_pen, self.w_floor, self.compress_on = K, lam_pen, w_floor, compress
        self.rebuilds = 0
        self.pl_prec = plastic_precision
        self.el_prec = elastic_precision
        self.stiff_method = stiffness_method   # dmn_stiffness method (None: tangent seeds with an FP64 tangent)
        self.side = torch.cuda.Stream()   # the plastic samples' stream (see loss)
        self.alpha = (alpha_min, alpha_max)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(self.dev)
        # initial parameters as in Sec. 4.4
        self.p = d(rng.uniform(0.0, 2 * np.pi, (N, M))).requires_grad_()
        self.q = d(rng.uniform(0.0, 2 * np.pi, (N, M))).requires_grad_()
        v0 = rng.uniform(0.0, 1.0, L)
        self.v = d(v0 / v0.sum()).requires_grad_()
        self.lr_scale = [1.0, min(1.0, 8.0 / L) if lr_scale_v is None else lr_scale_v]
        self.opt = torch.optim.Adam([{"params": [self.p, self.q]}, {"params": [self.v]}], lr=alpha_max, amsgrad=True)
        el_phases = (W.FIBER, elastic_matrix)
        self.el_phases = el_phases
        self.pl_phases = None if plastic is None else (W.FIBER, plastic)
        start = W.TreeParams(K, M, self.p.detach().cpu().numpy(), self.q.detach().cpu().numpy(), v0 / v0.sum(),
                             el_phases)
        # the stiffness samples' update at zero strain meets the criterion at its first evaluation: an
        # all-FP32 first stage would only add a pass
        self.m_el = dmn.DMN(start, precision=elastic_precision, first_stage=False)
        self.pattern = v0 > 0
        tgt_el = dmn.DMN(W.TreeParams(K, M, target.p, target.q, target.w, el_phases))
        A2, lam, Q = W.orientation_field(n_stiff, seed=seed + 1)
        self.lam_e, self.Q_e = d(lam), d(Q)
        with torch.no_grad():
            self.C_t = ag.dmn_stiffness(tgt_el, self.lam_e, self.Q_e, d(target.p), d(target.q), d(target.w))
        tgt_el.close()
        self.m_pl = None
        if plastic is not None and n_plastic > 0:
            pl_phases = (W.FIBER, plastic)
            self.m_pl = dmn.DMN(W.TreeParams(K, M, start.p, start.q, start.w, pl_phases), line_search=True,
                                precision=plastic_precision)
            tgt_pl = dmn.DMN(W.TreeParams(K, M, target.p, target.q, target.w, pl_phases), line_search=True)
            A2, lam, Q = W.orientation_field(n_plastic, seed=seed + 2)
            self.lam_p, self.Q_p = d(lam), d(Q)
            E = W.random6_path_final(n_plastic, 1.0, seed=seed + 3) * rng.uniform(0.01, 0.03, (n_plastic, 1))
            self.E_p = d(E)
            self.zE = torch.zeros_like(self.E_p)
            self.z_st = torch.zeros((self.m_pl.state_size, n_plastic), dtype=torch.float64, device=self.dev)
            with torch.no_grad():
                self.s_t = ag.dmn_stress(tgt_pl, self.lam_p, self.Q_p, self.zE, self.E_p, self.z_st, d(target.p),
                                         d(target.q), d(target.w))[0]
            tgt_pl.close()
        self.epoch = 0
        self.history = []

    def weights(self):
        """w = <v>_+ (compressing), or floored at w_floor (the floor carries no gradient)."""
        import torch
        return torch.clamp(self.v, min=0.0 if self.compress_on else self.w_floor)

    def _recompress(self, w):
        """New handles when the set of zero weights has changed (another compressed tree)."""
        import torch
        pattern = (w.detach() > 0).cpu().numpy()
        if (pattern == self.pattern).all():
            return
        self.pattern = pattern
        self.rebuilds += 1
        p, q, wn = (x.detach().cpu().numpy() for x in (self.p, self.q, w))
        self.m_el.close()
        self.m_el = dmn.DMN(W.TreeParams(self.K, 3, p, q, wn, self.el_phases), precision=self.el_prec,
                            first_stage=False)
        if self.m_pl is not None:
            self.m_pl.close()
            self.m_pl = dmn.DMN(W.TreeParams(self.K, 3, p, q, wn, self.pl_phases), line_search=True,
                                precision=self.pl_prec)
            self.z_st = torch.zeros((self.m_pl.state_size, self.E_p.shape[0]), dtype=torch.float64,
                                    device=self.dev)

    def loss(self):
        import torch
        w = self.weights()
        if self.compress_on:
            self._recompress(w)
        # The plastic samples (few points, many Newton steps, latency-bound) run on a stream of their
        # own, beside the stiffness samples; autograd runs each backward on its forward's stream, so
        # the two adjoints overlap too.  Parameter uploads synchronise the device: both come first.
        ag.sync_params(self.m_el, self.p, self.q, w)
        if self.m_pl is not None:
            ag.sync_params(self.m_pl, self.p, self.q, w)
            main = torch.cuda.current_stream()
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                s, _, stat = ag.dmn_stress(self.m_pl, self.lam_p, self.Q_p, self.zE, self.E_p, self.z_st, self.p,
                                           self.q, w)
                # unconverged samples contribute 0 (a mask by indexing would stop the host until the
                # solve ends, and the stiffness samples could not be queued beside it)
                e = torch.linalg.norm(s - self.s_t, dim=1) / torch.linalg.norm(self.s_t, dim=1)
                e = torch.where(stat == 0, e, torch.zeros_like(e))
                J_pl = torch.linalg.vector_norm(e, ord=10) / s.shape[0]
        C = ag.dmn_stiffness(self.m_el, self.lam_e, self.Q_e, self.p, self.q, w, method=self.stiff_method)
        J = stiffness_loss(C, self.C_t)
        if self.m_pl is not None:
            torch.cuda.current_stream().wait_stream(self.side)
            J = J + J_pl
        pen = self.lam_pen * (torch.clamp(self.v, min=0.0).sum() - 1.0) ** 2
        return J + pen, C

    def step(self):
        """One epoch (the whole sample set as one batch): returns (loss, max sample error, mean)."""
        import torch
        for g, f in zip(self.opt.param_groups, self.lr_scale):
            g["lr"] = f * lr_schedule(self.epoch, *self.alpha)
        self.opt.zero_grad()
        L, C = self.loss()
        L.backward()
        self.opt.step()
        with torch.no_grad():
            e = sample_errors(C, self.C_t)
        self.epoch += 1
        rec = (float(L.item()), float(e.max().item()), float(e.mean().item()))
        self.history.append(rec)
        return rec

    def train(self, epochs):
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(epochs):
            self.step()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def compress(self, rel=1e-6):
        """TreeParams of the trained DMN, weights below rel * max set to zero (tree compression)."""
        w = self.weights().detach().cpu().numpy().copy()
        w[w < rel * w.max()] = 0.0
        return W.TreeParams(self.K, 3, self.p.detach().cpu().numpy(), self.q.detach().cpu().numpy(), w,
                            (W.FIBER, W.MATRIX))

    def close(self):
        self.m_el.close()
        if self.m_pl is not None:
            self.m_pl.close()
