"""torch.autograd bindings of the DMN update and its adjoint (dmn_grad).

`dmn_stress(m, lam, Q, E_n, dE, state_in, p, q, w)` returns the converged
effective stress of an update and, in the backward pass, gradients with
respect to the DMN parameters p, q (angle coefficients, Sec. 2.3), w (leaf
weights) and the macro strain, from the implicit-function adjoint of the
converged Newton solution (the condensation at the converged jumps is
recomputed; nothing from the iterations is stored).

`dmn_stiffness(m, lam, Q, p, q, w)` returns the effective stiffness of a DMN
with linear elastic phases (the offline-training quantity of Sec. 3.1).  By
default (a handle whose tangent is FP64: precision "f64" or "mixed") it is the
tangent of one update from the virgin state at zero strain, and its backward
pass is dmn_grad with a tangent seed: one reverse pass through the laminate
recursion per sample.  method="stress" takes instead the six stresses at the
Mandel unit strains (sigma_bar = C_bar E holds exactly for elastic phases) and
six stress adjoints, <G, C_bar> = sum_k G[:, k] . sigma_bar(E = e_k); the
handles of the FP32-tangent form use it, since their stresses, not their
tangents, are FP64.

Both run every step through the C ABI; the parameters are uploaded with
dmn_set_params when they differ from the ones the handle holds.
"""
from __future__ import annotations

import torch


def sync_params(m, p, q, w):
    """Upload p, q, w to the handle if they differ from the ones it holds (synchronises the device)."""
    key = tuple(x.detach().double().cpu().numpy().tobytes() for x in (p, q, w))
    if getattr(m, "_param_key", None) != key:
        m.set_params(p.detach().double().cpu().numpy(), q.detach().double().cpu().numpy(),
                     w.detach().double().cpu().numpy())
        m._param_key = key


class _Stress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, lam, Q, E_n, dE, state_in, p, q, w):
        sync_params(m, p, q, w)
        out = m.update(lam, Q, E_n.detach(), dE.detach(), state_in)
        ctx.m = m
        ctx.save_for_backward(lam, Q, E_n.detach(), dE.detach(), state_in, out["state_out"], out["status"])
        ctx.shapes = (p.shape, q.shape, w.shape)
        ctx.mark_non_differentiable(out["state_out"], out["status"])
        return out["stress"], out["state_out"], out["status"]

    @staticmethod
    def backward(ctx, g_stress, _g_state, _g_status):
        lam, Q, E_n, dE, state_in, state_out, status = ctx.saved_tensors
        g = torch.where((status == 0)[:, None], g_stress, torch.zeros_like(g_stress)).contiguous()
        g_p, g_q, g_w, g_E = ctx.m.grad(lam, Q, E_n, dE, state_in, state_out, g)
        sp, sq, sw = ctx.shapes
        return (None, None, None, g_E, g_E, None, g_p.reshape(sp), g_q.reshape(sq), g_w.reshape(sw))


def dmn_stress(m, lam, Q, E_n, dE, state_in, p, q, w):
    """(stress [n, 6], state_out, status) of one update; differentiable in E_n, dE, p, q, w."""
    return _Stress.apply(m, lam, Q, E_n, dE, state_in, p, q, w)


class _Stiffness(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, lam, Q, p, q, w):
        sync_params(m, p, q, w)
        n = lam.shape[0]
        dev = lam.device
        S = m.state_size
        zero_state = torch.zeros((S, 6 * n), dtype=torch.float64, device=dev)
        lam6, Q6 = lam.repeat(6, 1), Q.repeat(6, 1)
        E0 = torch.zeros((6 * n, 6), dtype=torch.float64, device=dev)
        dE = torch.eye(6, dtype=torch.float64, device=dev).repeat_interleave(n, dim=0)
        out = m.update(lam6, Q6, E0, dE, zero_state)
        C = out["stress"].reshape(6, n, 6).permute(1, 2, 0).contiguous()   # C[:, :, k] = sigma(e_k)
        ctx.m = m
        ctx.save_for_backward(lam6, Q6, E0, dE, zero_state, out["state_out"])
        ctx.n = n
        ctx.shapes = (p.shape, q.shape, w.shape)
        return C

    @staticmethod
    def backward(ctx, G):
        lam6, Q6, E0, dE, st_in, st_out = ctx.saved_tensors
        n = ctx.n
        g = G.permute(2, 0, 1).reshape(6 * n, 6).contiguous()   # row block k: G[:, :, k]
        g_p, g_q, g_w, _ = ctx.m.grad(lam6, Q6, E0, dE, st_in, st_out, g, want_E=False)
        sp, sq, sw = ctx.shapes
        return None, None, None, g_p.reshape(sp), g_q.reshape(sq), g_w.reshape(sw)


class _StiffnessTangent(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, lam, Q, p, q, w):
        sync_params(m, p, q, w)
        n = lam.shape[0]
        dev = lam.device
        zero_state = torch.zeros((m.state_size, n), dtype=torch.float64, device=dev)
        E0 = torch.zeros((n, 6), dtype=torch.float64, device=dev)
        out = m.update(lam, Q, E0, E0, zero_state)
        ctx.m = m
        ctx.save_for_backward(lam, Q)
        ctx.shapes = (p.shape, q.shape, w.shape)
        return out["tangent"]

    @staticmethod
    def backward(ctx, G):
        lam, Q = ctx.saved_tensors
        g_p, g_q, g_w, _ = ctx.m.grad(lam, Q, None, None, None, None, None, want_E=False,
                                      g_tangent=G.contiguous())
        sp, sq, sw = ctx.shapes
        return None, None, None, g_p.reshape(sp), g_q.reshape(sq), g_w.reshape(sw)


def dmn_stiffness(m, lam, Q, p, q, w, method=None):
    """Effective stiffness [n, 6, 6] (global frame) of a DMN with elastic phases; differentiable in p, q, w.
    method: "tangent" (the update's tangent, a tangent-seeded adjoint), "stress" (six stresses and six
    stress adjoints) or None (tangent unless the handle's tangent is FP32)."""
    for ph in m.phases:
        if ph.kind != 0:
            raise ValueError("dmn_stiffness needs linear elastic phases")
    if method is None:
        method = "stress" if m.precision == "mixed-f32-tangent" else "tangent"
    if method == "tangent":
        if m.precision == "mixed-f32-tangent":
            raise ValueError("method='tangent' needs an FP64 tangent (precision 'f64' or 'mixed')")
        return _StiffnessTangent.apply(m, lam, Q, p, q, w)
    if method != "stress":
        raise ValueError("method must be 'tangent' or 'stress'")
    return _Stiffness.apply(m, lam, Q, p, q, w)


def macaulay(v):
    """w = <v>_+ = max(v, 0): the weight parametrisation of Sec. 3.1."""
    return torch.clamp(v, min=0.0)


__all__ = ["dmn_stress", "dmn_stiffness", "macaulay"]
