"""Offline training through the GPU adjoint (Sec. 3.1 loss, AMSGrad with the
schedule of Sec. 4.4) against a seeded target DMN."""
import pytest
import torch

from paper_2103_08253_gb300 import dmn, training as T, workloads as W

pytestmark = pytest.mark.gpu
EL_MATRIX = W.Phase(0, 3000.0, 0.35)


@pytest.mark.parametrize("n_plastic", [0, 64])
def test_training_lowers_the_loss(n_plastic):
    """80 epochs lower the loss; weights that reach zero compress the tree (Sec. 3.1)."""
    K = 4
    target = W.tree_d10_fit(K, seed=2)
    tr = T.Trainer(K, target, 128, seed=3, elastic_matrix=EL_MATRIX, plastic=W.MATRIX, n_plastic=n_plastic)
    first = tr.step()
    tr.train(80)
    last = tr.history[-1]
    assert last[0] < 0.75 * first[0], (first, last)
    assert last[2] < 0.9 * first[2], (first, last)
    # weights driven to zero compress the tree: the handles follow the set of zero weights
    assert (tr.weights() > 0).sum().item() == int(tr.pattern.sum())
    # the trained (and compressed) tree runs online
    t = tr.compress()
    m = dmn.DMN(t)
    n = 16
    A2, lam, Q = W.orientation_field(n, seed=4)
    dev = torch.device("cuda:0")
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=dev)
    E = torch.from_numpy(W.random6_path_final(n, 0.01, seed=5)).to(dev)
    o = m.update(torch.from_numpy(lam).to(dev), torch.from_numpy(Q).to(dev), torch.zeros_like(E), E, st)
    assert (o["status"] == 0).all()
    m.close()
    tr.close()


def test_optimiser_steps_follow_amsgrad_and_the_schedule():
    """Three epochs: the learning rates are those of the schedule of Sec. 4.4 (the weights' rate
    scaled by lr_scale_v), and every parameter update equals a numpy restatement of AMSGrad
    (the maximum of the second-moment estimates in the denominator) in the bias-corrected form
    of Adam, on the gradients the adjoint produced for that epoch."""
    import numpy as np
    K = 3
    target = W.tree_d10_fit(K, seed=12)
    tr = T.Trainer(K, target, 64, seed=13, elastic_matrix=EL_MATRIX, plastic=W.MATRIX, n_plastic=16)
    b1, b2, eps = 0.9, 0.999, 1e-8
    seen = []
    orig = tr.opt.step

    def spy():
        seen.append(dict(g=[x.grad.detach().cpu().numpy().copy() for x in (tr.p, tr.q, tr.v)],
                         x=[x.detach().cpu().numpy().copy() for x in (tr.p, tr.q, tr.v)],
                         lr=[grp["lr"] for grp in tr.opt.param_groups]))
        orig()
    tr.opt.step = spy
    m = v = vmax = None
    for epoch in range(3):
        tr.step()
        rec = seen[-1]
        sched = T.lr_schedule(epoch)
        assert abs(rec["lr"][0] - sched) <= 1e-15 * sched
        assert abs(rec["lr"][1] - min(1.0, 8.0 / (1 << K)) * sched) <= 1e-15 * sched
        if m is None:
            m = [np.zeros_like(x) for x in rec["x"]]
            v = [np.zeros_like(x) for x in rec["x"]]
            vmax = [np.zeros_like(x) for x in rec["x"]]
        t = epoch + 1
        after = [x.detach().cpu().numpy() for x in (tr.p, tr.q, tr.v)]
        for k in range(3):
            g = rec["g"][k]
            lr = rec["lr"][0 if k < 2 else 1]
            m[k] = b1 * m[k] + (1 - b1) * g
            v[k] = b2 * v[k] + (1 - b2) * g * g
            vmax[k] = np.maximum(vmax[k], v[k])
            step = lr / (1 - b1 ** t) * m[k] / (np.sqrt(vmax[k]) / np.sqrt(1 - b2 ** t) + eps)
            np.testing.assert_allclose(after[k], rec["x"][k] - step, rtol=1e-13, atol=1e-15)
    tr.close()
