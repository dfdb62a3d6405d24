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
