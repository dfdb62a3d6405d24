"""dmn_update_host: the update with host arrays, chunked and pipelined.

Each point is computed by the same kernels as in dmn_update, on its own inputs,
so the results must be bit-identical to dmn_update on device copies of the same
arrays, whatever the chunking.  The FP64 results are also checked against the
CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def host(x, pin=True):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory() if pin else t


def rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("prec,chunk,pin", [("f64", 300, True), ("mixed", 257, True), ("f64", 0, False)])
def test_host_update_is_bitwise_the_device_update(prec, chunk, pin):
    K, n, steps = 8, 1000, 3
    tree = W.tree_d10_fit(K, seed=41)
    A2, lam, Q = W.orientation_field(n, seed=42)
    Ef = W.random6_path_final(n, 0.03, seed=43)
    m = dmn.DMN(tree, precision=prec)
    S = m.state_size
    st_h = host(np.zeros((S, n)), pin)                 # updated in place on the host
    st_d = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    out_h = m.alloc_host_outputs(n, pin=pin)
    lam_h, Q_h = host(lam, pin), host(Q, pin)
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, 5)        # plastic from the second call on
        out_h["state_out"] = st_h
        m.update_host(lam_h, Q_h, host(En, pin), host(dE, pin), st_h, out=out_h, chunk=chunk)
        out_d = m.update(lam_h.to(DEV), Q_h.to(DEV), host(En).to(DEV), host(dE).to(DEV), st_d)
        st_d = out_d["state_out"]
        for k in ("stress", "tangent", "iters", "status"):
            assert same(out_h[k].numpy(), out_d[k].cpu().numpy()), k
        assert same(st_h.numpy(), st_d.cpu().numpy())
    stat = out_h["status"].numpy()
    assert (stat == 0).mean() > 0.95
    if prec == "f64":
        st_o = np.zeros((S, n))
        for s in range(1, steps + 1):
            En, dE = W.proportional_increment(Ef, s, 5)
            st_o, so, Co, io, sto, gap = oracle.update(tree, lam, Q, En, dE, st_o)
        assert (stat == sto).mean() > 0.95
        ok = (stat == 0) & (sto == 0)
        assert rel(out_h["stress"].numpy()[ok], so[ok]).max() <= 1e-10
        ok &= gap > 1e-9
        assert rel(out_h["tangent"].numpy()[ok], Co[ok]).max() <= 1e-10


def test_host_update_with_tree_ids_and_a_bad_tree():
    depths = (5, 6, 7, 8)
    n = 900
    trees = [W.tree_d10_fit(K, seed=60 + K) for K in depths]
    tid, elastic = W.mixed_depth_batch(n, 61, depths)
    tid[[5, 400]] = [7, -2]
    A2, lam, Q = W.orientation_field(n, seed=62)
    Edir = W.random6_path_final(n, 1.0, seed=63)
    amp = np.where(elastic, 0.001, 0.02)[:, None] * Edir
    m = dmn.DMN(trees, precision="f64")
    S = m.state_size
    st0 = np.full((S, n), 0.0)
    st_h = host(st0)
    out_h = m.alloc_host_outputs(n)
    out_h["state_out"] = st_h
    st_d = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    for s in (1, 2):
        En, dE = W.cyclic_increment(amp, s, 16)
        m.update_host(host(lam), host(Q), host(En), host(dE), st_h, out=out_h, tree_id=host(tid), chunk=128)
        out_d = m.update(host(lam).to(DEV), host(Q).to(DEV), host(En).to(DEV), host(dE).to(DEV), st_d,
                         tree_id=host(tid).to(DEV))
        good = (tid >= 0) & (tid < len(trees))
        stat = out_h["status"].numpy()
        assert (stat[~good] == dmn.STATUS_BAD_TREE).all() and (stat[good] == 0).mean() > 0.95
        for k in ("stress", "tangent"):
            assert same(out_h[k].numpy()[good], out_d[k].cpu().numpy()[good]), k
        assert same(out_h["iters"].numpy(), out_d["iters"].cpu().numpy())
        sd = out_d["state_out"].cpu().numpy()
        for k in range(len(trees)):             # a point of tree k owns the first S_k state fields
            idx = np.nonzero(tid == k)[0]
            Sk = m.tree_state_sizes[k]
            assert same(st_h.numpy()[:Sk, idx], sd[:Sk, idx])
        # a point of an unknown tree keeps its state (in place: the input)
        assert (st_h.numpy()[:, ~good] == 0.0).all()
        st_d = out_d["state_out"].clone()
        st_d[:, torch.from_numpy(~good).to(DEV)] = 0.0


def test_host_update_argument_errors():
    tree = W.tree_constant_normals(3, seed=1)
    m = dmn.DMN(tree)
    n = 4
    lam, Q = (host(x) for x in W.identity_orientation(n))
    z = host(np.zeros((n, 6)))
    with pytest.raises(TypeError):
        m.update_host(lam.to(DEV), Q, z, z, host(np.zeros((m.state_size, n))))
    with pytest.raises(ValueError):
        m.update_host(lam, Q, z, z, host(np.zeros((m.state_size + 1, n))))
