"""The Python bindings reject wrong arrays before anything reaches the library.

Every array the kernels read or write is checked for dtype, contiguity, shape
and device (the handle's), so a caller's mistake raises on the host instead of
handing the library a buffer it would read or write out of bounds.  No call
here launches a kernel with a bad array: each one raises first.
"""
import numpy as np
import pytest
import torch

from paper_2103_08253_gb300 import dmn, fe, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def handle():
    tree = W.tree_d10_fit(3, seed=5)
    m = dmn.DMN(tree)
    yield m, tree
    m.close()


def test_handle_records_its_device(handle):
    m, _ = handle
    assert m.device == torch.device("cuda", torch.cuda.current_device())


@pytest.mark.parametrize("case", ["f32", "cpu", "noncontig", "shape", "state_rows", "tangent_flat", "iters_i64"])
def test_update_rejects_wrong_arrays(handle, case):
    m, _ = handle
    n = 8
    args = dict(lam=f64(n, 2), Q=f64(n, 9), E_n=f64(n, 6), dE=f64(n, 6), state_in=f64(m.state_size, n))
    out = m.alloc_outputs(n, DEV)
    err = ValueError
    if case == "f32":
        args["lam"] = args["lam"].float(); err = TypeError
    elif case == "cpu":
        args["dE"] = args["dE"].cpu(); err = TypeError
    elif case == "noncontig":
        args["Q"] = f64(9, n).t()
    elif case == "shape":
        args["E_n"] = f64(n + 1, 6)
    elif case == "state_rows":
        args["state_in"] = f64(m.state_size - 1, n)
    elif case == "tangent_flat":
        out["tangent"] = f64(n, 36)
    elif case == "iters_i64":
        out["iters"] = torch.zeros(n, dtype=torch.int64, device=DEV); err = TypeError
    with pytest.raises(err):
        m.update(args["lam"], args["Q"], args["E_n"], args["dE"], args["state_in"], out=out)


def test_grad_rejects_wrong_accumulators(handle):
    m, tree = handle
    n = 4
    N = (1 << tree.K) - 1
    a = (f64(n, 2), f64(n, 9), f64(n, 6), f64(n, 6), f64(m.state_size, n), f64(m.state_size, n), f64(n, 6))
    with pytest.raises(ValueError, match="g_p"):
        m.grad(*a, g_p=f64(N + 1, tree.M))
    with pytest.raises(ValueError, match="g_w"):
        m.grad(*a, g_w=f64(1 << (tree.K - 1)))
    with pytest.raises(TypeError, match="g_q"):
        m.grad(*a, g_q=torch.zeros((N, tree.M), dtype=torch.float32, device=DEV))


def test_set_params_rejects_wrong_sizes(handle):
    m, tree = handle
    with pytest.raises(ValueError, match="p has"):
        m.set_params(tree.p[:-1], tree.q, tree.w)
    with pytest.raises(ValueError, match="w has"):
        m.set_params(tree.p, tree.q, np.append(tree.w, 0.1))
    with pytest.raises(ValueError, match="tree_id"):
        m.set_params(tree.p, tree.q, tree.w, tree_id=1)


def test_update_host_rejects_device_arrays(handle):
    m, _ = handle
    n = 4
    with pytest.raises(TypeError):
        m.update_host(f64(n, 2), f64(n, 9).cpu(), f64(n, 6).cpu(), f64(n, 6).cpu(), f64(m.state_size, n).cpu())


def test_fe_mesh_rejects_wrong_arrays():
    pm = W.plate_with_hole_mesh(4, 2, 1, R=2.0, H=6.0, T=2.0)
    g = fe.Hex8Mesh(pm.xyz, pm.conn)
    nd, ng = g.n_dofs, g.n_gp
    with pytest.raises(TypeError):
        g.strain(torch.zeros(nd, dtype=torch.float32, device=DEV))
    with pytest.raises(ValueError):
        g.strain(f64(nd - 3))
    with pytest.raises(ValueError):
        g.internal_force(f64(ng, 5))
    with pytest.raises(ValueError):
        g.apply_tangent(f64(ng, 35), f64(nd))
    with pytest.raises(TypeError):
        g.dot(f64(nd), f64(nd).cpu())
    with pytest.raises(ValueError):
        g.pcg(f64(ng, 6, 6), f64(nd), f64(nd), f64(nd), f64(nd + 1))
    with pytest.raises(ValueError):
        g.axpy(1.0, f64(nd), f64(nd), free=f64(2 * nd)[::2])
    # the accepted tangent layouts, [n_gp, 36] and [n_gp, 6, 6], give the same product
    C = torch.eye(6, dtype=torch.float64, device=DEV).expand(ng, 6, 6).contiguous()
    u = torch.linspace(0.0, 1e-3, nd, dtype=torch.float64, device=DEV)
    assert torch.equal(g.apply_tangent(C, u), g.apply_tangent(C.reshape(ng, 36), u))
    g.close()
    with pytest.raises(ValueError):
        fe.Hex8Mesh(pm.xyz[:, :2], pm.conn)


def test_noalloc_binding_rejects_wrong_state():
    tree = W.tree_d10_fit(3, seed=6)
    n = 4
    S = W.state_size(3)
    with pytest.raises(ValueError, match="state_in"):
        dmn.update_noalloc(tree, f64(n, 2), f64(n, 9), f64(n, 6), f64(n, 6), f64(S + 1, n))
