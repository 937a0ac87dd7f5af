"""The learned right preconditioner's network and its flexible solver.

The network's forward pass, loss and gradients (hand-written kernels) are
compared with a plain PyTorch CPU float64 restatement of the same network
(same BF16-rounded weights), on a lattice with odd sizes (partial 2x2x2
cells at every level); the kernels are deterministic; training lowers the
loss; and the flexible Bi-CGSTAB reaches the exact (dense) solution with and
without the network.
"""
import numpy as np
import pytest

from oracle import system
from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu, rel_l2, twin

pytestmark = pytest.mark.gpu

LAYERS = ((7, 16, 3), (16, 32, 3), (32, 160, 3), (160, 160, 3), (192, 32, 3), (48, 16, 3), (16, 6, 1))


def _split(w):
    """Flat parameter array -> [(weight (cout, cin, k, k, k), bias (cout,))]."""
    out, o = [], 0
    for cin, cout, k in LAYERS:
        n = cout * cin * k ** 3
        W = w[o:o + n].reshape(cout, cin, k, k, k)
        o += n
        b = w[o:o + cout]
        o += cout
        out.append((W, b))
    assert o == w.size
    return out


def _reference(torch, w, occ, v):
    """The network restated with torch CPU float64 ops; returns (z, tensors
    needing gradients)."""
    F = torch.nn.functional
    occ = occ > 0
    nz, ny, nx = occ.shape
    params = []
    for W, b in _split(w):
        Wt = torch.tensor(W, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).requires_grad_(True)
        bt = torch.tensor(b, dtype=torch.float64).requires_grad_(True)
        params.append((Wt, bt))
    idx = np.argwhere(occ)                            # (z, y, x) in scan order (x fastest)
    vt = torch.tensor(v)
    scale = torch.sqrt((vt.abs() ** 2).sum() / vt.numel())
    grid = torch.zeros(7, nz + nz % 2, ny + ny % 2, nx + nx % 2, dtype=torch.float64)
    for c in range(3):
        grid[2 * c, idx[:, 0], idx[:, 1], idx[:, 2]] = vt[c].real / scale
        grid[2 * c + 1, idx[:, 0], idx[:, 1], idx[:, 2]] = vt[c].imag / scale
    grid[6, idx[:, 0], idx[:, 1], idx[:, 2]] = 1.0
    f0 = F.avg_pool3d(grid[None], 2)[0]                # sum / 8 over the 2x2x2 cell

    def conv(x, L, relu=True):
        W, b = params[L]
        y = F.conv3d(x[None], W, b, padding=W.shape[-1] // 2)[0]
        return torch.relu(y) if relu else y

    def pool(x):
        d, h, wd = x.shape[1:]
        xp = F.pad(x, (0, wd % 2, 0, h % 2, 0, d % 2))
        ones = F.pad(torch.ones(1, d, h, wd, dtype=x.dtype), (0, wd % 2, 0, h % 2, 0, d % 2))
        return F.avg_pool3d(xp[None], 2)[0] / F.avg_pool3d(ones[None], 2)[0]

    def up(x, shape):
        y = x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)
        return y[:, :shape[0], :shape[1], :shape[2]]

    a0 = conv(f0, 0)
    a1 = conv(pool(a0), 1)
    a3 = conv(conv(pool(a1), 2), 3)
    a4 = conv(torch.cat([up(a3, a1.shape[1:]), a1]), 4)
    a5 = conv(torch.cat([up(a4, a0.shape[1:]), a0]), 5)
    o6 = conv(a5, 6, relu=False)
    cz, cy, cx = idx[:, 0] // 2, idx[:, 1] // 2, idx[:, 2] // 2
    z = torch.stack([torch.complex(o6[2 * c, cz, cy, cx], o6[2 * c + 1, cz, cy, cx]) for c in range(3)])
    return vt + z * scale, params


@pytest.fixture(scope="module")
def lattice():
    torch, dda = need_gpu()
    occ = inputs.ellipsoid(13, 11, 9)
    p, prob = twin(occ, [1.6 + 0.02j], 0.45)
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
    yield p, prob, occ
    p.close()


def test_network_forward_and_gradients_match_reference(lattice):
    torch, dda = need_gpu()
    p, prob, occ = lattice
    net = dda.PcNet(seed=5)
    assert net.nparam == 1033430
    w = net.weights()
    r = inputs.random_vectors(31, 1, p.n_occ)[0]
    e = inputs.random_vectors(32, 1, p.n_occ)[0]
    rd = torch.from_numpy(r).cuda()
    ed = torch.from_numpy(e).cuda()
    zd = torch.empty_like(rd)
    net.apply(p.h, rd, zd)
    z_ref, params = _reference(torch, w, occ, r)
    assert rel_l2(zd.cpu().numpy(), z_ref.detach().numpy()) < 1e-4
    # deterministic
    zd2 = torch.empty_like(rd)
    net.apply(p.h, rd, zd2)
    assert torch.equal(zd, zd2)
    # one training step: loss and gradients before the update
    z1 = torch.empty_like(rd)
    loss = net.train_step(p.h, rd, ed, z1, 1e-4)
    et = torch.tensor(e)
    loss_ref = ((z_ref - et).abs() ** 2).sum() / (et.abs() ** 2).sum()
    assert abs(loss - loss_ref.item()) < 1e-5 * loss_ref.item()
    loss_ref.backward()
    g = net.grads()
    o = 0
    for (W, b), (cin, cout, k) in zip(params, LAYERS):
        n = cout * cin * k ** 3
        assert rel_l2(g[o:o + n], W.grad.numpy().ravel()) < 1e-3, (cin, cout)
        o += n
        assert rel_l2(g[o:o + cout], b.grad.numpy()) < 1e-3, (cin, cout)
        o += cout
    net.close()


def test_training_lowers_the_loss(lattice):
    torch, dda = need_gpu()
    p, prob, occ = lattice
    net = dda.PcNet(seed=1)
    beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
    dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
    # a pair of the system itself: e a smooth field (the network's output is
    # constant over 2x2x2 cells, so white noise could not be fitted), r = A e
    e = system.incident_field(prob.pos, prob.kd, (0.6, 0.0, 0.8), (0.8, 0.3j, -0.6))
    r = prob.matvec(beta, "fft")(e)
    rd = torch.from_numpy(r).cuda()
    ed = torch.from_numpy(e).cuda()
    z = torch.empty_like(rd)
    losses = [net.train_step(p.h, rd, ed, z, 1e-3) for _ in range(40)]
    assert np.mean(losses[-5:]) < 0.8 * np.mean(losses[:5]), losses[::8]
    net.close()


@pytest.mark.parametrize("with_net", [False, True])
def test_flexible_bicgstab_reaches_the_exact_solution(with_net):
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    p, prob = twin(occ, [1.5], None, volume_x=3.0)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
        b = system.rhs(beta, prob.pos, prob.kd, (0, 0, 1), (1, 0, 0))
        exact = beta * system.solve_dense(prob.pos, beta, prob.kd, b)
        net = dda.PcNet(seed=3) if with_net else None
        P = torch.zeros((3, p.n_occ), dtype=torch.complex128, device="cuda")
        st, info, hist = dda.dda_solve_pc(p.h, net, dict(pol=dda.DDA_LDR, tol=1e-9, maxiter=400),
                                          [(0, 0, 1)], [(1, 0, 0)], P, 64)
        assert st == dda.DDA_OK, info
        assert info["rel_res_true"] < 1e-9
        assert rel_l2(P.cpu().numpy(), exact) < 1e-7
        assert hist[0] == 1.0
        if net is not None:
            net.close()
