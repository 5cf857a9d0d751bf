"""Host logic of the device inversion loop, on CPU tensors (no engine involved):
the Tikhonov term and its autograd gradient against the oracle's numpy statement,
and the two-loop recursion against the oracle's (Sec. 3.5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import inversion as oinv  # noqa: E402
from paper_2211_16665_gb300.inversion import Inversion, Tikhonov  # noqa: E402
from paper_2211_16665_gb300.workloads import stretched_axis  # noqa: E402


def grid():
    xn = stretched_axis(100.0, 6, 2, 2, 2, 1.2, -600.0)
    yn = stretched_axis(80.0, 5, 1, 1, 2, 1.1, -400.0)
    zn = stretched_axis(50.0, 4, 1, 2, 1, 1.3, 0.0)
    return xn, yn, zn


@pytest.mark.parametrize("lead", [(), (2,)])
def test_tikhonov_matches_oracle(lead):
    xn, yn, zn = grid()
    shape = lead + (zn.size - 1, yn.size - 1, xn.size - 1)
    rng = np.random.default_rng(7)
    m = rng.normal(size=shape)
    ref = rng.normal(size=shape)
    free = rng.random(shape) > 0.25
    alpha = (1.0, 0.7, 0.1)
    phi_o, g_o = oinv.tikhonov(m, ref, free, xn, yn, zn, alpha)
    reg = Tikhonov(xn, yn, zn, torch.as_tensor(free), torch.as_tensor(ref), alpha)
    mt = torch.as_tensor(m).requires_grad_(True)
    phi = reg(mt)
    phi.backward()
    assert abs(float(phi.detach()) - phi_o) <= 1e-12 * phi_o
    np.testing.assert_allclose(mt.grad.numpy(), g_o, rtol=1e-10, atol=1e-12)


def test_two_loop_direction_matches_oracle():
    rng = np.random.default_rng(3)
    n = 9
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    pairs = []
    for _ in range(4):
        s = rng.normal(size=n)
        pairs.append((s, A @ s))
    g = rng.normal(size=n)
    d_o = oinv.lbfgs_direction(g, pairs)
    d = Inversion._direction(Inversion.__new__(Inversion), torch.as_tensor(g),
                             [(torch.as_tensor(s), torch.as_tensor(y)) for s, y in pairs])
    np.testing.assert_allclose(d.numpy(), d_o, rtol=1e-12, atol=1e-14)
