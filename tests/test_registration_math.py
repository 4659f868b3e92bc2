"""Pose parameterisation and error measures of the registration driver (no GPU)."""
import numpy as np
import torch

from paper_2406_02518_gb300 import registration as reg


def test_rodrigues_and_errors_on_cpu_tensors():
    w = torch.tensor([[0.0, 0.0, 0.0], [0.1, -0.2, 0.3]], dtype=torch.float64)
    R = reg.rodrigues(w).numpy()
    assert np.allclose(R[0], np.eye(3))
    assert np.allclose(R[1] @ R[1].T, np.eye(3), atol=1e-12)
    assert abs(reg.rotation_error_deg(R[1], np.eye(3)) - np.degrees(np.linalg.norm(w[1]))) < 1e-9


def test_compose_is_a_rotation_about_the_isocenter():
    R0 = torch.eye(3, dtype=torch.float64)[None]
    t0 = torch.tensor([[0.0, 0.0, 800.0]], dtype=torch.float64)
    w = torch.tensor([[0.0, 0.0, 0.2]], dtype=torch.float64)
    d = torch.zeros((1, 3), dtype=torch.float64)
    P = reg.compose(R0, t0, w, d, 10.0)[0].numpy()
    # the isocenter (world origin) stays at t0; a point on the x axis rotates about z
    assert np.allclose(P[:, 3], [0, 0, 800])
    x = P[:, :3] @ np.array([10.0, 0, 0]) + P[:, 3]
    assert np.allclose(x, [10 * np.cos(0.2), 10 * np.sin(0.2), 800])
    P2 = reg.compose(R0, t0, torch.zeros_like(w), torch.tensor([[1.0, 0, 0]], dtype=torch.float64), 10.0)
    assert np.allclose(P2[0, :, 3].numpy(), [10, 0, 800])
    assert abs(reg.translation_error_mm(P, P2[0].numpy()) - 10) < 1e-9



def test_rodrigues_gradient_is_finite_at_identity():
    w = torch.zeros((2, 3), dtype=torch.float64, requires_grad=True)
    R = reg.rodrigues(w)
    (R * torch.arange(9, dtype=torch.float64).view(3, 3)).sum().backward()
    assert torch.isfinite(w.grad).all()
    # d exp([w]x) / dw at 0 is the generator: compare with finite differences
    eps = 1e-6
    for i in range(3):
        wp = torch.zeros(3, dtype=torch.float64)
        wp[i] = eps
        fd = ((reg.rodrigues(wp) - reg.rodrigues(-wp)) / (2 * eps) * torch.arange(9, dtype=torch.float64).view(3, 3)).sum()
        assert abs(float(fd) - float(w.grad[0, i])) < 1e-6


def test_device_adam_matches_torch_adam():
    """The graph-capturable Adam of the registration loop takes the same steps
    as torch.optim.Adam (same defaults) on a small quadratic."""
    torch.manual_seed(0)
    target = torch.randn(5, 3, dtype=torch.float64)
    p_ref = torch.zeros(5, 3, dtype=torch.float64, requires_grad=True)
    p_our = torch.zeros(5, 3, dtype=torch.float64, requires_grad=True)
    ref = torch.optim.Adam([p_ref], lr=0.05)
    our = reg._Adam([p_our], lr=0.05)
    for _ in range(25):
        for p, opt in ((p_ref, ref), (p_our, our)):
            opt.zero_grad()
            loss = ((p - target) ** 2 * torch.arange(1, 4, dtype=torch.float64)).sum()
            loss.backward()
            opt.step()
    assert torch.allclose(p_ref, p_our, rtol=0, atol=1e-12)


def test_coarse_targets_pool_and_blur():
    rng = np.random.default_rng(0)
    t = torch.as_tensor(rng.uniform(0, 1, (2, 16, 24)), dtype=torch.float32)
    # block means only
    c = reg.coarse_targets(t, 4, 0.0)
    assert c.shape == (2, 4, 6)
    assert torch.allclose(c[1, 2, 3], t[1, 8:12, 12:16].mean())
    # a blur keeps a constant image and spreads a centred spike with the given variance
    const = torch.full((1, 20, 20), 0.7)
    assert torch.allclose(reg.coarse_targets(const, 1, 2.0), const, atol=1e-6)
    spike = torch.zeros((1, 41, 41))
    spike[0, 20, 20] = 1.0
    b = reg.coarse_targets(spike, 1, 2.0)[0].double()
    assert abs(float(b.sum()) - 1.0) < 1e-5
    x = torch.arange(41, dtype=torch.float64) - 20
    var_x = float((b.sum(0) * x * x).sum())
    assert abs(var_x - 2.0) < 0.05
