"""Host logic of the fitting loop: gradient descent, power iteration and
checkpoint/resume, on a quadratic objective with CPU tensors (no GPU)."""
import pytest
import torch

from paper_2304_06340_b300.fit import gradient_descent, hessian_max_eig


def quadratic(n=12, seed=3):
    # D(v) = 1/2 (v - c)^T H (v - c) with H = Q diag(lam) Q^T, lam_max = 5
    g = torch.Generator().manual_seed(seed)
    q, _ = torch.linalg.qr(torch.randn(3 * n, 3 * n, generator=g, dtype=torch.float64))
    lam = torch.linspace(0.1, 5.0, 3 * n, dtype=torch.float64)
    H = q @ torch.diag(lam) @ q.T
    c = torch.randn(n, 3, generator=g, dtype=torch.float64)

    def f(v):
        d = (v - c).flatten()
        hd = H @ d
        return 0.5 * float(d @ hd), hd.reshape(n, 3)

    return f, c, n


def test_power_iteration_finds_largest_eigenvalue():
    f, c, n = quadratic()
    lam = hessian_max_eig(f, torch.zeros(n, 3, dtype=torch.float64), iters=200, eps=1e-3)
    assert abs(lam - 5.0) < 1e-3


def test_descent_decreases_and_converges():
    f, c, n = quadratic()
    r = gradient_descent(f, torch.zeros(n, 3, dtype=torch.float64), 400, 1.0 / 5.0)
    assert r.step == 400 and len(r.history) == 401
    assert all(b <= a for a, b in zip(r.history, r.history[1:]))
    # slowest mode contracts by (1 - 0.1/5) per step
    assert r.history[-1] < r.history[0] * (1 - 0.02) ** 800 * 1.01
    assert torch.allclose(r.verts, c, atol=1e-3)


def test_resume_gives_the_same_trajectory(tmp_path):
    f, c, n = quadratic()
    v0 = torch.zeros(n, 3, dtype=torch.float64)
    full = gradient_descent(f, v0, 30, 0.15)
    ck = str(tmp_path / "fit.pt")
    part = gradient_descent(f, v0, 13, 0.15, checkpoint=ck, checkpoint_every=5, meta={"k": 1})
    assert part.step == 13
    rest = gradient_descent(f, v0, 30, 0.15, checkpoint=ck, checkpoint_every=5, meta={"k": 1})
    assert rest.resumed_from == 13 and rest.step == 30
    assert torch.equal(rest.verts, full.verts)
    assert rest.history == full.history


def test_resume_from_a_periodic_checkpoint(tmp_path):
    # a run that stopped after the step-10 save (its end-of-run save lost)
    f, c, n = quadratic()
    v0 = torch.zeros(n, 3, dtype=torch.float64)
    full = gradient_descent(f, v0, 20, 0.15)
    ck = str(tmp_path / "fit.pt")
    seen = []

    def stop_at_12(step, d):
        seen.append(step)
        if step == 12:
            raise KeyboardInterrupt

    with pytest.raises(KeyboardInterrupt):
        gradient_descent(f, v0, 20, 0.15, checkpoint=ck, checkpoint_every=10, callback=stop_at_12)
    assert torch.load(ck, weights_only=False)["step"] == 10
    rest = gradient_descent(f, v0, 20, 0.15, checkpoint=ck, checkpoint_every=10)
    assert rest.resumed_from == 10
    assert torch.equal(rest.verts, full.verts) and rest.history == full.history


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    f, c, n = quadratic()
    v0 = torch.zeros(n, 3, dtype=torch.float64)
    ck = str(tmp_path / "fit.pt")
    gradient_descent(f, v0, 3, 0.1, checkpoint=ck, meta={"tris_crc32": 1})
    with pytest.raises(ValueError, match="another problem"):
        gradient_descent(f, v0, 6, 0.1, checkpoint=ck, meta={"tris_crc32": 2})
    with pytest.raises(ValueError, match="lr"):
        gradient_descent(f, v0, 6, 0.2, checkpoint=ck, meta={"tris_crc32": 1})
    with pytest.raises(ValueError, match="past"):
        gradient_descent(f, v0, 2, 0.1, checkpoint=ck, meta={"tris_crc32": 1})
    with pytest.raises(ValueError):
        gradient_descent(f, v0, 2, float("nan"))
