"""Adjoint parity: the CUDA gradient of D against the oracle's analytic
gradient and against central finite differences of the CUDA distance.
Bars: float64 1e-10 relative (2-norm); mixed forward 1e-6."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402
from paper_2304_06340_b300.autograd import weak_distance  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


CASES = [
    (2, 0.01, (8.0, 12, 8, 10, True), None, 1.0),
    (3, 0.02, (12.0, 9, 6, 7, False), ("sphere", 0.9, (0.05, -0.1, 0.02)), 2.0),
    (4, 0.005, (24.0, 16, 8, 12, True), None, 1.0),  # 320 triangles: several triangle blocks
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [wd.WD_FP64, wd.WD_MIXED])
def test_gradient_matches_oracle(ctx, case, prec):
    n, sig, desc, nu, s = case
    v, t = synth.icosphere(n)
    v = synth.jitter_isotropic(v, sig, n)
    rule = ctx.rule(*desc)
    xo, wo = oracle.ball_rule(*desc)
    d_or, g_or = oracle.distance_grad(xo, wo, s, v, t, nu=nu)
    d, g = ctx.distance_grad(rule, v, t, nu, s, prec)
    tol = 1e-10 if prec == wd.WD_FP64 else 1e-6
    assert abs(d - d_or) < max(tol, 1e-12) * d_or
    assert np.linalg.norm(g - g_or) < tol * np.linalg.norm(g_or), np.linalg.norm(g - g_or) / np.linalg.norm(g_or)


def test_gradient_matches_finite_differences(ctx):
    v, t = synth.icosphere(2)
    v = synth.jitter_isotropic(v, 0.01, 7)
    rule = ctx.rule(10.0, 10, 6, 8, True)
    _, g = ctx.distance_grad(rule, v, t, None, 1.0, wd.WD_FP64)
    h = 1e-6
    fd = np.zeros_like(v)
    for i in range(len(v)):
        for j in range(3):
            vp, vm = v.copy(), v.copy()
            vp[i, j] += h
            vm[i, j] -= h
            fd[i, j] = (ctx.distance(rule, vp, t) - ctx.distance(rule, vm, t)) / (2 * h)
    assert np.linalg.norm(fd - g) < 1e-7 * np.linalg.norm(g)


def test_gradient_zero_for_identical_measures(ctx):
    v, t = synth.icosphere(3)
    rule = ctx.rule(12.0, 8, 6, 8, True)
    d, g = ctx.distance_grad(rule, v, t, ("mesh", v, t), 1.0, wd.WD_FP64)
    assert d < 1e-24 and np.abs(g).max() < 1e-12


def test_autograd_function(ctx):
    v, t = synth.icosphere(3)
    v = synth.jitter_isotropic(v, 0.02, 1)
    rule = ctx.rule(12.0, 8, 6, 8, True)
    dv = torch.tensor(v, device="cuda", requires_grad=True)
    dt = torch.tensor(t, device="cuda")
    D = weak_distance(ctx, rule, dv, dt, 1.0)
    (3.0 * D).backward()
    _, g = ctx.distance_grad(rule, v, t, None, 1.0, wd.WD_FP64)
    assert abs(D.item() - ctx.distance(rule, v, t)) <= 1e-14 * D.item()
    assert np.allclose(dv.grad.cpu().numpy(), 3.0 * g, rtol=1e-12, atol=1e-14)


def test_gradient_of_a_far_mesh(ctx):
    """A common translation c of the mesh and the sphere leaves D, and so its
    vertex gradient, unchanged (translation theorem). At |c| = 1e3 and 1e5 the
    radial adjoint's phases reach 1e4 and 1e6 turns, where it folds the
    phase's rounding error into the reduced phase; its gradient must match
    the untranslated float64 gradient at the mixed bar."""
    v, t = synth.icosphere(8)
    v = synth.jitter_isotropic(v, 0.01, 11)
    rule = ctx.rule(64.0, 64, 16, 32, True)
    d0, g0 = ctx.distance_grad(rule, v, t, None, 1.0, wd.WD_FP64)
    for c in (np.array([600.0, 800.0, 0.0]), np.array([0.0, 6.0e4, -8.0e4])):
        d, g = ctx.distance_grad(rule, v + c, t, ("sphere", 1.0, c), 1.0, wd.WD_MIXED)
        assert abs(d - d0) < 1e-6 * d0, (c, d, d0)
        assert np.linalg.norm(g - g0) < 1e-6 * np.linalg.norm(g0), (c, np.linalg.norm(g - g0) / np.linalg.norm(g0))
