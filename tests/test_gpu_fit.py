"""Adjoint configuration on the GPU: bitwise-reproducible gradients, the
gradient of a 5,120-triangle jittered mesh against the oracle on a sampled
explicit sub-rule of the 1,179,648-node ball rule (per-node adjoint) and on a
ball rule with the same 192 radii (radial adjoint), and the gradient-descent
fit toward the unit sphere with checkpoint/resume."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402
from paper_2304_06340_b300.fit import fit_mesh  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


def _dev(v, t):
    return torch.tensor(v, device="cuda"), torch.tensor(t, device="cuda", dtype=torch.int32)


def _grad(ctx, rule, dv, dt, prec):
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros_like(dv)
    wd.wd_distance_grad_dev(ctx.handle, rule, dv, dt, None, 1.0, prec, out, g)
    torch.cuda.synchronize()
    return out, g


@pytest.mark.parametrize("prec", [wd.WD_FP64, wd.WD_MIXED])
def test_gradient_is_bitwise_reproducible(ctx, prec):
    v, t = synth.icosphere(4)
    v = synth.jitter_isotropic(v, 0.01, 5)
    dv, dt = _dev(v, t)
    rule = ctx.rule(24.0, 16, 8, 12, True)
    d0, g0 = _grad(ctx, rule, dv, dt, prec)
    for _ in range(3):
        d1, g1 = _grad(ctx, rule, dv, dt, prec)
        assert torch.equal(d0, d1) and torch.equal(g0, g1)


def test_adjoint_config_gradient_vs_oracle(ctx):
    # n=16 (5,120 triangles), sigma=0.01, seed 0; every 96th node of the
    # oracle's 192 x 64 x 96 Hermitian ball rule at R=128 (6,144 nodes)
    R = synth.ADJOINT_RULE
    v, t = synth.adjoint_mesh(16, 0)
    xo, wo = oracle.ball_rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    xs, ws = np.ascontiguousarray(xo[::96]), np.ascontiguousarray(wo[::96])
    d_or, g_or = oracle.distance_grad(xs, ws, 1.0, v, t)
    rule = ctx.rule_from_nodes(xs, ws)
    dv, dt = _dev(v, t)
    for prec, tol in ((wd.WD_FP64, 1e-10), (wd.WD_MIXED, 1e-6)):
        d, g = _grad(ctx, rule, dv, dt, prec)
        g = g.cpu().numpy()
        assert abs(d.item() - d_or) < tol * d_or
        err = np.linalg.norm(g - g_or) / np.linalg.norm(g_or)
        assert err < tol, (prec, err)


def test_adjoint_config_radial_gradient_vs_oracle(ctx):
    # the radial (ball-rule) mixed adjoint over the adjoint rule's full radial
    # range: R=128 with its 192 radii, on 2 x 6 directions (2,304 nodes),
    # n=16 mesh, sigma=0.01, seed 3
    v, t = synth.adjoint_mesh(16, 3)
    desc = (128.0, 192, 4, 6, True)
    xo, wo = oracle.ball_rule(*desc)
    d_or, g_or = oracle.distance_grad(xo, wo, 1.0, v, t)
    rule = ctx.rule(*desc)
    dv, dt = _dev(v, t)
    for prec, tol in ((wd.WD_FP64, 1e-10), (wd.WD_MIXED, 1e-6)):
        d, g = _grad(ctx, rule, dv, dt, prec)
        g = g.cpu().numpy()
        assert abs(d.item() - d_or) < tol * d_or
        err = np.linalg.norm(g - g_or) / np.linalg.norm(g_or)
        assert err < tol, (prec, err)


def test_fit_descends_and_resumes_bitwise(ctx, tmp_path):
    v, t = synth.icosphere(2)
    v = synth.jitter_isotropic(v, 0.02, 3)
    dv, dt = _dev(v, t)
    rule = ctx.rule(16.0, 12, 8, 12, True)
    full = fit_mesh(ctx, rule, dv, dt, steps=24, precision=wd.WD_MIXED)
    h = full.history
    assert len(h) == 25 and all(b <= a for a, b in zip(h, h[1:])) and h[-1] < 0.5 * h[0]
    ck = str(tmp_path / "fit.pt")
    part = fit_mesh(ctx, rule, dv, dt, steps=9, precision=wd.WD_MIXED, lr=full.lr, checkpoint=ck,
                    checkpoint_every=4)
    assert part.step == 9
    rest = fit_mesh(ctx, rule, dv, dt, steps=24, precision=wd.WD_MIXED, checkpoint=ck, checkpoint_every=4)
    assert rest.resumed_from == 9 and rest.lr == full.lr
    assert torch.equal(rest.verts, full.verts) and rest.history == full.history
    # a checkpoint of another mesh is refused
    v2, t2 = synth.icosphere(3)
    dv2, dt2 = _dev(v2, t2)
    with pytest.raises(ValueError):
        fit_mesh(ctx, rule, dv2, dt2, steps=30, precision=wd.WD_MIXED, lr=full.lr, checkpoint=ck)


def test_adjoint_config_fit_200_steps(ctx):
    # the adjoint configuration's fitting run: n=16, sigma=0.01, seed 0, mixed
    R = synth.ADJOINT_RULE
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    v, t = synth.adjoint_mesh(16, 0)
    dv, dt = _dev(v, t)
    r = fit_mesh(ctx, rule, dv, dt, steps=200, precision=wd.WD_MIXED)
    h = r.history
    assert all(b <= a for a, b in zip(h, h[1:]))
    assert h[-1] < 1e-3 * h[0]
    # the fitted vertices lie close to the sphere (start: radial spread 1e-2)
    assert r.verts.norm(dim=1).std().item() < 1e-3
    # D of the final mesh, re-evaluated in float64, agrees with the mixed history
    d64 = ctx.distance(rule, r.verts.cpu().numpy(), t, None, 1.0, wd.WD_FP64)
    assert abs(d64 - h[-1]) < 1e-6 * d64
