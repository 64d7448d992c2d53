"""Mixed-precision D from the timed kernel, at the sizes it is timed at,
against the float64 path and the oracle.

The benchmark times wd_distance in mixed precision on ball rules, which runs
the radial pair kernel with its whole-row Taylor variants. These tests call
that same entry point with the benchmark's rules and meshes and compare D with
float64 at the stated bar of 1e-6 relative:

* the n = 64 refinement-sweep query on the full 192 x 96 x 192 Hermitian rule
  (1,769,472 nodes, 1.45e11 pairs), s = 1 and s = 2;
* the n = 128 large query (327,680 triangles, radial jitter 1e-4, seed 7) on
  radial-shell windows of the 256 x 128 x 256 Hermitian rule at R = 256. A
  window whose bounds are multiples of 32 gives every node the same float32
  operations as the full-rule launch (same warp radii, same dither), which
  the first test checks bit for bit, so D over a window is a sample of the
  timed computation itself.

The float64 transforms are checked against the oracle at sampled nodes
(1e-13 of the mesh area), so the float64 side is pinned independently of
the CUDA path. The per-node mixed error eps_k is also bounded at a tolerance
tied to D rather than to the mesh area. To first order D moves by
sum_k 2 W_k Re(conj(Delta_k) eps_k), Delta = mu^ - nu^. The float32
roundings are made independent across nodes (per-node phase dither), so the
spread of that sum is sigma_D = 2 sqrt(sum_k W_k^2 |Delta_k|^2 |eps_k|^2),
which must stay a decade below the bar: sigma_D < 1e-7 D. A per-node error
large enough to move D shows there even where D itself happens to cancel.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402

FP64, MIXED = wd.WD_FP64, wd.WD_MIXED


@pytest.fixture(scope="module")
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


def area(v, t):
    return 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1).sum()


def weights(xi, wg, s):
    return wg * (1.0 + (xi * xi).sum(1)) ** (-s)


def device_ft(ctx, rule, v, t, prec):
    n, _ = wd.wd_rule_info(rule)
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(t, device="cuda")
    re = torch.empty(n, dtype=torch.float64, device="cuda")
    im = torch.empty(n, dtype=torch.float64, device="cuda")
    wd.wd_mesh_ft_dev(ctx.handle, rule, dv, dt, prec, re, im)
    wd.wd_sync(ctx.handle)
    return re.cpu().numpy() + 1j * im.cpu().numpy()


def device_distance(ctx, rule, v, t, s, prec):
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(t, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    wd.wd_distance_dev(ctx.handle, rule, dv, dt, None, s, prec, out)
    wd.wd_sync(ctx.handle)
    return out.item()


def check_fp64_against_oracle(v, t, xi, m64, k=24, seed=0):
    idx = np.random.default_rng(seed).choice(len(xi), k, replace=False)
    want = oracle.mesh_ft(v, t, xi[idx])
    assert np.abs(m64[idx] - want).max() < 1e-13 * area(v, t)


def check_per_node_error_bound(W, delta, eps, D):
    """sigma_D = 2 sqrt(sum W^2 |Delta|^2 |eps|^2) below a decade under the bar."""
    sigma = 2.0 * math.sqrt(float(np.sum((W * np.abs(delta) * np.abs(eps)) ** 2)))
    assert sigma < 1e-7 * D, (sigma / D, D)


def test_sweep_n64_full_rule(ctx):
    R = synth.SWEEP_RULE
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    xi, wg = wd.wd_rule_copy_nodes(rule)
    v, t = synth.icosphere(64)
    nu = ctx.sphere_ft(rule)
    m64 = device_ft(ctx, rule, v, t, FP64)
    check_fp64_against_oracle(v, t, xi, m64)
    mmx = device_ft(ctx, rule, v, t, MIXED)
    for s in synth.SWEEP_SS:
        W = weights(xi, wg, s)
        d64 = float(np.sum(W * np.abs(m64 - nu) ** 2))
        dmx = device_distance(ctx, rule, v, t, s, MIXED)  # the benchmark's call
        assert abs(dmx - d64) < 1e-6 * d64, (s, dmx, d64, (dmx - d64) / d64)
        # the distance launch and the transform launch give the same D
        assert abs(float(np.sum(W * np.abs(mmx - nu) ** 2)) - dmx) < 1e-12 * dmx
        check_per_node_error_bound(W, m64 - nu, mmx - m64, d64)


@pytest.fixture(scope="module")
def large(ctx):
    R = synth.LARGE_RULE
    v, t = synth.large_mesh()
    return R, v, t


def test_large_window_is_the_full_launch(ctx, large):
    """A 32-aligned window of the large rule evaluates every node with the
    same float32 operations as the full rule: identical mixed transforms."""
    R, v, t = large
    full = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    win = ctx.rule_shells(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian, 32, 64)
    n_win, _ = wd.wd_rule_info(win)
    per = n_win // 32
    ft_full = device_ft(ctx, full, v, t, MIXED)
    ft_win = device_ft(ctx, win, v, t, MIXED)
    assert np.array_equal(ft_win, ft_full[32 * per:64 * per])
    xi_full, w_full = wd.wd_rule_copy_nodes(full)
    xi_win, w_win = wd.wd_rule_copy_nodes(win)
    assert np.array_equal(xi_win, xi_full[32 * per:64 * per]) and np.array_equal(w_win, w_full[32 * per:64 * per])


@pytest.mark.parametrize("shells", [(0, 32), (128, 160)])
def test_large_window_mixed_vs_fp64(ctx, large, shells):
    R, v, t = large
    win = ctx.rule_shells(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian, *shells)
    xi, wg = wd.wd_rule_copy_nodes(win)
    nu = ctx.sphere_ft(win)
    W = weights(xi, wg, synth.LARGE_S)
    m64 = device_ft(ctx, win, v, t, FP64)
    check_fp64_against_oracle(v, t, xi, m64, k=8)
    d64 = float(np.sum(W * np.abs(m64 - nu) ** 2))
    dmx = device_distance(ctx, win, v, t, synth.LARGE_S, MIXED)
    assert abs(dmx - d64) < 1e-6 * d64, (shells, dmx, d64, (dmx - d64) / d64)
    mmx = device_ft(ctx, win, v, t, MIXED)
    check_per_node_error_bound(W, m64 - nu, mmx - m64, d64)
