"""Parity at the full size of the large workload: icosahedral n = 128
(327,680 triangles, radial jitter 1e-4, seed 7) against the unit sphere,
ball rule R = 256 with 256 x 128 x 256 nodes and Hermitian halving. The
oracle cannot evaluate the full rule, so: (1) the mixed transform over the
full rule, in the launch configuration the benchmark times, is compared with
the oracle at sampled nodes; (2) mixed against float64 on a four-shell
sub-rule at the 1e-6 bar; (3) float64 against the oracle per node, at 1e-13 of
the mesh area."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    ctx = wd.Context(0)
    R = synth.LARGE_RULE
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    v, t = synth.large_mesh()
    xi, w = wd.wd_rule_copy_nodes(rule)
    yield ctx, R, rule, v, t, xi, w
    ctx.close()


def test_full_rule_sampled_nodes_match_oracle(setup):
    ctx, R, rule, v, t, xi, w = setup
    n, _ = wd.wd_rule_info(rule)
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(t, device="cuda")
    re = torch.empty(n, dtype=torch.float64, device="cuda")
    im = torch.empty(n, dtype=torch.float64, device="cuda")
    wd.wd_mesh_ft_dev(ctx.handle, rule, dv, dt, wd.WD_MIXED, re, im)
    wd.wd_sync(ctx.handle)
    idx = np.random.default_rng(7).choice(n, 48, replace=False)
    got = re.cpu().numpy()[idx] + 1j * im.cpu().numpy()[idx]
    want = oracle.mesh_ft(v, t, xi[idx])
    area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1).sum()
    assert np.abs(got - want).max() < 2e-6 * area


def test_subrule_mixed_matches_fp64_and_fp64_matches_oracle(setup):
    ctx, R, rule, v, t, xi, w = setup
    per = len(xi) // R.n_r
    shells = [0, 40, 128, 255]
    idx = np.concatenate([np.arange(s * per, (s + 1) * per) for s in shells])
    sub = ctx.rule_from_nodes(xi[idx], w[idx])
    d64 = ctx.distance(sub, v, t, None, synth.LARGE_S, wd.WD_FP64)
    dmx = ctx.distance(sub, v, t, None, synth.LARGE_S, wd.WD_MIXED)
    assert abs(dmx - d64) < 1e-6 * d64, (dmx, d64)
    # float64 per node against the oracle (the D of a few dozen nodes would be
    # limited by random per-node rounding, ~sqrt(T) eps |F|, that only averages
    # out over many nodes)
    small = idx[:: len(idx) // 64][:64]
    sub2 = ctx.rule_from_nodes(xi[small], w[small])
    m64 = ctx.mesh_ft(sub2, v, t, wd.WD_FP64)
    mo = oracle.mesh_ft(v, t, xi[small])
    area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1).sum()
    assert np.abs(m64 - mo).max() < 1e-13 * area
