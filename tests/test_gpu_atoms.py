"""The paper's 64-atom approximation of the mesh transform (Sec. 3.1) on the
GPU: parity with the oracle's atomic transform, and its error against the
exact transform, small where |xi| h is small."""
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
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


def area(v, t):
    e1 = v[t[:, 1]] - v[t[:, 0]]
    e2 = v[t[:, 2]] - v[t[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_atoms_match_oracle(ctx, n):
    v, t = synth.icosphere(n)
    v = synth.jitter_isotropic(v, 0.01, n)
    rule = ctx.rule(40.0, 7, 6, 9, False)  # 378 nodes: a full and a ragged node block
    xi, _ = wd.wd_rule_copy_nodes(rule)
    got = ctx.mesh_ft_atoms(rule, v, t)
    want = oracle.mesh_ft_atoms(v, t, xi)
    assert np.abs(got - want).max() < 1e-13 * area(v, t)


def test_atoms_error_against_the_exact_transform(ctx):
    v, t = synth.icosphere_recursive(3)
    h = synth.mean_edge_length(v, t)
    rule = ctx.rule(60.0, 24, 8, 12, True)
    xi, _ = wd.wd_rule_copy_nodes(rule)
    kh = np.linalg.norm(xi, axis=1) * h
    err = np.abs(ctx.mesh_ft_atoms(rule, v, t) - ctx.mesh_ft(rule, v, t, wd.WD_FP64)) / area(v, t)
    assert err[kh < 1.0].max() < 1e-13
    assert err[kh < 3.0].max() < 1e-9
    # the approximation grows with |xi| h (3e-10 of the area at |xi| h ~ 9 here)
    assert err[kh > 6.0].max() > 100 * err[kh < 1.0].max()
