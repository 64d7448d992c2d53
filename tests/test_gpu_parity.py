"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the float64 path must match the oracle to 1e-12 relative on the
distance and to 1e-13 of the mesh area per node on the transform; the mixed
path to 1e-6 relative on the distance (the stated mixed-precision bar) and to
2e-6 of the area per node.
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


# ------------------------------------------------------------------ rule and sphere
@pytest.mark.parametrize("desc", [(32.0, 48, 24, 48, False), (128.0, 192, 96, 192, True), (5.0, 7, 6, 9, True),
                                  (3.0, 1, 1, 1, False)])
def test_rule_matches_oracle(ctx, desc):
    rule = ctx.rule(*desc)
    xi, w = wd.wd_rule_copy_nodes(rule)
    xo, wo = oracle.ball_rule(*desc)
    assert xi.shape == xo.shape
    assert np.abs(xi - xo).max() <= 4e-16 * desc[0]
    assert np.abs(w - wo).max() <= 1e-14 * np.abs(wo).max()
    n_eval, n_total = wd.wd_rule_info(rule)
    assert n_eval == len(xo) and n_total == desc[1] * desc[2] * desc[3]
    assert ctx.rule(*desc).value == rule.value  # cached by descriptor


def test_sphere_ft_matches_oracle(ctx):
    rule = ctx.rule(64.0, 24, 12, 16, False)
    xi, _ = wd.wd_rule_copy_nodes(rule)
    for rho, c in ((1.0, (0, 0, 0)), (0.37, (0.1, -2.0, 0.5))):
        got = ctx.sphere_ft(rule, rho, c)
        want = oracle.sphere_ft(xi, rho, c)
        assert np.abs(got - want).max() < 1e-13 * 4 * math.pi * rho * rho


# ------------------------------------------------------------------ mesh transform
MESHES = {
    "ico4": lambda: synth.icosphere(4),
    "flat5_jit": lambda: (synth.jitter_isotropic(synth.icosphere(5)[0], 0.01, 1), synth.icosphere(5)[1]),
    "ico1_rot": lambda: (synth.icosphere(1)[0] @ synth.haar_rotation(3).T, synth.icosphere(1)[1]),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_mesh_ft_matches_oracle(ctx, name, prec):
    v, t = MESHES[name]()
    # 7 x 6 x 9 = 378 nodes: one full node block and a ragged one
    rule = ctx.rule(40.0, 7, 6, 9, False)
    xi, _ = wd.wd_rule_copy_nodes(rule)
    got = ctx.mesh_ft(rule, v, t, prec)
    want = oracle.mesh_ft(v, t, xi)
    err = np.abs(got - want).max() / area(v, t)
    assert err < (1e-13 if prec == FP64 else 2e-6), err


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_mesh_ft_special_frequencies(ctx, prec):
    """Zero frequency (area), axis-aligned and normal-aligned nodes (exact
    phase coincidences), and frequencies straddling the Taylor seams."""
    v, t = synth.icosphere(2)
    nrm = np.cross(v[t[0, 1]] - v[t[0, 0]], v[t[0, 2]] - v[t[0, 0]])
    nrm /= np.linalg.norm(nrm)
    e = v[t[0, 1]] - v[t[0, 0]]
    nodes = [np.zeros(3), [1, 0, 0], [0, 0, 7], [0, 3, 0], 50 * nrm, 1e-9 * nrm, [1e-12, 0, 0]]
    for s in (0.99, 1.0, 1.01, 1.49, 1.5, 1.51, 3.0):
        nodes.append(s / np.abs(e).max() * np.array([1.0, 0.0, 0.0]))
        nodes.append(s * e / np.linalg.norm(e) ** 2)
    nodes = np.array(nodes, dtype=float)
    rule = ctx.rule_from_nodes(nodes, np.ones(len(nodes)))
    got = ctx.mesh_ft(rule, v, t, prec)
    want = oracle.mesh_ft(v, t, nodes)
    err = np.abs(got - want).max() / area(v, t)
    assert err < (1e-13 if prec == FP64 else 2e-6), err
    assert abs(got[0].real - area(v, t)) < (1e-13 if prec == FP64 else 2e-6) * area(v, t)


# ------------------------------------------------------------------ distance
def test_distance_small_config_fp64(ctx):
    """320 triangles vs the unit sphere, s = 1, R = 32, 48 x 24 x 48 nodes."""
    R = synth.SMALL_RULE
    v, t = synth.icosphere(synth.SMALL_N)
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    xo, wo = oracle.ball_rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    want = oracle.distance(xo, wo, synth.SMALL_S, v, t)
    got = ctx.distance(rule, v, t, None, synth.SMALL_S, FP64)
    assert abs(got - want) < 1e-12 * want, (got, want)
    got2 = ctx.distance(rule, v, t, None, synth.SMALL_S, FP64)
    assert got2 == got  # fixed reduction order: reproducible bit for bit


def test_distance_small_config_mixed(ctx):
    R = synth.SMALL_RULE
    v, t = synth.icosphere(synth.SMALL_N)
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    xo, wo = oracle.ball_rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    want = oracle.distance(xo, wo, synth.SMALL_S, v, t)
    got = ctx.distance(rule, v, t, None, synth.SMALL_S, MIXED)
    assert abs(got - want) < 1e-6 * want, (got, want, abs(got - want) / want)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_distance_variants_match_oracle(ctx, prec):
    tol = 1e-12 if prec == FP64 else 1e-6
    v, t = synth.icosphere(3)
    v = synth.jitter_isotropic(v, 0.02, 11)
    desc = (20.0, 13, 8, 11, True)
    rule = ctx.rule(*desc)
    xo, wo = oracle.ball_rule(*desc)
    for nu, s in ((("sphere", 1.0, (0.0, 0.0, 0.0)), 1.0), (("sphere", 0.9, (0.05, -0.02, 0.1)), 2.0),
                  (("mesh",) + synth.icosphere(2), 1.5)):
        want = oracle.distance(xo, wo, s, v, t, nu=nu)
        got = ctx.distance(rule, v, t, nu, s, prec)
        assert abs(got - want) < tol * want, (nu[0], s, got, want)


def test_distance_degenerate_inputs(ctx):
    rule = ctx.rule(16.0, 8, 4, 8, False)
    xo, wo = oracle.ball_rule(16.0, 8, 4, 8, False)
    empty_v, empty_t = np.zeros((0, 3)), np.zeros((0, 3), np.int32)
    scale = oracle.distance(xo, wo, 1.0, empty_v, empty_t)  # the sphere's own norm on the rule
    for prec in (FP64, MIXED):
        # no triangles
        assert abs(ctx.distance(rule, empty_v, empty_t, None, 1.0, prec) - scale) < 1e-13 * scale
        # identical measures: zero up to the rounding of the per-node sums
        v, t = synth.icosphere(3)
        d = ctx.distance(rule, v, t, ("mesh", v, t), 1.0, prec)
        assert 0.0 <= d < (1e-24 if prec == FP64 else 1e-12) * scale, d
        # a degenerate (zero-area) triangle contributes nothing
        v2 = np.vstack([v, [[0.3, 0.3, 0.3], [0.6, 0.6, 0.6]]])
        t2 = np.vstack([t, [[len(v), len(v) + 1, len(v)]]]).astype(np.int32)
        a = ctx.distance(rule, v, t, None, 1.0, prec)
        b = ctx.distance(rule, v2, t2, None, 1.0, prec)
        assert abs(a - b) <= 1e-14 * a
    # no nodes
    r0 = ctx.rule_from_nodes(np.zeros((0, 3)), np.zeros(0))
    v, t = synth.icosphere(2)
    assert ctx.distance(r0, v, t, None, 1.0, FP64) == 0.0


def test_invalid_inputs_are_rejected(ctx):
    rule = ctx.rule(8.0, 4, 4, 4, False)
    v, t = synth.icosphere(1)
    bad = t.copy()
    bad[2, 0] = len(v)
    with pytest.raises(wd.WDError) as e:
        ctx.distance(rule, v, bad)
    assert e.value.status == wd.WD_EINVAL
    vn = v.copy()
    vn[0, 1] = np.nan
    with pytest.raises(wd.WDError):
        ctx.distance(rule, vn, t)
    for s in (0.0, -1.0, float("nan")):
        with pytest.raises(wd.WDError):
            ctx.distance(rule, v, t, None, s)
    with pytest.raises(wd.WDError):
        ctx.rule(8.0, 4, 5, 4, True)
    with pytest.raises(wd.WDError):
        ctx.distance(rule, v, t, None, 1.0, 7)
    # the device path records bad indices and reports them at wd_sync
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(bad, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    wd.wd_distance_dev(ctx.handle, rule, dv, dt, None, 1.0, FP64, out)
    with pytest.raises(wd.WDError) as e:
        wd.wd_sync(ctx.handle)
    assert e.value.status == wd.WD_EINVAL
    wd.wd_sync(ctx.handle)  # flag cleared
    # and the context is still usable
    assert ctx.distance(rule, v, t) > 0


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_device_path_matches_host_path(ctx, prec):
    v, t = synth.icosphere(8)
    rule = ctx.rule(64.0, 24, 16, 24, True)
    host = ctx.distance(rule, v, t, None, 1.0, prec)
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(t, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    wd.wd_distance_dev(ctx.handle, rule, dv, dt, None, 1.0, prec, out)
    wd.wd_sync(ctx.handle)
    assert out.item() == host
    n, _ = wd.wd_rule_info(rule)
    re = torch.empty(n, dtype=torch.float64, device="cuda")
    im = torch.empty(n, dtype=torch.float64, device="cuda")
    wd.wd_mesh_ft_dev(ctx.handle, rule, dv, dt, prec, re, im)
    wd.wd_sync(ctx.handle)
    host_ft = ctx.mesh_ft(rule, v, t, prec)
    assert np.array_equal(re.cpu().numpy(), host_ft.real) and np.array_equal(im.cpu().numpy(), host_ft.imag)


@pytest.mark.parametrize("n, shells", [(32, None), (64, 32)])
@pytest.mark.parametrize("s", [1.0, 2.0])
def test_mixed_matches_fp64_on_the_refinement_sweep(ctx, n, shells, s):
    """Mixed vs float64 on the sweep rule (R = 128, 192 x 96 x 192, Hermitian):
    the full rule for n = 32, and for n = 64 the 32 lowest radial shells, where
    D for s = 2 is small next to the mesh transform and any coherent float32
    error would show first. Bar: 1e-6 relative."""
    R = synth.SWEEP_RULE
    rule = ctx.rule(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian)
    if shells is not None:
        xi, w = wd.wd_rule_copy_nodes(rule)
        per = len(xi) // R.n_r
        rule = ctx.rule_from_nodes(xi[: shells * per], w[: shells * per])
    v, t = synth.icosphere(n)
    d64 = ctx.distance(rule, v, t, None, s, FP64)
    dmx = ctx.distance(rule, v, t, None, s, MIXED)
    assert abs(dmx - d64) < 1e-6 * d64, (dmx, d64, (dmx - d64) / d64)


def test_radial_shell_windows(ctx):
    """A ball rule split into radial-shell windows: the windows' nodes and
    weights are the full rule's, in order; D over a partition of the shells
    adds up to D over the full rule (both precisions); and a 32-aligned
    window's mixed transform is the full rule's, bit for bit."""
    desc = (24.0, 96, 8, 12, True)
    full = ctx.rule(*desc)
    xi, w = wd.wd_rule_copy_nodes(full)
    per = len(xi) // desc[1]
    v, t = synth.icosphere(6)
    v = synth.jitter_isotropic(v, 0.01, 3)
    # float64: any partition; mixed: 32-aligned windows (the same float32
    # operations per node as the full rule, so only the final sums differ)
    for prec, bounds in ((FP64, [(0, 7), (7, 40), (40, 96)]), (MIXED, [(0, 32), (32, 64), (64, 96)])):
        parts = []
        for a, b in bounds:
            win = ctx.rule_shells(*desc, a, b)
            xw, ww = wd.wd_rule_copy_nodes(win)
            assert np.array_equal(xw, xi[a * per:b * per]) and np.array_equal(ww, w[a * per:b * per])
            assert wd.wd_rule_info(win) == ((b - a) * per, (b - a) * desc[2] * desc[3])
            parts.append(ctx.distance(win, v, t, None, 1.0, prec))
        d_full = ctx.distance(full, v, t, None, 1.0, prec)
        assert abs(sum(parts) - d_full) < 1e-13 * d_full, (prec, sum(parts), d_full)
    win = ctx.rule_shells(*desc, 32, 64)
    assert np.array_equal(ctx.mesh_ft(win, v, t, MIXED), ctx.mesh_ft(full, v, t, MIXED)[32 * per:64 * per])
    assert ctx.rule_shells(*desc, 32, 64).value == win.value  # cached by descriptor and window
    for a, b in ((-1, 4), (4, 4), (90, 97)):
        with pytest.raises(wd.WDError) as e:
            ctx.rule_shells(*desc, a, b)
        assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WDError):
        wd.wd_build_freq_rule_shells(ctx.handle, 5.0, 16, 0, 0, True, 0, 4)  # no windows of n_polar = 0


def test_far_mesh_reaches_the_reduced_phase_rows(ctx):
    """Meshes 10^3 and 10^5 units from the origin on a ball rule at R = 64: their
    phases reach 10^4 and 10^6 turns, past the 2^13 turns up to which the radial kernel feeds
    the unreduced phase to the table lookup, so the outer rows take the form
    that reduces the phase mod 1 first, and the inner ones use the lookup near
    the top of its range. A common translation c of the mesh and the sphere
    multiplies both transforms by exp(-i xi.c) (translation theorem), so D is
    unchanged: the translated D must equal the untranslated float64 D, and
    the mixed D must stay within the 1e-6 bar of it."""
    desc = (64.0, 64, 32, 64, True)
    rule = ctx.rule(*desc)
    v, t = synth.icosphere(16)
    v = synth.jitter_isotropic(v, 0.01, 5)
    d0 = ctx.distance(rule, v, t, None, 1.0, FP64)
    dmx0 = ctx.distance(rule, v, t, None, 1.0, MIXED)
    # |c| = 1e3: phases to 1e4 turns; |c| = 1e5: to 1e6 turns, where the high
    # product's rounding error alone spans table steps
    # (float64 itself rounds phases of 6e6 rad at 7e-10 rad: 1e-7 there)
    for c, tol64 in ((np.array([600.0, 800.0, 0.0]), 1e-8), (np.array([0.0, 6.0e4, -8.0e4]), 1e-7)):
        d64 = ctx.distance(rule, v + c, t, ("sphere", 1.0, c), 1.0, FP64)
        dmx = ctx.distance(rule, v + c, t, ("sphere", 1.0, c), 1.0, MIXED)
        assert abs(d64 - d0) < tol64 * d0, (c, d64, d0)
        assert abs(dmx - d0) < 1e-6 * d0, (c, dmx, d0, (dmx - d0) / d0)
        assert abs(dmx - dmx0) < 1e-6 * d0, (c, dmx, dmx0)

