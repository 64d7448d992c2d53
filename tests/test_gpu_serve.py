"""Serving loop: continuous batching gives every query the same result alone
and in the mix, and the same as wd_distance and the oracle; admission, queue
limits, bounded waits and cancellation."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402

RULES = [(16.0, 12, 8, 12, True), (24.0, 16, 8, 16, True)]


@pytest.fixture(scope="module")
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


def queries(k, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(2, 14))
        v, t = synth.icosphere(n)
        v = synth.jitter_isotropic(v @ synth.haar_rotation(int(rng.integers(1 << 30))).T, 0.01, i)
        out.append((v, t, float(rng.integers(1, 3)), RULES[int(rng.integers(0, 2))][0]))
    return out


@pytest.mark.parametrize("prec", [wd.WD_MIXED, wd.WD_FP64])
def test_results_alone_and_in_the_mix(ctx, prec):
    qs = queries(24)
    rules = {R[0]: ctx.rule(*R) for R in RULES}
    alone = [ctx.distance(rules[R], v, t, None, s, prec) for (v, t, s, R) in qs]
    # small launch budget: the queries are spread over several launches and share them
    sv = wd.wd_serve_start(ctx.handle, RULES, precision=prec, max_slots=8, pairs_per_launch=20_000_000)
    try:
        one_by_one = []
        for (v, t, s, R) in qs[:4]:
            one_by_one.append(wd.wd_serve_wait(sv, wd.wd_serve_submit(sv, v, t, s, R), 60000))
        tickets = [wd.wd_serve_submit(sv, v, t, s, R) for (v, t, s, R) in qs]
        mixed = [wd.wd_serve_wait(sv, tk, 60000) for tk in tickets]
        st = wd.wd_serve_stats(sv)
    finally:
        wd.wd_serve_stop(sv)
    # every query runs the items of its own wd_distance plan, summed in the
    # plan's fixed order: the same bits alone, in the mix and from wd_distance
    assert mixed == alone and one_by_one == alone[:4]
    assert st["completed"] == 28 and st["launches"] >= 2 and st["failed"] == 0


@pytest.mark.parametrize("prec", [wd.WD_MIXED, wd.WD_FP64])
def test_served_results_match_the_oracle(ctx, prec):
    """Served D against the CPU oracle on the serving rules' shapes (R = 64:
    64 x 32 x 64 and R = 128: 128 x 48 x 96, Hermitian), small meshes mixed
    with a large one so that the small queries share launches with it."""
    rules = [(R.R, R.n_r, R.n_polar, R.n_azim, R.hermitian) for R in synth.SERVE_RULES.values()]
    small = []
    for i, (n, R) in enumerate(((2, 64.0), (3, 128.0), (5, 64.0))):
        v, t = synth.icosphere(n)
        v = synth.jitter_isotropic(v @ synth.haar_rotation(40 + i).T, 1e-3 * synth.mean_edge_length(v, t), 40 + i)
        small.append((v, t, 1.0 + (i % 2), R))
    big_v, big_t = synth.icosphere(40)
    sv = wd.wd_serve_start(ctx.handle, rules, precision=prec, max_slots=8, pairs_per_launch=2_000_000_000)
    try:
        tk_big = wd.wd_serve_submit(sv, big_v, big_t, 1.0, 128.0)
        tks = [wd.wd_serve_submit(sv, v, t, s, R) for (v, t, s, R) in small]
        served = [wd.wd_serve_wait(sv, tk, 600000) for tk in tks]
        wd.wd_serve_wait(sv, tk_big, 600000)
    finally:
        wd.wd_serve_stop(sv)
    tol = 1e-12 if prec == wd.WD_FP64 else 1e-6
    for (v, t, s, R), got in zip(small, served):
        xo, wo = oracle.ball_rule(*next(r for r in rules if r[0] == R))
        want = oracle.distance(xo, wo, s, v, t)
        assert abs(got - want) <= tol * want, (R, len(t), got, want, (got - want) / want)


def test_admission_limits_waits_and_cancel(ctx):
    v_small, t_small = synth.icosphere(2)
    v_big, t_big = synth.icosphere(32)
    # memory cap below the large query's footprint
    sv = wd.wd_serve_start(ctx.handle, RULES, mem_cap_bytes=1 << 20, max_slots=2, max_pending=3,
                           pairs_per_launch=2_000_000)
    try:
        with pytest.raises(wd.WDError) as e:
            wd.wd_serve_submit(sv, v_big, t_big, 1.0, 16.0)
        assert e.value.status == wd.WD_ENOMEM
        with pytest.raises(wd.WDError) as e:
            wd.wd_serve_submit(sv, v_small, t_small, 1.0, 99.0)  # no rule for R
        assert e.value.status == wd.WD_EINVAL
        tickets = []
        busy = 0
        for _ in range(40):
            try:
                tickets.append(wd.wd_serve_submit(sv, v_small, t_small, 1.0, 16.0))
            except wd.WDError as err:
                assert err.status == wd.WD_EBUSY
                busy += 1
        for tk in tickets:
            wd.wd_serve_wait(sv, tk, 60000)
        st = wd.wd_serve_stats(sv)
        assert st["completed"] == len(tickets) and st["rejected"] == 1 + busy  # ENOMEM + queue-full refusals
    finally:
        wd.wd_serve_stop(sv)
    # bounded wait and cancellation on a slow query
    sv = wd.wd_serve_start(ctx.handle, RULES, max_slots=1, pairs_per_launch=1_000_000)
    try:
        v, t = synth.icosphere(24)
        tk = wd.wd_serve_submit(sv, v, t, 1.0, 24.0)
        tk2 = wd.wd_serve_submit(sv, v, t, 1.0, 24.0)
        t0 = time.perf_counter()
        with pytest.raises(wd.WDError) as e:
            wd.wd_serve_wait(sv, tk, 1)
        assert e.value.status == wd.WD_ETIMEOUT and time.perf_counter() - t0 < 5.0
        wd.wd_serve_cancel(sv, tk2)
        d = wd.wd_serve_wait(sv, tk, 60000)
        assert d > 0
        deadline = time.time() + 60
        while True:
            done, _, status = wd.wd_serve_poll(sv, tk2)
            if done or time.time() > deadline:
                break
            time.sleep(0.01)
        assert done and status == wd.WD_ECANCELLED
    finally:
        wd.wd_serve_stop(sv)


def test_queued_queries_time_out(ctx):
    sv = wd.wd_serve_start(ctx.handle, RULES, max_slots=1, timeout_ms=1, pairs_per_launch=500_000)
    try:
        v, t = synth.icosphere(24)
        tks = [wd.wd_serve_submit(sv, v, t, 1.0, 24.0) for _ in range(4)]
        outcomes = []
        for tk in tks:
            try:
                wd.wd_serve_wait(sv, tk, 60000)
                outcomes.append(wd.WD_OK)
            except wd.WDError as err:
                outcomes.append(err.status)
        assert outcomes[0] == wd.WD_OK and wd.WD_ETIMEOUT in outcomes[1:]
        assert wd.wd_serve_stats(sv)["timeouts"] >= 1
    finally:
        wd.wd_serve_stop(sv)


@pytest.mark.parametrize("prec", [wd.WD_MIXED, wd.WD_FP64])
def test_lattice_rule_queries(ctx, prec):
    # a cube (lattice) rule in the server: its per-node path (tile shifts, the
    # origin node) gives what wd_distance gives on the same rule
    rules = [(5.0, 16, 0, 0, True, wd.WD_RULE_CUBE_TRAP)]
    cube = ctx.cube_rule(5.0, 16, True)
    qs = [(synth.icosphere_recursive(k)[0], synth.icosphere_recursive(k)[1], 10.0) for k in (1, 2, 3)]
    alone = [ctx.distance(cube, v, t, None, s, prec) for (v, t, s) in qs]
    sv = wd.wd_serve_start(ctx.handle, rules, precision=prec, max_slots=4, pairs_per_launch=2_000_000)
    try:
        tickets = [wd.wd_serve_submit(sv, v, t, s, 5.0) for (v, t, s) in qs]
        served = [wd.wd_serve_wait(sv, tk, 60000) for tk in tickets]
    finally:
        wd.wd_serve_stop(sv)
    assert served == alone


def test_paper_lattice_rule_queries(ctx):
    """The paper's M = 128 lattice in the server: its lattice-line form and
    extended-precision blocks give wd_distance's bits, alone and in the mix."""
    rules = [(synth.PAPER_XI_MAX, synth.PAPER_M, 0, 0, True, wd.WD_RULE_CUBE_TRAP)]
    cube = ctx.cube_rule(synth.PAPER_XI_MAX, synth.PAPER_M, True)
    qs = [(synth.icosphere_recursive(k)[0], synth.icosphere_recursive(k)[1], s) for k, s in ((1, 10.0), (3, 10.0),
                                                                                            (2, 3.0))]
    alone = [ctx.distance(cube, v, t, None, s, wd.WD_MIXED) for (v, t, s) in qs]
    sv = wd.wd_serve_start(ctx.handle, rules, precision=wd.WD_MIXED, max_slots=4, pairs_per_launch=200_000_000)
    try:
        tickets = [wd.wd_serve_submit(sv, v, t, s, synth.PAPER_XI_MAX) for (v, t, s) in qs]
        served = [wd.wd_serve_wait(sv, tk, 600000) for tk in tickets]
        st = wd.wd_serve_stats(sv)
    finally:
        wd.wd_serve_stop(sv)
    assert served == alone and st["launches"] >= 2
