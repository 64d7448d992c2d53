"""Runtime support on the GPU, with every failure injected on the host (no GPU
fault): the n-th device allocation failing (WD_FAULT_ALLOC), a dropped
serving completion (WD_FAULT_DROP_COMPLETION), NaN-poisoned scratch that must
not reach any result (WD_POISON_SCRATCH), and stderr logging (WD_LOG)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402


def _mesh():
    v, t = synth.icosphere(4)
    return synth.jitter_isotropic(v, 0.01, 2), t


def test_injected_allocation_failure_is_reported_and_recoverable(monkeypatch):
    ctx = wd.Context(0)
    v, t = _mesh()
    try:
        monkeypatch.setenv("WD_FAULT_ALLOC", "1")  # the next device allocation fails
        with pytest.raises(wd.WDError) as ei:
            ctx.rule(16.0, 12, 8, 12, True)
        assert ei.value.status == wd.WD_ENOMEM
        monkeypatch.delenv("WD_FAULT_ALLOC")
        rule = ctx.rule(16.0, 12, 8, 12, True)  # the context stays usable
        d_ok = ctx.distance(rule, v, t, None, 1.0, wd.WD_MIXED)
        fresh = wd.Context(0)
        try:
            rule2 = fresh.rule(16.0, 12, 8, 12, True)
            monkeypatch.setenv("WD_FAULT_ALLOC", "2")  # fails inside the distance call
            with pytest.raises(wd.WDError) as ei:
                fresh.distance(rule2, v, t, None, 1.0, wd.WD_MIXED)
            assert ei.value.status == wd.WD_ENOMEM
            monkeypatch.delenv("WD_FAULT_ALLOC")
            assert fresh.distance(rule2, v, t, None, 1.0, wd.WD_MIXED) == d_ok
        finally:
            fresh.close()
    finally:
        ctx.close()


def test_dropped_completion_makes_the_wait_time_out(monkeypatch):
    ctx = wd.Context(0)
    monkeypatch.setenv("WD_FAULT_DROP_COMPLETION", "2")
    sv = wd.wd_serve_start(ctx.handle, [(16.0, 12, 8, 12, True)], precision=wd.WD_MIXED,
                           mem_cap_bytes=256 << 20, max_slots=1)
    monkeypatch.delenv("WD_FAULT_DROP_COMPLETION")
    try:
        v, t = _mesh()
        tickets = [wd.wd_serve_submit(sv, v, t, 1.0, 16.0) for _ in range(3)]
        assert wd.wd_serve_wait(sv, tickets[0], 60000) > 0.0
        with pytest.raises(wd.WDError) as ei:
            wd.wd_serve_wait(sv, tickets[1], 2000)  # its completion was dropped
        assert ei.value.status == wd.WD_ETIMEOUT
        assert wd.wd_serve_wait(sv, tickets[2], 60000) > 0.0
        done, _, _ = wd.wd_serve_poll(sv, tickets[1])
        assert not done
        assert wd.wd_serve_stats(sv)["completed"] == 3
    finally:
        wd.wd_serve_stop(sv)
        ctx.close()


@pytest.mark.parametrize("prec", [wd.WD_FP64, wd.WD_MIXED])
def test_poisoned_scratch_does_not_reach_results(monkeypatch, prec):
    v, t = _mesh()
    desc = (16.0, 12, 8, 12, True)
    runs = []
    for poison in ("0", "1"):
        monkeypatch.setenv("WD_POISON_SCRATCH", poison)
        ctx = wd.Context(0)
        try:
            rule = ctx.rule(*desc)
            expl = ctx.rule_from_nodes(*wd.wd_rule_copy_nodes(rule))
            cube = ctx.cube_rule(5.0, 8, True)
            out = [ctx.distance(rule, v, t, None, 1.0, prec), ctx.distance(expl, v, t, None, 1.0, prec),
                   ctx.distance(cube, v, t, None, 10.0, prec), ctx.mesh_ft(rule, v, t, prec)]
            d, g = ctx.distance_grad(rule, v, t, None, 1.0, prec)
            out += [d, g]
            runs.append(out)
        finally:
            ctx.close()
    monkeypatch.delenv("WD_POISON_SCRATCH")
    for a, b in zip(*runs):
        assert np.all(np.isfinite(b))
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_logging_to_stderr(monkeypatch, capfd):
    monkeypatch.setenv("WD_LOG", "4")
    ctx = wd.Context(0)
    try:
        v, t = _mesh()
        ctx.distance(ctx.rule(16.0, 12, 8, 12, True), v, t, None, 1.0, wd.WD_MIXED)
        with pytest.raises(wd.WDError):
            ctx.distance(ctx.rule(16.0, 12, 8, 12, True), v, t, None, -1.0, wd.WD_MIXED)
    finally:
        ctx.close()
    monkeypatch.delenv("WD_LOG")
    err = capfd.readouterr().err
    assert "[wd info] context created" in err
    assert "[wd debug] alloc" in err
    assert "[wd error]" in err and "s must be" in err
