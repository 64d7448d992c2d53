"""The allocation-free distance entry point against the regular one.

wd_distance_dev_noalloc exists for callers that may not allocate device
memory while they run (an application whose memory manager owns the device,
a latency-critical loop that must not hit cudaMalloc/cudaFree, a plugin that
only receives buffers). It keeps its intermediates in a fixed static array
shared by all calls, so the checks below call it twice in a row on each case:
the second call must not see stale counters or partial sums from the first.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2304_06340_b300 as wd  # noqa: E402

TOL = {wd.WD_FP64: 1e-12, wd.WD_MIXED: 1e-6}  # the parity tolerances of the other GPU tests


@pytest.fixture(scope="module")
def ctx():
    c = wd.Context(0)
    yield c
    c.close()


# (rule, mesh n): many node blocks and one triangle chunk; a single node block
# whose triangles are split into chunks (exercises the partial sums and the
# completion counters kept in the static array)
CASES = [((64.0, 24, 16, 24, True), 8), ((16.0, 8, 4, 8, False), 8), ((20.0, 5, 6, 7, False), 3)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [wd.WD_FP64, wd.WD_MIXED])
def test_noalloc_matches_regular_entry_point(ctx, case, prec):
    desc, n = case
    rule = ctx.rule(*desc)
    xi, w = wd.wd_rule_copy_nodes(rule)
    v, t = synth.icosphere(n)
    v = synth.jitter_isotropic(v, 0.005, 2)
    dv = torch.tensor(v, device="cuda")
    dt = torch.tensor(t, device="cuda")
    dxi = torch.tensor(np.ascontiguousarray(xi.T), device="cuda")
    dw = torch.tensor(w, device="cuda")
    center = (0.01, -0.02, 0.03)
    for s in (1.0, 2.0):
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        wd.wd_distance_dev(ctx.handle, rule, dv, dt, ("sphere", 0.98, center), s, prec, ref)
        wd.wd_sync(ctx.handle)
        want = ref.item()
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            wd.wd_distance_dev_noalloc(dxi, dw, dv, dt, s, 0.98, center, prec, out)
            torch.cuda.synchronize()
            got = out.item()
            assert abs(got - want) <= TOL[prec] * want, (got, want)


def test_noalloc_rejects_oversized_problems():
    # sized far beyond the fixed scratch: refused before anything is launched
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    di = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    dv = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    lib = wd.library()
    import ctypes
    c = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    st = lib.wd_distance_dev_noalloc(dummy.data_ptr(), dummy.data_ptr(), 1 << 30, dv.data_ptr(), 3,
                                     di.data_ptr(), 1, 1.0, 1.0, c, wd.WD_FP64, dummy.data_ptr(), None)
    assert st == wd.WD_EINVAL
    assert "scratch" in wd.wd_last_error()
