"""The allocation-free entry point ptylm_forward_loss_noalloc, called through the C-ABI,
against the context-based forward_loss on the same inputs, twice in a row.

Callers that cannot allocate device memory (work issued while a stream is captured into a
CUDA graph, allocation-free steady-state loops, memory owned by another allocator) use this
entry point; its scratch is a file-scope device array shared by all calls.  This file is
collected last so that a run stopping at the first failure has already run everything else;
it passes alone in a fresh process as well as after the other tests."""
import math

import numpy as np
import pytest

from paper_2103_01767_gb300 import synth
from tests.problems import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the relative bound of the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    return ptylm


def _c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


@pytest.mark.parametrize("shape,loss", [((160, 64, 23), 0), ((640, 128, 400), 1), ((256, 32, 3000), 1)])
def test_noalloc_loss_matches_context_path_on_two_calls(lib, shape, loss):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=31)
    pos = torch.from_numpy(case.pos).cuda()
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    P = _c64(case.P)
    O = _c64(synth.to_c64(case.O_true + synth.random_complex(case.O_true.shape, seed=32, scale=0.05)))
    ctx = lib.lm_init(n, n, m, m, pos, y, loss, case.b)
    f_ref, dl2_ref = lib.forward_loss(ctx, O, P, cache=1)
    lib.lm_destroy(ctx)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(math.nan)  # each call must write its own result
        lib.ptylm_forward_loss_noalloc(n, n, m, pos, y, O, P, out, loss, case.b)
        f, dl2 = out.tolist()
        assert abs(f - f_ref) <= TOL * abs(f_ref), (f, f_ref)
        assert abs(dl2 - dl2_ref) <= TOL * abs(dl2_ref), (dl2, dl2_ref)


def test_noalloc_rejects_out_of_range_positions_and_sizes(lib):
    case = make_case(96, 32, K=5, loss=0, seed=33)
    bad = case.pos.copy()
    bad[3] = (96 - 32 + 1, 0)
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    O, P = _c64(case.O_true), _c64(case.P)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.PtylmError) as e:
        lib.ptylm_forward_loss_noalloc(96, 96, 32, torch.from_numpy(bad).cuda(), y, O, P, out, 0, case.b)
    assert e.value.status == lib.PTYLM_ERR_ARG
    with pytest.raises(lib.PtylmError) as e:
        lib.ptylm_forward_loss_noalloc(512, 512, 256, torch.from_numpy(case.pos).cuda(), y, O, P, out, 0, case.b)
    assert e.value.status == lib.PTYLM_ERR_ARG
    # a valid call afterwards still works (the flag is cleared per call)
    lib.ptylm_forward_loss_noalloc(96, 96, 32, torch.from_numpy(case.pos).cuda(), y, O, P, out, 0, case.b)
    assert math.isfinite(out[0].item())
