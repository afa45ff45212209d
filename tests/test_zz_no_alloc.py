"""The allocation-free entry point ptylm_forward_loss_noalloc, called through the C-ABI, on two
calls in a row: against the context-based forward_loss (cache = 0, the call the header says it
equals, and cache = 1) on the same inputs at 1e-5, and against the FP64 oracle's error metric
with the checks of the parity tests (test_gpu_parity.compare).

Callers that must not allocate device memory use this entry point: serving or real-time loops
that reserve all their memory at start-up (cudaMalloc and cudaFree can synchronise the device
and take unbounded time), plug-ins inside a host framework whose memory pool already holds
nearly all of the device memory, and code whose device bytes must all be accounted to another
allocator.  Its scratch is a file-scope device array shared by all calls.  This file is
collected last so that a run stopping at the first failure has already run everything else;
it passes alone in a fresh process as well as after the other tests."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.fp32_eval import ORDERS
from tests.problems import make_case
from tests.test_gpu_parity import compare, fp32_model

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


@pytest.mark.parametrize("side_stream", [False, True])
@pytest.mark.parametrize("shape,loss", [((160, 64, 23), 0), ((640, 128, 400), 1), ((256, 32, 3000), 1)])
def test_noalloc_loss_matches_context_path_on_two_calls(lib, shape, loss, side_stream):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=31)
    pos = torch.from_numpy(case.pos).cuda()
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    P = _c64(case.P)
    O_np = synth.to_c64(case.O_true + synth.random_complex(case.O_true.shape, seed=32, scale=0.05))
    O = _c64(O_np)
    ctx = lib.lm_init(n, n, m, m, pos, y, loss, case.b)
    f0, dl2_0 = lib.forward_loss(ctx, O, P, cache=0)
    f1, dl2_1 = lib.forward_loss(ctx, O, P, cache=1)
    lib.lm_destroy(ctx)
    pb = case.problem()
    case.at_truth = False
    mdl = fp32_model(case)
    f_orc, dl2_orc = oracle.loss(pb, O_np, return_dl_norm2=True)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream() if side_stream else None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        out.fill_(math.nan)  # each call must write its own result
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                lib.ptylm_forward_loss_noalloc(n, n, m, pos, y, O, P, out, loss, case.b, stream=stream)
            torch.cuda.current_stream().wait_stream(stream)
        else:
            lib.ptylm_forward_loss_noalloc(n, n, m, pos, y, O, P, out, loss, case.b)
        f, dl2 = out.tolist()
        # the existing entry point on the same inputs: the same arithmetic, 1e-5
        parity.check("noalloc f vs forward_loss(cache=0)", f, f0)
        parity.check("noalloc ||dl||^2 vs forward_loss(cache=0)", dl2, dl2_0)
        parity.check("noalloc f vs forward_loss(cache=1)", f, f1)
        parity.check("noalloc ||dl||^2 vs forward_loss(cache=1)", dl2, dl2_1)
        # the FP64 oracle, with the checks of the parity tests (Poisson counts away from the
        # truth: the FP32 conditioning bound and the independent FP32 evaluation)
        compare("noalloc f vs oracle", f, f_orc, case, lambda A: oracle.loss(pb, A), (O_np,),
                lambda: [mdl.loss_value(O_np, order=o)[0] for o in ORDERS])
        compare("noalloc ||dl||^2 vs oracle", dl2, dl2_orc, case,
                lambda A: oracle.loss(pb, A, return_dl_norm2=True)[1], (O_np,),
                lambda: [mdl.loss_value(O_np, order=o)[1] for o in ORDERS])


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
    big = torch.zeros((512, 512), dtype=torch.complex64, device="cuda")
    P256 = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
    y256 = torch.zeros(5 * 256 * 256, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.PtylmError) as e:
        lib.ptylm_forward_loss_noalloc(512, 512, 256, torch.from_numpy(case.pos).cuda(), y256, big, P256, out, 0,
                                       case.b)
    assert e.value.status == lib.PTYLM_ERR_ARG
    # a valid call afterwards still works (the flag is cleared per call)
    lib.ptylm_forward_loss_noalloc(96, 96, 32, torch.from_numpy(case.pos).cuda(), y, O, P, out, 0, case.b)
    assert math.isfinite(out[0].item())
