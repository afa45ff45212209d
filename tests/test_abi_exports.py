"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function
that include/ptylm.h declares (no compute calls are made)."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "ptylm.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lm_init", "forward_loss", "jvp", "jtvp", "ggn_matvec", "lm_solve", "lm_destroy",
              "ptylm_strerror", "gradient"):
        assert n in names, n


def test_library_exports_every_declared_symbol():
    from paper_2103_01767_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    assert ptylm.ptylm_strerror(0) == "success"
    assert "argument" in ptylm.ptylm_strerror(1)


def test_calls_fail_cleanly_without_a_gpu():
    """Without a usable GPU the library reports errors instead of crashing: argument
    errors are found on the host first, CUDA failures come back as PTYLM_ERR_CUDA."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the path taken when no GPU is present")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    pos = torch.zeros((4, 2), dtype=torch.int32)
    y = torch.zeros((4, 32, 32), dtype=torch.float32)
    with pytest.raises(ptylm.PtylmError) as e:
        ptylm.lm_init(64, 64, 30, 30, pos, y)
    assert e.value.status == ptylm.PTYLM_ERR_ARG
    with pytest.raises(ptylm.PtylmError) as e:
        ptylm.lm_init(64, 64, 32, 32, pos, y)
    assert e.value.status == ptylm.PTYLM_ERR_CUDA and "CUDA" in str(e.value)


def test_noalloc_wrapper_rejects_bad_arguments_before_the_library():
    """The context-free entry point has no context holding sizes or types, so the binding
    checks dtypes, sizes and device placement itself and raises ValueError before any
    pointer reaches the library."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2103_01767_gb300 import ptylm
    n, m, K = 64, 32, 3
    good = dict(positions=torch.zeros((K, 2), dtype=torch.int32),
                y=torch.zeros((K, m, m), dtype=torch.float32),
                O=torch.zeros((n, n), dtype=torch.complex64),
                P=torch.zeros((m, m), dtype=torch.complex64),
                out=torch.zeros(2, dtype=torch.float64))
    bad_cases = [
        ("positions", torch.zeros((K, 2), dtype=torch.int64)),            # int64 read as int2
        ("positions", torch.zeros((K, 3), dtype=torch.int32)),
        ("O", torch.zeros((n, n), dtype=torch.complex128)),
        ("O", torch.zeros((n, n - 1), dtype=torch.complex64)),
        ("P", torch.zeros((m, m), dtype=torch.float32)),
        ("y", torch.zeros((K, m, m), dtype=torch.float64)),
        ("y", torch.zeros((K - 1, m, m), dtype=torch.float32)),
        ("out", torch.zeros(2, dtype=torch.float32)),                      # 16-byte store into 8 bytes
        ("out", torch.zeros(1, dtype=torch.float64)),
        ("O", torch.zeros((n, 2 * n), dtype=torch.complex64)[:, ::2]),     # not contiguous
        ("O", np.zeros((n, n), np.complex64)),                             # host numpy array
    ]
    for name, bad in bad_cases:
        args = dict(good)
        args[name] = bad
        with pytest.raises(ValueError):
            ptylm.ptylm_forward_loss_noalloc(n, n, m, args["positions"], args["y"], args["O"], args["P"],
                                             args["out"])
    # well-typed host tensors are rejected too: the kernels would read host pointers
    with pytest.raises(ValueError, match="CUDA"):
        ptylm.ptylm_forward_loss_noalloc(n, n, m, good["positions"], good["y"], good["O"], good["P"], good["out"])


def test_batch_schedule_table():
    """The 24 autotuner schedules: index = order/positions schedule + 6 x (tile of the 32^2
    problems + 2 x tile of the 64^2 problems), every combination once."""
    from paper_2103_01767_gb300 import ptylm
    seen = set()
    for c in range(ptylm.N_SCHEDULES):
        d = ptylm.schedule_desc(c)
        assert d["order"] in (0, 1) and d["positions_per_team"] in (1, 2, 4)
        assert d["values_per_thread_32"] in (16, 32) and d["values_per_thread_64"] in (16, 32)
        seen.add(tuple(sorted(d.items())))
    assert len(seen) == ptylm.N_SCHEDULES == 24
    assert ptylm.schedule_desc(0) == {"order": 0, "positions_per_team": 1, "values_per_thread_32": 32,
                                      "values_per_thread_64": 32}
    assert ptylm.schedule_desc(18)["values_per_thread_32"] == 16 and ptylm.schedule_desc(18)["values_per_thread_64"] == 16


def test_batch_calls_reject_null_handles():
    """The batch entry points check their handles and arguments on the host."""
    import ctypes
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    lib = ptylm.load_library()
    assert lib.ptylm_batch_ggn_diag(None, None, ctypes.c_double(0.0)) == ptylm.PTYLM_ERR_ARG
    assert lib.ptylm_batch_set_schedule(None, 0) == ptylm.PTYLM_ERR_ARG
    assert lib.ptylm_batch_tune(None, None, None, 0) == ptylm.PTYLM_ERR_ARG
