"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function
that include/ptylm.h declares (no compute calls are made)."""
import ctypes
import os
import re

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
