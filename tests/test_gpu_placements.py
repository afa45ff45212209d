"""The 128^2 GGN matvec against the FP64 oracle at scan placements that stress its
addressing: patches touching every border of a rectangular object (rows and columns
swapped would show), even and odd first columns, odd and even object widths, and vectors
that start 8 bytes into their allocations.  All agree with the oracle to the FP32 bound
1e-5 (Gaussian metric, well conditioned)."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.problems import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
M = 128


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    return ptylm


def border_positions(ny, nx, extra, seed):
    """Corners and edges with both column parities, then `extra` uniform positions."""
    r_hi, c_hi = ny - M, nx - M
    pts = [(0, 0), (0, 1), (0, c_hi), (0, c_hi - 1), (r_hi, 0), (r_hi, 1), (r_hi, c_hi), (r_hi, c_hi - 1),
           (r_hi // 2, c_hi // 2), (r_hi // 2, c_hi // 2 | 1), (1, 2), (2, 3)]
    rng = np.random.default_rng(seed)
    rnd = np.stack([rng.integers(0, r_hi + 1, extra), rng.integers(0, c_hi + 1, extra)], axis=1)
    return np.concatenate([np.array(pts), rnd]).astype(np.int32)


def setup(lib, ny, nx, extra, seed):
    pos = border_positions(ny, nx, extra, seed)
    O_true = synth.to_c64(synth.object_texture(max(ny, nx), seed=seed)[:ny, :nx])
    P = synth.to_c64(synth.probe_disk_defocus(M, 40.0))
    pb = oracle.Problem((ny, nx), P, pos, None, 0, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true))
    O = synth.to_c64(O_true + synth.random_complex(O_true.shape, seed=seed + 1, scale=0.05))
    ctx = lib.lm_init(ny, nx, M, M, torch.from_numpy(pos).cuda(), f32(pb.y), 0, 1e-8)
    lib.forward_loss(ctx, c64(O), c64(P), cache=1)
    return pb, ctx, O


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("ny,nx,extra", [(260, 266, 30), (300, 268, 500), (259, 267, 30)])
def test_matvec_border_placements(lib, ny, nx, extra):
    pb, ctx, O = setup(lib, ny, nx, extra, seed=ny + nx)
    v = synth.to_c64(synth.random_complex((ny, nx), seed=7))
    vd = c64(v)
    out = torch.empty_like(vd)
    for lam in (0.0, 0.29):
        lib.ggn_matvec(ctx, vd, out, lam)
        ref = oracle.ggn_matvec(pb, O, v, lam=lam)
        parity.check("(G + lam I) v (border placements)", host(out), ref, TOL)
        parity.check("(G + lam I) v (border placements)", host(out), ref, TOL, norm="max")


def test_matvec_vectors_at_8_byte_offsets(lib):
    ny, nx = 260, 266
    pb, ctx, O = setup(lib, ny, nx, 30, seed=3)
    v = synth.to_c64(synth.random_complex((ny, nx), seed=8))
    # views starting 8 bytes into their allocations: not 16-byte aligned
    vbuf = torch.zeros(ny * nx + 1, dtype=torch.complex64, device="cuda")
    obuf = torch.zeros(ny * nx + 1, dtype=torch.complex64, device="cuda")
    vd = vbuf[1:].view(ny, nx)
    vd.copy_(c64(v))
    out = obuf[1:].view(ny, nx)
    assert vd.data_ptr() % 16 == 8 and out.data_ptr() % 16 == 8
    lib.ggn_matvec(ctx, vd, out, 0.11)
    ref = oracle.ggn_matvec(pb, O, v, lam=0.11)
    parity.check("(G + lam I) v (border placements)", host(out), ref, TOL)
    parity.check("(G + lam I) v (border placements)", host(out), ref, TOL, norm="max")
    aligned = torch.empty((ny, nx), dtype=torch.complex64, device="cuda")
    lib.ggn_matvec(ctx, c64(v), aligned, 0.11)
    parity.check("(G + lam I) v, 8-byte vs 16-byte aligned", host(aligned), host(out), 2 * TOL, basis="2 x 1e-5 (two GPU results)")


def test_matvec_launches_are_profiled(lib):
    ny, nx = 260, 266
    _, ctx, _ = setup(lib, ny, nx, 10, seed=4)
    v = c64(synth.random_complex((ny, nx), seed=9))
    out = torch.empty_like(v)
    lib.ptylm_profile(ctx, 1)
    for _ in range(3):
        lib.ggn_matvec(ctx, v, out, 0.0)
    ms, n = lib.ptylm_profile_read(ctx, lib.KERNEL_GGN_MATVEC)
    lib.ptylm_profile(ctx, 0)
    assert n == 3 and ms > 0.0


def test_profile_select_times_only_the_chosen_kernel(lib):
    ny, nx = 260, 266
    pb, ctx, O_np = setup(lib, ny, nx, 10, seed=5)
    O, P = c64(O_np), c64(pb.P)
    v = c64(synth.random_complex((ny, nx), seed=10))
    out = torch.empty_like(v)
    lib.ptylm_profile_select(ctx, [lib.KERNEL_GGN_MATVEC])
    for _ in range(2):
        lib.forward_loss(ctx, O, P, cache=1)
        lib.ggn_matvec(ctx, v, out, 0.0)
    mv = lib.ptylm_profile_read(ctx, lib.KERNEL_GGN_MATVEC)
    fc = lib.ptylm_profile_read(ctx, lib.KERNEL_FORWARD_CACHE)
    _, launches = lib.ptylm_profile_read(ctx, -1)
    lib.ptylm_profile_select(ctx, [])
    assert mv[1] == 2 and mv[0] > 0.0
    assert fc == (0.0, 0)                 # not timed
    assert launches >= 4                  # but every launch is counted
