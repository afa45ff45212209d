"""Learned initialisation on the GPU against its FP64 oracle (oracle/learned.py): physics
input, training pairs, network forward and gradients (bfloat16 weights on both sides; on the
GPU tensor-core convolutions with FP32 accumulation and activations carried as bfloat16
pairs), the stitched initial object, and training that lowers the loss.

Tolerances: 1e-5 relative for the FFT-based inputs (the FP32 bound of the forward model);
1e-4 for network outputs and gradients, whose FP32 sums run over up to 2304 products per
output and 2 x 128^2 x 9 products per weight gradient, and whose activation pairs carry
2^-18 relative representation error per layer."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.problems import make_case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M = 128
WIDTHS = (32, 64, 96)
FULL = (64, 128, 256)   # 740,226 parameters


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    return ptylm


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def probe():
    return synth.to_c64(synth.probe_disk_defocus(M, 40.0))


def flat_params(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def bf16_params(params):
    return [(L.to_bf16(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in params]


def test_training_pairs_match_the_oracle(lib):
    pool = np.stack([synth.to_c64(synth.object_texture(160, seed=s)) for s in (1, 2)])
    P = probe()
    samples = np.array([[0, 5, 7], [1, 20, 31], [0, 32, 0], [1, 0, 32]], np.int32)
    net = lib.net_create(WIDTHS, max_batch=4)
    X = torch.empty((4, 2, M, M), dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    lib.net_pairs(net, c64(pool), 160, torch.from_numpy(samples).cuda(), c64(P), X, T)
    for i, (o, r, c) in enumerate(samples):
        patch = pool[o, r:r + M, c:c + M].astype(np.complex128)
        y = np.abs(np.fft.fft2(P * patch, norm="ortho")) ** 2
        ref = L.physics_input(y[None], P)[0]
        assert rel_err(X[i].cpu().numpy(), ref) <= 1e-5, i
        assert np.array_equal(T[i, 0].cpu().numpy(), patch.real.astype(np.float32))
        assert np.array_equal(T[i, 1].cpu().numpy(), patch.imag.astype(np.float32))
    bad = torch.from_numpy(np.array([[0, 40, 0]], np.int32)).cuda()   # 40 + 128 > 160
    with pytest.raises(lib.PtylmError):
        lib.net_pairs(net, c64(pool), 160, bad, c64(P), X, T)


@pytest.mark.parametrize("loss", [0, 1])
def test_physics_inputs_from_a_context(lib, loss):
    case = make_case(288, M, K=9, loss=loss, peak=1e3 if loss else 0.0, seed=60 + loss, noisy=False)
    ctx = lib.lm_init(288, 288, M, M, torch.from_numpy(case.pos).cuda(), f32(case.y), loss, case.b)
    net = lib.net_create(WIDTHS, max_batch=4)
    idx = np.array([0, 4, 8], np.int32)
    X = torch.empty((3, 2, M, M), dtype=torch.float32, device="cuda")
    lib.learned_inputs(ctx, net, c64(case.P), torch.from_numpy(idx).cuda(), X)
    ref = L.physics_input(case.y[idx], case.P)
    assert rel_err(X.cpu().numpy(), ref) <= 1e-5


# (96, 64, 96): a first width that does not divide 256 keeps the last layer on the tensor
# cores; the others run it on the CUDA cores (conv_last.cu)
@pytest.mark.parametrize("widths,N", [(WIDTHS, 3), (FULL, 2), ((96, 64, 96), 2)])
def test_network_forward_and_gradients_match_the_oracle(lib, widths, N):
    params = L.init_params(widths, seed=3)
    # non-zero biases so they take part in the comparison
    params = [(W, 0.05 * np.random.default_rng(10 + l).standard_normal(b.shape)) for l, (W, b) in enumerate(params)]
    net = lib.net_create(widths, max_batch=4, seed=1)
    assert net.num_params == flat_params(params).size
    lib.net_set_params(net, flat_params(params))
    rng = np.random.default_rng(4)
    X = rng.standard_normal((N, 2, M, M)).astype(np.float32)
    T = rng.standard_normal((N, 2, M, M)).astype(np.float32)
    mask = (np.abs(probe()) > 0).astype(np.float32)
    out = torch.empty((N, 2, M, M), dtype=torch.float32, device="cuda")
    lib.net_forward(net, f32(X), out)
    pb = bf16_params(params)
    acts = L.net_forward(pb, X.astype(np.float64), widths)
    tag = f"net {widths} N={N}"
    parity.check(f"{tag} output", out.cpu().numpy(), acts[-1], 1e-4, basis="1e-4 (network)")
    parity.check(f"{tag} output", out.cpu().numpy(), acts[-1], 1e-4, norm="max", basis="1e-4 (network)")
    loss = lib.net_loss_grad(net, f32(X), f32(T), f32(mask))
    # Hidden activations: each layer against the oracle, and the ReLU decisions.  Activations
    # travel between layers as bfloat16 pairs (2^-18 relative), so a pre-activation within that
    # precision of zero can land on the other side of the kink than in FP64; the backward pass
    # of the oracle takes the network's own decisions (a discrete choice made in the kernel's
    # precision), after checking that every disagreement sits at such a near-zero value.
    relu_masks = []
    for l in range(1, 6):
        a_gpu = lib.net_activation(net, l, N).cpu().numpy().astype(np.float64)
        a_ref = acts[l]
        parity.check(f"{tag} activation {l}", a_gpu, a_ref, 1e-4, basis="1e-4 (network)")
        m_gpu, m_ref = a_gpu > 0.0, a_ref > 0.0
        diff = m_gpu != m_ref
        if diff.any():
            near = np.maximum(np.abs(a_gpu[diff]), np.abs(a_ref[diff])).max() / np.abs(a_ref).max()
            assert near <= 1e-4, (l, int(diff.sum()), near)
        relu_masks.append(m_gpu)
    loss_ref, grads_ref = L.net_loss_and_grads(pb, X.astype(np.float64), T.astype(np.float64), mask.astype(np.float64),
                                               widths, relu_masks=relu_masks)
    parity.check(f"{tag} loss", loss, loss_ref, 1e-4, basis="1e-4 (network)")
    _, g = lib.net_get_params(net)
    off = 0
    for l, (dW, db) in enumerate(grads_ref):
        gw = g[off:off + dW.size].reshape(dW.shape)
        off += dW.size
        gb = g[off:off + db.size]
        off += db.size
        parity.check(f"{tag} dW{l + 1}", gw, dW, 1e-4, basis="1e-4 (network)")
        parity.check(f"{tag} dW{l + 1}", gw, dW, 1e-4, norm="max", basis="1e-4 (network)")
        parity.check(f"{tag} db{l + 1}", gb, db, 1e-4, basis="1e-4 (network)")


def test_forward_is_independent_of_the_batch_it_runs_in(lib):
    """Every image's output is the same whether it runs alone or inside a batch (the grid,
    the phases per CTA and the pipeline depth change with N; the arithmetic per output does
    not)."""
    net = lib.net_create(FULL, max_batch=8, seed=5)
    X = np.random.default_rng(8).standard_normal((8, 2, M, M)).astype(np.float32)
    out8 = torch.empty((8, 2, M, M), dtype=torch.float32, device="cuda")
    lib.net_forward(net, f32(X), out8)
    out1 = torch.empty((1, 2, M, M), dtype=torch.float32, device="cuda")
    for i in (0, 5, 7):
        lib.net_forward(net, f32(X[i:i + 1]), out1)
        assert torch.equal(out1[0], out8[i]), i


def test_stitched_initial_object_matches_the_oracle(lib):
    case = make_case(256, M, K=12, loss=0, seed=70, noisy=False)
    ctx = lib.lm_init(256, 256, M, M, torch.from_numpy(case.pos).cuda(), f32(case.y), 0, case.b)
    params = L.init_params(WIDTHS, seed=5)
    net = lib.net_create(WIDTHS, max_batch=5, seed=2)   # 12 positions -> chunks of 5, 5, 2
    lib.net_set_params(net, flat_params(params))
    idx = np.arange(12, dtype=np.int32)
    O0 = torch.empty((256, 256), dtype=torch.complex64, device="cuda")
    lib.learned_init(ctx, net, c64(case.P), torch.from_numpy(idx).cuda(), O0)
    e = L.physics_input(case.y, case.P)
    acts = L.net_forward(bf16_params(params), e, WIDTHS)
    patches = acts[-1][:, 0] + 1j * acts[-1][:, 1]
    ref = L.stitch(patches, case.pos, case.P, (256, 256))
    assert rel_err(O0.cpu().numpy(), ref) <= 1e-4


def test_training_lowers_the_loss(lib):
    pool = np.stack([synth.to_c64(synth.object_texture(256, seed=s)) for s in range(4)])
    net = lib.net_create(WIDTHS, max_batch=16, seed=7)
    hist = lib.net_train(net, c64(pool), 4, 256, c64(probe()), steps=300, batch=16, lr=2e-3, seed=11)
    assert np.all(np.isfinite(hist))
    assert hist[-30:].mean() < 0.5 * hist[:10].mean(), (hist[:10].mean(), hist[-30:].mean())


def test_learned_argument_errors(lib):
    with pytest.raises(lib.PtylmError) as e:
        lib.net_create((32, 48, 64))
    assert e.value.status == lib.PTYLM_ERR_ARG
    with pytest.raises(lib.PtylmError):
        lib.net_create(WIDTHS, m=64)


def test_trained_network_gains_over_the_flat_start(lib):
    """What the trained network gains over the method without it: on a held-out object its
    stitched estimate is much closer to the truth than the flat start, and Algorithm 1 from
    it reaches 1e-3 object error in no more outer iterations (noiseless amplitude data)."""
    n = 384
    pool = np.stack([synth.to_c64(synth.object_texture(n, seed=200 + s)) for s in range(4)])
    P = probe()
    net = lib.net_create(FULL, max_batch=32, seed=3)
    hist = lib.net_train(net, c64(pool), 4, n, c64(P), steps=800, batch=32, lr=2e-3, seed=9)
    assert hist[-50:].mean() < 0.05 * hist[:10].mean()
    O_true = synth.to_c64(synth.object_texture(n, seed=7))
    pos, _ = synth.raster_positions(n, M, 12, 20, 0, seed=8)
    pb = oracle.Problem((n, n), P, pos, None, 0, 1e-8)
    y = oracle.intensity(pb, O_true)
    ctx = lib.lm_init(n, n, M, M, torch.from_numpy(pos).cuda(), f32(y), 0, 1e-8)
    mask = synth.illumination_mask(n, P, pos, 0.1)
    maskd = torch.from_numpy(mask.astype(np.uint8)).cuda()
    O0 = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    lib.learned_init(ctx, net, c64(P), torch.from_numpy(np.arange(pos.shape[0], dtype=np.int32)).cuda(), O0)
    flat = synth.flat_object(n) * np.abs(O_true).mean()
    e_learned = oracle.object_error(O0.cpu().numpy(), O_true, mask)
    e_flat = oracle.object_error(flat, O_true, mask)
    assert e_learned < 0.6 * e_flat, (e_learned, e_flat)
    outer = {}
    for name, start in (("flat", c64(flat)), ("learned", O0.clone())):
        _, info = lib.lm_solve(ctx, start, c64(P), hist_len=100, O_ref=c64(O_true), mask=maskd, max_outer=100,
                               target_err=1e-3)
        assert info["err"][-1] <= 1e-3, name
        outer[name] = info["n_outer"]
    assert outer["learned"] <= outer["flat"], outer
