"""Learned warm start on the GPU against the oracle.

Tolerances: BF16 stores 8 significant bits (unit roundoff 2^-8); the network
inputs are compared at 4e-3 relative.

The network (forward output, loss, every weight and bias gradient) is
compared with the FP64 oracle in two ways:
- bit for bit, on integer-valued weights, biases and inputs chosen so that
  every hidden activation and every back-propagated value is exactly
  representable in BF16 and every sum exactly in FP32: the GPU's rounding
  steps are then all exact, so any wrong tap, channel, site, wrap or mask
  shows up as a difference.  The test asserts that precondition on the
  oracle's own intermediate values before it compares.  Lattices: 8x16x4x4
  and 16x32x4x4 (periodic wrap inside one halo tile, several tiles),
  32x4x4x3, the ragged 6x4x6x10 (1440 sites, not a multiple of the 128-site
  tile) and 16x16x8x8 (where each CTA of the x-line weight-gradient kernel
  runs several stages through its buffer ring), each with the per-tap gather
  kernels, the x-line and halo-tile kernels and the CUDA-core kernels;
- element by element on random weights, within 8 standard deviations of
  the rounding error, which is propagated through the layers from the
  arithmetic: the BF16 rounding of every stored activation and the FP32
  accumulation of every sum, independent and zero mean, carried forward
  through W^2 (a worst-case bound through |W| is vacuous for random signs).

The applied gauge transformation is stored as FP32 and reprojected onto SU(3)
in FP64, so it differs from the exact exponential by ~1e-7; it is still an
exact FP64 gauge transformation (plaquette to 1e-13).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, learned, synth

pytestmark = pytest.mark.gpu


def cpu_field(dims, seed=1, gseed=2):
    return synth.as_numpy(synth.make_field(dims, 0.60, seed, gseed))


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_features_match_oracle():
    dims = (6, 4, 6, 8)
    U = cpu_field(dims, 3, 4)
    oracle.or_sweeps(U, 1.7, 0, 20)
    c = gf.gf_create(dims, 0)
    gf.gf_upload(c, torch.from_numpy(U).cuda(), gf.GF_FP64)
    s = math.sqrt(oracle.theta(U, 0))
    V = int(np.prod(dims))
    f = torch.empty(V, 80, dtype=torch.bfloat16, device="cuda")
    gf.gf_features(c, s, f)
    got = f.float().cpu().numpy().astype(np.float64)
    want = oracle.features(U, s)
    assert np.all(np.abs(got - want) <= 4e-3 * np.abs(want) + 1e-30)


def test_apply_algebra_is_exact_gauge_transform():
    dims = (4, 6, 4, 8)
    U = cpu_field(dims, 5, 6)
    V = int(np.prod(dims))
    rng = np.random.default_rng(0)
    for scale in (1e-3, 0.7):
        cc = rng.standard_normal((V, 8)).astype(np.float32)
        ctx = gf.gf_create(dims, 0)
        d = torch.from_numpy(U).cuda()
        gf.gf_upload(ctx, d, gf.GF_FP64)
        gf.gf_apply_algebra(ctx, torch.from_numpy(cc).cuda(), scale)
        gf.gf_download(ctx, d)
        W = U.copy()
        g = oracle.expmap(cc.astype(np.float64), scale).reshape(U.shape[:4] + (3, 3))
        oracle.gauge_transform(W, g)
        assert np.abs(d.cpu().numpy() - W).max() < 1e-6
        assert gf.gf_plaquette(ctx, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)


def test_tracked_gauge_and_labels():
    dims = (8, 8, 8, 8)
    U0 = cpu_field(dims, 7, 8)
    for prec in (gf.GF_FP32, gf.GF_FP64):
        ctx = gf.gf_create(dims, 0)
        gf.gf_set_option(ctx, "track", 1)
        d = torch.from_numpy(U0).cuda()
        gf.gf_upload(ctx, d, prec)
        gf.gf_gauge_reset(ctx)
        gf.gf_or_sweeps(ctx, 1.7, 30)
        gf.gf_download(ctx, d)
        g = np.zeros(U0.shape[:4] + (3, 3), dtype=np.complex128)
        gf.gf_get_gauge(ctx, g)
        W = U0.copy()
        oracle.gauge_transform(W, g)  # U_now must equal g U0 g^+ (g tracked in FP32)
        assert np.abs(d.cpu().numpy() - W).max() < (2e-5 if prec == gf.GF_FP32 else 2e-6)
        s = 0.01
        lab = torch.empty(int(np.prod(dims)), 8, dtype=torch.float32, device="cuda")
        gf.gf_gauge_algebra(ctx, s, lab)
        want = oracle.algebra_log(g.reshape(-1, 3, 3), s)
        np.testing.assert_allclose(lab.cpu().numpy(), want, rtol=1e-5, atol=1e-4)


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def test_network_forward_and_gradient_match_oracle():
    dims = (4, 4, 4, 6)
    V = int(np.prod(dims))
    rng = np.random.default_rng(1)
    ch = gf.NET_CHANNELS
    P = gf.gf_net_param_count()
    assert P == oracle.net_param_count(ch)
    params = learned.init_params(3, scale_last=1.0)
    # biases non-zero to exercise them
    off = 0
    for l in range(4):
        off += 81 * ch[l + 1] * ch[l]
        params[off:off + ch[l + 1]] = rng.standard_normal(ch[l + 1]) * 0.1
        off += ch[l + 1]
    feats = bf16_round(rng.standard_normal((V, 80)))
    target = rng.standard_normal((V, 8)).astype(np.float32)
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, params)
    fd = torch.from_numpy(feats).to(torch.bfloat16).cuda()
    td = torch.from_numpy(target).cuda()
    out = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(net, fd, out)
    grad = np.zeros(P, dtype=np.float32)
    loss = gf.gf_net_gradient(net, fd, td, grad)
    # oracle on the BF16-rounded weights (biases stay FP32)
    pq = params.astype(np.float64).copy()
    off = 0
    for l in range(4):
        n = 81 * ch[l + 1] * ch[l]
        pq[off:off + n] = bf16_round(params[off:off + n])
        off += n + ch[l + 1]
    oloss, ograd, oout = oracle.net_loss(feats, target, pq, dims, ch)
    assert rel_l2(out.cpu().numpy(), oout) < 2e-2
    assert loss == pytest.approx(oloss, rel=2e-2)
    off = 0
    for l in range(4):
        n = 81 * ch[l + 1] * ch[l]
        assert rel_l2(grad[off:off + n], ograd[off:off + n]) < 5e-2, l
        assert rel_l2(grad[off + n:off + n + ch[l + 1]], ograd[off + n:off + n + ch[l + 1]]) < 5e-2, l
        off += n + ch[l + 1]


CHANNELS = (80, 32, 32, 32, 8)


def exact_network(dims, seed, nnz=(12, 6, 3, 6)):
    """Integer weights (nnz entries of +-1 per output channel), integer biases
    in {-1, 0, 1} and inputs in {-1, 0, 1}; the target differs from the
    output by q * {-1, 0, 1}, q the odd part of the output count, so that the
    loss gradient 2 (out - target) / (8 V) is a power of two times an integer."""
    rng = np.random.default_rng(seed)
    V = int(np.prod(dims))
    Ws, bs, flat = [], [], []
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W = np.zeros((81, co, ci))
        for o in range(co):
            idx = rng.choice(81 * ci, nnz[l], replace=False)
            W[idx // ci, o, idx % ci] = rng.choice([-1.0, 1.0], nnz[l])
        b = rng.integers(-1, 2, co).astype(np.float64)
        Ws.append(W)
        bs.append(b)
        flat += [W.ravel(), b]
    X0 = rng.integers(-1, 2, (V, 80)).astype(np.float64)
    acts = [X0]
    for l in range(4):
        Y = oracle.conv_forward(acts[-1], Ws[l], bs[l], dims)
        acts.append(np.maximum(Y, 0.0) if l < 3 else Y)
    nout = V * 8
    q = nout >> ((nout & -nout).bit_length() - 1)
    target = acts[4] - q * rng.integers(-1, 2, (V, 8)).astype(np.float64)
    # precondition: every value the GPU rounds to BF16 is exactly representable
    g = 2.0 * (acts[4] - target) / nout
    rounded = [acts[1], acts[2], acts[3], g]
    for l in (3, 2, 1):
        g = oracle.conv_backward_data(g, Ws[l], dims) * (acts[l] > 0)
        rounded.append(g)
    for a in rounded:
        assert np.array_equal(bf16_round(a).astype(np.float64), a), "design not exact in BF16"
    return np.concatenate(flat).astype(np.float32), X0, target, acts[4]


# net option conv_halo of each convolution path: 1 = x-line kernel where Lx is
# 8, 16 or 32, 2 = halo-tile kernel (Lx % 8, Ly % 16, Lz % 2), both falling back
# to the per-tap gather kernel (0) where the extents do not allow them.  On the
# x-line path every layer writes the next one's ghost-padded input itself; with
# Lz odd, (16, 8, 3, 4), conv_halo 1 runs the x-line weight-gradient kernel
# beside the gather convolutions instead.
CONV_HALO = {"gather": 0, "xline": 1, "halo_tile": 2, "cuda_cores": 0}


@pytest.mark.parametrize(
    "dims", [(8, 16, 4, 4), (16, 32, 4, 4), (32, 4, 4, 3), (6, 4, 6, 10), (16, 16, 8, 8), (16, 8, 3, 4)]
)
@pytest.mark.parametrize("path", ["gather", "xline", "halo_tile", "cuda_cores"])
def test_network_exact_arithmetic_matches_oracle_bit_for_bit(dims, path):
    params, X0, target, out_exact = exact_network(dims, seed=sum(dims))
    V = int(np.prod(dims))
    loss_o, grad_o, out_o = oracle.net_loss(X0, target, params.astype(np.float64), dims, CHANNELS)
    assert np.array_equal(out_o, out_exact)
    assert np.array_equal(grad_o.astype(np.float32).astype(np.float64), grad_o)  # exact in FP32
    net = gf.gf_net_create(dims)
    gf.gf_net_set_option(net, "tensor_cores", 0 if path == "cuda_cores" else 1)
    gf.gf_net_set_option(net, "conv_halo", CONV_HALO[path])
    gf.gf_net_set_params(net, params)
    fd = torch.from_numpy(X0.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(target.astype(np.float32)).cuda()
    out = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(net, fd, out)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), out_o)
    grad = np.zeros(gf.gf_net_param_count(), dtype=np.float32)
    loss = gf.gf_net_gradient(net, fd, td, grad)
    assert loss == pytest.approx(loss_o, rel=1e-14)
    bad = np.flatnonzero(grad.astype(np.float64) != grad_o)
    assert bad.size == 0, (bad[:10], grad[bad[:10]], grad_o[bad[:10]])


def test_network_exact_arithmetic_persistent_tiles_bit_for_bit():
    """The persistent x-line convolution walks 512 tiles with 152 CTAs or
    fewer, so every CTA runs three or four tiles: both accumulator sets are
    reused and the buffer ring wraps across tiles.  Forward output and all
    gradients bit for bit against the oracle, as above, on 32x32x16x8."""
    dims = (32, 32, 16, 8)
    params, X0, target, out_exact = exact_network(dims, seed=sum(dims))
    V = int(np.prod(dims))
    loss_o, grad_o, out_o = oracle.net_loss(X0, target, params.astype(np.float64), dims, CHANNELS)
    assert np.array_equal(out_o, out_exact)
    assert np.array_equal(grad_o.astype(np.float32).astype(np.float64), grad_o)
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, params)
    fd = torch.from_numpy(X0.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(target.astype(np.float32)).cuda()
    out = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(net, fd, out)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), out_o)
    grad = np.zeros(gf.gf_net_param_count(), dtype=np.float32)
    loss = gf.gf_net_gradient(net, fd, td, grad)
    assert loss == pytest.approx(loss_o, rel=1e-14)
    bad = np.flatnonzero(grad.astype(np.float64) != grad_o)
    assert bad.size == 0, (bad[:10], grad[bad[:10]], grad_o[bad[:10]])


def forward_error_sigma(X0, Ws, bs, dims):
    """Element-wise standard deviation of GPU output - FP64 output, from the
    arithmetic: every stored activation is rounded to BF16 (an error uniform
    within half a unit in the last place, at most 2^-8 of the value, variance
    (2^-7 |x|)^2 / 12), every sum of K products accumulates in FP32 (variance
    at most K (2^-24 sum |W||X|)^2 / 3); the errors are independent and zero
    mean, so their variances propagate through the next layer as W^2, and
    through ReLU only where the activation is positive."""
    X, VarE = X0, np.zeros_like(X0)
    for l in range(4):
        K = 81 * X.shape[1]
        Y = oracle.conv_forward(X, Ws[l], bs[l], dims)
        mag = oracle.conv_forward(np.abs(X), np.abs(Ws[l]), np.abs(bs[l]), dims)
        VarD = oracle.conv_forward(VarE, Ws[l] ** 2, None, dims) + K * (2.0 ** -24 * mag) ** 2 / 3.0
        if l == 3:
            return Y, np.sqrt(VarD)
        X = np.maximum(Y, 0.0)
        VarE = VarD * (Y > 0) + (2.0 ** -7 * X) ** 2 / 12.0


@pytest.mark.parametrize("dims", [(8, 16, 4, 4), (32, 4, 4, 3), (6, 4, 6, 10)])
@pytest.mark.parametrize("path", ["gather", "xline", "halo_tile", "cuda_cores"])
def test_network_forward_within_rounding_bound_elementwise(dims, path):
    V = int(np.prod(dims))
    rng = np.random.default_rng(7)
    params = learned.init_params(21, scale_last=1.0)
    Ws, bs, off = [], [], 0
    for l in range(4):
        n = 81 * CHANNELS[l + 1] * CHANNELS[l]
        params[off + n:off + n + CHANNELS[l + 1]] = rng.standard_normal(CHANNELS[l + 1]) * 0.1
        Ws.append(bf16_round(params[off:off + n]).astype(np.float64).reshape(81, CHANNELS[l + 1], CHANNELS[l]))
        bs.append(params[off + n:off + n + CHANNELS[l + 1]].astype(np.float64))
        off += n + CHANNELS[l + 1]
    X0 = bf16_round(rng.standard_normal((V, 80))).astype(np.float64)
    Y, sigma = forward_error_sigma(X0, Ws, bs, dims)
    D = 8.0 * sigma + 1e-7 * np.abs(Y)
    net = gf.gf_net_create(dims)
    gf.gf_net_set_option(net, "tensor_cores", 0 if path == "cuda_cores" else 1)
    gf.gf_net_set_option(net, "conv_halo", CONV_HALO[path])
    gf.gf_net_set_params(net, params)
    out = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(net, torch.from_numpy(X0.astype(np.float32)).to(torch.bfloat16).cuda(), out)
    err = np.abs(out.cpu().numpy().astype(np.float64) - Y)
    assert np.all(err <= D), (err.max(), D[err > D][:5])
    # the bound is not vacuous: it is about 6 % of the output's scale, while a
    # single wrong tap (one of 81) moves an output by about a ninth of it
    assert np.median(D) < 0.1 * np.median(np.abs(Y))


def test_training_reduces_loss():
    """A student network fits the outputs of a teacher network (a target the
    architecture can represent)."""
    dims = (4, 4, 4, 4)
    V = 256
    rng = np.random.default_rng(2)
    feats = torch.from_numpy(bf16_round(rng.standard_normal((V, 80)))).to(torch.bfloat16).cuda()
    teacher = gf.gf_net_create(dims)
    gf.gf_net_set_params(teacher, learned.init_params(11, scale_last=1.0))
    target = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(teacher, feats, target)
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, learned.init_params(4))
    l0 = gf.gf_net_gradient(net, feats, target)
    for _ in range(150):
        gf.gf_net_train_step(net, feats, target, 1e-3)
    assert gf.gf_net_gradient(net, feats, target) < 0.5 * l0


@pytest.mark.parametrize("dims", [(32, 4, 4, 3), (6, 4, 6, 10)])
def test_train_step_weight_copies_match_a_fresh_cast(dims):
    """The Adam kernel writes each updated weight into the four BF16 copies the
    convolutions read; setting the same FP32 parameters again casts them anew.
    Both must give the same network, bit for bit (x-line and gather paths)."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(7)
    feats = torch.from_numpy(bf16_round(rng.standard_normal((V, 80)))).to(torch.bfloat16).cuda()
    target = torch.from_numpy(rng.standard_normal((V, 8)).astype(np.float32)).cuda()
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, learned.init_params(5))
    for _ in range(3):
        gf.gf_net_train_step(net, feats, target, 1e-2)
    out_step = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(net, feats, out_step)
    params = np.zeros(gf.gf_net_param_count(), dtype=np.float32)
    gf.gf_net_get_params(net, params)
    fresh = gf.gf_net_create(dims)
    gf.gf_net_set_params(fresh, params)
    out_fresh = torch.empty(V, 8, dtype=torch.float32, device="cuda")
    gf.gf_net_forward(fresh, feats, out_fresh)
    assert torch.equal(out_step, out_fresh)
    assert out_step.abs().max().item() > 0


def test_tensor_core_and_cuda_core_convolutions_agree():
    dims = (4, 6, 4, 8)
    V = int(np.prod(dims))
    rng = np.random.default_rng(3)
    feats = torch.from_numpy(bf16_round(rng.standard_normal((V, 80)))).to(torch.bfloat16).cuda()
    target = torch.from_numpy(rng.standard_normal((V, 8)).astype(np.float32)).cuda()
    params = learned.init_params(12, scale_last=1.0)
    outs, grads = [], []
    for tc in (0, 1):
        net = gf.gf_net_create(dims)
        gf.gf_net_set_option(net, "tensor_cores", tc)
        gf.gf_net_set_params(net, params)
        out = torch.empty(V, 8, dtype=torch.float32, device="cuda")
        gf.gf_net_forward(net, feats, out)
        g = np.zeros(gf.gf_net_param_count(), dtype=np.float32)
        gf.gf_net_gradient(net, feats, target, g)
        outs.append(out.cpu().numpy())
        grads.append(g)
    # same BF16 operands, FP32 accumulation in a different order
    assert rel_l2(outs[1], outs[0]) < 1e-2
    assert rel_l2(grads[1], grads[0]) < 3e-2


def test_zero_network_leaves_the_mixed_solver_unchanged():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, 9, 10)
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, np.zeros(gf.gf_net_param_count(), dtype=np.float32))
    res = []
    for attach in (False, True):
        c = gf.gf_create(dims, 0)
        gf.gf_set_option(c, "precision", gf.GF_MIXED)
        gf.gf_set_option(c, "check_every", 10)
        if attach:
            gf.gf_set_net(c, net)
        d = torch.from_numpy(U).cuda()
        res.append(gf.gf_overrelax(c, d, 1.7, 1e-14, 20000))
    assert res[0][0] and res[1][0]
    assert res[0][1] == res[1][1]
    assert res[0][2] == pytest.approx(res[1][2], abs=1e-13)


def test_learned_warm_start_pipeline_small():
    """Train on solver pairs from 8^4 fields, then fix fresh fields with and
    without the network; both must converge to the same F, and the network
    must save FP64 sweeps (the full-size measurement is in bench.py)."""
    dims = (8, 8, 8, 8)
    ctx = gf.gf_create(dims, 0)
    pairs = []
    for k in range(6):
        U = synth.make_field(dims, 0.60, 1000 + k, 3000 + k, device="cuda")
        pairs.append(learned.make_pair(ctx, U, label_theta=1e-11))
    net = gf.gf_net_create(dims)
    gf.gf_net_set_params(net, learned.init_params(5))
    hist = learned.train(net, pairs[:5], epochs=30, lr=1e-3)
    assert hist[-1] < hist[0]
    sweeps = {}
    for attach in (False, True, "repeat"):
        c = gf.gf_create(dims, 0)
        gf.gf_set_option(c, "precision", gf.GF_MIXED)
        gf.gf_set_option(c, "check_every", 10)
        if attach:
            gf.gf_set_net(c, net)
        if attach == "repeat":  # applied again at every hundredfold drop of theta
            gf.gf_set_option(c, "learned_repeat", 3)
        U = synth.make_field(dims, 0.60, 5000, 6000, device="cuda")
        conv, it, F, th = gf.gf_overrelax(c, U, 1.7, 1e-14, 50000)
        assert conv and th < 1e-14
        sweeps[attach] = (gf.gf_get_stat(c, "sweeps_fp64"), F)
        if attach == "repeat":
            assert gf.gf_get_stat(c, "learned_applications") >= 1
    assert abs(sweeps["repeat"][1] - sweeps[False][1]) < 1e-9
    assert abs(sweeps[True][1] - sweeps[False][1]) < 1e-9
    print("fp64 sweeps without / with the network:", sweeps[False][0], sweeps[True][0])
    # what the trained network gains: fewer FP64 sweeps to the same final F
    assert sweeps[True][0] < sweeps[False][0]



def test_learned_warm_start_only_in_landau_gauge():
    net = gf.gf_net_create((4, 4, 4, 4))
    for gauge in (gf.GF_COULOMB, gf.GF_MAG):
        c = gf.gf_create((4, 4, 4, 4), gauge)
        with pytest.raises(gf.GFError) as e:
            gf.gf_set_net(c, net)
        assert e.value.code == gf.GF_EINVAL
    c = gf.gf_create((4, 4, 4, 4), gf.GF_LANDAU)
    gf.gf_set_net(c, net)
    gf.gf_set_net(c, None)
