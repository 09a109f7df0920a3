"""Reunitarisation and the precision policies built on it, against the oracle.

Reunitarisation (the projection back onto SU(3) that keeps FP32 and 12-real
fields unitary; Sec. 4.1 rebuilds the third row from the first two): the
resident field of every storage format is reunitarised by the library and
compared element by element with oracle.reunitarize of the same links, on
links perturbed off SU(3), so that the Gram-Schmidt step, its row order and
the conjugate in the rebuilt third row all act.

FP32 restarts of the mixed policy (option "fp32_restarts"): the result is an
exact FP64 gauge transform of the input (plaquette unchanged to 1e-13), it
reaches theta < 1e-14, and its F equals the all-FP64 solve's and the oracle's
to 1e-13 (the same maximum).

Tolerances: FP64 storage 1e-14 (Gram-Schmidt is a few dozen operations per
row); double-float storage holds 48 significand bits (2^-48 ~ 3.6e-15 per
element on input and output), 1e-13; FP32 storage rounds the input and the
output to FP32 (6e-8 of O(1) values each), 2e-7 absolute, with the oracle
run on the FP32-rounded input.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu


def cpu_field(dims, seed, gseed, plaq=0.60):
    return synth.as_numpy(synth.make_field(dims, plaq, seed, gseed))


def perturbed(dims, seed, eps):
    U = cpu_field(dims, seed, seed + 1)
    rng = np.random.default_rng(seed)
    U = U + eps * (rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    return np.ascontiguousarray(U)


def unitarity(U):
    M = U.reshape(-1, 3, 3)
    d = M @ np.conj(np.swapaxes(M, -1, -2)) - np.eye(3)
    return np.abs(d).max(), np.abs(np.linalg.det(M) - 1.0).max()


FORMATS = [  # (name, precision, options, tolerance, input rounding)
    ("fp64_18", gf.GF_FP64, {}, 1e-14, None),
    ("fp64_12", gf.GF_FP64, {"storage64": 12}, 1e-14, None),
    ("df64_18", gf.GF_FP64, {"fp64_arith": 1}, 1e-13, None),
    ("fp32_12", gf.GF_FP32, {"storage32": 12}, 2e-7, np.complex64),
    ("fp32_18", gf.GF_FP32, {"storage32": 18}, 2e-7, np.complex64),
]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
@pytest.mark.parametrize("fmt", range(len(FORMATS)))
@pytest.mark.parametrize("eps", [1e-3, 0.1])
def test_reunitarize_matches_oracle_elementwise(dims, fmt, eps):
    name, prec, opts, tol, rnd = FORMATS[fmt]
    U = perturbed(dims, 11, eps)
    assert unitarity(U)[0] > eps / 10  # really off SU(3)
    want = U.astype(rnd).astype(np.complex128) if rnd is not None else U.copy()
    oracle.reunitarize(want.reshape(-1, 3, 3))
    c = gf.gf_create(dims, gf.GF_LANDAU)
    for k, v in opts.items():
        gf.gf_set_option(c, k, v)
    d = torch.from_numpy(U).cuda()
    gf.gf_upload(c, d, prec)
    gf.gf_reunitarize(c)
    gf.gf_download(c, d)
    got = d.cpu().numpy()
    err = np.abs(got - want).max()
    assert err < tol, (name, err)
    assert unitarity(got)[0] < (1e-6 if rnd is not None else 1e-14)


def test_reunitarize_is_idempotent_on_su3():
    """Links already in SU(3) are left as they are (to rounding)."""
    dims = (4, 4, 4, 4)
    U = cpu_field(dims, 5, 6)
    c = gf.gf_create(dims, gf.GF_LANDAU)
    d = torch.from_numpy(U).cuda()
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_reunitarize(c)
    gf.gf_download(c, d)
    assert np.abs(d.cpu().numpy() - U).max() < 1e-15 * 10


def fix(U, dims, **opts):
    c = gf.gf_create(dims, gf.GF_LANDAU)
    gf.gf_set_option(c, "check_every", 10)
    for k, v in opts.items():
        gf.gf_set_option(c, k, v)
    d = torch.from_numpy(U).cuda()
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-14, 40000)
    return c, conv, it, F, th, d.cpu().numpy()


@pytest.mark.parametrize("dims,restarts", [((8, 8, 8, 8), 2), ((6, 4, 6, 10), 1), ((8, 8, 8, 8), 0)])
def test_fp32_restarts_reach_the_fp64_result(dims, restarts):
    U = cpu_field(dims, 3, 4)
    P0 = oracle.plaquette(U)
    _, conv64, it64, F64, th64, _ = fix(U, dims, precision=gf.GF_FP64)
    assert conv64
    opts = {"precision": gf.GF_MIXED, "fp32_restarts": restarts}
    if restarts:
        opts["theta_switch"] = 1e-30  # the first FP32 stage also runs to its rounding floor
    c, conv, it, F, th, W = fix(U, dims, **opts)
    assert conv and th < 1e-14
    if restarts:
        assert gf.gf_get_stat(c, "fp32_restarts_done") >= 1
        assert gf.gf_get_stat(c, "theta_after_restarts") < 1e-9
        # the restarts replace FP64 sweeps by FP32 ones
        assert gf.gf_get_stat(c, "sweeps_fp64") < it64
    assert abs(F - F64) <= 1e-13
    # an exact gauge transform of the input, checked by the oracle on the returned field
    assert oracle.plaquette(W) == pytest.approx(P0, abs=1e-13)
    assert oracle.theta(W, 0) < 1e-14
    assert oracle.functional(W, 0) == pytest.approx(F, abs=1e-14)
    assert unitarity(W)[0] < 1e-13
    # the same maximum as the oracle's own solve from the same input
    Uo = U.copy()
    conv_o, it_o, F_o, th_o = oracle.overrelax(Uo, 0, 1.7, 1e-14, 40000, 10)
    assert conv_o and abs(F - F_o) <= 1e-13


@pytest.mark.parametrize("gauge", [gf.GF_LANDAU, gf.GF_COULOMB])
@pytest.mark.parametrize("policy", ["fp64", "mixed", "mixed_restarts"])
def test_double_float_finish_is_an_exact_fp64_gauge_transform(gauge, policy):
    """fp64_arith 1: the double-float sweeps work on a copy and track E = g - 1;
    g is applied to the FP64 field in FP64, so the returned field is a gauge
    transform of the input to FP64 rounding: the plaquette to 1e-14, the same
    F as the native FP64 solve to 1e-14 (|dF| was 1.3e-13 while the links
    themselves were double-float), theta < 1e-14 by the oracle."""
    dims = (8, 8, 8, 8) if gauge == gf.GF_LANDAU else (6, 4, 6, 10)
    U = cpu_field(dims, 3, 4)
    P0 = oracle.plaquette(U)
    opts = {"precision": gf.GF_FP64 if policy == "fp64" else gf.GF_MIXED}
    if policy == "mixed_restarts":
        opts.update(fp32_restarts=2, theta_switch=1e-30)
    res = {}
    for arith in (0, 1):
        c = gf.gf_create(dims, gauge)
        gf.gf_set_option(c, "check_every", 10)
        for k, v in opts.items():
            gf.gf_set_option(c, k, v)
        gf.gf_set_option(c, "fp64_arith", arith)
        d = torch.from_numpy(U).cuda()
        conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-14, 40000)
        assert conv and th < 1e-14, (arith, th)
        W = d.cpu().numpy()
        res[arith] = (F, it, W)
        if arith == 1:
            assert gf.gf_get_stat(c, "sweeps_df64") > 0
            assert oracle.plaquette(W) == pytest.approx(P0, abs=1e-14)
            assert oracle.theta(W, gauge) < 1e-14
            assert oracle.functional(W, gauge) == pytest.approx(F, abs=1e-14)  # summation order
            assert unitarity(W)[0] < 1e-13
    assert abs(res[1][0] - res[0][0]) <= 1e-14
    # the same maximum, reached in about the same number of sweeps
    assert abs(res[1][1] - res[0][1]) <= 20 + res[0][1] // 20


def test_fma_peak_is_plausible():
    """The measured FMA rates that the ALU rooflines divide by: positive, and
    within a factor of a few of the nominal figures (FP64: 152 SMs x 4 flop
    per clock x about 2 GHz = 1.26 TFLOP/s; FP32: 152 x 256 x 2 GHz = 80)."""
    t64, ms64 = gf.gf_fma_peak(True, 2000)
    t32, ms32 = gf.gf_fma_peak(False, 50000)
    assert 0.3 < t64 < 3.0 and ms64 > 0
    assert 20.0 < t32 < 200.0 and ms32 > 0
    assert t32 > 10 * t64
    with pytest.raises(gf.GFError):
        gf.gf_fma_peak(True, 0)


@pytest.mark.parametrize("gauge", [gf.GF_LANDAU, gf.GF_COULOMB])
def test_double_float_annealing_is_an_exact_fp64_gauge_transform(gauge):
    """gf_anneal with fp64_arith 1: heatbath sweeps on a double-float copy with
    E = g - 1 tracked, g applied to the FP64 field in FP64.  A 12-sweep
    schedule equals the oracle's (same Philox draws, Sec. 1 annealing) to
    1e-10; after 300 sweeps the field is unitary to 1e-13 and its plaquette
    is the input's to 1e-14."""
    dims = (8, 8, 8, 16)
    U = cpu_field(dims, 27, 28, plaq=0.58)
    P0 = oracle.plaquette(U)
    c = gf.gf_create(dims, gauge)
    gf.gf_set_option(c, "fp64_arith", 1)
    d = torch.from_numpy(U).cuda()
    gf.gf_anneal(c, d, 1.45, 0.01, 12, 77)
    W = U.copy()
    assert oracle.anneal(W, gauge, 1.45, 0.01, 12, 77) == 0
    got = d.cpu().numpy()
    assert np.abs(got - W).max() / np.abs(W).max() < 1e-10
    d = torch.from_numpy(U).cuda()
    gf.gf_anneal(c, d, 1.45, 0.01, 300, 77)
    got = d.cpu().numpy()
    assert unitarity(got)[0] < 1e-13
    assert oracle.plaquette(got) == pytest.approx(P0, abs=1e-14)


@pytest.fixture
def oracle_sa_draw():
    yield oracle.set_sa_draw
    oracle.set_sa_draw(0)


SA_FORMS = {"acc": {"variant": 2}, "tps2": {"variant": 1, "threads_per_site": 2}, "df64": {"fp64_arith": 1}}


@pytest.mark.parametrize("gauge", [gf.GF_LANDAU, gf.GF_COULOMB])
@pytest.mark.parametrize("form", sorted(SA_FORMS))
@pytest.mark.parametrize("T", [1.45, 0.3, 0.01])
def test_fp32_heatbath_draw_half_sweep_parity(oracle_sa_draw, gauge, form, T):
    """The FP32 reading of the heatbath draw (option sa_draw 1) against the
    oracle's FP32 reading, same Philox draws.  Both decide accept/reject in FP32;
    their FP32 exp/log/cos/sin (CUDA's, the C library's) may differ by an ulp,
    which moves the drawn element by ~1e-7 relative: links agree to 1e-5 per
    half-sweep, and no decision differs on these seeds (a differing decision
    would change a whole site by O(1))."""
    oracle_sa_draw(1)
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, 35, 36)
    c = gf.gf_create(dims, gauge)
    for k, v in {**SA_FORMS[form], "sa_draw": 1}.items():
        gf.gf_set_option(c, k, v)
    d = torch.from_numpy(U).cuda()
    gf.gf_upload(c, d, gf.GF_FP64)
    for parity in (0, 1):
        gf.gf_sa_half_sweep(c, parity, T, 99, 4)
        assert oracle.sa_half_sweep(U, parity, T, gauge, 99, 4) == 0
    gf.gf_download(c, d)
    diff = np.abs(d.cpu().numpy() - U).reshape(-1, 18).max(axis=1)
    assert diff.max() < 1e-5, (int((diff > 1e-5).sum()), diff.max())


def test_fp32_draw_annealing_is_exact_and_matches_oracle(oracle_sa_draw):
    """gf_anneal with the double-float sweeps (E tracked, g applied in FP64) and
    the FP32 draw: a 6-sweep schedule 1.45 -> 0.01 equals the oracle's FP32
    reading to 1e-4 (differences of ~1e-7 per draw grow along the chain), and
    300 sweeps keep the plaquette to 1e-14 and unitarity to 1e-13."""
    oracle_sa_draw(1)
    dims = (8, 8, 8, 16)
    U = cpu_field(dims, 27, 28, plaq=0.58)
    P0 = oracle.plaquette(U)
    c = gf.gf_create(dims, gf.GF_COULOMB)
    gf.gf_set_option(c, "fp64_arith", 1)
    gf.gf_set_option(c, "sa_draw", 1)
    d = torch.from_numpy(U).cuda()
    gf.gf_anneal(c, d, 1.45, 0.01, 6, 77)
    W = U.copy()
    assert oracle.anneal(W, gf.GF_COULOMB, 1.45, 0.01, 6, 77) == 0
    assert np.abs(d.cpu().numpy() - W).max() < 1e-4
    d = torch.from_numpy(U).cuda()
    gf.gf_anneal(c, d, 1.45, 0.01, 300, 77)
    got = d.cpu().numpy()
    assert unitarity(got)[0] < 1e-13
    assert oracle.plaquette(got) == pytest.approx(P0, abs=1e-14)
