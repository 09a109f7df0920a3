"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Tolerances
----------
FP64 storage: 1e-12 relative per half-sweep/sweep, element by element (the
two sides differ only in rounding order and FMA contraction, ~1e-16 per
operation over a few hundred operations).
FP32 storage: the input is rounded to FP32 (relative 6e-8) and each link
update is ~150 FP32 operations; the bound used is 5e-6 absolute per link
element (|U_ab| <= 1) per half-sweep, 2e-5 after a few sweeps.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
SMALL = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 6, 10), (10, 6, 4, 8)]


def cpu_field(dims, seed=1, gseed=2, plaq=0.60, pure=False):
    return synth.as_numpy(synth.make_field(dims, plaq, seed, gseed, pure_gauge=pure))


def dev(U):
    return torch.from_numpy(U).to(DEV)


def host(T):
    return T.cpu().numpy()


def ctx_for(dims, gauge=0, **opts):
    c = gf.gf_create(dims, gauge)
    # threads_per_site = 0 in these tests selects the accumulate-form variant
    if opts.get("threads_per_site", None) == 0:
        opts = dict(opts)
        del opts["threads_per_site"]
        opts["variant"] = 2
    for k, v in opts.items():
        gf.gf_set_option(c, k, v)
    return c


def max_rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------------------
# FP64 half-sweeps and sweeps, every threads-per-site variant
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", SMALL)
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("tps", [0, 1, 2, 4, 8])
def test_fp64_half_sweep_parity(dims, gauge, tps):
    U = cpu_field(dims, seed=3, gseed=4)
    c = ctx_for(dims, gauge, threads_per_site=tps)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    for parity in (0, 1):
        gf.gf_or_half_sweep(c, parity, 1.7)
        oracle.or_half_sweep(U, parity, 1.7, gauge)
        gf.gf_download(c, d)
        assert max_rel(host(d), U) < 1e-12


@pytest.mark.parametrize("storage", [18, 12])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10)])
@pytest.mark.parametrize("variant", [1, 2])
def test_fp64_sweeps_parity(storage, dims, variant):
    U = cpu_field(dims, seed=5, gseed=6)
    c = ctx_for(dims, 0, storage64=storage, variant=variant)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_or_sweeps(c, 1.7, 10)
    oracle.or_sweeps(U, 1.7, 0, 10)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-12


@pytest.mark.parametrize("block", [32, 64, 256])
def test_fp64_block_shapes(block):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=7, gseed=8)
    c = ctx_for(dims, 0, block=block, threads_per_site=2)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_or_sweeps(c, 1.3, 3)
    oracle.or_sweeps(U, 1.3, 0, 3)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-12


# ---------------------------------------------------------------------------
# FP32 storage
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", [12, 18])
@pytest.mark.parametrize("tps", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("gauge", [0, 1])
def test_fp32_half_sweep_parity(storage, tps, gauge):
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=9, gseed=10)
    c = ctx_for(dims, gauge, storage32=storage, threads_per_site=tps)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP32)
    gf.gf_or_half_sweep(c, 0, 1.7)
    gf.gf_or_half_sweep(c, 1, 1.7)
    oracle.or_sweeps(U, 1.7, gauge, 1)
    gf.gf_download(c, d)
    assert np.abs(host(d) - U).max() < 5e-6
    gf.gf_or_sweeps(c, 1.7, 4)
    oracle.or_sweeps(U, 1.7, gauge, 4)
    gf.gf_download(c, d)
    assert np.abs(host(d) - U).max() < 2e-5


# ---------------------------------------------------------------------------
# reductions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", SMALL)
@pytest.mark.parametrize("gauge", [0, 1])
def test_functional_theta_plaquette(dims, gauge):
    U = cpu_field(dims, seed=11, gseed=12)
    oracle.or_sweeps(U, 1.7, gauge, 3)  # a field with smaller theta as well
    c = ctx_for(dims, gauge)
    d = dev(U)
    assert gf.gf_functional(c, d) == pytest.approx(oracle.functional(U, gauge), rel=1e-13, abs=1e-15)
    assert gf.gf_theta(c, d) == pytest.approx(oracle.theta(U, gauge), rel=1e-12)
    assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), rel=1e-13)
    # resident-field measurement, FP64 storage 18 and 12
    for st in (18, 12):
        gf.gf_set_option(c, "storage64", st)
        gf.gf_upload(c, d, gf.GF_FP64)
        F, th = gf.gf_measure(c)
        assert F == pytest.approx(oracle.functional(U, gauge), rel=1e-13, abs=1e-15)
        assert th == pytest.approx(oracle.theta(U, gauge), rel=1e-11)
    # host (numpy) input takes the same path through a staging copy
    assert gf.gf_theta(c, U) == pytest.approx(oracle.theta(U, gauge), rel=1e-12)


def test_measure_is_deterministic():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=13, gseed=14)
    c = ctx_for(dims, 0)
    d = dev(U)
    vals = {gf.gf_theta(c, d) for _ in range(5)}
    assert len(vals) == 1


# ---------------------------------------------------------------------------
# the whole method
# ---------------------------------------------------------------------------
def test_overrelax_fp64_matches_oracle_sweep_count():
    """Config: Landau, omega = 1.7, 8^4, theta < 1e-12, seeds 1/2."""
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=1, gseed=2)
    c = ctx_for(dims, 0, check_every=10)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-12, 5000)
    oconv, oit, oF, oth = oracle.overrelax(U, 0, 1.7, 1e-12, 5000, 10)
    assert conv and oconv
    assert it == oit
    assert F == pytest.approx(oF, rel=1e-12)
    assert th == pytest.approx(oth, rel=1e-6)
    assert max_rel(host(d), U) < 1e-10


def test_pure_gauge_reaches_unit_functional_on_gpu():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, gseed=2, pure=True)
    c = ctx_for(dims, 0, check_every=10)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-24, 20000)
    assert conv and th < 1e-24
    assert F == pytest.approx(1.0, abs=1e-12)


def test_plaquette_invariant_under_gpu_sweeps():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=15, gseed=16)
    P = oracle.plaquette(U)
    c = ctx_for(dims, 0)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_or_sweeps(c, 1.7, 200)
    gf.gf_download(c, d)
    assert gf.gf_plaquette(c, d) == pytest.approx(P, abs=1e-13)


def test_host_pointer_path_equals_device_path():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=17, gseed=18)
    c = ctx_for(dims, 0, check_every=10)
    d = dev(U)
    Uh = U.copy()
    r1 = gf.gf_overrelax(c, d, 1.7, 1e-10, 2000)
    r2 = gf.gf_overrelax(c, Uh, 1.7, 1e-10, 2000)
    assert r1 == r2
    np.testing.assert_array_equal(host(d), Uh)


def test_not_converged_is_reported_with_valid_outputs():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=19, gseed=20)
    c = ctx_for(dims, 0, check_every=10)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-14, 25)
    assert not conv and it == 25 and th > 1e-14
    assert th == pytest.approx(gf.gf_theta(c, d), rel=1e-12)


@pytest.mark.parametrize("variant", [1, 2])
def test_mixed_precision_reaches_same_functional(variant):
    """FP32 (12-real) sweeps to theta < 1e-6, then FP64 to 1e-14 (config on 8^4)."""
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=3, gseed=4)
    c64 = ctx_for(dims, 0, check_every=10)
    d64 = dev(U)
    conv, it64, F64, th64 = gf.gf_overrelax(c64, d64, 1.7, 1e-14, 20000)
    assert conv
    for track in (1, 0):
        c = ctx_for(dims, 0, check_every=10, precision=gf.GF_MIXED, track_gauge=track, variant=variant)
        d = dev(U)
        conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-14, 20000)
        assert conv and th < 1e-14
        assert gf.gf_get_stat(c, "sweeps_fp32") > 0 and gf.gf_get_stat(c, "sweeps_fp64") > 0
        if track:
            # a gauge transform of the exact input: same F as all-FP64, plaquette exact
            assert abs(F - F64) < 1e-10
            assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)
        else:
            assert abs(F - F64) < 1e-6


def test_fp32_policy_converges_to_fp32_precision():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=3, gseed=4)
    c = ctx_for(dims, 0, check_every=10, precision=gf.GF_FP32)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-8, 20000)
    assert conv and th < 1e-8


# ---------------------------------------------------------------------------
# simulated annealing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("tps", [0, 1, 2, 8])
@pytest.mark.parametrize("T", [1.45, 0.3, 0.01])
def test_sa_half_sweep_parity(gauge, tps, T):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=21, gseed=22)
    c = ctx_for(dims, gauge, threads_per_site=tps)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_sa_half_sweep(c, 0, T, 1234, 7)
    gf.gf_sa_half_sweep(c, 1, T, 1234, 7)
    assert oracle.sa_half_sweep(U, 0, T, gauge, 1234, 7) == 0
    assert oracle.sa_half_sweep(U, 1, T, gauge, 1234, 7) == 0
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-11


def test_anneal_schedule_parity():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=23, gseed=24)
    c = ctx_for(dims, 1, sa_sweep_offset=100)
    d = dev(U)
    gf.gf_anneal(c, d, 1.45, 0.01, 12, 99)
    assert oracle.anneal(U, 1, 1.45, 0.01, 12, 99, 100) == 0
    assert max_rel(host(d), U) < 1e-10


def test_anneal_rejection_cap_reports_error():
    dims = (4, 4, 4, 4)
    U = cpu_field(dims, seed=25, gseed=26)
    c = ctx_for(dims, 0, sa_cap=1)
    d = dev(U)
    rc = gf.gf_anneal(c, d, 0.05, 0.05, 1, 5, allow_reject=True)
    assert rc == gf.GF_EREJECT
    assert gf.gf_get_stat(c, "sa_rejects") > 0
    P = oracle.plaquette(U)
    assert gf.gf_plaquette(c, d) == pytest.approx(P, abs=1e-13)


# ---------------------------------------------------------------------------
# argument errors surface as GFError, no device fault
# ---------------------------------------------------------------------------
def test_argument_errors():
    dims = (4, 4, 4, 4)
    U = cpu_field(dims)
    c = ctx_for(dims, 0)
    d = dev(U)
    with pytest.raises(gf.GFError) as e:
        gf.gf_overrelax(c, d, 2.5, 1e-12, 10)
    assert e.value.code == gf.GF_EINVAL
    with pytest.raises(gf.GFError):
        gf.gf_overrelax(c, d, float("nan"), 1e-12, 10)
    with pytest.raises(gf.GFError):
        gf.gf_anneal(c, d, -1.0, 0.1, 3, 1)
    with pytest.raises(ValueError):
        gf.gf_theta(c, torch.zeros(10, dtype=torch.float64, device=DEV))


def test_autotune_picks_a_valid_config_and_keeps_parity():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=27, gseed=28)
    c = ctx_for(dims, 0)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    tps, block = gf.gf_autotune(c)
    assert tps in (0, 1, 2, 4, 8) and block in (64, 128, 256)  # 0: accumulate form
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_or_sweeps(c, 1.7, 3)
    oracle.or_sweeps(U, 1.7, 0, 3)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-12


# ---------------------------------------------------------------------------
# FP64-class double-float storage and arithmetic (option fp64_arith = 1): each
# double-float operation has relative error ~2^-47 (7e-15) and the input is
# rounded to a 48-bit significand; a link update is ~100 operations, so the
# bound is 1e-12 relative per half-sweep, growing linearly with the number of
# half-sweeps compared (2e-12 per sweep).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 6, 10)])
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("variant", [2, 1])
def test_df64_half_sweeps_parity(dims, gauge, variant):
    U = cpu_field(dims, seed=31, gseed=32)
    c = ctx_for(dims, gauge, fp64_arith=1, variant=variant)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-14  # 48-bit storage round trip
    for parity in (0, 1):
        gf.gf_or_half_sweep(c, parity, 1.7)
        oracle.or_half_sweep(U, parity, 1.7, gauge)
        gf.gf_download(c, d)
        assert max_rel(host(d), U) < 1e-12
    gf.gf_or_sweeps(c, 1.7, 10)
    oracle.or_sweeps(U, 1.7, gauge, 10)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 2e-12 * 11  # 11 sweeps in total


@pytest.mark.parametrize("gauge", [0, 1])
def test_df64_heatbath_parity(gauge):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=33, gseed=34)
    c = ctx_for(dims, gauge, fp64_arith=1)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    for parity in (0, 1):
        gf.gf_sa_half_sweep(c, parity, 0.7, 99, 4)
        assert oracle.sa_half_sweep(U, parity, 0.7, gauge, 99, 4) == 0
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-11


def test_mixed_with_df64_phase_matches_native():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=3, gseed=4)
    res = {}
    for arith in (0, 1):
        c = ctx_for(dims, 0, check_every=10, precision=gf.GF_MIXED, fp64_arith=arith)
        d = dev(U)
        res[arith] = gf.gf_overrelax(c, d, 1.7, 1e-14, 20000)
        assert res[arith][0] and res[arith][3] < 1e-14
        assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)
    assert abs(res[0][2] - res[1][2]) < 1e-12
    assert abs(res[0][1] - res[1][1]) <= 10


# ---------------------------------------------------------------------------
# stochastic relaxation (Sec. 1): same Philox draws on both sides
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("tps", [0, 2, 8])
@pytest.mark.parametrize("p", [0.0, 0.5, 1.0])
def test_sr_half_sweep_parity(gauge, tps, p):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=41, gseed=42)
    c = ctx_for(dims, gauge, threads_per_site=tps)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    for parity in (0, 1):
        gf.gf_sr_half_sweep(c, parity, p, 77, 9)
        oracle.sr_half_sweep(U, parity, p, gauge, 77, 9)
    gf.gf_download(c, d)
    assert max_rel(host(d), U) < 1e-12


@pytest.mark.parametrize("arith", [0, 1])
def test_sr_df64_parity(arith):
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=43, gseed=44)
    c = ctx_for(dims, 0, fp64_arith=arith)
    d = dev(U)
    gf.gf_upload(c, d, gf.GF_FP64)
    for n in range(3):
        for parity in (0, 1):
            gf.gf_sr_half_sweep(c, parity, 0.6, 5, n)
            oracle.sr_half_sweep(U, parity, 0.6, 0, 5, n)
    gf.gf_download(c, d)
    # native FP64: 1e-12; double-float: 1e-12 per half-sweep (6 here)
    assert max_rel(host(d), U) < (1e-12 if arith == 0 else 6e-12)


def test_overrelax_with_stochastic_relaxation_converges():
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=1, gseed=2)
    c = ctx_for(dims, 0, check_every=10, stochastic_p=0.85, sr_seed=3)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-12, 20000)
    assert conv and th < 1e-12
    assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)
    # the same number of stochastic sweeps in the oracle gives the same field
    V = U.copy()
    for n in range(it):
        for parity in (0, 1):
            oracle.sr_half_sweep(V, parity, 0.85, 0, 3, n)
    assert max_rel(host(d), V) < 1e-9


# ---------------------------------------------------------------------------
# in-graph kernel timing (used for the benchmark's roofline)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("graphs", [1, 0])
def test_kernel_timing_counts_every_sweep_launch(graphs):
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=3, gseed=4)
    c = ctx_for(dims, 0, check_every=10, precision=gf.GF_MIXED, use_graphs=graphs, kernel_timing=1)
    ref = ctx_for(dims, 0, check_every=10, precision=gf.GF_MIXED, use_graphs=graphs)
    d, e = dev(U), dev(U)
    r = gf.gf_overrelax(c, d, 1.7, 1e-14, 20000)
    r0 = gf.gf_overrelax(ref, e, 1.7, 1e-14, 20000)
    assert r[0] and r[1] == r0[1]
    assert torch.equal(d, e)  # the events change nothing in the result
    for ph in ("fp32", "fp64"):
        n = gf.gf_get_stat(c, f"sweep_launches_{ph}")
        assert n == 2 * gf.gf_get_stat(c, f"sweeps_{ph}")
        ms = gf.gf_get_stat(c, f"ms_sweep_kernels_{ph}")
        assert 0.0 < ms <= gf.gf_get_stat(c, f"ms_{ph}")


# ---------------------------------------------------------------------------
# accumulate form with a register budget (FP64 storage)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10)])
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("storage", [18, 12])
@pytest.mark.parametrize("regs", [168, 128])
def test_acc_register_budget_parity(dims, gauge, storage, regs):
    U = cpu_field(dims, seed=3, gseed=4)
    c = ctx_for(dims, gauge, variant=2, acc_registers=regs, storage64=storage, block=128)
    gf.gf_upload(c, dev(U), gf.GF_FP64)
    W = U.copy()
    for p in (0, 1):
        gf.gf_or_half_sweep(c, p, 1.7)
        oracle.or_half_sweep(W, p, 1.7, gauge)
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    assert max_rel(host(d), W) < 1e-12
    # heatbath through the same kernels
    gf.gf_sa_half_sweep(c, 0, 0.7, 5, 3)
    oracle.sa_half_sweep(W, 0, 0.7, gauge, 5, 3)
    gf.gf_download(c, d)
    assert max_rel(host(d), W) < 1e-11


# ---------------------------------------------------------------------------
# readings of g -> g^omega (option or_variant), same reading on both sides
# ---------------------------------------------------------------------------
@pytest.fixture
def oracle_or_variant():
    yield oracle.set_or_variant
    oracle.set_or_variant(0)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("form", ["acc", "tps2", "df64", "fp32"])
def test_or_variant_parity(oracle_or_variant, variant, gauge, form):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=3, gseed=4)
    opts = {"or_variant": variant}
    prec = gf.GF_FP64
    if form == "acc":
        opts["variant"] = 2
    elif form == "tps2":
        opts.update(variant=1, threads_per_site=2)
    elif form == "df64":
        opts["fp64_arith"] = 1
    else:
        prec = gf.GF_FP32
    c = ctx_for(dims, gauge, **opts)
    gf.gf_upload(c, dev(U), prec)
    oracle_or_variant(variant)
    W = U.copy()
    for p in (0, 1):
        gf.gf_or_half_sweep(c, p, 1.7)
        oracle.or_half_sweep(W, p, 1.7, gauge)
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    if prec == gf.GF_FP32:
        assert np.abs(host(d) - W).max() < 5e-6 * 2
    else:
        assert max_rel(host(d), W) < 1e-12


@pytest.mark.parametrize("variant", [1, 2])
def test_or_variant_solver_converges_with_oracle_sweep_count(oracle_or_variant, variant):
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=3, gseed=4)
    c = ctx_for(dims, 0, or_variant=variant, check_every=10)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-12, 20000)
    oracle_or_variant(variant)
    W = U.copy()
    oconv, oit, oF, oth = oracle.overrelax(W, 0, 1.7, 1e-12, 20000, 10)
    assert conv and oconv and it == oit
    assert abs(F - oF) < 1e-12


# ---------------------------------------------------------------------------
# per-timeslice F and theta (Coulomb gauge fixes each timeslice on its own)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10), (10, 6, 4, 8)])
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("prec", [gf.GF_FP64, gf.GF_FP32])
def test_timeslice_measurement_matches_oracle(dims, gauge, prec):
    U = cpu_field(dims, seed=21, gseed=22)
    c = ctx_for(dims, gauge)
    gf.gf_upload(c, dev(U), prec)
    F_t, th_t = gf.gf_measure_timeslices(c)
    oF, oth = oracle.timeslices(U, gauge)
    if prec == gf.GF_FP64:
        np.testing.assert_allclose(F_t, oF, rtol=1e-13)
        np.testing.assert_allclose(th_t, oth, rtol=1e-12)
    else:  # FP32 storage: the links are rounded to FP32 (6e-8)
        np.testing.assert_allclose(F_t, oF, atol=1e-6)
        np.testing.assert_allclose(th_t, oth, rtol=1e-5)
    F, th = gf.gf_measure(c)
    assert F == pytest.approx(F_t.mean(), rel=1e-12)


def test_coulomb_converges_every_timeslice():
    dims = (8, 8, 8, 6)
    U = cpu_field(dims, seed=23, gseed=24)
    c = ctx_for(dims, 1, check_every=10, theta_per_timeslice=1)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-12, 20000)
    assert conv
    W = host(d)
    oF, oth = oracle.timeslices(W, 1)
    assert oth.max() < 1e-12
    assert th == pytest.approx(oth.max(), rel=1e-9)
    # the global criterion stops no later (its theta is the mean)
    c2 = ctx_for(dims, 1, check_every=10)
    conv2, it2, F2, th2 = gf.gf_overrelax(c2, dev(U), 1.7, 1e-12, 20000)
    assert conv2 and it2 <= it


# ---------------------------------------------------------------------------
# a long annealing schedule down to T = 0.01 through every site-update form
# ---------------------------------------------------------------------------
FORMS = [dict(variant=1, threads_per_site=2), dict(variant=2), dict(variant=2, acc_registers=168, block=64),
         dict(variant=2, acc_registers=168, block=128), dict(variant=2, acc_registers=128, block=128),
         dict(variant=2, acc_registers=128, block=256), dict(fp64_arith=1), dict(variant=2, storage64=12),
         dict(variant=1, threads_per_site=2, storage64=12)]


def unitarity(U):
    M = U.reshape(-1, 3, 3)
    return np.abs(M @ np.conj(np.swapaxes(M, -1, -2)) - np.eye(3)).max()


@pytest.mark.parametrize("form", range(len(FORMS)))
@pytest.mark.parametrize("gauge", [0, 1])
def test_anneal_long_schedule_every_form(form, gauge):
    """(1) a 10-sweep schedule 1.45 -> 0.01 matches the oracle (same draws);
    (2) 300 sweeps of the schedule stay unitary and keep the plaquette.  Long
    runs are not compared link by link: heatbath trajectories with the same
    random numbers separate exponentially from rounding-level differences, so
    only the final F is compared, loosely."""
    dims = (8, 8, 8, 16)
    U = cpu_field(dims, seed=27, gseed=28, plaq=0.58)
    P = oracle.plaquette(U)
    c = ctx_for(dims, gauge, **FORMS[form])
    d = dev(U)
    gf.gf_anneal(c, d, 1.45, 0.01, 10, 77)
    W = U.copy()
    assert oracle.anneal(W, gauge, 1.45, 0.01, 10, 77) == 0
    assert max_rel(host(d), W) < 1e-10
    d = dev(U)
    gf.gf_anneal(c, d, 1.45, 0.01, 300, 77)  # raises on a rejection-cap hit
    out = host(d)
    assert np.isfinite(out).all() and unitarity(out) < 1e-12
    assert gf.gf_plaquette(c, d) == pytest.approx(P, abs=1e-12)
    W = U.copy()
    assert oracle.anneal(W, gauge, 1.45, 0.01, 300, 77) == 0
    assert gf.gf_functional(c, d) == pytest.approx(oracle.functional(W, gauge), abs=0.02)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-10, 5000)  # overrelaxation continues from there
    assert conv and np.isfinite(F)


def test_anneal_autotuned_heatbath_config():
    """gf_anneal tunes its own launch configuration (heatbath timing); the
    result is that of any fixed configuration up to rounding."""
    dims = (8, 8, 8, 8)
    U = cpu_field(dims, seed=29, gseed=30)
    a = ctx_for(dims, 1, autotune=1)
    b = ctx_for(dims, 1, variant=1, threads_per_site=4)
    da, db = dev(U), dev(U)
    gf.gf_anneal(a, da, 1.2, 0.1, 6, 5)
    gf.gf_anneal(b, db, 1.2, 0.1, 6, 5)
    assert max_rel(host(da), host(db)) < 1e-11
    assert gf.gf_get_stat(a, "sweeps") == 6


# ---------------------------------------------------------------------------
# maximally Abelian gauge (Sec. 6): the same subgroup relaxation on both sides
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
@pytest.mark.parametrize("tps", [1, 2, 4, 8])
@pytest.mark.parametrize("storage", [18, 12])
def test_mag_half_sweep_parity(dims, tps, storage):
    U = cpu_field(dims, seed=61, gseed=62)
    c = ctx_for(dims, gf.GF_MAG, threads_per_site=tps, storage64=storage)
    gf.gf_upload(c, dev(U), gf.GF_FP64)
    W = U.copy()
    for p, om in ((0, 1.0), (1, 1.7), (0, 1.7)):
        gf.gf_or_half_sweep(c, p, om)
        oracle.mag_half_sweep(W, p, om)
        d = torch.empty_like(dev(U))
        gf.gf_download(c, d)
        assert max_rel(host(d), W) < 1e-12


def test_mag_fp32_half_sweep():
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=63, gseed=64)
    c = ctx_for(dims, gf.GF_MAG, threads_per_site=2)
    gf.gf_upload(c, dev(U), gf.GF_FP32)
    W = U.copy()
    gf.gf_or_half_sweep(c, 0, 1.7)
    oracle.mag_half_sweep(W, 0, 1.7)
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    # the MAG step is an eigenvector of H: FP32 rounding of H (~1e-6 of |H|)
    # is amplified by |H| / (eigenvalue gap), up to ~10 on random fields
    assert np.abs(host(d) - W).max() < 2e-5


@pytest.mark.parametrize("prec", [gf.GF_FP64, gf.GF_FP32])
def test_mag_measurement_matches_oracle(prec):
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=65, gseed=66)
    c = ctx_for(dims, gf.GF_MAG)
    F_aos, th_aos = gf.gf_functional(c, dev(U)), gf.gf_theta(c, dev(U))
    assert F_aos == pytest.approx(oracle.mag_functional(U), rel=1e-13)
    assert th_aos == pytest.approx(oracle.mag_theta(U), rel=1e-12)
    gf.gf_upload(c, dev(U), prec)
    F, th = gf.gf_measure(c)
    tol = 1e-12 if prec == gf.GF_FP64 else 1e-5
    assert F == pytest.approx(oracle.mag_functional(U), rel=tol)
    assert th == pytest.approx(oracle.mag_theta(U), rel=tol)


def test_mag_overrelax_matches_oracle_sweep_count():
    dims = (4, 4, 4, 6)
    U = cpu_field(dims, seed=67, gseed=68)
    c = ctx_for(dims, gf.GF_MAG, check_every=10)
    d = dev(U)
    conv, it, F, th = gf.gf_overrelax(c, d, 1.7, 1e-10, 4000)
    assert conv and th < 1e-10
    W = U.copy()
    n = 0
    while not oracle.mag_theta(W) < 1e-10 and n < 4000:
        oracle.mag_sweeps(W, 1.7, 10)
        n += 10
    assert n == it
    assert F == pytest.approx(oracle.mag_functional(W), abs=1e-12)
    assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)


def test_mag_mixed_precision_is_exact_gauge_transform():
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=69, gseed=70)
    res = {}
    for prec in (gf.GF_FP64, gf.GF_MIXED):
        c = ctx_for(dims, gf.GF_MAG, check_every=10, precision=prec, theta_switch=1e-5)
        d = dev(U)
        res[prec] = gf.gf_overrelax(c, d, 1.7, 1e-11, 10000)
        assert res[prec][0]
        assert gf.gf_plaquette(c, d) == pytest.approx(oracle.plaquette(U), abs=1e-13)
    assert abs(res[gf.GF_FP64][2] - res[gf.GF_MIXED][2]) < 1e-6  # same local maximum region


def test_mag_unsupported_paths_raise():
    dims = (4, 4, 4, 4)
    U = cpu_field(dims)
    c = ctx_for(dims, gf.GF_MAG)
    with pytest.raises(gf.GFError):
        gf.gf_anneal(c, dev(U), 1.0, 0.1, 2, 1)
    with pytest.raises(gf.GFError):
        gf.gf_set_option(c, "fp64_arith", 1)
    with pytest.raises(gf.GFError):
        gf.gf_set_option(c, "stochastic_p", 0.5)
    gf.gf_upload(c, dev(U), gf.GF_FP64)
    with pytest.raises(gf.GFError):
        gf.gf_measure_timeslices(c)
    gf.gf_or_half_sweep(c, 0, 1.5)  # still usable afterwards


# ---------------------------------------------------------------------------
# Wilson-action generation: the same Cabibbo-Marinari updates on both sides
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
@pytest.mark.parametrize("storage", [18, 12])
def test_wilson_update_parity(dims, storage):
    U = cpu_field(dims, seed=81, gseed=82, plaq=0.59)
    c = ctx_for(dims, 0, storage64=storage)
    gf.gf_upload(c, dev(U), gf.GF_FP64)
    W = U.copy()
    for mu in range(4):
        for p in (0, 1):
            for mode in (0, 1):
                gf.gf_wilson_update(c, mu, p, 6.1, mode, 11, 3)
                assert oracle.wilson_update(W, mu, p, 6.1, mode, 11, 3) == 0
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    assert max_rel(host(d), W) < 1e-11


def test_generate_matches_oracle_and_thermalises():
    dims = (6, 4, 6, 10)
    U = cpu_field(dims, seed=83, gseed=84, plaq=0.5)
    c = ctx_for(dims, 0)
    d = dev(U)
    gf.gf_generate(c, d, 6.0, 2, 2, 13, 0)
    W = U.copy()
    for k in range(2):
        oracle.wilson_sweep(W, 6.0, 0, 13, k)
        for _ in range(2):
            oracle.wilson_sweep(W, 6.0, 1, 13, 0)
    assert max_rel(host(d), W) < 1e-10
    # thermalised plaquette at beta = 6.0 (0.5937 in the literature; 8^4)
    d8 = dev(cpu_field((8, 8, 8, 8), seed=85, gseed=86, plaq=0.5))
    c8 = ctx_for((8, 8, 8, 8), 0)
    gf.gf_generate(c8, d8, 6.0, 30, 2, 17, 0)
    vals = []
    for k in range(20):
        gf.gf_generate(c8, d8, 6.0, 1, 2, 17, 30 + k)
        vals.append(gf.gf_plaquette(c8, d8))
    assert np.mean(vals) == pytest.approx(0.5937, abs=6e-3)
    M = host(d8).reshape(-1, 3, 3)
    assert np.abs(M @ np.conj(np.swapaxes(M, -1, -2)) - np.eye(3)).max() < 1e-12


# ---------------------------------------------------------------------------
# degenerate subgroups: k = 0 and k along -1 (a constant diagonal field)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("form", ["acc", "tps1", "tps8", "df64", "fp32"])
def test_degenerate_subgroups_match_oracle(oracle_or_variant, variant, form):
    """All links diag(i, i, -1): subgroup (0,1) has k = 0 (no change) and
    subgroup (1,2) has k = (-8, 0, 0, 0) (rotation by pi, or no change for the
    exact power); the oracle pins give the result, diag(i, -i, 1) everywhere
    after one half-sweep for the rational and first-order readings."""
    dims = (4, 4, 4, 6)
    Lx, Ly, Lz, Lt = dims
    D = np.diag([1j, 1j, -1.0])
    U = np.broadcast_to(D, (Lt, Lz, Ly, Lx, 4, 3, 3)).copy()
    opts = {"or_variant": variant}
    prec = gf.GF_FP64
    if form == "acc":
        opts["variant"] = 2
    elif form.startswith("tps"):
        opts.update(variant=1, threads_per_site=int(form[3:]))
    elif form == "df64":
        opts["fp64_arith"] = 1
    else:
        prec = gf.GF_FP32
    c = ctx_for(dims, 0, **opts)
    gf.gf_upload(c, dev(U), prec)
    oracle_or_variant(variant)
    W = U.copy()
    for p in (0, 1, 0, 1):
        gf.gf_or_half_sweep(c, p, 1.7)
        oracle.or_half_sweep(W, p, 1.7, 0)
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    # FP32: the reciprocal square root of the rotation by pi rounds (6e-8 per step, a
    # few dozen steps): the multi-sweep FP32 bound of this file
    tol = 2e-5 if prec == gf.GF_FP32 else 1e-12
    expect = np.broadcast_to(D if variant == 2 else np.diag([1j, -1j, 1.0]), U.shape)
    assert np.abs(W - expect).max() < 1e-15
    assert np.abs(host(d) - W).max() < tol
    gf.gf_destroy(c)


# ---------------------------------------------------------------------------
# the smallest extents: with L = 2, x + mu and x - mu are the same site
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6)])
@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("form", ["acc", "tps2", "tps8", "df64", "fp32"])
def test_extent_two_half_sweeps_match_oracle(dims, gauge, form):
    U = cpu_field(dims, seed=5, gseed=6)
    opts = {}
    prec = gf.GF_FP64
    if form == "acc":
        opts["variant"] = 2
    elif form.startswith("tps"):
        opts.update(variant=1, threads_per_site=int(form[3:]))
    elif form == "df64":
        opts["fp64_arith"] = 1
    else:
        prec = gf.GF_FP32
    c = ctx_for(dims, gauge, **opts)
    gf.gf_upload(c, dev(U), prec)
    W = U.copy()
    for p in (0, 1):
        gf.gf_or_half_sweep(c, p, 1.7)
        oracle.or_half_sweep(W, p, 1.7, gauge)
    d = torch.empty_like(dev(U))
    gf.gf_download(c, d)
    if prec == gf.GF_FP32:
        assert np.abs(host(d) - W).max() < 5e-6 * 2
    else:
        assert max_rel(host(d), W) < 1e-12
    F, th = gf.gf_measure(c)
    # FP32 storage is measured from its FP32 values (row 2 rebuilt in FP32)
    assert F == pytest.approx(oracle.functional(host(d), gauge), abs=1e-6 if prec == gf.GF_FP32 else 1e-13)
    gf.gf_destroy(c)
