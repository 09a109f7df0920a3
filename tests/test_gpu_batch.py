"""Batched persistent launch: many lattices of uneven volume in one kernel.

Parity: every lattice of a batch against the oracle (FP64: identical sweep
counts, fields within 1e-10 after hundreds of sweeps -- the per-sweep bound
is 1e-12 relative, FP64 rounding differences grow slowly over the solve), and
against the single-lattice library path.  Failure path: a grid barrier that
cannot complete (test hook: one block more than exist) must end with
GF_ETIMEOUT after its bounded wait, and the batch must work again afterwards.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 6, 10), (8, 8, 8, 8), (4, 6, 4, 8)]


def fields(dims_list, seed0=100):
    out = []
    for k, d in enumerate(dims_list):
        plaq = synth.batched_plaquettes(len(dims_list))[k]
        out.append(synth.as_numpy(synth.make_field(d, plaq, seed0 + k, seed0 + 50 + k)))
    return out


@pytest.mark.parametrize("gauge", [gf.GF_LANDAU, gf.GF_COULOMB])
@pytest.mark.parametrize("tps", [0, -1])
def test_batch_fp64_matches_oracle(gauge, tps):
    host = fields(DIMS)
    dev = [torch.from_numpy(u).cuda() for u in host]
    b = gf.gf_batch_create(DIMS, gauge)
    gf.gf_batch_set_option(b, "threads_per_site", tps)  # -1: accumulate form
    gf.gf_batch_set_option(b, "precision", gf.GF_FP64)
    gf.gf_batch_set_option(b, "check_every", 10)
    rc, iters, F, th = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 3000)
    assert rc == gf.GF_OK
    for k, u in enumerate(host):
        conv, oit, oF, oth = oracle.overrelax(u, gauge, 1.7, 1e-12, 3000, 10)
        assert conv
        assert iters[k] == oit
        assert F[k] == pytest.approx(oF, rel=1e-12)
        assert th[k] == pytest.approx(oth, rel=1e-6)
        d = dev[k].cpu().numpy()
        assert np.abs(d - u).max() < 1e-10


def test_batch_mixed_matches_single_lattice_path():
    host = fields(DIMS, seed0=200)
    dev = [torch.from_numpy(u).cuda() for u in host]
    b = gf.gf_batch_create(DIMS, gf.GF_LANDAU)
    gf.gf_batch_set_option(b, "precision", gf.GF_MIXED)
    gf.gf_batch_set_option(b, "check_every", 10)
    rc, iters, F, th = gf.gf_batch_overrelax(b, dev, 1.7, 1e-14, 20000)
    assert rc == gf.GF_OK
    for k, u in enumerate(host):
        c = gf.gf_create(DIMS[k], gf.GF_LANDAU)
        gf.gf_set_option(c, "check_every", 10)
        d = torch.from_numpy(u).cuda()
        conv, it64, F64, th64 = gf.gf_overrelax(c, d, 1.7, 1e-14, 20000)
        assert conv and th[k] < 1e-14
        assert abs(F[k] - F64) < 1e-10
        # the batch result is an exact gauge transform of its input
        assert gf.gf_plaquette(c, dev[k]) == pytest.approx(oracle.plaquette(u), abs=1e-13)
        assert abs(iters[k] - it64) <= max(200, 0.2 * it64)


def test_batch_graph_replay_is_reproducible():
    host = fields(DIMS[:3], seed0=300)
    b = gf.gf_batch_create(DIMS[:3], gf.GF_LANDAU)
    gf.gf_batch_set_option(b, "check_every", 10)
    dev = [torch.from_numpy(u).cuda() for u in host]
    r1 = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 5000)
    out1 = [d.clone() for d in dev]
    for d, u in zip(dev, host):
        d.copy_(torch.from_numpy(u))
    r2 = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 5000)  # replays the captured graph
    assert r1 == r2
    for a, c in zip(out1, dev):
        assert torch.equal(a, c)


def test_batch_barrier_timeout_is_reported_and_recoverable():
    host = fields(DIMS[:2], seed0=400)
    dev = [torch.from_numpy(u).cuda() for u in host]
    b = gf.gf_batch_create(DIMS[:2], gf.GF_LANDAU)
    gf.gf_batch_set_option(b, "precision", gf.GF_FP64)
    gf.gf_batch_set_option(b, "barrier_timeout_ms", 200)
    gf.gf_batch_set_option(b, "barrier_extra_blocks", 1)
    rc, *_ = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 100, raise_on_error=False)
    assert rc == gf.GF_ETIMEOUT
    gf.gf_batch_set_option(b, "barrier_extra_blocks", 0)
    for d, u in zip(dev, host):
        d.copy_(torch.from_numpy(u))
    rc, iters, F, th = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 5000)
    assert rc == gf.GF_OK and max(th) < 1e-12


def test_batch_autotune_keeps_results():
    host = fields(DIMS[:3], seed0=500)
    dev = [torch.from_numpy(u).cuda() for u in host]
    b = gf.gf_batch_create(DIMS[:3], gf.GF_LANDAU)
    tps, block = gf.gf_batch_autotune(b, dev)
    assert tps in (0, 1, 2, 4, 8) and block in (64, 128, 256)  # 0: accumulate form
    for d, u in zip(dev, host):
        assert torch.equal(d.cpu(), torch.from_numpy(u))  # autotuning leaves fields alone
    gf.gf_batch_set_option(b, "precision", gf.GF_FP64)
    gf.gf_batch_set_option(b, "check_every", 10)
    rc, iters, F, th = gf.gf_batch_overrelax(b, dev, 1.7, 1e-12, 3000)
    assert rc == gf.GF_OK
    for k, u in enumerate(host):
        conv, oit, oF, oth = oracle.overrelax(u, 0, 1.7, 1e-12, 3000, 10)
        assert iters[k] == oit and F[k] == pytest.approx(oF, rel=1e-12)


def test_batch_rejects_host_fields():
    host = fields(DIMS[:1])
    b = gf.gf_batch_create(DIMS[:1], gf.GF_LANDAU)
    rc, *_ = gf.gf_batch_overrelax(b, host, 1.7, 1e-12, 10, raise_on_error=False)
    assert rc == gf.GF_EINVAL


def test_one_call_batched_entry_point():
    """gf_overrelax_batched (the one-call form): the same per-lattice results,
    bit for bit, as a batch object with the default options; every returned
    field checked by the oracle: theta below the target, plaquette kept, and
    F equal to the oracle's own FP64 solve from the same input (the same
    maximum; Alg. 1 with the checks of Sec. 4.1)."""
    host = fields(DIMS, seed0=300)
    one = [torch.from_numpy(u).cuda() for u in host]
    rc, iters, F, th = gf.gf_overrelax_batched(DIMS, one, 1.7, 1e-13, 20000)
    assert rc == gf.GF_OK
    obj = [torch.from_numpy(u).cuda() for u in host]
    b = gf.gf_batch_create(DIMS, gf.GF_LANDAU)
    gf.gf_batch_set_option(b, "use_graphs", 0)
    rc2, iters2, F2, th2 = gf.gf_batch_overrelax(b, obj, 1.7, 1e-13, 20000)
    assert rc2 == gf.GF_OK and iters2 == iters and F2 == F and th2 == th
    for k, u in enumerate(host):
        W = one[k].cpu().numpy()
        assert np.array_equal(W, obj[k].cpu().numpy())
        assert oracle.theta(W, 0) < 1e-13
        assert oracle.plaquette(W) == pytest.approx(oracle.plaquette(u), abs=1e-13)
        conv, oit, oF, oth = oracle.overrelax(u.copy(), 0, 1.7, 1e-13, 20000, 25)
        assert conv and F[k] == pytest.approx(oF, abs=1e-12)
    # argument errors come back as codes
    with pytest.raises(gf.GFError):
        gf.gf_overrelax_batched([(4, 4, 4, 5)], one[:1], 1.7, 1e-13, 10)


@pytest.mark.parametrize("precision", [gf.GF_MIXED, gf.GF_FP64])
def test_batch_double_float_phase_is_exact(precision):
    """Batch option fp64_arith 1: the FP64 phase as double-float sweeps with
    E = g - 1 tracked per lattice and applied in FP64.  Every lattice reaches
    theta < 1e-14 (the oracle on the returned field), keeps its plaquette
    (an exact FP64 gauge transform) and ends at the native batch's F."""
    host = fields(DIMS, seed0=400)
    res = {}
    for arith in (0, 1):
        dev = [torch.from_numpy(u).cuda() for u in host]
        b = gf.gf_batch_create(DIMS, gf.GF_LANDAU)
        gf.gf_batch_set_option(b, "precision", precision)
        gf.gf_batch_set_option(b, "check_every", 10)
        gf.gf_batch_set_option(b, "fp64_arith", arith)
        rc, iters, F, th = gf.gf_batch_overrelax(b, dev, 1.7, 1e-14, 20000)
        assert rc == gf.GF_OK
        res[arith] = (iters, F, [d.cpu().numpy() for d in dev])
        if arith:
            assert gf.gf_batch_get_stat(b, "grid_df64") > 0
    for k, u in enumerate(host):
        W = res[1][2][k]
        assert oracle.theta(W, 0) < 1e-14
        assert oracle.plaquette(W) == pytest.approx(oracle.plaquette(u), abs=1e-13)
        assert res[1][1][k] == pytest.approx(res[0][1][k], abs=1e-13)
        assert abs(res[1][0][k] - res[0][0][k]) <= 20 + res[0][0][k] // 20
