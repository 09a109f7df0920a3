"""gf_measure_noalloc: F and theta without any device allocation.

Some callers cannot allocate device memory at the moment they need a
measurement: code running while another thread captures a CUDA graph (an
allocation there would break or serialise the capture), code inside a
framework whose own pool owns all device memory, and services that forbid
allocation after start-up.  The allocation-free entry point keeps its
reduction scratch in a fixed device array instead.  This file checks, on two
calls in a row (different lattices and gauges, so stale scratch contents from
the first call would show up in the second), that it gives the oracle's F and
theta (Sec. 2, eqs. F_g and theta) and the same values as the context-based
gf_functional / gf_theta, that repeated calls leave the device's free memory
unchanged, and that it refuses what it cannot hold: volumes
beyond its fixed scratch, host memory (pageable or pinned), odd extents, and
tensors of the wrong type or size.

The file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu


def test_noalloc_measure_matches_oracle_and_context_entry_points():
    cases = [((8, 8, 8, 8), gf.GF_LANDAU, (1, 2)), ((6, 4, 6, 10), gf.GF_COULOMB, (3, 4))]
    for dims, gauge, seeds in cases:
        U = synth.make_field(dims, 0.60, *seeds)
        Un = synth.as_numpy(U)
        Ud = U.to("cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = gf.gf_measure_noalloc(dims, gauge, Ud, out)
        assert rc == gf.GF_OK
        torch.cuda.synchronize()
        F_na, th_na = out[0].item(), out[1].item()
        # against the oracle (same definitions, FP64, different summation order)
        assert F_na == pytest.approx(oracle.functional(Un, gauge), rel=1e-13, abs=1e-15)
        assert th_na == pytest.approx(oracle.theta(Un, gauge), rel=1e-12)
        # and against the context entry points
        ctx = gf.gf_create(dims, gauge)
        F = gf.gf_functional(ctx, Ud)
        th = gf.gf_theta(ctx, Ud)
        gf.gf_destroy(ctx)
        assert F_na == pytest.approx(F, rel=1e-13, abs=1e-15)
        assert th_na == pytest.approx(th, rel=1e-12)


def test_noalloc_measure_leaves_free_device_memory_unchanged():
    """The first call on a device looks up the scratch array's address and
    loads the kernels; after it, calls move no device memory at all: the
    free memory the driver reports is the same before and after three calls
    (an allocation would take at least its 2 MiB granule)."""
    dims = (8, 8, 8, 8)
    Ud = synth.make_field(dims, 0.60, 1, 2).to("cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert gf.gf_measure_noalloc(dims, gf.GF_LANDAU, Ud, out) == gf.GF_OK
    torch.cuda.synchronize()
    first = out.cpu().numpy().copy()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert gf.gf_measure_noalloc(dims, gf.GF_LANDAU, Ud, out) == gf.GF_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    np.testing.assert_array_equal(out.cpu().numpy(), first)


def test_noalloc_measure_rejects_what_it_cannot_hold():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    U = synth.make_field((4, 4, 4, 4), 0.60, 1, 2).to("cuda")
    # a volume beyond the fixed scratch (2^21 sites): 48^4 = 5,308,416 (checked before any pointer is read)
    assert gf.gf_measure_noalloc((48, 48, 48, 48), gf.GF_LANDAU, U.data_ptr(), out) == gf.GF_EINVAL
    # host fields, pageable or pinned, cannot be read without a staging allocation
    assert gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U.cpu(), out) == gf.GF_EINVAL
    assert gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U.cpu().pin_memory(), out) == gf.GF_EINVAL
    assert gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U, torch.zeros(2, dtype=torch.float64).pin_memory()) \
        == gf.GF_EINVAL
    # an odd extent reaches the library as raw addresses (the binding checks sizes of tensors only)
    assert gf.gf_measure_noalloc((4, 4, 4, 5), gf.GF_LANDAU, U.data_ptr(), out.data_ptr()) == gf.GF_EINVAL
    # the binding refuses tensors the library would read or write out of bounds
    with pytest.raises(ValueError):
        gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U, torch.zeros(2, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U, torch.zeros(1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U.float(), out)
    with pytest.raises(ValueError):
        gf.gf_measure_noalloc((4, 4, 4, 6), gf.GF_LANDAU, U, out)


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second device to hold the foreign field")
def test_noalloc_measure_rejects_memory_of_another_device():
    U = synth.make_field((4, 4, 4, 4), 0.60, 1, 2).to("cuda:1")
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        assert gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U, out) == gf.GF_EINVAL
    assert np.isfinite(out.cpu().numpy()).all()
