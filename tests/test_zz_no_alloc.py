"""gf_measure_noalloc: F and theta without any device allocation.

Some callers cannot allocate device memory at the moment they need a
measurement: code running while another thread captures a CUDA graph (an
allocation there would break or serialise the capture), code inside a
framework whose own pool owns all device memory, and services that forbid
allocation after start-up.  The allocation-free entry point keeps its
reduction scratch in a fixed device array instead; this file checks that it
gives the same F and theta as the context-based gf_functional / gf_theta, on
two calls in a row (different lattices and gauges, so stale scratch contents
from the first call would show up in the second), and that it refuses
volumes beyond its fixed scratch size and host pointers.

The file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import pytest
import torch

from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu


def test_noalloc_measure_matches_context_entry_points():
    cases = [((8, 8, 8, 8), gf.GF_LANDAU, (1, 2)), ((6, 4, 6, 10), gf.GF_COULOMB, (3, 4))]
    for dims, gauge, seeds in cases:
        U = synth.make_field(dims, 0.60, *seeds).to("cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = gf.gf_measure_noalloc(dims, gauge, U, out)
        assert rc == gf.GF_OK
        torch.cuda.synchronize()
        ctx = gf.gf_create(dims, gauge)
        F = gf.gf_functional(ctx, U)
        th = gf.gf_theta(ctx, U)
        gf.gf_destroy(ctx)
        assert out[0].item() == pytest.approx(F, rel=1e-13, abs=1e-15)
        assert out[1].item() == pytest.approx(th, rel=1e-12)


def test_noalloc_measure_rejects_what_it_cannot_hold():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    U = synth.make_field((4, 4, 4, 4), 0.60, 1, 2).to("cuda")
    # a volume beyond the fixed scratch (2^21 sites): 48^4 = 5,308,416
    assert gf.gf_measure_noalloc((48, 48, 48, 48), gf.GF_LANDAU, U, out) == gf.GF_EINVAL
    # a host field cannot be read without a staging allocation
    assert gf.gf_measure_noalloc((4, 4, 4, 4), gf.GF_LANDAU, U.cpu(), out) == gf.GF_EINVAL
    assert gf.gf_measure_noalloc((4, 4, 4, 5), gf.GF_LANDAU, U, out) == gf.GF_EINVAL
