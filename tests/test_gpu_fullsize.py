"""Full-size parity on sampled sites.

The lattices of the benchmark (32^4 Landau) and of the Coulomb configuration
(48^3 x 96, 6.1 GB of FP64 links) are too large for the oracle to sweep whole;
the oracle instead recomputes the update of randomly sampled sites one by one
from the same input field (sites of one parity are independent, Sec. 2), and
the 8 links of each sampled site after the GPU half-sweep must match.  The GPU
runs in the launch configuration the benchmark uses (autotuned).
Tolerances as in test_gpu_parity.py: 1e-12 relative for FP64 and double-float, 5e-6 absolute
per element for FP32-12 storage; SA 1e-11.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import gf, synth

pytestmark = pytest.mark.gpu


def sampled_links(U_after, dims, sites):
    """The 8 links of each listed site from a canonical field (numpy)."""
    flat = U_after.reshape(-1, 4, 3, 3)
    out = np.empty((len(sites), 8, 3, 3), dtype=np.complex128)
    for j, i in enumerate(sites):
        for mu in range(4):
            out[j, mu] = flat[i, mu]
            out[j, 4 + mu] = flat[oracle.backward_site(dims, i, mu), mu]
    return out


def sites_of_parity(dims, parity, n, seed):
    rng = np.random.default_rng(seed)
    V = int(np.prod(dims))
    out = []
    while len(out) < n:
        i = int(rng.integers(V))
        if oracle.site_parity(dims, i) == parity:
            out.append(i)
    return out


@pytest.mark.parametrize("prec,storage,tol", [(gf.GF_FP64, 18, 1e-12), (gf.GF_FP32, 12, 5e-6),
                                              (gf.GF_FP64, "df64", 1e-12)])
def test_landau_32x32x32x32_half_sweep_sampled(prec, storage, tol):
    dims = (32, 32, 32, 32)
    U = synth.make_field(dims, 0.60, 3, 4, device="cuda")
    host = synth.as_numpy(U)
    c = gf.gf_create(dims, gf.GF_LANDAU)
    if storage == "df64":  # double-float storage, the mixed policy's alternative finish
        gf.gf_set_option(c, "fp64_arith", 1)
    else:
        gf.gf_set_option(c, "storage64" if prec == gf.GF_FP64 else "storage32", storage)
    gf.gf_upload(c, U, prec)
    gf.gf_autotune(c)
    gf.gf_upload(c, U, prec)
    gf.gf_or_half_sweep(c, 0, 1.7)
    gf.gf_download(c, U)
    after = synth.as_numpy(U)
    sites = sites_of_parity(dims, 0, 3000, 1)
    want = oracle.or_update_sites(host, sites, 1.7, 0)
    got = sampled_links(after, dims, sites)
    err = np.abs(got - want).max()
    assert err < tol, err


def test_coulomb_48x48x48x96_or_and_sa_sampled():
    dims = (48, 48, 48, 96)
    U = synth.make_field(dims, 0.58, 11, 12, device="cuda")
    host = synth.as_numpy(U)
    c = gf.gf_create(dims, gf.GF_COULOMB)
    gf.gf_upload(c, U, gf.GF_FP64)
    gf.gf_autotune(c)
    gf.gf_upload(c, U, gf.GF_FP64)
    # overrelaxation half-sweep on the odd sites
    gf.gf_or_half_sweep(c, 1, 1.7)
    gf.gf_download(c, U)
    after = synth.as_numpy(U)
    sites = sites_of_parity(dims, 1, 2000, 2)
    want = oracle.or_update_sites(host, sites, 1.7, 1)
    assert np.abs(sampled_links(after, dims, sites) - want).max() < 1e-12
    # heatbath half-sweep (T = 1.45, the start of the annealing schedule) on the even sites
    gf.gf_sa_half_sweep(c, 0, 1.45, 11, 0)
    gf.gf_download(c, U)
    after2 = synth.as_numpy(U)
    sites = sites_of_parity(dims, 0, 2000, 3)
    want = oracle.sa_update_sites(after, sites, 1.45, 1, 11, 0)
    assert np.abs(sampled_links(after2, dims, sites) - want).max() < 1e-11
    # both steps are gauge transformations: spatial and temporal plaquettes unchanged
    assert gf.gf_plaquette(c, U) == pytest.approx(gf.gf_plaquette(c, torch.from_numpy(host).cuda()), abs=1e-12)


def test_landau_32x32x32x32_fp32_restarts_equal_fp64_solve():
    """The mixed policy with FP32 restarts on the benchmark field: the same F as
    the all-FP64 solve (to 1e-13), theta < 1e-14, plaquette of the input kept
    (an exact FP64 gauge transform)."""
    dims = (32, 32, 32, 32)
    U0 = synth.make_field(dims, 0.60, 3, 4, device="cuda")
    res = {}
    for name, opts in (("fp64", {"precision": gf.GF_FP64}),
                       ("restarts", {"precision": gf.GF_MIXED, "fp32_restarts": 2, "theta_switch": 1e-30})):
        c = gf.gf_create(dims, gf.GF_LANDAU)
        gf.gf_set_option(c, "check_every", 25)
        for k, v in opts.items():
            gf.gf_set_option(c, k, v)
        U = U0.clone()
        conv, it, F, th = gf.gf_overrelax(c, U, 1.7, 1e-14, 20000)
        assert conv and th < 1e-14, name
        res[name] = (F, gf.gf_plaquette(c, U), gf.gf_theta(c, U), gf.gf_get_stat(c, "sweeps_fp64"))
        if name == "restarts":
            assert gf.gf_get_stat(c, "fp32_restarts_done") >= 1
        P0 = gf.gf_plaquette(c, U0)
    assert abs(res["restarts"][0] - res["fp64"][0]) <= 1e-13
    assert res["restarts"][1] == pytest.approx(P0, abs=1e-13)
    assert res["restarts"][2] < 1e-14
    assert res["restarts"][3] < res["fp64"][3]
