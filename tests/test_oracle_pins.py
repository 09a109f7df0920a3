"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (Alg. 1 flop counts), published known answers (Philox), closed
forms and textbook routines (SU(2) local solution, eq. localsolution),
invariants (gauge invariance of the plaquette, unitarity), brute force
(no SU(2) rotation beats the closed-form subgroup maximum), monotonicity of
plain relaxation, and the distribution a heatbath must sample.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1209_4008_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SUBGROUPS = [(0, 1), (1, 2), (0, 2)]


def field(dims, seed=1, gseed=2, plaq=0.60, pure=False):
    return synth.as_numpy(synth.make_field(dims, plaq, seed, gseed, pure_gauge=pure))


def su2_from_quaternion(r):
    """Independent construction: R = r0 1 + i (r1 s1 + r2 s2 + r3 s3)."""
    s1 = np.array([[0, 1], [1, 0]], complex)
    s2 = np.array([[0, -1j], [1j, 0]], complex)
    s3 = np.array([[1, 0], [0, -1]], complex)
    return r[0] * np.eye(2) + 1j * (r[1] * s1 + r[2] * s2 + r[3] * s3)


def embed(R2, a, b):
    G = np.eye(3, dtype=complex)
    G[np.ix_([a, b], [a, b])] = R2
    return G


def site_star(U, dims, i):
    """The 8 links of site i: U_mu(x), U_mu(x - mu) (numpy views of copies)."""
    Lx, Ly, Lz, Lt = dims
    flat = U.reshape(-1, 4, 3, 3)
    fwd = [flat[i, mu].copy() for mu in range(4)]
    bwd = [flat[oracle.backward_site(dims, i, mu), mu].copy() for mu in range(4)]
    return fwd, bwd


def local_objective(G, fwd, bwd, nk=4):
    """sum_mu Re tr[G U_mu(x)] + Re tr[U_mu(x-mu) G^dagger] -- the part of F that
    depends on g(x) (eq. F_g[U] with the update of eq. 1 at one site)."""
    return sum(np.trace(G @ fwd[m]).real + np.trace(bwd[m] @ G.conj().T).real for m in range(nk))


def haarsu2_from_quaternion(n, rng):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# values the paper prints
# --------------------------------------------------------------------------
def test_flop_counts_match_alg1():
    gold = json.load(open(os.path.join(GOLDEN, "paper_flop_counts.json")))
    ps = gold["per_subgroup"]
    per_sub = ps["assemble_K"] + ps["omega_and_project"] + 4 * (
        ps["update_forward_link"] + ps["update_backward_link"])
    assert per_sub == gold["per_site_per_subgroup"]
    assert 3 * per_sub == gold["per_site_su3"]
    dims = (4, 4, 4, 4)
    U = field(dims)
    V = 4 ** 4
    flops = oracle.count_flops_half_sweep(U, 0, 1.7, 0)
    assert flops == gold["per_site_su3"] * (V // 2)


# --------------------------------------------------------------------------
# Philox4x32-10 known answers (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# --------------------------------------------------------------------------
# SU(2) subgroup algebra
# --------------------------------------------------------------------------
def test_quaternion_projection_is_re_trace():
    rng = np.random.default_rng(5)
    for _ in range(200):
        w = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        r = haarsu2_from_quaternion(1, rng)[0]
        k = oracle.block_quaternion(w)
        assert np.trace(su2_from_quaternion(r) @ w).real == pytest.approx(r @ k, abs=1e-13)


def test_overrelax_quaternion_properties():
    rng = np.random.default_rng(6)
    for _ in range(200):
        k = rng.standard_normal(4) * rng.uniform(0.1, 10)
        r1 = oracle.overrelax_quaternion(k, 1.0)
        np.testing.assert_allclose(r1, k / np.linalg.norm(k), atol=1e-15)  # relaxation
        r = oracle.overrelax_quaternion(k, 1.7)
        assert abs(np.linalg.norm(r) - 1) < 1e-15
        # same axis, larger rotation angle in the direction of k (tan phi' = b tan phi)
        kh = k / np.linalg.norm(k)
        phi = math.atan2(np.linalg.norm(kh[1:]), kh[0])
        phip = math.atan2(np.linalg.norm(r[1:]), r[0])
        b = (1.7 * kh[0] ** 2 + (1 - kh[0] ** 2))
        assert math.tan(phip) == pytest.approx(b * math.tan(phi), rel=1e-10, abs=1e-12)
        np.testing.assert_allclose(np.cross(r[1:], k[1:]), 0, atol=1e-12)
    # small angles: g^omega to first order, angle multiplied by omega
    k = np.array([1.0, 1e-4, -2e-4, 3e-4])
    r = oracle.overrelax_quaternion(k, 1.7)
    ang = lambda q: 2 * math.atan2(np.linalg.norm(q[1:]), q[0])
    assert ang(r) == pytest.approx(1.7 * ang(k / np.linalg.norm(k)), rel=1e-6)
    assert oracle.overrelax_quaternion(np.zeros(4), 1.7) is None


def test_brute_force_no_su2_beats_subgroup_maximum():
    """North-star test (c): random SU(2) rotations never raise Re tr[g K]
    past the closed-form maximum |k| of the subgroup."""
    dims = (4, 4, 4, 4)
    U = field(dims, seed=11, gseed=12)
    rng = np.random.default_rng(7)
    for i in (0, 37, 101):
        fwd, bwd = site_star(U, dims, i)
        for sg, (a, b) in enumerate(SUBGROUPS):
            k = oracle.site_quaternion(U, i, 0, sg)
            rbest = oracle.overrelax_quaternion(k, 1.0)
            base = local_objective(np.eye(3), fwd, bwd)
            best = local_objective(embed(su2_from_quaternion(rbest), a, b), fwd, bwd)
            # the identity's block contributes k0, the maximum |k|
            assert best - base == pytest.approx(np.linalg.norm(k) - k[0], abs=1e-12)
            qs = haarsu2_from_quaternion(100_000, rng)
            # objective is affine in r: base + (r - 1).k ; evaluate a sample exactly too
            vals = base + qs @ k - k[0]
            assert vals.max() <= best + 1e-12
            assert vals.max() > best - 0.1 * np.linalg.norm(k)
            for q in qs[:50]:
                v = local_objective(embed(su2_from_quaternion(q), a, b), fwd, bwd)
                assert v == pytest.approx(base + q @ k - k[0], abs=1e-12)
                assert v <= best + 1e-12


def test_stationary_after_relaxation_step():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=13, gseed=14)
    for i in (3, 64, 200):
        for sg in range(3):
            k = oracle.site_quaternion(U, i, 0, sg)
            r = oracle.overrelax_quaternion(k, 1.0)
            oracle.site_rotate(U, i, sg, r)
            k2 = oracle.site_quaternion(U, i, 0, sg)
            assert np.linalg.norm(k2[1:]) <= 1e-13 * np.linalg.norm(k)
            assert k2[0] == pytest.approx(np.linalg.norm(k), rel=1e-14)


def test_su2_reduction_matches_textbook_local_solution():
    """Links block-diag(SU(2), 1): the SU(3) update at omega = 1 is SU(2)
    relaxation g = K^+ / sqrt(det K^+) (eq. localsolution)."""
    dims = (4, 4, 4, 4)
    rng = np.random.default_rng(8)
    V = 4 ** 4
    q = haarsu2_from_quaternion(V * 4, rng)
    U = np.zeros((4, 4, 4, 4, 4, 3, 3), complex)
    flat = U.reshape(-1, 3, 3)
    for n in range(V * 4):
        flat[n] = embed(su2_from_quaternion(q[n]), 0, 1)
    ref = U.copy()
    oracle.or_half_sweep(U, 0, 1.0, 0)
    rflat = ref.reshape(-1, 4, 3, 3)
    for i in range(V):
        if oracle.site_parity(dims, i) != 0:
            continue
        K = np.zeros((2, 2), complex)
        for mu in range(4):
            K += rflat[i, mu, :2, :2]
            K += rflat[oracle.backward_site(dims, i, mu), mu, :2, :2].conj().T
        Kd = K.conj().T
        g2 = Kd / np.sqrt(np.linalg.det(Kd))
        G = embed(g2, 0, 1)
        for mu in range(4):
            rflat[i, mu] = G @ rflat[i, mu]
            j = oracle.backward_site(dims, i, mu)
            rflat[j, mu] = rflat[j, mu] @ G.conj().T
    np.testing.assert_allclose(U, ref, atol=1e-13)


# --------------------------------------------------------------------------
# functional and precision
# --------------------------------------------------------------------------
def test_functional_and_theta_special_cases():
    dims = (4, 4, 4, 6)
    U = np.zeros((6, 4, 4, 4, 4, 3, 3), complex)
    U[...] = np.eye(3)
    assert oracle.functional(U, 0) == pytest.approx(1.0, abs=1e-15)
    assert oracle.theta(U, 0) == 0.0
    assert oracle.plaquette(U) == pytest.approx(1.0, abs=1e-15)
    # a constant field: F = Re tr U0 / 3, divergence zero
    rng = np.random.default_rng(3)
    U0 = synth.as_numpy(synth.haar_su3((1,), 77))[0]
    U[...] = U0
    assert oracle.functional(U, 0) == pytest.approx(np.trace(U0).real / 3, abs=1e-14)
    assert oracle.theta(U, 0) < 1e-28
    # centre element: F = Re(z) for z = exp(2 pi i / 3)
    z = np.exp(2j * np.pi / 3)
    U[...] = z * np.eye(3)
    assert oracle.functional(U, 0) == pytest.approx(z.real, abs=1e-15)
    del rng


def test_theta_two_routes_agree():
    for dims, gauge in (((4, 4, 4, 4), 0), ((4, 6, 4, 8), 0), ((4, 4, 4, 6), 1)):
        U = field(dims, seed=21, gseed=22)
        a, b = oracle.theta(U, gauge), oracle.theta_from_M(U, gauge)
        assert a == pytest.approx(b, rel=1e-13)


def test_theta_single_link_closed_form():
    """One non-trivial link W at site 0 in direction mu, unit field elsewhere:
    Delta = +A(W) at x = 0 and -A(W) at x + mu, so theta = 2 |A(W)|^2 / (3V)."""
    dims = (4, 4, 4, 4)
    U = np.zeros((4, 4, 4, 4, 4, 3, 3), complex)
    U[...] = np.eye(3)
    W = synth.as_numpy(synth.haar_su3((1,), 5))[0]
    U[0, 0, 0, 0, 2] = W
    A = (W - W.conj().T) / 2j
    A -= np.trace(A) / 3 * np.eye(3)
    expect = 2 * np.sum(np.abs(A) ** 2) / (3 * 256)
    assert oracle.theta(U, 0) == pytest.approx(expect, rel=1e-13)
    # Coulomb: a temporal link does not enter theta
    U[...] = np.eye(3)
    U[0, 0, 0, 0, 3] = W
    assert oracle.theta(U, 1) == 0.0
    assert oracle.functional(U, 1) == pytest.approx(1.0, abs=1e-15)


def test_plaquette_target_of_the_generator():
    U = field((8, 8, 8, 8), seed=1, gseed=2, plaq=0.60)
    assert abs(oracle.plaquette(U) - 0.60) < 0.004


def test_generator_is_seeded_and_its_fields_are_su3():
    """Same seeds, same field (bit for bit); another field seed or gauge seed
    gives another field; every link is in SU(3); the gauge rotation leaves the
    plaquette of the unrotated field unchanged."""
    dims = (4, 4, 4, 6)
    a = field(dims, seed=7, gseed=8)
    np.testing.assert_array_equal(a, field(dims, seed=7, gseed=8))
    assert np.abs(a - field(dims, seed=9, gseed=8)).max() > 0.1
    assert np.abs(a - field(dims, seed=7, gseed=9)).max() > 0.1
    assert unitarity_error(a) < 1e-13
    # same field seed, different gauge seeds: gauge-equivalent fields
    assert oracle.plaquette(a) == pytest.approx(oracle.plaquette(field(dims, seed=7, gseed=9)), abs=1e-13)


# --------------------------------------------------------------------------
# invariants of the sweep
# --------------------------------------------------------------------------
def unitarity_error(U):
    M = U.reshape(-1, 3, 3)
    e = np.abs(M @ M.conj().transpose(0, 2, 1) - np.eye(3)).max()
    d = np.abs(np.linalg.det(M) - 1).max()
    return max(e, d)


@pytest.mark.parametrize("gauge", [0, 1])
def test_plaquette_invariant_and_unitarity(gauge):
    """North-star test (b): every sweep is a gauge transformation."""
    dims = (4, 4, 6, 4)
    U = field(dims, seed=31, gseed=32)
    P0 = oracle.plaquette(U)
    for n in range(20):
        oracle.or_sweeps(U, 1.7, gauge, 5)
        assert abs(oracle.plaquette(U) - P0) < 1e-13
    assert unitarity_error(U) < 1e-13


@pytest.mark.parametrize("gauge", [0, 1])
def test_relaxation_is_monotone(gauge):
    """North-star test (d): at omega = 1, F never decreases."""
    dims = (4, 4, 4, 4)
    U = field(dims, seed=41, gseed=42)
    F = oracle.functional(U, gauge)
    for n in range(30):
        oracle.or_half_sweep(U, n % 2, 1.0, gauge)
        F2 = oracle.functional(U, gauge)
        assert F2 >= F - 1e-15
        F = F2


def test_half_sweep_touches_each_link_once_and_only_its_parity():
    """Sites of one parity are independent: the site-by-site update equals the
    half-sweep, and links between two sites of the other parity do not exist."""
    dims = (4, 4, 4, 4)
    U = field(dims, seed=51, gseed=52)
    sites = [i for i in range(256) if oracle.site_parity(dims, i) == 1]
    per_site = oracle.or_update_sites(U, sites, 1.7, 0)
    W = U.copy()
    oracle.or_half_sweep(W, 1, 1.7, 0)
    flat = W.reshape(-1, 4, 3, 3)
    for j, i in enumerate(sites):
        for mu in range(4):
            np.testing.assert_array_equal(per_site[j, mu], flat[i, mu])
            np.testing.assert_array_equal(per_site[j, 4 + mu],
                                          flat[oracle.backward_site(dims, i, mu), mu])


@pytest.mark.parametrize("gauge", [0, 1])
def test_heatbath_site_by_site_equals_the_half_sweep(gauge):
    """The sampled-site heatbath used at full sizes draws the same numbers as
    the half-sweep (the Philox counter depends on the site, not on the order)."""
    dims = (4, 4, 6, 4)
    U = field(dims, seed=53, gseed=54)
    V = int(np.prod(dims))
    sites = [i for i in range(V) if oracle.site_parity(dims, i) == 0][::3]
    per_site = oracle.sa_update_sites(U, sites, 0.7, gauge, 99, 5)
    W = U.copy()
    assert oracle.sa_half_sweep(W, 0, 0.7, gauge, 99, 5) == 0
    flat = W.reshape(-1, 4, 3, 3)
    assert np.abs(W - U).max() > 1e-2
    for j, i in enumerate(sites):
        for mu in range(4):
            np.testing.assert_array_equal(per_site[j, mu], flat[i, mu])
            np.testing.assert_array_equal(per_site[j, 4 + mu],
                                          flat[oracle.backward_site(dims, i, mu), mu])


def constant_field(dims, D):
    Lx, Ly, Lz, Lt = dims
    return np.broadcast_to(np.asarray(D, complex), (Lt, Lz, Ly, Lx, 4, 3, 3)).copy()


@pytest.mark.parametrize("or_variant", [0, 1, 2])
def test_unit_field_is_a_fixed_point(or_variant):
    """Every subgroup quaternion of the unit field is (4, 0, 0, 0) > 0, whose
    relaxation element is the identity: sweeps leave it exactly unchanged."""
    U = constant_field((4, 4, 4, 6), np.eye(3))
    assert oracle.functional(U, 0) == 1.0 and oracle.theta(U, 0) == 0.0
    W = U.copy()
    try:
        oracle.set_or_variant(or_variant)
        oracle.or_sweeps(W, 1.7, 0, 3)
    finally:
        oracle.set_or_variant(0)
    np.testing.assert_array_equal(W, U)


@pytest.mark.parametrize("or_variant", [0, 1, 2])
def test_degenerate_subgroups_of_a_constant_diagonal_field(or_variant):
    """All links D = diag(i, i, -1): M(x) = 4 D + 4 D^dagger = diag(0, 0, -8).
    Subgroup (0,1): the block vanishes, k = 0, no change.  Subgroup (1,2):
    k = (-8, 0, 0, 0), relaxation element -1 (a rotation by pi); the rational
    and first-order readings give R = -1 (rows 1, 2 of forward links and
    columns 1, 2 of backward links change sign), the exact power has no axis
    there and changes nothing.  Every link touches one even site, so after the
    even half-sweep every link is D' = diag(i, -i, 1) (readings 0, 1), whose
    subgroup quaternions are all 0 or positive: a fixed point with theta = 0
    but F = 1/3 -- theta vanishes at stationary points that are not maxima."""
    dims = (4, 4, 4, 6)
    D = np.diag([1j, 1j, -1.0])
    Dp = np.diag([1j, -1j, 1.0])
    U = constant_field(dims, D)
    assert oracle.theta(U, 0) == 0.0 and oracle.functional(U, 0) == pytest.approx(-1 / 3, abs=1e-15)
    W = U.copy()
    try:
        oracle.set_or_variant(or_variant)
        oracle.or_half_sweep(W, 0, 1.7, 0)
        expect = constant_field(dims, D if or_variant == 2 else Dp)
        np.testing.assert_allclose(W, expect, atol=1e-15)
        oracle.or_sweeps(W, 1.7, 0, 2)
        np.testing.assert_allclose(W, expect, atol=1e-15)
    finally:
        oracle.set_or_variant(0)
    assert oracle.theta(W, 0) == 0.0
    assert oracle.functional(W, 0) == pytest.approx(-1 / 3 if or_variant == 2 else 1 / 3, abs=1e-15)


def test_pure_gauge_reaches_unit_functional():
    """North-star test (a): U = g(x) g(x+mu)^dagger fixes to F = 1, theta -> 0."""
    # (extent 2 is the smallest lattice: x + mu and x - mu are the same site)
    for dims, seed in (((4, 4, 4, 4), 2), ((8, 8, 8, 8), 2), ((4, 6, 4, 8), 3), ((2, 2, 2, 2), 2),
                       ((2, 4, 2, 6), 3)):
        U = field(dims, gseed=seed, pure=True)
        conv, it, F, th = oracle.overrelax(U, 0, 1.7, 1e-24, 20000, 10)
        assert conv and th < 1e-24
        assert F == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(np.abs(U.reshape(-1, 3, 3)[:, range(3), range(3)]), 1, atol=1e-10)


def test_coulomb_converges_per_timeslice():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=61, gseed=62)
    conv, it, F, th = oracle.overrelax(U, 1, 1.7, 1e-13, 5000, 10)
    assert conv and th < 1e-13
    assert oracle.theta(U, 0) > 1e-6  # Landau violation remains: different gauge


def test_overrelax_driver_checks_cadence():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=71, gseed=72)
    conv, it, F, th = oracle.overrelax(U.copy(), 0, 1.7, 1e-10, 5000, 7)
    assert conv and it % 7 == 0
    # the same number of sweeps by hand reproduces the result exactly
    W = U.copy()
    oracle.or_sweeps(W, 1.7, 0, it)
    assert oracle.theta(W, 0) == th
    conv2, it2, F2, th2 = oracle.overrelax(U.copy(), 0, 1.7, 1e-10, it - 7, 7)
    assert not conv2 and it2 == it - 7 and th2 >= 1e-10
    # already converged input: zero sweeps
    conv3, it3, _, _ = oracle.overrelax(W, 0, 1.7, 1e-10, 100, 7)
    assert conv3 and it3 == 0


def test_reunitarize_projects_onto_su3():
    M = synth.as_numpy(synth.haar_su3((500,), 9))
    P = M.copy()
    oracle.reunitarize(P)
    np.testing.assert_allclose(P, M, atol=1e-14)  # idempotent on SU(3)
    rng = np.random.default_rng(1)
    N = M + 1e-3 * (rng.standard_normal(M.shape) + 1j * rng.standard_normal(M.shape))
    oracle.reunitarize(N)
    assert unitarity_error(N) < 1e-14
    assert np.abs(N - M).max() < 1e-2


def test_gauge_transform_preserves_plaquette():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=81, gseed=82)
    g = synth.as_numpy(synth.haar_su3((4, 4, 4, 4), 83))
    P = oracle.plaquette(U)
    oracle.gauge_transform(U, g)
    assert oracle.plaquette(U) == pytest.approx(P, abs=1e-14)


# --------------------------------------------------------------------------
# heatbath (simulated annealing)
# --------------------------------------------------------------------------
def s0_cdf(alpha):
    x = np.linspace(-1, 1, 200_001)
    dens = np.sqrt(np.clip(1 - x * x, 0, None)) * np.exp(alpha * (x - 1))
    c = np.concatenate([[0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(x))])
    return x, c / c[-1]


@pytest.fixture
def sa_draw():
    """Select the heatbath draw's reading (0 FP64, 1 FP32) for one test."""
    def set_(v):
        oracle.set_sa_draw(v)
    yield set_
    oracle.set_sa_draw(0)


@pytest.mark.parametrize("alpha", [0.3, 1.9, 2.1, 8.0, 150.0])
@pytest.mark.parametrize("draw", [0, 1])
def test_heatbath_samples_weighted_haar(alpha, draw, sa_draw):
    """r . k/|k| must follow sqrt(1 - s^2) exp(alpha s) (weight exp(Re tr[gK]/T)
    times the SU(2) Haar measure); the perpendicular part must be isotropic.
    Both readings of the draw (FP64, and FP32 with the element renormalised in
    FP64) sample the same density."""
    sa_draw(draw)
    rng = np.random.default_rng(int(alpha * 10))
    k = rng.standard_normal(4)
    kn = np.linalg.norm(k)
    T = kn / alpha
    n = 6000
    s = np.empty(n)
    perp = np.empty((n, 3))
    kh = k / kn
    for j in range(n):
        st, r = oracle.heatbath_quaternion(k, T, j, 17, j % 3, 64, 1234)
        assert st == 1
        assert abs(np.linalg.norm(r) - 1) < 1e-14
        s[j] = r @ kh
        # s = r kbar-hat (quaternion product) carries the isotropic direction
        q0 = r[0] * kh[0] + r[1:] @ kh[1:]
        qv = -r[0] * kh[1:] + kh[0] * r[1:] - np.cross(r[1:], -kh[1:])
        assert q0 == pytest.approx(s[j], abs=1e-13)
        perp[j] = qv / max(np.linalg.norm(qv), 1e-300)
    x, cdf = s0_cdf(alpha)
    emp = np.sort(s)
    model = np.interp(emp, x, cdf)
    ks = np.abs(model - (np.arange(1, n + 1) / n)).max()
    assert ks < 1.63 / math.sqrt(n)  # 1% KS critical value
    assert np.abs(perp.mean(axis=0)).max() < 0.06
    np.testing.assert_allclose(np.diag(perp.T @ perp / n), 1 / 3, atol=0.04)


@pytest.mark.parametrize("draw", [0, 1])
def test_heatbath_zero_temperature_is_relaxation(draw, sa_draw):
    sa_draw(draw)
    rng = np.random.default_rng(3)
    for j in range(20):
        k = rng.standard_normal(4)
        st, r = oracle.heatbath_quaternion(k, 1e-9 * np.linalg.norm(k), j, 0, 0, 64, 9)
        np.testing.assert_allclose(r, k / np.linalg.norm(k), atol=1e-3)


def test_heatbath_fp32_reading_follows_the_fp64_draw(sa_draw):
    """The FP32 reading takes the same steps as the FP64 definition from the
    same Philox words (23 of their 32 bits): draw by draw, the two elements
    agree to FP32 rounding unless an accept/reject decision falls within that
    rounding of its threshold, which is rare.  A dropped term, a wrong sign or
    a swapped uniform in either reading moves most draws far apart."""
    rng = np.random.default_rng(5)
    far = 0
    n = 3000
    for j in range(n):
        k = rng.standard_normal(4) * rng.choice([0.05, 0.5, 3.0])
        T = np.linalg.norm(k) / rng.choice([0.2, 1.0, 1.99, 2.01, 5.0, 60.0])
        sa_draw(0)
        st0, r0 = oracle.heatbath_quaternion(k, T, j, 3, j % 3, 64, 77)
        sa_draw(1)
        st1, r1 = oracle.heatbath_quaternion(k, T, j, 3, j % 3, 64, 77)
        assert st0 == 1 and st1 == 1
        assert abs(np.linalg.norm(r1) - 1) < 1e-15
        d = np.abs(r1 - r0).max()
        if d > 2e-4:
            far += 1
    assert far <= n // 500, far


def test_anneal_fp32_draw_is_gauge_transformation(sa_draw):
    sa_draw(1)
    dims = (4, 4, 4, 4)
    for gauge in (0, 1):
        U = field(dims, seed=93, gseed=94)
        P = oracle.plaquette(U)
        assert oracle.anneal(U, gauge, 1.45, 0.01, 30, 77) == 0
        assert oracle.plaquette(U) == pytest.approx(P, abs=1e-13)
        assert unitarity_error(U) < 1e-13


def test_heatbath_rejection_cap_reported():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=91, gseed=92)
    W = U.copy()
    fails = oracle.sa_half_sweep(W, 0, 0.05, 0, 5, 0, cap=1)
    assert fails > 0
    fails = oracle.sa_half_sweep(U, 0, 0.05, 0, 5, 0, cap=64)
    assert fails == 0


def test_anneal_is_gauge_transformation():
    dims = (4, 4, 4, 4)
    for gauge in (0, 1):
        U = field(dims, seed=93, gseed=94)
        P = oracle.plaquette(U)
        assert oracle.anneal(U, gauge, 1.45, 0.01, 30, 77) == 0
        assert oracle.plaquette(U) == pytest.approx(P, abs=1e-13)
        assert unitarity_error(U) < 1e-13


def test_anneal_resumes_from_a_sweep_offset():
    """A schedule split in two calls -- the second starting at the next
    temperature with the Philox sweep counter offset by the sweeps done --
    equals the schedule run at once, bit for bit (counter-based draws)."""
    dims = (4, 4, 4, 4)
    T0, T1, n = 1.2, 0.3, 4
    Tk = [T0 + (T1 - T0) * k / (n - 1) for k in range(n)]
    A = field(dims, seed=69, gseed=70)
    B = A.copy()
    assert oracle.anneal(A, 0, T0, T1, n, 11) == 0
    assert oracle.anneal(B, 0, Tk[0], Tk[1], 2, 11, 0) == 0
    assert oracle.anneal(B, 0, Tk[2], Tk[3], 2, 11, 2) == 0
    np.testing.assert_array_equal(A, B)


def test_anneal_schedule_ends_at_t1():
    """T falls linearly from T0 to T1 inclusive: with T1 -> 0 the last sweep is a
    relaxation, so every site of the parity updated last ends at the maximum of
    its last subgroup (quaternion real and positive); an end temperature above
    T1 would leave a heatbath spread of order sqrt(T / |k|)."""
    dims = (4, 4, 4, 4)
    U = field(dims, seed=61, gseed=62)
    assert oracle.anneal(U, 0, 1.0, 1e-12, 2, 5) == 0
    worst = 0.0
    for i in range(int(np.prod(dims))):
        if oracle.site_parity(dims, i) != 1:
            continue
        k = oracle.site_quaternion(U, i, 0, 2)
        assert k[0] > 0
        worst = max(worst, np.linalg.norm(k[1:]) / np.linalg.norm(k))
    assert worst < 1e-4


def test_haar_generator_moments():
    M = synth.haar_su3((40_000,), 3)
    tr = torch.diagonal(M, dim1=-2, dim2=-1).sum(-1)
    assert abs(tr.mean().item()) < 0.02
    assert (tr.abs() ** 2).mean().item() == pytest.approx(1.0, abs=0.03)


def test_plaquette_single_link_closed_form():
    """Unit field with one link W: the 6 plaquettes through it give Re tr W,
    the other 6V - 6 give 3, so P = (18 V - 18 + 6 Re tr W) / (18 V)."""
    dims = (4, 4, 6, 4)
    V = 4 * 4 * 6 * 4
    U = np.zeros((4, 6, 4, 4, 4, 3, 3), complex)
    U[...] = np.eye(3)
    W = synth.as_numpy(synth.haar_su3((1,), 6))[0]
    U[1, 2, 3, 0, 1] = W
    expect = (18 * V - 18 + 6 * np.trace(W).real) / (18 * V)
    assert oracle.plaquette(U) == pytest.approx(expect, abs=1e-15)
    del dims


def test_stochastic_relaxation_limits():
    """p = 0 is plain relaxation (the omega = 1 update); p = 1 applies the
    microcanonical step at every subgroup, which leaves each subgroup's
    Re tr[g K] and hence F unchanged; every step is a gauge transformation."""
    dims = (4, 4, 4, 4)
    U = field(dims, seed=95, gseed=96)
    W = U.copy()
    oracle.sr_half_sweep(U, 0, 0.0, 0, 7, 3)
    oracle.or_half_sweep(W, 0, 1.0, 0)
    np.testing.assert_allclose(U, W, atol=1e-14)
    P = oracle.plaquette(U)
    for gauge in (0, 1):
        F = oracle.functional(U, gauge)
        X = U.copy()
        oracle.sr_half_sweep(X, 1, 1.0, gauge, 7, 4)
        assert oracle.functional(X, gauge) == pytest.approx(F, abs=1e-13)
        assert oracle.plaquette(X) == pytest.approx(P, abs=1e-13)
        assert np.abs(X - U).max() > 1e-3  # it did move the links
    # intermediate p: F between the two limits is not monotone but the draw is seeded
    A, B = U.copy(), U.copy()
    oracle.sr_half_sweep(A, 0, 0.5, 0, 11, 5)
    oracle.sr_half_sweep(B, 0, 0.5, 0, 11, 5)
    np.testing.assert_array_equal(A, B)


def test_stochastic_relaxation_fixes_the_gauge():
    dims = (4, 4, 4, 4)
    U = field(dims, seed=97, gseed=98)
    for n in range(400):
        oracle.sr_half_sweep(U, n % 2, 0.8, 0, 3, n // 2)
    assert oracle.theta(U, 0) < 1e-8


# ---------------------------------------------------------------------------
# readings of g -> g^omega (Sec. 2 leaves the order of the exponent open)
# ---------------------------------------------------------------------------
@pytest.fixture
def or_variant():
    yield oracle.set_or_variant
    oracle.set_or_variant(0)


def test_or_variants_reduce_to_relaxation_at_omega_one(or_variant):
    rng = np.random.default_rng(31)
    for v in (0, 1, 2):
        or_variant(v)
        for _ in range(50):
            k = rng.standard_normal(4) * rng.uniform(0.1, 5)
            r = oracle.overrelax_quaternion(k, 1.0)
            np.testing.assert_allclose(r, k / np.linalg.norm(k), atol=1e-15)


def test_or_exact_power_is_the_matrix_power(or_variant):
    """Reading 2 equals G^omega of the relaxation element G (principal
    branch), computed by scipy's fractional matrix power."""
    from scipy.linalg import fractional_matrix_power
    or_variant(2)
    rng = np.random.default_rng(32)
    for _ in range(40):
        k = rng.standard_normal(4)
        k[0] = abs(k[0]) + 0.05  # rotation angle below pi/2 .. pi: principal branch well defined
        omega = rng.uniform(0.2, 1.95)
        G = su2_from_quaternion(k / np.linalg.norm(k))
        want = fractional_matrix_power(G, omega)
        got = su2_from_quaternion(oracle.overrelax_quaternion(k, omega))
        np.testing.assert_allclose(got, want, atol=1e-12)


def test_or_first_order_is_projected_linear_combination(or_variant):
    """Reading 1 is (1 - omega) 1 + omega G projected back onto SU(2):
    proportional to that matrix with a positive factor, and unitary."""
    or_variant(1)
    rng = np.random.default_rng(33)
    for _ in range(40):
        k = rng.standard_normal(4)
        omega = rng.uniform(0.2, 1.95)
        G = su2_from_quaternion(k / np.linalg.norm(k))
        Mlin = (1 - omega) * np.eye(2) + omega * G
        R = su2_from_quaternion(oracle.overrelax_quaternion(k, omega))
        np.testing.assert_allclose(R @ R.conj().T, np.eye(2), atol=1e-14)
        ratio = Mlin / R
        np.testing.assert_allclose(ratio, ratio[0, 0] * np.ones((2, 2)), atol=1e-12)
        assert ratio[0, 0].real > 0 and abs(ratio[0, 0].imag) < 1e-12


def test_or_readings_agree_at_small_angles(or_variant):
    """All readings rotate by omega * phi + O(phi^3) (first order in the
    exponent's angle): the three agree to O(phi^3)."""
    omega = 1.7
    n = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    for phi in (1e-2, 1e-3):
        k = np.concatenate([[np.cos(phi)], np.sin(phi) * n])
        rs = []
        for v in (0, 1, 2):
            or_variant(v)
            rs.append(oracle.overrelax_quaternion(k, omega))
        for r in rs:
            ang = np.arctan2(np.linalg.norm(r[1:]), r[0])
            assert abs(ang - omega * phi) < 2 * phi ** 3


@pytest.mark.parametrize("v", [1, 2])
def test_or_variants_fix_the_gauge_and_keep_the_plaquette(or_variant, v):
    dims = (4, 4, 4, 4)
    or_variant(v)
    U = field(dims, seed=1, gseed=2, pure=True)
    oracle.or_sweeps(U, 1.5, 0, 300)
    assert oracle.theta(U, 0) < 1e-24
    assert oracle.functional(U, 0) == pytest.approx(1.0, abs=1e-12)
    W = field(dims, seed=5, gseed=6)
    P = oracle.plaquette(W)
    oracle.or_sweeps(W, 1.7, 0, 20)
    assert oracle.plaquette(W) == pytest.approx(P, abs=1e-13)


# ---------------------------------------------------------------------------
# per-timeslice F and theta (Coulomb gauge fixes each timeslice on its own)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gauge", [0, 1])
def test_timeslice_means_are_the_global_values(gauge):
    U = field((4, 4, 6, 8), seed=41, gseed=42)
    F_t, th_t = oracle.timeslices(U, gauge)
    assert len(F_t) == 8
    assert F_t.mean() == pytest.approx(oracle.functional(U, gauge), rel=1e-14)
    assert th_t.mean() == pytest.approx(oracle.theta(U, gauge), rel=1e-13)


def test_timeslice_values_are_local_in_time():
    """A gauge rotation confined to timeslice t0 of the unit field leaves every
    other timeslice at F_t = 1, theta_t = 0 in Coulomb gauge (spatial links of
    t0 only are touched; temporal links do not enter F and theta)."""
    import torch
    dims = (4, 4, 4, 6)
    Lx, Ly, Lz, Lt = dims
    t0 = 2
    one = torch.eye(3, dtype=torch.complex128).expand(Lt, Lz, Ly, Lx, 4, 3, 3).contiguous()
    g = torch.eye(3, dtype=torch.complex128).expand(Lt, Lz, Ly, Lx, 3, 3).clone()
    g[t0] = synth.haar_su3((Lz, Ly, Lx), 43)
    U = synth.as_numpy(synth.rotate_field(one, g))
    F_t, th_t = oracle.timeslices(U, 1)
    for t in range(Lt):
        if t == t0:
            assert th_t[t] > 1e-3 and F_t[t] < 0.99
        else:
            assert th_t[t] < 1e-28 and F_t[t] == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------------------
# maximally Abelian gauge (Sec. 6; functional sum |U_ii|^2 of the literature)
# ---------------------------------------------------------------------------
def _diag_weight_after(star_links, a, b, R):
    """sum over the 8 links of |diag_a|^2 + |diag_b|^2 after the subgroup
    rotation R (forward links R U, backward links U R^dagger), with numpy."""
    G = np.eye(3, dtype=complex)
    G[np.ix_([a, b], [a, b])] = R
    q = 0.0
    for f in star_links[0]:
        V = G @ f
        q += abs(V[a, a]) ** 2 + abs(V[b, b]) ** 2
    for w in star_links[1]:
        V = w @ G.conj().T
        q += abs(V[a, a]) ** 2 + abs(V[b, b]) ** 2
    return q


def _star(U, site):
    dims = oracle.dims_of(U)
    flat = U.reshape(-1, 4, 3, 3)
    fwd = [flat[site, mu] for mu in range(4)]
    bwd = [flat[oracle.backward_site(tuple(int(d) for d in dims), site, mu), mu] for mu in range(4)]
    return fwd, bwd


def block_su2_field(dims, seed):
    """Every link block-diag(R, 1), R Haar-random in SU(2)."""
    rng = np.random.default_rng(seed)
    V = int(np.prod(dims))
    q = haarsu2_from_quaternion(V * 4, rng)
    Lx, Ly, Lz, Lt = dims
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), complex)
    flat = U.reshape(-1, 3, 3)
    for n in range(V * 4):
        flat[n] = embed(su2_from_quaternion(q[n]), 0, 1)
    return U


def test_mag_local_matrix_is_the_quadratic_form_and_its_maximum():
    """q(r) = r^T A r for unit and non-unit r (numpy evaluation of the diagonal
    weight); no random SU(2) element beats the chosen maximiser, which reaches
    the largest eigenvalue of A."""
    U = field((4, 4, 4, 4), seed=51, gseed=52)
    rng = np.random.default_rng(53)
    for site, sg in ((0, 0), (37, 1), (101, 2)):
        a, b = [(0, 1), (1, 2), (0, 2)][sg]
        A = oracle.mag_local_matrix(U, site, sg)
        st = _star(U, site)
        for _ in range(5):
            r = rng.standard_normal(4)
            assert r @ A @ r == pytest.approx(_diag_weight_after(st, a, b, su2_from_quaternion(r)), rel=1e-12)
        r = oracle.mag_maximiser(A)
        best = _diag_weight_after(st, a, b, su2_from_quaternion(r))
        assert best == pytest.approx(np.linalg.eigvalsh(A).max(), rel=1e-12)
        trials = rng.standard_normal((20000, 4))
        trials /= np.linalg.norm(trials, axis=1, keepdims=True)
        vals = np.einsum("ni,ij,nj->n", trials, A, trials)
        assert vals.max() <= best + 1e-12


def test_mag_maximiser_is_the_su2_textbook_solution():
    """For links block-diag(SU(2), 1) the subgroup-(0,1) MAG step is the SU(2)
    one: g rotates X = sum_mu [U s3 U^+ + U_b^+ s3 U_b] onto +|X| s3 (numpy)."""
    U = block_su2_field((4, 4, 4, 4), 55)
    s3 = np.diag([1.0, -1.0])
    for site in (0, 77):
        fwd, bwd = _star(U, site)
        X = sum(f[:2, :2] @ s3 @ f[:2, :2].conj().T for f in fwd) + \
            sum(w[:2, :2].conj().T @ s3 @ w[:2, :2] for w in bwd)
        R = su2_from_quaternion(oracle.mag_maximiser(oracle.mag_local_matrix(U, site, 0)))
        Y = R @ X @ R.conj().T
        assert abs(X[0, 1]) > 1e-3  # a non-trivial rotation
        assert abs(Y[0, 1]) < 1e-12 and Y[0, 0].real > 0
        assert Y[0, 0].real == pytest.approx(np.sqrt(0.5 * np.trace(X @ X).real), rel=1e-12)


def test_mag_overrelaxation_applies_the_exponent_to_the_relaxation_step():
    """Links block-diag(SU(2), 1): only subgroup (0,1) acts, and the step maps
    X = sum_mu [U s3 U^+ + U_b^+ s3 U_b] (numpy) to R X R^+.  Relaxation turns X
    onto +s3 (angle 2 phi -> 0); with omega the element is the rational map of
    the relaxation element, tan phi' = b tan phi, b = omega cos^2 phi + sin^2 phi,
    so the angle between R X R^+ and s3 becomes |2 phi' - 2 phi|."""
    omega = 1.7
    U = block_su2_field((4, 4, 4, 4), 67)
    s3 = np.diag([1.0, -1.0])

    def X_of(W, site):
        fwd, bwd = _star(W, site)
        return sum(f[:2, :2] @ s3 @ f[:2, :2].conj().T for f in fwd) + \
            sum(w[:2, :2].conj().T @ s3 @ w[:2, :2] for w in bwd)

    def angle(X):
        n = np.sqrt(0.5 * np.trace(X @ X).real)
        return np.arccos(np.clip(0.5 * np.trace(X @ s3).real / n, -1, 1)), n

    W = U.copy()
    oracle.mag_half_sweep(W, 0, omega)
    checked = 0
    for site in range(256):
        if oracle.site_parity((4, 4, 4, 4), site) != 0:
            continue
        a0, n0 = angle(X_of(U, site))
        a1, n1 = angle(X_of(W, site))
        phi = a0 / 2
        b = omega * np.cos(phi) ** 2 + np.sin(phi) ** 2
        phi1 = np.arctan2(b * np.sin(phi), np.cos(phi))
        assert a0 > 1e-3  # a non-trivial rotation
        assert n1 == pytest.approx(n0, rel=1e-12)
        assert a1 == pytest.approx(abs(2 * phi1 - 2 * phi), abs=1e-9)
        checked += 1
    assert checked == 128


def test_mag_relaxation_is_monotone_and_a_gauge_transformation():
    U = field((4, 4, 4, 6), seed=57, gseed=58)
    P = oracle.plaquette(U)
    F = oracle.mag_functional(U)
    for n in range(6):
        oracle.mag_half_sweep(U, n % 2, 1.0)
        F1 = oracle.mag_functional(U)
        assert F1 >= F - 1e-14
        F = F1
    assert oracle.plaquette(U) == pytest.approx(P, abs=1e-13)


def test_mag_theta_is_the_squared_gradient_of_the_diagonal_weight():
    """theta_MAG = 1/(3V) sum_x sum_subgroups |grad q|^2 / 4, q the star's
    diagonal weight after R = exp(i eps sigma_j) (numpy, central differences):
    dq/deps_j = 2 A_j0.  The third direction is the residual U(1), along which
    q is flat."""
    U = field((4, 4, 4, 4), seed=63, gseed=64)
    V = 256
    eps = 1e-5
    sig = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
           np.array([[1, 0], [0, -1]], complex)]
    total = 0.0
    for site in range(V):
        st = _star(U, site)
        for sg, (a, b) in enumerate([(0, 1), (1, 2), (0, 2)]):
            g = []
            for j in range(3):
                Rp = np.cos(eps) * np.eye(2) + 1j * np.sin(eps) * sig[j]
                Rm = np.cos(eps) * np.eye(2) - 1j * np.sin(eps) * sig[j]
                g.append((_diag_weight_after(st, a, b, Rp) - _diag_weight_after(st, a, b, Rm)) / (2 * eps))
            assert abs(g[2]) < 1e-6 * (1 + abs(g[0]) + abs(g[1]))
            total += (g[0] ** 2 + g[1] ** 2) / 4
    assert oracle.mag_theta(U) == pytest.approx(total / (3 * V), rel=1e-6)


def test_mag_maximiser_is_the_one_closest_to_the_identity():
    """The maximisers of the subgroup's diagonal weight form a circle (the
    residual U(1)); the chosen one has alpha real and positive, i.e. r3 = 0,
    r0 > 0, and r0 equal to the largest identity component on that circle: the
    norm of the projection of e0 onto the top eigenspace (numpy eigh)."""
    U = field((4, 4, 4, 4), seed=65, gseed=66)
    for site, sg in ((3, 0), (77, 1), (150, 2), (201, 0)):
        A = oracle.mag_local_matrix(U, site, sg)
        w, Q = np.linalg.eigh(A)
        top = Q[:, w > w.max() - 1e-10 * max(1.0, abs(w.max()))]
        r = oracle.mag_maximiser(A)
        assert abs(r[3]) < 1e-12 and r[0] > 0
        assert r[0] == pytest.approx(np.linalg.norm(top.T @ np.eye(4)[0]), rel=1e-12)
        assert r @ A @ r == pytest.approx(w.max(), rel=1e-12)


def test_mag_fixed_points():
    """Diagonal links are maximal (F = 1, theta = 0) and left unchanged; a
    gauge-rotated diagonal field is brought back to F = 1, theta -> 0."""
    import torch
    dims = (4, 4, 4, 4)
    rng = np.random.default_rng(59)
    ph = rng.uniform(0, 2 * np.pi, (4, 4, 4, 4, 4, 2))
    D = np.zeros((4, 4, 4, 4, 4, 3, 3), complex)
    D[..., 0, 0] = np.exp(1j * ph[..., 0])
    D[..., 1, 1] = np.exp(1j * ph[..., 1])
    D[..., 2, 2] = np.exp(-1j * (ph[..., 0] + ph[..., 1]))
    assert oracle.mag_functional(D) == pytest.approx(1.0, abs=1e-15)
    assert oracle.mag_theta(D) < 1e-28
    W = D.copy()
    oracle.mag_sweeps(W, 1.7, 2)
    np.testing.assert_allclose(W, D, atol=1e-14)
    g = synth.haar_su3((4, 4, 4, 4), 60)
    R = synth.as_numpy(synth.rotate_field(torch.from_numpy(D), g))
    assert oracle.mag_functional(R) < 0.6
    oracle.mag_sweeps(R, 1.7, 300)
    assert oracle.mag_theta(R) < 1e-20
    assert oracle.mag_functional(R) == pytest.approx(1.0, abs=1e-10)


# ---------------------------------------------------------------------------
# Wilson-action generation (heatbath + microcanonical overrelaxation)
# ---------------------------------------------------------------------------
def _plaquettes_with_link(U, site, mu):
    """sum over the 6 plaquettes containing U_mu(x) of Re tr U_P, with numpy."""
    dims = tuple(int(d) for d in oracle.dims_of(U))
    flat = U.reshape(-1, 4, 3, 3)

    def shift(i, nu, d):
        c = list(np.unravel_index(i, dims[::-1])[::-1])
        c[nu] = (c[nu] + d) % dims[nu]
        return int(np.ravel_multi_index(c[::-1], dims[::-1]))
    tot = 0.0
    for nu in range(4):
        if nu == mu:
            continue
        xp, xn, xm = shift(site, mu, 1), shift(site, nu, 1), shift(site, nu, -1)
        P = flat[site, mu] @ flat[xp, nu] @ flat[xn, mu].conj().T @ flat[site, nu].conj().T
        Q = flat[xm, mu] @ flat[shift(xm, mu, 1), nu] @ flat[site, mu].conj().T @ flat[xm, nu].conj().T
        tot += np.trace(P).real + np.trace(Q).real
    return tot


def test_staple_gives_the_plaquettes_of_the_link():
    """Re tr(U A) equals the sum over the six plaquettes containing U (numpy)."""
    U = field((4, 4, 4, 6), seed=71, gseed=72)
    flat = U.reshape(-1, 4, 3, 3)
    for site, mu in ((0, 0), (57, 2), (300, 3)):
        A = oracle.staple(U, site, mu)
        assert np.trace(flat[site, mu] @ A).real == pytest.approx(_plaquettes_with_link(U, site, mu), rel=1e-12)


def test_wilson_overrelaxation_conserves_the_action():
    U = field((4, 4, 4, 4), seed=73, gseed=74)
    P = oracle.plaquette(U)
    V = U.copy()
    for mu in range(4):
        for p in (0, 1):
            oracle.wilson_update(V, mu, p, 6.0, 1, 1, 0)
    assert oracle.plaquette(V) == pytest.approx(P, abs=1e-13)
    assert np.abs(V - U).max() > 1e-2  # the links did move


def test_wilson_heatbath_zero_temperature_is_relaxation():
    """beta -> infinity: each subgroup is set to the maximiser of Re tr(R U A),
    so the local action Re tr(U A) reaches its subgroup maxima and the
    plaquette rises."""
    U = field((4, 4, 4, 4), seed=75, gseed=76)
    P0 = oracle.plaquette(U)
    flat_before = U.reshape(-1, 4, 3, 3).copy()
    oracle.wilson_update(U, 0, 0, 1e15, 0, 3, 0)  # heatbath spread ~ sqrt(3 / (beta |k|)) ~ 1e-8
    assert oracle.plaquette(U) > P0
    # the updated link maximises the last subgroup (0, 2): its quaternion is real
    A = oracle.staple(U, 0, 0)
    W = U.reshape(-1, 4, 3, 3)[0, 0] @ A
    k = oracle.block_quaternion(np.array([[W[0, 0], W[0, 2]], [W[2, 0], W[2, 2]]]))
    assert np.linalg.norm(k[1:]) < 1e-6 * np.linalg.norm(k) and k[0] > 0
    assert not np.allclose(flat_before[0, 0], U.reshape(-1, 4, 3, 3)[0, 0])


def test_wilson_strong_coupling_plaquette():
    """beta = 0.3: <Re tr U_P / 3> = beta/18 + O(beta^2) for SU(3)."""
    beta = 0.3
    U = field((4, 4, 4, 4), seed=77, gseed=78, plaq=0.1)
    vals = []
    for n in range(60):
        assert oracle.wilson_sweep(U, beta, 0, 5, n) == 0
        if n >= 20:
            vals.append(oracle.plaquette(U))
    assert np.mean(vals) == pytest.approx(beta / 18, abs=3e-3)


def test_wilson_beta6_plaquette():
    """beta = 6.0 on 8^4: the average plaquette of the thermalised Wilson
    theory, 0.5937 (a standard value of the literature), within 0.006."""
    U = field((8, 8, 8, 8), seed=79, gseed=80, plaq=0.59)
    vals = []
    for n in range(40):
        oracle.wilson_sweep(U, 6.0, 0, 7, n)
        oracle.wilson_sweep(U, 6.0, 1, 7, n)
        if n >= 15:
            vals.append(oracle.plaquette(U))
    assert np.mean(vals) == pytest.approx(0.5937, abs=6e-3)
