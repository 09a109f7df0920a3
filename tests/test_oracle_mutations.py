"""The pins pin: plausible mistakes planted in a copy of the oracle make them fail.

Each case copies the oracle's C sources to a temporary directory, replaces one
line with a plausible mistake (a dropped term, a wrong sign or index, a
transposed operand, a wrong constant), checks that the copy still compiles,
and runs the oracle pin tests against it (environment ORACLE_SOURCE_DIR).
The case passes when the pins fail.  All on the CPU; nothing here touches a
GPU or the library.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SOURCES = ("gf_oracle.c", "conv_oracle.c")

# (name, file, original text, planted mistake)
MUTATIONS = [
    ("quaternion sign", "gf_oracle.c",
     "k[1] = -(w01.im + w10.im);", "k[1] = (w01.im + w10.im);"),
    ("quaternion transposed operands", "gf_oracle.c",
     "k[2] = w10.re - w01.re;", "k[2] = w01.re - w10.re;"),
    ("su2 matrix sign", "gf_oracle.c",
     "R[1][0] = c_make(-r[2], r[1]);", "R[1][0] = c_make(r[2], r[1]);"),
    ("omega on the wrong term", "gf_oracle.c",
     "double b = (omega * a0sq + aisq) / (a0sq + aisq);", "double b = (a0sq + omega * aisq) / (a0sq + aisq);"),
    ("backward rotation without dagger", "gf_oracle.c",
     "cplx r00 = c_conj(R[0][0]), r01 = c_conj(R[0][1]);", "cplx r00 = R[0][0], r01 = R[0][1];"),
    ("backward link at x + mu", "gf_oracle.c",
     "s->bwd[mu] = mat_load(link_cptr(U, site_shift(g, i, mu, -1), mu));",
     "s->bwd[mu] = mat_load(link_cptr(U, site_shift(g, i, mu, +1), mu));"),
    ("backward block not transposed", "gf_oracle.c",
     "block_quaternion(c_conj(w->m[a][a]), c_conj(w->m[b][a]), c_conj(w->m[a][b]),",
     "block_quaternion(c_conj(w->m[a][a]), c_conj(w->m[a][b]), c_conj(w->m[b][a]),"),
    ("Coulomb gauge with temporal links", "gf_oracle.c",
     "static int gauge_nk(int gauge) { return gauge == 1 ? 3 : 4; }",
     "static int gauge_nk(int gauge) { return gauge == 1 ? 4 : 4; }"),
    ("functional normalisation", "gf_oracle.c",
     "return sum / (3.0 * nk * (double)g.V);", "return sum / (3.0 * 4 * (double)g.V);"),
    ("theta without the 1/2", "gf_oracle.c",
     "A.m[a][b] = c_make(0.5 * z.im, -0.5 * z.re);", "A.m[a][b] = c_make(z.im, -z.re);"),
    ("theta not traceless", "gf_oracle.c",
     "c_sub(Af.m[a][b], Ab.m[a][b]));\n        }\n        make_traceless(&D);",
     "c_sub(Af.m[a][b], Ab.m[a][b]));\n        }"),
    ("gauge transform with g(x) on both ends", "gf_oracle.c",
     "mat3 gy = mat_load(gfield + site_shift(&g, i, mu, +1) * 18);", "mat3 gy = mat_load(gfield + i * 18);"),
    ("Philox key schedule constant", "gf_oracle.c",
     "k[1] += 0xBB67AE85u;", "k[1] += 0xBB67AE87u;"),
    ("Creutz draw support", "gf_oracle.c",
     "double e = exp(-2.0 * alpha);", "double e = exp(-alpha);"),
    ("Kennedy-Pendleton scale", "gf_oracle.c",
     "double lam2 = -(log(u01(w[0])) + c * c * log(u01(w[2]))) / (2.0 * alpha);",
     "double lam2 = -(log(u01(w[0])) + c * c * log(u01(w[2]))) / alpha;"),
    ("heatbath direction not on the sphere", "gf_oracle.c",
     "double s[4] = { s0, rho * st * cos(phi), rho * st * sin(phi), rho * ct };",
     "double s[4] = { s0, rho * cos(phi), rho * sin(phi), rho * ct };"),
    ("stochastic relaxation probability inverted", "gf_oracle.c",
     "if (u01(w[0]) < p) {", "if (u01(w[0]) >= p) {"),
    ("maximally Abelian weight of an off-diagonal entry", "gf_oracle.c",
     "return c_abs2(u->m[a][a]) + c_abs2(u->m[b][b]);", "return c_abs2(u->m[a][a]) + c_abs2(u->m[a][b]);"),
    ("maximally Abelian polarisation factor", "gf_oracle.c",
     "A[k][m] = A[m][k] = 0.25 * (", "A[k][m] = A[m][k] = 0.5 * ("),
    ("lower staple product order", "gf_oracle.c",
     "mat3 t2 = mat_mul(&dd, &ed);", "mat3 t2 = mat_mul(&ed, &dd);"),
    ("exact-power reading ignores omega", "gf_oracle.c",
     "double c = cos(omega * phi), sn = sin(omega * phi);", "double c = cos(phi), sn = sin(phi);"),
    ("first-order reading drops omega on k", "gf_oracle.c",
     "double v[4] = { (1.0 - omega) + omega * (k[0] / n),", "double v[4] = { (1.0 - omega) + (k[0] / n),"),
    ("timeslice functional normalisation", "gf_oracle.c",
     "F_t[t] = fs / (3.0 * nk * (double)Ls);", "F_t[t] = fs / (3.0 * 4 * (double)Ls);"),
    ("convergence loop sweeps once per check", "gf_oracle.c",
     "oracle_or_sweeps(U, dims, omega, gauge, n);", "oracle_or_sweeps(U, dims, omega, gauge, 1);"),
    ("microcanonical step replaced by relaxation", "gf_oracle.c",
     "    quat_mul(h, h, r);\n    return 1;", "    memcpy(r, h, sizeof h);\n    return 1;"),
    ("network inputs without the backward dagger", "gf_oracle.c",
     "for (int b = 0; b < 3; ++b) M.m[a][b] = c_add(M.m[a][b], c_add(uf.m[a][b], ubd.m[a][b]));",
     "for (int b = 0; b < 3; ++b) M.m[a][b] = c_add(M.m[a][b], c_add(uf.m[a][b], ub.m[a][b]));"),
    ("network inputs with the link reals out of order", "gf_oracle.c",
     "for (int r = 0; r < 18; ++r) o[mu * 18 + r] = p[r];",
     "for (int r = 0; r < 18; ++r) o[mu * 18 + r] = p[(r + 2) % 18];"),
    ("exponential map without the 1/2 of lambda/2", "gf_oracle.c",
     "double w = 0.5 * scale * c[j * 8 + a];", "double w = scale * c[j * 8 + a];"),
    ("exponential map Taylor divisor", "gf_oracle.c",
     "T.m[x][y] = c_make(P.m[x][y].re / k, P.m[x][y].im / k);",
     "T.m[x][y] = c_make(P.m[x][y].re / (k + 1), P.m[x][y].im / (k + 1));"),
    ("algebra coefficients multiplied by the scale", "gf_oracle.c",
     "for (int a = 0; a < 8; ++a) c[j * 8 + a] = re_tr_lambda(a, &A) / scale;",
     "for (int a = 0; a < 8; ++a) c[j * 8 + a] = re_tr_lambda(a, &A) * scale;"),
    ("plaquette second link at x", "gf_oracle.c",
     "mat3 b = mat_load(link_cptr(U, site_shift(&g, i, mu, +1), nu));", "mat3 b = mat_load(link_cptr(U, i, nu));"),
    ("reunitarised third row not conjugated", "gf_oracle.c",
     "            u.m[2][c] = c_conj(x);\n        }\n        mat_store(M + j * 18, &u);",
     "            u.m[2][c] = x;\n        }\n        mat_store(M + j * 18, &u);"),
    ("Gram-Schmidt projection conjugated wrongly", "gf_oracle.c",
     "ip = c_add(ip, c_mul(c_conj(u.m[0][c]), u.m[1][c]));", "ip = c_add(ip, c_mul(u.m[0][c], c_conj(u.m[1][c])));"),
    ("annealing schedule misses T1", "gf_oracle.c",
     "double T = steps > 1 ? T0 + (T1 - T0) * (double)k / (double)(steps - 1) : T0;",
     "double T = steps > 1 ? T0 + (T1 - T0) * (double)k / (double)steps : T0;"),
    ("heatbath alpha = |k| T", "gf_oracle.c",
     "if (!heatbath_s0(kn / T, site, sweep, sg, cap, key, tag, &s0)) return 0;",
     "if (!heatbath_s0(kn * T, site, sweep, sg, cap, key, tag, &s0)) return 0;"),
    ("Wilson heatbath temperature 1/beta", "gf_oracle.c",
     "st = heatbath_quaternion_tag(k, 3.0 / beta,", "st = heatbath_quaternion_tag(k, 1.0 / beta,"),
    ("Wilson local matrix A U instead of U A", "gf_oracle.c",
     "mat3 W = mat_mul(&u, &A);", "mat3 W = mat_mul(&A, &u);"),
    ("maximally Abelian theta along the residual U(1)", "gf_oracle.c",
     "sum += A[1][0] * A[1][0] + A[2][0] * A[2][0];", "sum += A[1][0] * A[1][0] + A[3][0] * A[3][0];"),
    ("maximally Abelian maximiser projects e1", "gf_oracle.c",
     "const int e = target == 0 ? 0 : 2;", "const int e = target == 0 ? 1 : 2;"),
    ("microcanonical square without the -1", "gf_oracle.c",
     "r[0] = 2.0 * r0 * r0 - 1.0;", "r[0] = 2.0 * r0 * r0;"),
    ("loss gradient factor", "conv_oracle.c",
     "dY[i] = 2.0 * (act[4][i] - target[i]) / (double)n;", "dY[i] = 1.0 * (act[4][i] - target[i]) / (double)n;"),
    ("ReLU mask never applied", "conv_oracle.c",
     "if (!(act[l][i] > 0.0)) dX[i] = 0.0;", "if (!(act[l][i] >= 0.0)) dX[i] = 0.0;"),
    ("weight gradient with the backward shift", "conv_oracle.c",
     "        for (long s = 0; s < g.V; ++s) {\n            const double *x = X + shifted(&g, s, k, +1) * cin;",
     "        for (long s = 0; s < g.V; ++s) {\n            const double *x = X + shifted(&g, s, k, -1) * cin;"),
    ("temporal links of the star not rotated", "gf_oracle.c",
     "static void star_rotate(star *s, int a, int b, cplx R[2][2])\n{\n    for (int mu = 0; mu < 4; ++mu) {",
     "static void star_rotate(star *s, int a, int b, cplx R[2][2])\n{\n    for (int mu = 0; mu < 3; ++mu) {"),
    ("maximally Abelian step without the overrelaxation exponent", "gf_oracle.c",
     "if (!overrelax_quaternion(r, omega, ro)) continue;", "if (!overrelax_quaternion(r, 1.0, ro)) continue;"),
    ("network violation inputs not scaled", "gf_oracle.c",
     "for (int a = 0; a < 8; ++a) o[72 + a] = re_tr_lambda(a, &D) / scale;",
     "for (int a = 0; a < 8; ++a) o[72 + a] = re_tr_lambda(a, &D);"),
    ("stochastic-relaxation square drops a factor 2", "gf_oracle.c",
     "r[1] = 2.0 * r0 * r[1];", "r[1] = r0 * r[1];"),
    ("convolution taps transposed", "conv_oracle.c",
     "int d[4] = { k % 3 - 1, (k / 3) % 3 - 1, (k / 9) % 3 - 1, (k / 27) % 3 - 1 };",
     "int d[4] = { (k / 3) % 3 - 1, k % 3 - 1, (k / 9) % 3 - 1, (k / 27) % 3 - 1 };"),
    ("FP32 draw: Creutz support", "gf_oracle.c",
     "float e = expf(-2.0f * alpha);", "float e = expf(-alpha);"),
    ("FP32 draw: Kennedy-Pendleton uniforms swapped", "gf_oracle.c",
     "float lam2 = -(logf(u01f(w[0])) + c * c * logf(u01f(w[2]))) / (2.0f * alpha);",
     "float lam2 = -(logf(u01f(w[2])) + c * c * logf(u01f(w[0]))) / (2.0f * alpha);"),
    ("FP32 draw: direction without the sphere factor", "gf_oracle.c",
     "double s[4] = { (double)s0f, (double)(rho * st * cosf(phi)), (double)(rho * st * sinf(phi)),",
     "double s[4] = { (double)s0f, (double)(rho * cosf(phi)), (double)(rho * st * sinf(phi)),"),
    ("FP32 draw: uniform from the low bits", "gf_oracle.c",
     "static float u01f(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }",
     "static float u01f(uint32_t w) { return ((float)(w & 0x7FFFFFu) + 0.5f) * (1.0f / 8388608.0f); }"),
    ("convolution backward data with the forward shift", "conv_oracle.c",
     "const double *dy = dY + shifted(&g, s, k, -1) * cout;", "const double *dy = dY + shifted(&g, s, k, +1) * cout;"),
]


def _pins_on_copy(workdir, mutation=None):
    """Copy the sources (with the mutation applied), build them where the oracle
    module looks for them, run the pins against the copy; (pytest exit code, output)."""
    os.makedirs(workdir)
    for f in SOURCES:
        shutil.copy(os.path.join(ORACLE, f), os.path.join(workdir, f))
    if mutation is not None:
        fname, old, new = mutation
        path = os.path.join(workdir, fname)
        text = open(path).read()
        if text.count(old) != 1:
            return None, f"mutation site not unique or missing: {old!r}"
        open(path, "w").write(text.replace(old, new))
    # the copy must compile, so that a failing pin run means a caught mistake
    srcs = [os.path.join(workdir, f) for f in SOURCES]
    os.makedirs(os.path.join(workdir, "_build"))
    cc = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall",
                         "-Wno-unused-function", "-fopenmp", *srcs, "-o",
                         os.path.join(workdir, "_build", "liboracle.so"), "-lm"], capture_output=True, text=True)
    if cc.returncode != 0:
        return None, "does not compile:\n" + cc.stderr[-2000:]
    env = dict(os.environ, ORACLE_SOURCE_DIR=workdir, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
           os.path.join(ROOT, "tests", "test_conv_oracle.py"), "-x", "-q", "-m", "not gpu",
           "-p", "no:cacheprovider"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=workdir, env=env)
    return r.returncode, r.stdout


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every case (and the unmodified control) run up front, four at a time."""
    base = str(tmp_path_factory.mktemp("mutants"))
    jobs = {"control": None, **{m[0]: m[1:] for m in MUTATIONS}}
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        futs = {name: ex.submit(_pins_on_copy, os.path.join(base, f"case{i}"), mut)
                for i, (name, mut) in enumerate(jobs.items())}
        return {name: f.result() for name, f in futs.items()}


def test_unmodified_copy_passes_the_pins(outcomes):
    """Control: the same procedure on an unmodified copy passes, so a failure
    below is the planted mistake's doing."""
    rc, out = outcomes["control"]
    assert rc == 0, out[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_the_pins(outcomes, name):
    rc, out = outcomes[name]
    assert rc is not None, out
    # pytest exit code 1: tests ran and some failed (2+ would be an interrupted or broken run)
    assert rc == 1, f"the pins did not catch '{name}':\n{out[-3000:]}"
