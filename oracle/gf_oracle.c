/*
 * gf_oracle.c -- plain FP64 CPU oracle for SU(3) lattice gauge fixing by
 * checkerboard overrelaxation and simulated annealing.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Source: Schroeck & Vogt, "Gauge fixing using overrelaxation and simulated
 * annealing on GPUs" (Lattice 2012).  Every function cites the passage it
 * follows.  Points the paper leaves open are taken as follows (each is listed
 * with its reason in the design notes of the repository):
 *   - periodic boundaries, all extents even; RED = even parity, updated first;
 *   - SU(2) subgroups visited in the order (0,1), (1,2), (0,2);
 *   - the exponent g -> g^omega (Sec. 2 leaves its order open) is taken
 *     as the 19-flop rational form: b = (w a0^2 + |a|^2)/(a0^2 + |a|^2),
 *     r = (a0, b a)/sqrt(a0^2 + b^2 |a|^2) (equals relaxation at w = 1);
 *   - F is normalised by 1/(Nc Nd V) so that the unit field has F = 1;
 *   - the violation Delta(x) of eq. (theta) is the traceless part of
 *     sum_mu [A_mu(x) - A_mu(x-mu)], A = (U - U^dagger)/(2i);
 *   - Coulomb gauge: only spatial links enter K, F and theta, the temporal
 *     links are rotated by the same g so that the update stays a gauge
 *     transformation;
 *   - a subgroup whose projected quaternion vanishes is left unchanged;
 *   - two further readings of g -> g^omega are selectable (first order, exact
 *     power; oracle_set_or_variant);
 *   - the maximally Abelian gauge (Sec. 6, named only) maximises the
 *     literature's sum |U_ii|^2 by the same subgroup relaxation/overrelaxation;
 *   - thermalised inputs (Sec. 5) come from the Wilson action by
 *     Cabibbo-Marinari heatbath and microcanonical overrelaxation.
 *
 * Data layout (canonical, shared with the library's public API): a field is
 * double U[Lt][Lz][Ly][Lx][4][3][3][2] -- site index x fastest, then the four
 * link directions mu = x, y, z, t, then the 3x3 complex matrix row-major,
 * complex numbers as (re, im).  dims = {Lx, Ly, Lz, Lt}.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off (no fused multiply-add, so each
 * operation rounds as written).  With -DORACLE_COUNT_FLOPS (and without
 * OpenMP) every real floating-point operation of the overrelaxation update is
 * counted, to pin the per-step counts printed in Alg. 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 2 pi as the nearest double */
#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* flop counting (Alg. 1: 60 + 19 + 4 x (84 + 84) flop per subgroup)         */
/* ------------------------------------------------------------------------ */
#ifdef ORACLE_COUNT_FLOPS
static unsigned long long g_flops;
#define FLOPS(n) (g_flops += (unsigned long long)(n))
#else
#define FLOPS(n) ((void)0)
#endif

unsigned long long oracle_flops(void)
{
#ifdef ORACLE_COUNT_FLOPS
    return g_flops;
#else
    return 0ULL;
#endif
}

void oracle_reset_flops(void)
{
#ifdef ORACLE_COUNT_FLOPS
    g_flops = 0;
#endif
}

int oracle_counts_flops(void)
{
#ifdef ORACLE_COUNT_FLOPS
    return 1;
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* complex numbers and 3x3 matrices                                          */
/* ------------------------------------------------------------------------ */
typedef struct { double re, im; } cplx;
typedef struct { cplx m[3][3]; } mat3;

static cplx c_make(double re, double im) { cplx z; z.re = re; z.im = im; return z; }
static cplx c_conj(cplx a) { return c_make(a.re, -a.im); }
static cplx c_add(cplx a, cplx b) { FLOPS(2); return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { FLOPS(2); return c_make(a.re - b.re, a.im - b.im); }
static cplx c_mul(cplx a, cplx b)
{
    FLOPS(6);
    return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static double c_abs2(cplx a) { return a.re * a.re + a.im * a.im; }

static mat3 mat_load(const double *p)
{
    mat3 u;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            u.m[a][b] = c_make(p[2 * (3 * a + b)], p[2 * (3 * a + b) + 1]);
    return u;
}

static void mat_store(double *p, const mat3 *u)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            p[2 * (3 * a + b)] = u->m[a][b].re;
            p[2 * (3 * a + b) + 1] = u->m[a][b].im;
        }
}

static mat3 mat_dagger(const mat3 *u)
{
    mat3 d;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            d.m[a][b] = c_conj(u->m[b][a]);
    return d;
}

static mat3 mat_mul(const mat3 *x, const mat3 *y)
{
    mat3 z;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cplx s = c_make(0.0, 0.0);
            for (int c = 0; c < 3; ++c)
                s = c_add(s, c_mul(x->m[a][c], y->m[c][b]));
            z.m[a][b] = s;
        }
    return z;
}

static double mat_retrace(const mat3 *u)
{
    return u->m[0][0].re + u->m[1][1].re + u->m[2][2].re;
}

/* ------------------------------------------------------------------------ */
/* lattice geometry (Sec. 2: nearest neighbours, checkerboard RED/BLACK)     */
/* ------------------------------------------------------------------------ */
typedef struct { int L[4]; long V; } lattice;

static int lattice_init(lattice *g, const int dims[4])
{
    g->V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1)) return -1;
        g->L[mu] = dims[mu];
        g->V *= dims[mu];
    }
    return 0;
}

static void site_coords(const lattice *g, long i, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(i % g->L[mu]);
        i /= g->L[mu];
    }
}

static long site_index(const lattice *g, const int c[4])
{
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

static int site_parity(const lattice *g, long i)
{
    int c[4];
    site_coords(g, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* index of x + dir * mu-hat with periodic wrap */
static long site_shift(const lattice *g, long i, int mu, int dir)
{
    int c[4];
    site_coords(g, i, c);
    c[mu] = (c[mu] + dir + g->L[mu]) % g->L[mu];
    return site_index(g, c);
}

static double *link_ptr(double *U, long i, int mu) { return U + (i * 4 + mu) * 18; }
static const double *link_cptr(const double *U, long i, int mu) { return U + (i * 4 + mu) * 18; }

/* ------------------------------------------------------------------------ */
/* SU(2) subgroups (Sec. 2, Cabibbo-Marinari) in quaternion form             */
/* ------------------------------------------------------------------------ */
static const int SUBGROUP[3][2] = { { 0, 1 }, { 1, 2 }, { 0, 2 } };

/*
 * An SU(2) element r = (r0, r1, r2, r3), r.r = 1, is the matrix
 *     R = r0 1 + i (r1 s1 + r2 s2 + r3 s3)
 *       = [[ r0 + i r3,  r2 + i r1],
 *          [-r2 + i r1,  r0 - i r3]]      (s_k the Pauli matrices).
 * For any complex 2x2 block w, Re tr[R w] = r . k with the projection below,
 * so the maximum of Re tr[R w] over SU(2) is |k|, reached at r = k/|k| --
 * the quaternion form of the SU(2) local solution g = K^+/sqrt(det K^+) of
 * eq. (localsolution).  Costs 4 flop.
 */
static void block_quaternion(cplx w00, cplx w01, cplx w10, cplx w11, double k[4])
{
    FLOPS(4);
    k[0] = w00.re + w11.re;
    k[1] = -(w01.im + w10.im);
    k[2] = w10.re - w01.re;
    k[3] = -(w00.im - w11.im);
}

static void su2_matrix(const double r[4], cplx R[2][2])
{
    R[0][0] = c_make(r[0], r[3]);
    R[0][1] = c_make(r[2], r[1]);
    R[1][0] = c_make(-r[2], r[1]);
    R[1][1] = c_make(r[0], -r[3]);
}

/*
 * The paper leaves open to which order g^omega is formed (Sec. 2); three
 * readings are selectable (one process-wide setting):
 *   0: the 19-flop rational form b = (w a0^2 + |a|^2)/(a0^2 + |a|^2),
 *      r = (a0, b a)/sqrt(a0^2 + b^2 |a|^2) (default; Alg. 1's count);
 *   1: first order, r = normalise((1 - omega) 1 + omega k/|k|);
 *   2: the exact power: with k/|k| = (cos phi, sin phi n), r = (cos(omega phi),
 *      sin(omega phi) n), phi in [0, pi]; the subgroup is left unchanged when
 *      the direction n is undefined (k parallel to -1: phi = pi).
 * All three give the relaxation step r = k/|k| at omega = 1.
 */
static int g_or_variant = 0;

int oracle_set_or_variant(int v)
{
    if (v < 0 || v > 2) return -1;
    g_or_variant = v;
    return 0;
}

static int overrelax_first_order(const double k[4], double omega, double r[4])
{
    double n = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
    if (n == 0.0) return 0;
    double v[4] = { (1.0 - omega) + omega * (k[0] / n), omega * (k[1] / n), omega * (k[2] / n),
                    omega * (k[3] / n) };
    double m = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    if (m == 0.0) return 0;
    for (int c = 0; c < 4; ++c) r[c] = v[c] / m;
    return 1;
}

static int overrelax_exact_power(const double k[4], double omega, double r[4])
{
    double a = sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
    if (a == 0.0) {
        if (k[0] > 0.0) {  /* phi = 0: the relaxation step is the identity */
            r[0] = 1.0;
            r[1] = r[2] = r[3] = 0.0;
            return 1;
        }
        return 0;  /* k = 0, or phi = pi with no direction */
    }
    double phi = atan2(a, k[0]);
    double c = cos(omega * phi), sn = sin(omega * phi);
    r[0] = c;
    r[1] = sn * (k[1] / a);
    r[2] = sn * (k[2] / a);
    r[3] = sn * (k[3] / a);
    return 1;
}

/*
 * Overrelaxation exponent g -> g^omega followed by the projection back to
 * SU(2) (Alg. 1's 19-flop step; Sec. 2 on the overrelaxation of Mandula and
 * Ogilvie), in the reading selected above.  Input: the unnormalised
 * quaternion k.  Output: r in SU(2).  Returns 0 (and leaves r untouched)
 * when k = 0.
 */
static int overrelax_quaternion(const double k[4], double omega, double r[4])
{
    if (g_or_variant == 1) return overrelax_first_order(k, omega, r);
    if (g_or_variant == 2) return overrelax_exact_power(k, omega, r);
    double a0sq = k[0] * k[0];
    double aisq = k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    FLOPS(6);
    if (a0sq + aisq == 0.0) return 0;
    double b = (omega * a0sq + aisq) / (a0sq + aisq);
    FLOPS(4);
    double c = 1.0 / sqrt(a0sq + b * b * aisq);
    FLOPS(4);
    double bc = b * c;
    FLOPS(1);
    r[0] = c * k[0];
    r[1] = bc * k[1];
    r[2] = bc * k[2];
    r[3] = bc * k[3];
    FLOPS(4);
    return 1;
}

/* U <- G U, G the subgroup (a,b) embedding of R: rows a, b mix (84 flop). */
static void rotate_rows(mat3 *u, int a, int b, cplx R[2][2])
{
    for (int c = 0; c < 3; ++c) {
        cplx ua = u->m[a][c], ub = u->m[b][c];
        u->m[a][c] = c_add(c_mul(R[0][0], ua), c_mul(R[0][1], ub));
        u->m[b][c] = c_add(c_mul(R[1][0], ua), c_mul(R[1][1], ub));
    }
}

/* U <- U G^dagger: columns a, b mix (84 flop). */
static void rotate_cols_dagger(mat3 *u, int a, int b, cplx R[2][2])
{
    cplx r00 = c_conj(R[0][0]), r01 = c_conj(R[0][1]);
    cplx r10 = c_conj(R[1][0]), r11 = c_conj(R[1][1]);
    for (int row = 0; row < 3; ++row) {
        cplx ua = u->m[row][a], ub = u->m[row][b];
        u->m[row][a] = c_add(c_mul(ua, r00), c_mul(ub, r01));
        u->m[row][b] = c_add(c_mul(ua, r10), c_mul(ub, r11));
    }
}

/*
 * The eight links touching site x: forward U_mu(x) and backward U_mu(x-mu).
 * nk = 4 for Landau gauge, 3 for Coulomb gauge (spatial directions in K).
 */
typedef struct { mat3 fwd[4], bwd[4]; } star;

static void star_load(const double *U, const lattice *g, long i, star *s)
{
    for (int mu = 0; mu < 4; ++mu) {
        s->fwd[mu] = mat_load(link_cptr(U, i, mu));
        s->bwd[mu] = mat_load(link_cptr(U, site_shift(g, i, mu, -1), mu));
    }
}

static void star_store(double *U, const lattice *g, long i, const star *s)
{
    for (int mu = 0; mu < 4; ++mu) {
        mat_store(link_ptr(U, i, mu), &s->fwd[mu]);
        mat_store(link_ptr(U, site_shift(g, i, mu, -1), mu), &s->bwd[mu]);
    }
}

/*
 * Quaternion of the subgroup (a,b) block of
 *     M(x) = sum_mu [ U_mu(x) + U_mu(x-mu)^dagger ]
 * i.e. of K(x) of eq. (Kx) with the current gauge transformation already
 * absorbed into the links (Alg. 1 first step, 60 flop for nk = 4:
 * 8 x 4 flop per link, 7 x 4 flop to sum).
 */
static void star_quaternion(const star *s, int nk, int a, int b, double k[4])
{
    double q[4];
    int first = 1;
    for (int mu = 0; mu < nk; ++mu) {
        const mat3 *f = &s->fwd[mu];
        block_quaternion(f->m[a][a], f->m[a][b], f->m[b][a], f->m[b][b], q);
        if (first) {
            memcpy(k, q, sizeof q);
            first = 0;
        } else {
            for (int c = 0; c < 4; ++c) k[c] += q[c];
            FLOPS(4);
        }
        /* block of U^dagger: (U^dagger)_{ab} = conj(U_{ba}) */
        const mat3 *w = &s->bwd[mu];
        block_quaternion(c_conj(w->m[a][a]), c_conj(w->m[b][a]), c_conj(w->m[a][b]),
                         c_conj(w->m[b][b]), q);
        for (int c = 0; c < 4; ++c) k[c] += q[c];
        FLOPS(4);
    }
}

static void star_rotate(star *s, int a, int b, cplx R[2][2])
{
    for (int mu = 0; mu < 4; ++mu) {
        rotate_rows(&s->fwd[mu], a, b, R);
        rotate_cols_dagger(&s->bwd[mu], a, b, R);
    }
}

/*
 * One overrelaxation update of one site: Alg. 1 inner body.  For every SU(2)
 * subgroup: assemble the projected K, apply the exponent omega and project to
 * SU(2), then U_mu(x) <- g U_mu(x) and U_mu(x-mu) <- U_mu(x-mu) g^dagger for
 * all four mu.
 */
static void or_update_star(star *s, int nk, double omega)
{
    for (int sg = 0; sg < 3; ++sg) {
        int a = SUBGROUP[sg][0], b = SUBGROUP[sg][1];
        double k[4], r[4];
        cplx R[2][2];
        star_quaternion(s, nk, a, b, k);
        if (!overrelax_quaternion(k, omega, r)) continue;
        su2_matrix(r, R);
        star_rotate(s, a, b, R);
    }
}

static int gauge_nk(int gauge) { return gauge == 1 ? 3 : 4; }

/*
 * One half-sweep over the sites of one parity (Alg. 1, FORALL x of
 * sublattice).  Sites of one parity share no link (Sec. 2, checkerboard), so
 * they are updated independently and in any order.
 */
int oracle_or_half_sweep(double *U, const int dims[4], int parity, double omega, int gauge)
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
    int nk = gauge_nk(gauge);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long i = 0; i < g.V; ++i) {
        if (site_parity(&g, i) != parity) continue;
        star s;
        star_load(U, &g, i, &s);
        or_update_star(&s, nk, omega);
        star_store(U, &g, i, &s);
    }
    return 0;
}

/* nsweeps full sweeps: RED (parity 0) then BLACK (parity 1), Alg. 1. */
int oracle_or_sweeps(double *U, const int dims[4], double omega, int gauge, int nsweeps)
{
    for (int n = 0; n < nsweeps; ++n)
        for (int p = 0; p < 2; ++p)
            if (oracle_or_half_sweep(U, dims, p, omega, gauge)) return -1;
    return 0;
}

/*
 * The eight updated links of selected sites after one OR update of each,
 * computed from the unmodified field U (read only).  out holds, per site,
 * U_0..3(x) then U_0..3(x-mu), 18 doubles each.  Used to check a
 * half-sweep on a large lattice site by site.
 */
int oracle_or_update_sites(const double *U, const int dims[4], const long *sites, long n,
                           double omega, int gauge, double *out)
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
    int nk = gauge_nk(gauge);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long j = 0; j < n; ++j) {
        star s;
        star_load(U, &g, sites[j], &s);
        or_update_star(&s, nk, omega);
        for (int mu = 0; mu < 4; ++mu) {
            mat_store(out + (j * 8 + mu) * 18, &s.fwd[mu]);
            mat_store(out + (j * 8 + 4 + mu) * 18, &s.bwd[mu]);
        }
    }
    return 0;
}

/* Single-site helpers exposed for the pinning tests. */
void oracle_block_quaternion(const double w[8], double k[4])
{
    block_quaternion(c_make(w[0], w[1]), c_make(w[2], w[3]), c_make(w[4], w[5]),
                     c_make(w[6], w[7]), k);
}

int oracle_overrelax_quaternion(const double k[4], double omega, double r[4])
{
    return overrelax_quaternion(k, omega, r);
}

/* quaternion k of subgroup (a,b) of M(x) at site i, from the field U */
int oracle_site_quaternion(const double *U, const int dims[4], long i, int gauge, int sg,
                           double k[4])
{
    lattice g;
    if (lattice_init(&g, dims) || sg < 0 || sg > 2) return -1;
    star s;
    star_load(U, &g, i, &s);
    star_quaternion(&s, gauge_nk(gauge), SUBGROUP[sg][0], SUBGROUP[sg][1], k);
    return 0;
}

/*
 * Apply one SU(2) subgroup rotation r (quaternion) at site i:
 * U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dagger for all mu.
 */
int oracle_site_rotate(double *U, const int dims[4], long i, int sg, const double r[4])
{
    lattice g;
    if (lattice_init(&g, dims) || sg < 0 || sg > 2) return -1;
    star s;
    cplx R[2][2];
    star_load(U, &g, i, &s);
    su2_matrix(r, R);
    star_rotate(&s, SUBGROUP[sg][0], SUBGROUP[sg][1], R);
    star_store(U, &g, i, &s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* gauge functional F (eq. F_g[U]) and precision theta (eq. theta)           */
/* ------------------------------------------------------------------------ */

/* F = 1/(3 nk V) sum_{x, mu < nk} Re tr U_mu(x). */
double oracle_functional(const double *U, const int dims[4], int gauge)
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    int nk = gauge_nk(gauge);
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i)
        for (int mu = 0; mu < nk; ++mu) {
            mat3 u = mat_load(link_cptr(U, i, mu));
            sum += mat_retrace(&u);
        }
    return sum / (3.0 * nk * (double)g.V);
}

/* A = (U - U^dagger)/(2i) */
static mat3 antiherm_part(const mat3 *u)
{
    mat3 A;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cplx z = c_sub(u->m[a][b], c_conj(u->m[b][a]));
            A.m[a][b] = c_make(0.5 * z.im, -0.5 * z.re); /* z / (2i) */
        }
    return A;
}

static void make_traceless(mat3 *A)
{
    cplx tr = c_make(0.0, 0.0);
    for (int a = 0; a < 3; ++a) tr = c_add(tr, A->m[a][a]);
    for (int a = 0; a < 3; ++a) A->m[a][a] = c_sub(A->m[a][a], c_make(tr.re / 3.0, tr.im / 3.0));
}

static double frob2(const mat3 *A)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += c_abs2(A->m[a][b]);
    return s;
}

/*
 * theta = 1/(Nc V) sum_x tr[Delta(x) Delta(x)^dagger] with
 * Delta(x) = traceless part of sum_{mu<nk} [A_mu(x) - A_mu(x-mu)].
 * This is the lattice divergence of the gauge field.
 */
double oracle_theta(const double *U, const int dims[4], int gauge)
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    int nk = gauge_nk(gauge);
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i) {
        mat3 D;
        memset(&D, 0, sizeof D);
        for (int mu = 0; mu < nk; ++mu) {
            mat3 uf = mat_load(link_cptr(U, i, mu));
            mat3 ub = mat_load(link_cptr(U, site_shift(&g, i, mu, -1), mu));
            mat3 Af = antiherm_part(&uf), Ab = antiherm_part(&ub);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    D.m[a][b] = c_add(D.m[a][b], c_sub(Af.m[a][b], Ab.m[a][b]));
        }
        make_traceless(&D);
        sum += frob2(&D);
    }
    return sum / (3.0 * (double)g.V);
}

/*
 * F and theta of every timeslice t (the sites with time coordinate t; for
 * Coulomb gauge each timeslice is gauge fixed on its own, Sec. 2):
 * F_t = 1/(3 nk Ls) sum_{x in t, mu < nk} Re tr U_mu(x),
 * theta_t = 1/(3 Ls) sum_{x in t} tr Delta(x) Delta(x)^dagger, Ls = Lx Ly Lz.
 * The means over t are F and theta.
 */
int oracle_timeslices(const double *U, const int dims[4], int gauge, double *F_t, double *theta_t)
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
    int nk = gauge_nk(gauge);
    long Ls = (long)g.L[0] * g.L[1] * g.L[2];
    for (int t = 0; t < g.L[3]; ++t) {
        double fs = 0.0, ts = 0.0;
        for (long i = t * Ls; i < (t + 1) * Ls; ++i) {
            mat3 D;
            memset(&D, 0, sizeof D);
            for (int mu = 0; mu < nk; ++mu) {
                mat3 uf = mat_load(link_cptr(U, i, mu));
                mat3 ub = mat_load(link_cptr(U, site_shift(&g, i, mu, -1), mu));
                fs += mat_retrace(&uf);
                mat3 Af = antiherm_part(&uf), Ab = antiherm_part(&ub);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        D.m[a][b] = c_add(D.m[a][b], c_sub(Af.m[a][b], Ab.m[a][b]));
            }
            make_traceless(&D);
            ts += frob2(&D);
        }
        F_t[t] = fs / (3.0 * nk * (double)Ls);
        theta_t[t] = ts / (3.0 * (double)Ls);
    }
    return 0;
}

/*
 * The same theta through the local matrix of the update:
 * Delta(x) = traceless part of (M(x) - M(x)^dagger)/(2i),
 * M(x) = sum_mu [U_mu(x) + U_mu(x-mu)^dagger].  A second, independent route
 * used to pin oracle_theta.
 */
double oracle_theta_from_M(const double *U, const int dims[4], int gauge)
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    int nk = gauge_nk(gauge);
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i) {
        mat3 M;
        memset(&M, 0, sizeof M);
        for (int mu = 0; mu < nk; ++mu) {
            mat3 uf = mat_load(link_cptr(U, i, mu));
            mat3 ub = mat_load(link_cptr(U, site_shift(&g, i, mu, -1), mu));
            mat3 ubd = mat_dagger(&ub);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    M.m[a][b] = c_add(M.m[a][b], c_add(uf.m[a][b], ubd.m[a][b]));
        }
        mat3 D = antiherm_part(&M);
        make_traceless(&D);
        sum += frob2(&D);
    }
    return sum / (3.0 * (double)g.V);
}

/* average plaquette, 1/(18 V) sum_{x, mu<nu} Re tr[U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+] */
double oracle_plaquette(const double *U, const int dims[4])
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                mat3 a = mat_load(link_cptr(U, i, mu));
                mat3 b = mat_load(link_cptr(U, site_shift(&g, i, mu, +1), nu));
                mat3 c = mat_load(link_cptr(U, site_shift(&g, i, nu, +1), mu));
                mat3 d = mat_load(link_cptr(U, i, nu));
                mat3 cd = mat_dagger(&c), dd = mat_dagger(&d);
                mat3 ab = mat_mul(&a, &b);
                mat3 abc = mat_mul(&ab, &cd);
                mat3 p = mat_mul(&abc, &dd);
                sum += mat_retrace(&p);
            }
    return sum / (18.0 * (double)g.V);
}

/* ------------------------------------------------------------------------ */
/* gauge transformation (eq. 1) and reunitarisation                           */
/* ------------------------------------------------------------------------ */

/* U_mu(x) <- g(x) U_mu(x) g(x+mu)^dagger for all x, mu; g[V][3][3][2]. */
int oracle_gauge_transform(double *U, const double *gfield, const int dims[4])
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long i = 0; i < g.V; ++i) {
        mat3 gx = mat_load(gfield + i * 18);
        for (int mu = 0; mu < 4; ++mu) {
            mat3 gy = mat_load(gfield + site_shift(&g, i, mu, +1) * 18);
            mat3 gyd = mat_dagger(&gy);
            mat3 u = mat_load(link_cptr(U, i, mu));
            mat3 t = mat_mul(&gx, &u);
            mat3 r = mat_mul(&t, &gyd);
            mat_store(link_ptr(U, i, mu), &r);
        }
    }
    return 0;
}

/*
 * Project n 3x3 matrices back onto SU(3): Gram-Schmidt on rows 0 and 1, then
 * row 2 = conj(row0 x row1), which makes the determinant 1.
 */
void oracle_reunitarize(double *M, long n)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long j = 0; j < n; ++j) {
        mat3 u = mat_load(M + j * 18);
        double n0 = 0.0;
        for (int c = 0; c < 3; ++c) n0 += c_abs2(u.m[0][c]);
        n0 = 1.0 / sqrt(n0);
        for (int c = 0; c < 3; ++c) u.m[0][c] = c_make(u.m[0][c].re * n0, u.m[0][c].im * n0);
        cplx ip = c_make(0.0, 0.0); /* <row0, row1> */
        for (int c = 0; c < 3; ++c) ip = c_add(ip, c_mul(c_conj(u.m[0][c]), u.m[1][c]));
        for (int c = 0; c < 3; ++c) u.m[1][c] = c_sub(u.m[1][c], c_mul(ip, u.m[0][c]));
        double n1 = 0.0;
        for (int c = 0; c < 3; ++c) n1 += c_abs2(u.m[1][c]);
        n1 = 1.0 / sqrt(n1);
        for (int c = 0; c < 3; ++c) u.m[1][c] = c_make(u.m[1][c].re * n1, u.m[1][c].im * n1);
        for (int c = 0; c < 3; ++c) {
            int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            cplx x = c_sub(c_mul(u.m[0][c1], u.m[1][c2]), c_mul(u.m[0][c2], u.m[1][c1]));
            u.m[2][c] = c_conj(x);
        }
        mat_store(M + j * 18, &u);
    }
}

/* ------------------------------------------------------------------------ */
/* host convergence loop (Alg. 1 WHILE; Sec. 4.1: check every N iterations)  */
/* ------------------------------------------------------------------------ */

/*
 * Sweep until theta < theta_target, checking theta before the first sweep and
 * then after every check_every sweeps, at most max_iter sweeps.  Returns 0 if
 * converged, 1 if max_iter was reached, -1 on bad arguments.
 */
int oracle_overrelax(double *U, const int dims[4], int gauge, double omega, double theta_target,
                     int max_iter, int check_every, int *iters_out, double *F_out,
                     double *theta_out)
{
    lattice g;
    if (lattice_init(&g, dims) || check_every < 1 || max_iter < 0) return -1;
    int it = 0;
    double th = oracle_theta(U, dims, gauge);
    while (!(th < theta_target) && it < max_iter) {
        int n = check_every;
        if (n > max_iter - it) n = max_iter - it;
        oracle_or_sweeps(U, dims, omega, gauge, n);
        it += n;
        th = oracle_theta(U, dims, gauge);
    }
    if (iters_out) *iters_out = it;
    if (F_out) *F_out = oracle_functional(U, dims, gauge);
    if (theta_out) *theta_out = th;
    return th < theta_target ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11)                     */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = { ctr[0], ctr[1], ctr[2], ctr[3] };
    uint32_t k[2] = { key[0], key[1] };
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* open-interval uniform (0,1) from one 32-bit word: (w + 1/2) / 2^32 */
static double u01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------------ */
/* simulated annealing: SU(2)-subgroup heatbath on exp(Re tr[g K] / T)       */
/* (Sec. 1, simulated annealing as a preconditioner)                         */
/* ------------------------------------------------------------------------ */
#define SA_TAG 1u
#define SA_DIRECTION_DRAW 255u
#define SA_ALPHA_SWITCH 2.0

/*
 * Draw s0 in [-1,1] with density sqrt(1 - s0^2) exp(alpha s0), the
 * distribution of the real part of an SU(2) element under the Haar measure
 * weighted by exp(alpha s0).  alpha < 2: Creutz (1980), inverse-CDF draw of
 * exp(alpha s0) accepted with probability sqrt(1 - s0^2).  alpha >= 2:
 * Kennedy and Pendleton (1985), s0 = 1 - 2 lambda^2 with lambda^2 drawn from
 * lambda^2 exp(-2 alpha lambda^2) and accepted with probability
 * sqrt(1 - lambda^2).  Attempt a uses Philox counter (site, sweep,
 * sg * 256 + a, 1).  Returns 1 on success, 0 after cap rejections.
 */
static int heatbath_s0(double alpha, uint32_t site, uint32_t sweep, int sg, int cap,
                       const uint32_t key[2], uint32_t tag, double *s0_out)
{
    for (int a = 0; a < cap && a < (int)SA_DIRECTION_DRAW; ++a) {
        uint32_t ctr[4] = { site, sweep, (uint32_t)sg * 256u + (uint32_t)a, tag };
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        if (alpha < SA_ALPHA_SWITCH) {
            double u = u01(w[0]);
            double e = exp(-2.0 * alpha);
            double s0 = 1.0 + log(e + u * (1.0 - e)) / alpha;
            double v = u01(w[1]);
            if (v <= sqrt(1.0 - s0 * s0)) {
                *s0_out = s0;
                return 1;
            }
        } else {
            double c = cos(ORACLE_TWO_PI * u01(w[1]));
            double lam2 = -(log(u01(w[0])) + c * c * log(u01(w[2]))) / (2.0 * alpha);
            double v = u01(w[3]);
            if (v * v <= 1.0 - lam2) {
                *s0_out = 1.0 - 2.0 * lam2;
                return 1;
            }
        }
    }
    return 0;
}

/*
 * The FP32 reading of the same draw (oracle_set_sa_draw(1); annealing only,
 * the Wilson-action generation keeps FP64).  A preconditioner does not need
 * the draw's precision, and FP32 transcendental functions are far cheaper on
 * the GPU than FP64 ones, so the reading is stated here as its own
 * definition: alpha = |k|/T is computed in FP64 and rounded once to FP32;
 * uniforms are ((w >> 9) + 1/2) / 2^23 (exact in FP32, open interval); every
 * later operation -- expf, logf, cosf, sinf, sqrtf, products, sums, the
 * divisions, the accept/reject comparisons -- is one FP32 operation in the
 * order written; the four components of the drawn SU(2) element are then
 * widened to FP64 and normalised in FP64 before the product with k/|k|, so
 * that the rotation is unitary to FP64 rounding.
 */
static int g_sa_draw_fp32 = 0;

int oracle_set_sa_draw(int fp32)
{
    if (fp32 != 0 && fp32 != 1) return -1;
    g_sa_draw_fp32 = fp32;
    return 0;
}

static float u01f(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }

#define ORACLE_TWO_PI_F 6.28318530717958647692f

static int heatbath_s0_f32(float alpha, uint32_t site, uint32_t sweep, int sg, int cap,
                           const uint32_t key[2], uint32_t tag, float *s0_out)
{
    for (int a = 0; a < cap && a < (int)SA_DIRECTION_DRAW; ++a) {
        uint32_t ctr[4] = { site, sweep, (uint32_t)sg * 256u + (uint32_t)a, tag };
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        if (alpha < (float)SA_ALPHA_SWITCH) {
            float u = u01f(w[0]);
            float e = expf(-2.0f * alpha);
            float s0 = 1.0f + logf(e + u * (1.0f - e)) / alpha;
            float v = u01f(w[1]);
            if (v <= sqrtf(1.0f - s0 * s0)) {
                *s0_out = s0;
                return 1;
            }
        } else {
            float c = cosf(ORACLE_TWO_PI_F * u01f(w[1]));
            float lam2 = -(logf(u01f(w[0])) + c * c * logf(u01f(w[2]))) / (2.0f * alpha);
            float v = u01f(w[3]);
            if (v * v <= 1.0f - lam2) {
                *s0_out = 1.0f - 2.0f * lam2;
                return 1;
            }
        }
    }
    return 0;
}

/* quaternion product q = a b, the product of the SU(2) matrices */
static void quat_mul(const double a[4], const double b[4], double q[4])
{
    q[0] = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    double cx = a[2] * b[3] - a[3] * b[2];
    double cy = a[3] * b[1] - a[1] * b[3];
    double cz = a[1] * b[2] - a[2] * b[1];
    q[1] = a[0] * b[1] + b[0] * a[1] - cx;
    q[2] = a[0] * b[2] + b[0] * a[2] - cy;
    q[3] = a[0] * b[3] + b[0] * a[3] - cz;
}

/*
 * Heatbath choice of the subgroup element: r = s k/|k| with s drawn from
 * exp(alpha s0) dHaar(s), alpha = |k|/T, so that r has density
 * proportional to exp(Re tr[r w]/T) = exp(r.k/T).  The direction of the
 * imaginary part of s is uniform on the sphere, from Philox counter
 * (site, sweep, sg * 256 + 255, 1).
 */
static int heatbath_quaternion_tag(const double k[4], double T, uint32_t site, uint32_t sweep, int sg,
                                   int cap, const uint32_t key[2], uint32_t tag, double r[4])
{
    double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
    if (kn == 0.0) return 2; /* nothing to do */
    if (g_sa_draw_fp32 && tag == SA_TAG) {
        float s0f;
        if (!heatbath_s0_f32((float)(kn / T), site, sweep, sg, cap, key, tag, &s0f)) return 0;
        uint32_t ctr[4] = { site, sweep, (uint32_t)sg * 256u + SA_DIRECTION_DRAW, tag };
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        float ct = 2.0f * u01f(w[0]) - 1.0f;
        float phi = ORACLE_TWO_PI_F * u01f(w[1]);
        float st = sqrtf(1.0f - ct * ct);
        float rho = sqrtf(1.0f - s0f * s0f);
        double s[4] = { (double)s0f, (double)(rho * st * cosf(phi)), (double)(rho * st * sinf(phi)),
                        (double)(rho * ct) };
        double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
        for (int c = 0; c < 4; ++c) s[c] /= sn;
        double kh[4] = { k[0] / kn, k[1] / kn, k[2] / kn, k[3] / kn };
        quat_mul(s, kh, r);
        return 1;
    }
    double s0;
    if (!heatbath_s0(kn / T, site, sweep, sg, cap, key, tag, &s0)) return 0;
    uint32_t ctr[4] = { site, sweep, (uint32_t)sg * 256u + SA_DIRECTION_DRAW, tag };
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    double ct = 2.0 * u01(w[0]) - 1.0;
    double phi = ORACLE_TWO_PI * u01(w[1]);
    double st = sqrt(1.0 - ct * ct);
    double rho = sqrt(1.0 - s0 * s0);
    double s[4] = { s0, rho * st * cos(phi), rho * st * sin(phi), rho * ct };
    double kh[4] = { k[0] / kn, k[1] / kn, k[2] / kn, k[3] / kn };
    quat_mul(s, kh, r);
    return 1;
}

static int heatbath_quaternion(const double k[4], double T, uint32_t site, uint32_t sweep, int sg,
                               int cap, const uint32_t key[2], double r[4])
{
    return heatbath_quaternion_tag(k, T, site, sweep, sg, cap, key, SA_TAG, r);
}

int oracle_heatbath_quaternion(const double k[4], double T, uint32_t site, uint32_t sweep, int sg,
                               int cap, uint64_t seed, double r[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    return heatbath_quaternion(k, T, site, sweep, sg, cap, key, r);
}

static int sa_update_star(star *s, int nk, double T, uint32_t site, uint32_t sweep, int cap,
                          const uint32_t key[2])
{
    int ok = 1;
    for (int sg = 0; sg < 3; ++sg) {
        int a = SUBGROUP[sg][0], b = SUBGROUP[sg][1];
        double k[4], r[4];
        cplx R[2][2];
        star_quaternion(s, nk, a, b, k);
        int st = heatbath_quaternion(k, T, site, sweep, sg, cap, key, r);
        if (st == 0) ok = 0;
        if (st != 1) continue;
        su2_matrix(r, R);
        star_rotate(s, a, b, R);
    }
    return ok;
}

/*
 * One heatbath half-sweep at temperature T over the sites of one parity.
 * Returns the number of subgroup draws that hit the rejection cap (those
 * subgroups are left unchanged), or -1 on bad arguments.
 */
long oracle_sa_half_sweep(double *U, const int dims[4], int parity, double T, int gauge,
                          uint64_t seed, uint32_t sweep, int cap)
{
    lattice g;
    if (lattice_init(&g, dims) || !(T > 0.0) || cap < 1) return -1;
    int nk = gauge_nk(gauge);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    long failures = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : failures)
#endif
    for (long i = 0; i < g.V; ++i) {
        if (site_parity(&g, i) != parity) continue;
        star s;
        star_load(U, &g, i, &s);
        if (!sa_update_star(&s, nk, T, (uint32_t)i, sweep, cap, key)) failures += 1;
        star_store(U, &g, i, &s);
    }
    return failures;
}

/*
 * Simulated annealing: steps heatbath sweeps with T falling linearly from T0
 * to T1, T_k = T0 + (T1 - T0) k / (steps - 1); sweep k uses Philox sweep
 * counter sweep_offset + k.
 */
long oracle_anneal(double *U, const int dims[4], int gauge, double T0, double T1, int steps,
                   uint64_t seed, uint32_t sweep_offset, int cap)
{
    long failures = 0;
    for (int k = 0; k < steps; ++k) {
        double T = steps > 1 ? T0 + (T1 - T0) * (double)k / (double)(steps - 1) : T0;
        for (int p = 0; p < 2; ++p) {
            long f = oracle_sa_half_sweep(U, dims, p, T, gauge, seed, sweep_offset + (uint32_t)k, cap);
            if (f < 0) return -1;
            failures += f;
        }
    }
    return failures;
}

/* per-site heatbath updates of selected sites from an unmodified field */
int oracle_sa_update_sites(const double *U, const int dims[4], const long *sites, long n, double T,
                           int gauge, uint64_t seed, uint32_t sweep, int cap, double *out)
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
    int nk = gauge_nk(gauge);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long j = 0; j < n; ++j) {
        star s;
        star_load(U, &g, sites[j], &s);
        sa_update_star(&s, nk, T, (uint32_t)sites[j], sweep, cap, key);
        for (int mu = 0; mu < 4; ++mu) {
            mat_store(out + (j * 8 + mu) * 18, &s.fwd[mu]);
            mat_store(out + (j * 8 + 4 + mu) * 18, &s.bwd[mu]);
        }
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* learned warm start: network inputs, exp map, algebra coefficients         */
/* ------------------------------------------------------------------------ */

/* Gell-Mann matrices lambda_1..8, tr(lambda_a lambda_b) = 2 delta_ab */
static mat3 gell_mann(int a)
{
    mat3 L;
    memset(&L, 0, sizeof L);
    const double r3 = 1.0 / sqrt(3.0);
    switch (a) {
    case 0: L.m[0][1] = c_make(1, 0); L.m[1][0] = c_make(1, 0); break;
    case 1: L.m[0][1] = c_make(0, -1); L.m[1][0] = c_make(0, 1); break;
    case 2: L.m[0][0] = c_make(1, 0); L.m[1][1] = c_make(-1, 0); break;
    case 3: L.m[0][2] = c_make(1, 0); L.m[2][0] = c_make(1, 0); break;
    case 4: L.m[0][2] = c_make(0, -1); L.m[2][0] = c_make(0, 1); break;
    case 5: L.m[1][2] = c_make(1, 0); L.m[2][1] = c_make(1, 0); break;
    case 6: L.m[1][2] = c_make(0, -1); L.m[2][1] = c_make(0, 1); break;
    default:
        L.m[0][0] = c_make(r3, 0);
        L.m[1][1] = c_make(r3, 0);
        L.m[2][2] = c_make(-2 * r3, 0);
    }
    return L;
}

/* Re tr(lambda_a X) */
static double re_tr_lambda(int a, const mat3 *X)
{
    mat3 L = gell_mann(a);
    mat3 P = mat_mul(&L, X);
    return mat_retrace(&P);
}

/*
 * Network inputs of the learned warm start, per site (channels last, 80 per
 * site): the 72 reals of the four forward links U_mu(x) (row-major, re/im),
 * then tr(lambda_a Delta(x)) / scale for a = 1..8, with Delta(x) the
 * traceless part of (M - M^dagger)/(2i), M = sum_mu [U_mu(x) + U_mu(x-mu)^+]
 * (Landau), i.e. the gauge-fixing violation of eq. theta.
 */
int oracle_features(const double *U, const int dims[4], double scale, double *f)
{
    lattice g;
    if (lattice_init(&g, dims) || !(scale > 0)) return -1;
    for (long i = 0; i < g.V; ++i) {
        double *o = f + i * 80;
        mat3 M;
        memset(&M, 0, sizeof M);
        for (int mu = 0; mu < 4; ++mu) {
            const double *p = link_cptr(U, i, mu);
            for (int r = 0; r < 18; ++r) o[mu * 18 + r] = p[r];
            mat3 uf = mat_load(p);
            mat3 ub = mat_load(link_cptr(U, site_shift(&g, i, mu, -1), mu));
            mat3 ubd = mat_dagger(&ub);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M.m[a][b] = c_add(M.m[a][b], c_add(uf.m[a][b], ubd.m[a][b]));
        }
        mat3 D = antiherm_part(&M);
        make_traceless(&D);
        for (int a = 0; a < 8; ++a) o[72 + a] = re_tr_lambda(a, &D) / scale;
    }
    return 0;
}

/*
 * g = exp(i H), H = scale * sum_a c_a lambda_a / 2, for n sets of 8
 * coefficients.  Taylor series of order 12 after halving H until its
 * Frobenius norm is below 1/8, then repeated squaring (Moler and Van Loan,
 * "scaling and squaring").
 */
void oracle_expmap(const double *c, double scale, double *gout, long n)
{
    for (long j = 0; j < n; ++j) {
        mat3 H;
        memset(&H, 0, sizeof H);
        for (int a = 0; a < 8; ++a) {
            mat3 L = gell_mann(a);
            double w = 0.5 * scale * c[j * 8 + a];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y)
                    H.m[x][y] = c_add(H.m[x][y], c_make(w * L.m[x][y].re, w * L.m[x][y].im));
        }
        double nrm = sqrt(frob2(&H));
        int sq = 0;
        while (nrm > 0.125) {
            nrm *= 0.5;
            ++sq;
        }
        double s = ldexp(1.0, -sq);
        mat3 A; /* A = i H s */
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) A.m[x][y] = c_make(-H.m[x][y].im * s, H.m[x][y].re * s);
        mat3 E, T;
        memset(&E, 0, sizeof E);
        for (int x = 0; x < 3; ++x) E.m[x][x] = c_make(1, 0);
        T = E;
        for (int k = 1; k <= 12; ++k) {
            mat3 P = mat_mul(&T, &A);
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) T.m[x][y] = c_make(P.m[x][y].re / k, P.m[x][y].im / k);
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) E.m[x][y] = c_add(E.m[x][y], T.m[x][y]);
        }
        for (int k = 0; k < sq; ++k) E = mat_mul(&E, &E);
        mat_store(gout + j * 18, &E);
    }
}

/* c_a = tr(lambda_a (g - g^+)/(2i)) / scale: the algebra coefficients of
 * log g to first order (exact up to O(|log g|^3)). */
void oracle_algebra_log(const double *gin, double scale, double *c, long n)
{
    for (long j = 0; j < n; ++j) {
        mat3 gm = mat_load(gin + j * 18);
        mat3 A = antiherm_part(&gm);
        for (int a = 0; a < 8; ++a) c[j * 8 + a] = re_tr_lambda(a, &A) / scale;
    }
}

/* ------------------------------------------------------------------------ */
/* stochastic relaxation (Sec. 1; de Forcrand's relaxation against critical  */
/* slowing down): per subgroup the maximiser r* = k/|k| is used with         */
/* probability 1 - p and its square r*^2 with probability p.  r*^2 reflects  */
/* the current element through the maximum: it leaves Re tr[g K] of the      */
/* subgroup unchanged ("microcanonical").  The draw per (site, subgroup) is  */
/* the first word of Philox counter (site, sweep, 256 * subgroup, 2).        */
/* ------------------------------------------------------------------------ */
#define SR_TAG 2u

static int sr_quaternion(const double k[4], double p, uint32_t site, uint32_t sweep, int sg, const uint32_t key[2],
                         double r[4])
{
    double n2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    if (n2 == 0.0) return 0;
    double inv = 1.0 / sqrt(n2);
    for (int c = 0; c < 4; ++c) r[c] = k[c] * inv;
    uint32_t ctr[4] = { site, sweep, (uint32_t)sg * 256u, SR_TAG };
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    if (u01(w[0]) < p) { /* r <- r r (quaternion square) */
        double r0 = r[0];
        r[0] = 2.0 * r0 * r0 - 1.0;
        r[1] = 2.0 * r0 * r[1];
        r[2] = 2.0 * r0 * r[2];
        r[3] = 2.0 * r0 * r[3];
    }
    return 1;
}

int oracle_sr_half_sweep(double *U, const int dims[4], int parity, double p, int gauge, uint64_t seed,
                         uint32_t sweep)
{
    lattice g;
    if (lattice_init(&g, dims) || !(p >= 0.0 && p <= 1.0)) return -1;
    int nk = gauge_nk(gauge);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long i = 0; i < g.V; ++i) {
        if (site_parity(&g, i) != parity) continue;
        star s;
        star_load(U, &g, i, &s);
        for (int sg = 0; sg < 3; ++sg) {
            int a = SUBGROUP[sg][0], b = SUBGROUP[sg][1];
            double k[4], r[4];
            cplx R[2][2];
            star_quaternion(&s, nk, a, b, k);
            if (!sr_quaternion(k, p, (uint32_t)i, sweep, sg, key, r)) continue;
            su2_matrix(r, R);
            star_rotate(&s, a, b, R);
        }
        star_store(U, &g, i, &s);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Maximally Abelian gauge (named in Sec. 6 as the next application of the  */
/* method; the functional is the one of the gauge-fixing literature)        */
/* ------------------------------------------------------------------------ */
/*
 * F_MAG = 1/(3 Nd V) sum_{x, mu} sum_i |U_mu(x)_ii|^2   (Nd = 4; 1 for diagonal links)
 *
 * Local step at site x, subgroup (a,b), element R(r) = r0 + i r.sigma: the
 * site's part of F_MAG after U_mu(x) <- R U_mu(x), U_mu(x-mu) <- U_mu(x-mu) R^+
 * is a quadratic form q(r) = r^T A r in the quaternion r (R is linear in r).
 * A is read off q by polarisation; the maximiser over unit r is an eigenvector
 * of the largest eigenvalue (Jacobi rotations).  That eigenvalue is at least
 * two-fold: F_MAG does not change under the diagonal U(1) of the subgroup,
 * so among the maximisers the one closest to the identity (largest r0) is
 * taken.  The overrelaxation exponent is then applied to it as for Landau
 * gauge (overrelax_quaternion with k = r).
 */
static double diag_sq(const mat3 *u, int a, int b)
{
    return c_abs2(u->m[a][a]) + c_abs2(u->m[b][b]);
}

/* q(r): the (a,b) diagonal weight of the star after the (unnormalised) rotation R(r) */
static double mag_local_value(const star *s, int a, int b, const double r[4])
{
    cplx R[2][2];
    su2_matrix(r, R);
    double q = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        mat3 f = s->fwd[mu], w = s->bwd[mu];
        rotate_rows(&f, a, b, R);
        rotate_cols_dagger(&w, a, b, R);
        q += diag_sq(&f, a, b) + diag_sq(&w, a, b);
    }
    return q;
}

static void mag_local_matrix(const star *s, int a, int b, double A[4][4])
{
    for (int k = 0; k < 4; ++k)
        for (int m = k; m < 4; ++m) {
            double p[4] = { 0, 0, 0, 0 }, n[4] = { 0, 0, 0, 0 };
            p[k] += 1.0;
            p[m] += 1.0;
            n[k] += 1.0;
            n[m] -= 1.0;
            /* polarisation: A_km = (q(e_k + e_m) - q(e_k - e_m)) / 4 */
            A[k][m] = A[m][k] = 0.25 * (mag_local_value(s, a, b, p) - mag_local_value(s, a, b, n));
        }
}

/* eigen-decomposition of a symmetric 4x4 matrix by cyclic Jacobi rotations:
 * A <- V^T A V diagonal, columns of V the eigenvectors */
static void jacobi4(double A[4][4], double V[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                tot += A[i][j] * A[i][j];
                if (i != j) off += A[i][j] * A[i][j];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 4; ++k) { /* columns p, q */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) { /* rows p, q */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
}

/* The maximiser closest to the identity: e0 = (1,0,0,0) projected onto the
 * eigenspace of the largest eigenvalue (two-fold by the U(1) symmetry, four-
 * fold when A is a multiple of the identity).  When that eigenspace is
 * orthogonal to e0 (all maximisers have r0 = 0), e2 = (0,0,1,0) is projected
 * instead (beta real and positive).  Returns 0 when the result is the identity. */
static int mag_maximiser(double A[4][4], double r[4])
{
    double B[4][4], V[4][4];
    memcpy(B, A, sizeof B);
    jacobi4(B, V);
    double top = B[0][0];
    for (int i = 1; i < 4; ++i)
        if (B[i][i] > top) top = B[i][i];
    double scale = fabs(top) > 1.0 ? fabs(top) : 1.0;
    for (int target = 0; target < 2; ++target) {
        const int e = target == 0 ? 0 : 2;
        for (int c = 0; c < 4; ++c) r[c] = 0.0;
        for (int i = 0; i < 4; ++i)
            if (B[i][i] >= top - 1e-10 * scale)
                for (int c = 0; c < 4; ++c) r[c] += V[e][i] * V[c][i];
        double n = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
        if (n > 1e-12) {
            for (int c = 0; c < 4; ++c) r[c] /= n;
            return !(r[0] == 1.0 && r[1] == 0.0 && r[2] == 0.0 && r[3] == 0.0);
        }
    }
    r[0] = 1.0;
    r[1] = r[2] = r[3] = 0.0;
    return 0;
}

static void mag_update_star(star *s, double omega)
{
    for (int sg = 0; sg < 3; ++sg) {
        int a = SUBGROUP[sg][0], b = SUBGROUP[sg][1];
        double A[4][4], r[4], ro[4];
        cplx R[2][2];
        mag_local_matrix(s, a, b, A);
        if (!mag_maximiser(A, r)) continue;
        if (!overrelax_quaternion(r, omega, ro)) continue;
        su2_matrix(ro, R);
        star_rotate(s, a, b, R);
    }
}

int oracle_mag_half_sweep(double *U, const int dims[4], int parity, double omega)
{
    lattice g;
    if (lattice_init(&g, dims)) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long i = 0; i < g.V; ++i) {
        if (site_parity(&g, i) != parity) continue;
        star s;
        star_load(U, &g, i, &s);
        mag_update_star(&s, omega);
        star_store(U, &g, i, &s);
    }
    return 0;
}

double oracle_mag_functional(const double *U, const int dims[4])
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i)
        for (int mu = 0; mu < 4; ++mu) {
            mat3 u = mat_load(link_cptr(U, i, mu));
            for (int a = 0; a < 3; ++a) sum += c_abs2(u.m[a][a]);
        }
    return sum / (3.0 * 4.0 * (double)g.V);
}

/*
 * theta_MAG = 1/(3V) sum_x sum_{subgroups} (A_10^2 + A_20^2): the squared
 * gradient of the local functional at the identity along the two directions
 * that are not the residual U(1) (which has zero gradient); zero exactly at a
 * stationary point of every subgroup update.
 */
double oracle_mag_theta(const double *U, const int dims[4])
{
    lattice g;
    if (lattice_init(&g, dims)) return NAN;
    double sum = 0.0;
    for (long i = 0; i < g.V; ++i) {
        star s;
        star_load(U, &g, i, &s);
        for (int sg = 0; sg < 3; ++sg) {
            double A[4][4];
            mag_local_matrix(&s, SUBGROUP[sg][0], SUBGROUP[sg][1], A);
            sum += A[1][0] * A[1][0] + A[2][0] * A[2][0];
        }
    }
    return sum / (3.0 * (double)g.V);
}

/* the local matrix A of site i, subgroup sg (row-major 16 doubles), for the pins */
int oracle_mag_local_matrix(const double *U, const int dims[4], long i, int sg, double *A16)
{
    lattice g;
    if (lattice_init(&g, dims) || sg < 0 || sg > 2) return -1;
    star s;
    star_load(U, &g, i, &s);
    double A[4][4];
    mag_local_matrix(&s, SUBGROUP[sg][0], SUBGROUP[sg][1], A);
    memcpy(A16, A, sizeof A);
    return 0;
}

/* the maximiser of a given local matrix (closest to the identity) */
int oracle_mag_maximiser(const double *A16, double *r)
{
    double A[4][4];
    memcpy(A, A16, sizeof A);
    return mag_maximiser(A, r);
}

/* ------------------------------------------------------------------------ */
/* Gauge-field generation with the Wilson action (to give the gauge fixing  */
/* thermalised inputs like the paper's ensembles, Sec. 5)                   */
/* ------------------------------------------------------------------------ */
/*
 * S = beta sum_P (1 - Re tr U_P / 3).  The part of S that depends on the link
 * U = U_mu(x) is -(beta/3) Re tr(U A) with the staple sum
 *   A = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *                       + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ].
 * Cabibbo-Marinari: for each SU(2) subgroup the link is multiplied from the
 * left by R, and Re tr(R U A) = r.k with k the quaternion of the subgroup
 * block of W = U A; the heatbath draws r with weight exp((beta/3) r.k),
 * i.e. the SU(2) draw of the annealing at T = 3/beta, with Philox counter
 * (4 site + mu, sweep, 256 subgroup + draw, 3).  The overrelaxation step is
 * the microcanonical r = (k/|k|)^2, which leaves Re tr(U A) unchanged.
 * Links U_mu(x) of one direction and one parity share no staple, so they are
 * updated together.
 */
#define WILSON_TAG 3u

static mat3 staple_sum(const double *U, const lattice *g, long i, int mu)
{
    mat3 A;
    memset(&A, 0, sizeof A);
    long xp = site_shift(g, i, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long xn = site_shift(g, i, nu, +1), xm = site_shift(g, i, nu, -1);
        long xpm = site_shift(g, xp, nu, -1);
        /* upper staple U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
        mat3 a = mat_load(link_cptr(U, xp, nu));
        mat3 b = mat_load(link_cptr(U, xn, mu));
        mat3 c = mat_load(link_cptr(U, i, nu));
        mat3 bd = mat_dagger(&b), cd = mat_dagger(&c);
        mat3 t = mat_mul(&a, &bd);
        mat3 up = mat_mul(&t, &cd);
        /* lower staple U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) */
        mat3 d = mat_load(link_cptr(U, xpm, nu));
        mat3 e = mat_load(link_cptr(U, xm, mu));
        mat3 f = mat_load(link_cptr(U, xm, nu));
        mat3 dd = mat_dagger(&d), ed = mat_dagger(&e);
        mat3 t2 = mat_mul(&dd, &ed);
        mat3 lo = mat_mul(&t2, &f);
        for (int r = 0; r < 3; ++r)
            for (int c2 = 0; c2 < 3; ++c2) A.m[r][c2] = c_add(A.m[r][c2], c_add(up.m[r][c2], lo.m[r][c2]));
    }
    return A;
}

/* squared quaternion of the relaxation element: the microcanonical step */
static int micro_quaternion(const double k[4], double r[4])
{
    double n = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
    if (n == 0.0) return 0;
    double h[4] = { k[0] / n, k[1] / n, k[2] / n, k[3] / n };
    quat_mul(h, h, r);
    return 1;
}

/*
 * Update every link U_mu(x) with x of the given parity: mode 0 heatbath
 * (counter sweep), mode 1 overrelaxation.  Returns the number of heatbath
 * draws that hit the rejection cap (those subgroups are left unchanged), or
 * -1 on bad arguments.
 */
long oracle_wilson_update(double *U, const int dims[4], int mu, int parity, double beta, int mode,
                          uint64_t seed, uint32_t sweep, int cap)
{
    lattice g;
    if (lattice_init(&g, dims) || mu < 0 || mu > 3 || !(beta > 0.0) || cap < 1) return -1;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    long fails = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : fails)
#endif
    for (long i = 0; i < g.V; ++i) {
        if (site_parity(&g, i) != parity) continue;
        mat3 A = staple_sum(U, &g, i, mu);
        mat3 u = mat_load(link_cptr(U, i, mu));
        for (int sg = 0; sg < 3; ++sg) {
            int a = SUBGROUP[sg][0], b = SUBGROUP[sg][1];
            mat3 W = mat_mul(&u, &A);
            double k[4], r[4];
            block_quaternion(W.m[a][a], W.m[a][b], W.m[b][a], W.m[b][b], k);
            int st;
            if (mode == 0) {
                st = heatbath_quaternion_tag(k, 3.0 / beta, (uint32_t)(4 * i + mu), sweep, sg, cap, key,
                                             WILSON_TAG, r);
            } else {
                st = micro_quaternion(k, r);
            }
            if (mode == 0 && st == 0) ++fails;
            if (st != 1) continue;
            cplx R[2][2];
            su2_matrix(r, R);
            rotate_rows(&u, a, b, R);
        }
        mat_store(link_ptr(U, i, mu), &u);
    }
    return fails;
}

/* the staple sum A of link U_mu(x_i), for the pins (18 doubles) */
int oracle_staple(const double *U, const int dims[4], long i, int mu, double *out)
{
    lattice g;
    if (lattice_init(&g, dims) || mu < 0 || mu > 3) return -1;
    mat3 A = staple_sum(U, &g, i, mu);
    mat_store(out, &A);
    return 0;
}
