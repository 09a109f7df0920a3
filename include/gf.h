/*
 * gf.h -- C ABI of libgf.so: SU(3) lattice gauge fixing on one GB300 GPU by
 * checkerboard overrelaxation and simulated annealing.
 *
 * Method: Schroeck & Vogt, "Gauge fixing using overrelaxation and simulated
 * annealing on GPUs" (Lattice 2012).  Gauge fixing maximises the functional
 * F_g[U] = Re sum_{mu,x} tr[g(x) U_mu(x) g(x+mu)^dagger] (Sec. 2, eq. F_g)
 * over gauge transformations g(x) in SU(3); the overrelaxation algorithm
 * (Alg. 1) visits the sites of one checkerboard parity at a time and, for
 * each of the three SU(2) subgroups (Cabibbo-Marinari), rotates the 8 links
 * touching the site by the local maximiser raised to the power omega.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Field layout ("canonical"): double U[Lt][Lz][Ly][Lx][4][3][3][2], i.e. the
 *   site index runs x fastest, then the link direction mu = x, y, z, t, then
 *   the 3x3 complex matrix row-major, complex numbers as (re, im).
 *   dims = {Lx, Ly, Lz, Lt}; every extent must be even and >= 2 (the
 *   checkerboard needs it) and the volume below 2^31.  Boundaries are
 *   periodic.  Parity of a site is (x+y+z+t) mod 2; RED = 0 is swept first.
 * Pointers: a field argument may be device memory of the current device or
 *   host memory (pageable or pinned).  Host fields are copied in and out by
 *   the call; device fields are read (and, for in-place calls, written) on the
 *   context's stream.  Device memory of another device gives GF_EINVAL.
 *   The library never frees or keeps caller memory after a call returns.
 * Ownership: a gf_ctx owns its internal device buffers (the resident field in
 *   per-parity structure-of-arrays layout, reduction scratch, CUDA graphs);
 *   they are allocated on first use and freed by gf_destroy.
 * Streams: work is issued on the stream given by gf_set_stream (default: the
 *   legacy default stream).  Calls that return numbers synchronise that
 *   stream; the others are stream ordered.  A context is not thread safe.
 * Errors: every function returns GF_OK (0) or one of the codes below;
 *   gf_last_error returns a message for the most recent failure.
 * Normalisations: F is divided by Nc * Nd * V (Nd = 4 Landau, 3 Coulomb) so
 *   that the unit field has F = 1; theta (Sec. 2, eq. theta) is
 *   1/(Nc V) sum_x tr[Delta Delta^dagger] with Delta(x) the traceless part of
 *   sum_mu [A_mu(x) - A_mu(x-mu)], A = (U - U^dagger)/(2i), sum over the
 *   gauge's directions.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define GF_OK 0
#define GF_EINVAL 1         /* bad argument: odd/zero extent, omega outside (0,2), NULL, NaN */
#define GF_ECUDA 2          /* a CUDA runtime call failed (message in gf_last_error) */
#define GF_ETIMEOUT 3       /* a bounded device-side wait expired; the context stays usable */
#define GF_ENOTCONVERGED 4  /* max_iter reached before theta_target; outputs are valid */
#define GF_ENOMEM 5         /* device allocation failed */
#define GF_EREJECT 6        /* heatbath: some draws hit the rejection cap (left unchanged) */
#define GF_ESTATE 7         /* call needs a resident field and none is loaded */

/* gauges (Sec. 1: Landau d_mu A_mu = 0, Coulomb d_i A_i = 0; Sec. 6: the
 * maximally Abelian gauge, functional F = 1/(3 Nd V) sum_{x,mu} sum_i
 * |U_mu(x)_ii|^2, theta = 1/(3V) sum_x sum_subgroups |h12|^2, the squared
 * gradient of the local subgroup functional at the identity) */
#define GF_LANDAU 0
#define GF_COULOMB 1
#define GF_MAG 2

/* precision policy for gf_overrelax (option "precision") */
#define GF_FP64 0   /* FP64 storage and arithmetic throughout */
#define GF_MIXED 1  /* FP32 sweeps until theta < "theta_switch", then FP64 */
#define GF_FP32 2   /* FP32 storage and arithmetic; theta accumulated in FP64 */

typedef struct gf_ctx gf_ctx;

/* ---------------------------------------------------------------- context */

/* Create a context for a lattice of extents dims and the given gauge
 * (GF_LANDAU, GF_COULOMB or GF_MAG).  Allocates nothing on the device yet.
 * GF_MAG supports overrelaxation (gf_overrelax, gf_or_half_sweep,
 * gf_or_sweeps, gf_converge, all precision policies, per-subgroup site
 * update with 1-8 threads per site, native storage formats) and the
 * measurements; annealing, stochastic relaxation, double-float storage,
 * per-timeslice measurement and the learned warm start return GF_EINVAL.
 * *out receives the handle; release it with gf_destroy. */
int gf_create(const int dims[4], int gauge, gf_ctx **out);

/* Free the context and every device buffer it owns.  NULL is accepted. */
int gf_destroy(gf_ctx *ctx);

/* Message of the last failure on this context ("" if none).  The string
 * stays valid until the next call on the context. */
const char *gf_last_error(const gf_ctx *ctx);

/* Short name of a return code. */
const char *gf_error_string(int code);

/* Issue all work on stream (a cudaStream_t; NULL = legacy default stream). */
int gf_set_stream(gf_ctx *ctx, void *stream);

/* Options (numbers; unknown keys give GF_EINVAL):
 *   "precision"      GF_FP64 / GF_MIXED / GF_FP32 (default GF_FP64)
 *   "storage64"      18 or 12 reals per FP64 link (default 18; 12 stores two
 *                    rows and rebuilds the third from unitarity, Sec. 4.1)
 *   "storage32"      12 or 18 reals per FP32 link (default 12)
 *   "check_every"    sweeps between theta checks (default 100, Sec. 4.1)
 *   "theta_switch"   FP32 -> FP64 switch of GF_MIXED (default 1e-6)
 *   "track_gauge"    GF_MIXED: 1 = accumulate g(x) in the FP32 phase and
 *                    apply it to the caller's FP64 field at the switch, so
 *                    the result is a gauge transform of the exact input
 *                    (default 1); 0 = widen the FP32 links instead
 *   "reunitarize_every"  FP32 phase: reunitarise every n checks (default 1)
 *   "threads_per_site"   1, 2, 4 or 8; 0 = autotune (default 0)
 *   "variant"        site update: 1 = the three subgroup rotations applied to
 *                    the eight links held in registers (Alg. 1 literally,
 *                    1-8 threads per site), 2 = the same steps on M(x) =
 *                    sum of the links with G = R3 R2 R1 accumulated and applied
 *                    once per link (one thread per site; equal in exact
 *                    arithmetic), 0 = autotuned or default (default 0)
 *   "block"          threads per block (multiple of 32, <= 256; 0 = autotune)
 *   "learned_repeat" with an attached network (gf_set_net): apply it again,
 *                    up to this many times, each time theta has fallen by the
 *                    factor "learned_factor" (default 1e-2) during the FP64
 *                    phase (default 0: once, at the switch)
 *   "fp32_restarts"  GF_MIXED (track_gauge 1, reunitarize_every 1, else
 *                    gf_overrelax returns GF_EINVAL): after the switch, up to
 *                    n times (0..16, default 0), the FP32 field is re-encoded
 *                    from the FP64 field, g is reset to the identity, the FP32
 *                    sweeps run until theta (below 1e-8) falls by less than
 *                    10 % over 100 sweeps -- the FP32 rounding floor -- and g
 *                    is applied to the FP64 field in FP64; FP64 sweeps then
 *                    finish.  With n > 0 the first FP32 phase also stops at
 *                    that floor (a tiny "theta_switch", e.g. 1e-30, sweeps
 *                    it there).
 *                    The result stays a gauge transform of the exact input.
 *   "theta_per_timeslice"  1 = every theta the context reports or checks
 *                    (stopping rule, gf_overrelax's output, gf_measure) is the
 *                    largest timeslice value theta_t (gf_measure_timeslices),
 *                    so that every timeslice reaches the target (default 0)
 *   "or_variant"     reading of the exponent g -> g^omega (Sec. 2 leaves its
 *                    order open): 0 = the 19-flop rational form b =
 *                    (omega a0^2 + |a|^2)/(a0^2 + |a|^2), r = (a0, b a)/norm
 *                    (default; the count of Alg. 1), 1 = first order,
 *                    normalise((1 - omega) 1 + omega k/|k|), 2 = the exact
 *                    power (cos(omega phi), sin(omega phi) n); all equal
 *                    relaxation at omega = 1.  Batches use 0.
 *   "acc_registers"  accumulate form on FP64 storage: register budget per
 *                    thread, 255, 168 or 128 (0 = autotuned or 255; default 0)
 *   "autotune"       1 = time the candidate launch configurations (threads
 *                    per site, accumulate form and register budget, block)
 *                    of each storage format the first time a call sweeps it,
 *                    and cache the fastest per (extents, format, gauge,
 *                    overrelaxation or heatbath) for the process (default 0:
 *                    the fixed defaults, or "threads_per_site"/"block")
 *   "use_graphs"     1 = replay sweep loops as CUDA graphs (default 1)
 *   "kernel_timing"  1 = record CUDA events (inside the graphs) around the
 *                    sweep kernels of every check chunk of gf_overrelax and
 *                    report their time (default 0; creating the events may
 *                    fail with GF_ECUDA)
 *   "sa_cap"         heatbath rejection cap per draw (default 64, <= 255)
 *   "sa_draw"        heatbath draw of gf_anneal / gf_sa_half_sweep: 0 = FP64
 *                    throughout (default), 1 = the FP32 reading: alpha = |k|/T
 *                    rounded once to FP32, uniforms ((w >> 9) + 1/2) / 2^23,
 *                    the Creutz / Kennedy-Pendleton steps and the direction in
 *                    FP32 operations as written, the drawn element widened to
 *                    FP64 and normalised before the product with k/|k| (the
 *                    rotation stays unitary to FP64 rounding).  The decisions
 *                    follow the FP32 arithmetic; the library's FP32 exp, log,
 *                    cos and sin may differ from another implementation by an
 *                    ulp
 *   "sa_sweep_offset" Philox sweep counter of the first annealing sweep
 *   "stochastic_p"   > 0: gf_overrelax / gf_or_sweeps / gf_converge use
 *                    stochastic relaxation with this probability instead of
 *                    overrelaxation (omega unused; default 0)
 *   "sr_seed"        Philox key of those draws (resets their sweep counter)
 *   "fp64_arith"     FP64 phase and GF_FP64 policy: 0 = native FP64 (default),
 *                    1 = double-float values (pairs of FP32, 48-bit
 *                    significand, storage DF64_18) updated on the FP32 pipe;
 *                    per sweep within 1e-12 of FP64.  In gf_overrelax the
 *                    double-float sweeps run on a working copy of the FP64
 *                    field and track the gauge transformation they apply as
 *                    E = g - 1 in double-float; g = 1 + E (reunitarised in
 *                    FP64) is then applied to the FP64 field in FP64, so the
 *                    result is a gauge transform of the input to FP64
 *                    rounding; native FP64 sweeps finish if theta of that
 *                    field is not yet below the target.  With "stochastic_p"
 *                    > 0 the double-float field is used throughout instead
 *                    (stochastic sweeps do not track the transformation). */
int gf_set_option(gf_ctx *ctx, const char *key, double value);
int gf_get_option(const gf_ctx *ctx, const char *key, double *value);

/* Statistics of the last gf_overrelax / gf_anneal call:
 *   "sweeps", "sweeps_fp32", "sweeps_fp64", "checks", "ms_total",
 *   "ms_fp32", "ms_fp64", "threads_per_site", "block", "accumulate_form",
 *   "acc_registers", "sa_rejects";
 *   with "kernel_timing": "ms_sweep_kernels_fp32", "sweep_launches_fp32",
 *   "ms_sweep_kernels_fp64", "sweep_launches_fp64" (device time of the
 *   half-sweep kernels of each phase and the number of launches it covers);
 *   GF_MIXED: "theta_switch_measured" (theta of the FP64 field at the switch);
 *   with "fp64_arith" 1: "sweeps_df64" (double-float sweeps among "sweeps_fp64");
 *   with a network (gf_set_net): "theta_before_learned", "theta_after_learned"
 *   (around the first application), "ms_learned" (wall time of all
 *   applications), "learned_applications" (those after the first); with
 *   "fp32_restarts": "fp32_restarts_done", "theta_after_restarts" (theta of
 *   the FP64 field after the last restart), "ms_restarts". */
int gf_get_stat(const gf_ctx *ctx, const char *key, double *value);

/* ---------------------------------------------------- the method, one call */

/* Gauge-fix U in place by overrelaxation (Alg. 1; Sec. 2 overrelaxation with
 * exponent omega in (0, 2), omega = 1 is plain relaxation).  theta is
 * checked before the first sweep and every "check_every" sweeps (Sec. 4.1);
 * the call stops at the first check with theta < theta_target or after
 * max_iter sweeps.  U: canonical field, host or device, in/out.
 * Outputs (any may be NULL): sweeps done, final F, final theta.
 * Returns GF_OK when converged, GF_ENOTCONVERGED at max_iter. */
int gf_overrelax(gf_ctx *ctx, double *U, double omega, double theta_target, int max_iter,
                 int *iters_out, double *F_out, double *theta_out);

/* Simulated annealing (Sec. 1, as a preconditioner): steps heatbath sweeps
 * at temperatures T_k = T0 + (T1 - T0) k / (steps - 1).  Per site and SU(2)
 * subgroup the new subgroup element r is drawn with density proportional to
 * exp(Re tr[r K]/T) times the SU(2) Haar measure (Creutz for |k|/T < 2,
 * Kennedy-Pendleton otherwise) from Philox4x32-10 with key = seed and
 * counter = (lexicographic site, sweep_offset + k, 256 * subgroup + draw, 1).
 * With "fp64_arith" 1 (and a policy other than GF_FP32) the sweeps run in
 * double-float arithmetic on a copy of the FP64 field while the
 * transformation is tracked as E = g - 1, and g = 1 + E is applied to the
 * FP64 field in FP64 at the end: the annealed field stays a gauge transform
 * of the input to FP64 rounding.
 * U: canonical field, host or device, in/out.  Returns GF_EREJECT if some
 * draws hit "sa_cap" (those subgroups are left unchanged). */
int gf_anneal(gf_ctx *ctx, double *U, double T0, double T1, int steps, uint64_t seed);

/* F of a canonical field (host or device), FP64. */
int gf_functional(gf_ctx *ctx, const double *U, double *F_out);

/* theta of a canonical field (host or device), FP64. */
int gf_theta(gf_ctx *ctx, const double *U, double *theta_out);

/* average plaquette 1/(18 V) sum Re tr[U_mu U_nu U_mu^+ U_nu^+] (gauge
 * invariant; used to check that sweeps are gauge transformations). */
int gf_plaquette(gf_ctx *ctx, const double *U, double *P_out);

/* ----------------------------------------- resident field, explicit steps */

/* Copy a canonical field (host or device) into the context's resident field
 * in per-parity structure-of-arrays form (Sec. 4.1: RED and BLACK blocks,
 * site index fastest) at the precision given: GF_FP64 uses "storage64"
 * reals per link, GF_FP32 uses "storage32". */
int gf_upload(gf_ctx *ctx, const double *U, int precision);

/* Write the resident field back in canonical form (host or device).  A
 * 12-real field gets its third rows rebuilt in FP64. */
int gf_download(gf_ctx *ctx, double *U);

/* One OR half-sweep of the resident field over the sites of one parity
 * (Alg. 1 inner loops). */
int gf_or_half_sweep(gf_ctx *ctx, int parity, double omega);

/* nsweeps full OR sweeps (RED then BLACK) of the resident field, no checks;
 * replayed from a CUDA graph when "use_graphs" is set. */
int gf_or_sweeps(gf_ctx *ctx, double omega, int nsweeps);

/* One heatbath half-sweep of the resident field at temperature T with
 * Philox key seed and sweep counter sweep. */
int gf_sa_half_sweep(gf_ctx *ctx, int parity, double T, uint64_t seed, uint32_t sweep);

/* One stochastic-relaxation half-sweep (Sec. 1: relaxation against critical
 * slowing down): per subgroup the maximiser r* = k/|k| is applied, or with
 * probability p its square r*^2, which reflects the subgroup element through
 * the maximum and leaves Re tr[g K] unchanged.  The draw for (site, subgroup)
 * is the first word of Philox4x32-10 with key seed and counter
 * (lexicographic site, sweep, 256 * subgroup, 2), compared with p in FP64. */
int gf_sr_half_sweep(gf_ctx *ctx, int parity, double p, uint64_t seed, uint32_t sweep);

/* F and theta of the resident field (accumulated in FP64).  With the option
 * "theta_per_timeslice", theta_out is the largest theta_t (see below). */
int gf_measure(gf_ctx *ctx, double *F_out, double *theta_out);

/* F_t and theta_t of every timeslice t = 0..Lt-1 of the resident field
 * (Coulomb gauge fixes each timeslice on its own, Sec. 2):
 * F_t = 1/(3 nk Ls) sum_{x in t, mu < nk} Re tr U_mu(x), theta_t = 1/(3 Ls)
 * sum_{x in t} tr Delta Delta^dagger, Ls = Lx Ly Lz, nk = 3 (Coulomb) or 4;
 * their means over t are F and theta.  F_t, theta_t: Lt doubles each, host
 * or device, either may be NULL.  Synchronises the context's stream. */
int gf_measure_timeslices(gf_ctx *ctx, double *F_t, double *theta_t);

/* Project every resident link back onto SU(3) (Gram-Schmidt in FP64). */
int gf_reunitarize(gf_ctx *ctx);

/* Pick threads per site and block size for the resident field's storage by
 * timing every candidate on a scratch copy; the choice is cached per
 * (volume, storage, gauge) for the process.  Outputs may be NULL.
 * threads_per_site: 1, 2, 4, 8 = per-subgroup form with that many threads per
 * site; 0, -1, -2 = accumulate form, one thread per site, with at most 255,
 * 168 or 128 registers per thread (the budget of the last two is tried for
 * FP64 storage only). */
int gf_autotune(gf_ctx *ctx, int *threads_per_site, int *block);

/* ------------------------------------- Wilson-action gauge-field generation */

/* Thermalised inputs like the paper's ensembles (Sec. 5), S = beta sum_P
 * (1 - Re tr U_P / 3).  One update of every link U_mu(x), x of the given
 * parity, of the resident FP64 field (storage 18 or 12): mode 0 heatbath
 * (Cabibbo-Marinari on the SU(2) draw of gf_anneal at T = 3/beta, Philox
 * key seed, counter (4 x + mu, sweep, 256 subgroup + draw, 3)), mode 1
 * microcanonical overrelaxation (the squared relaxation element; the action
 * is unchanged).  Heatbath draws that hit "sa_cap" leave their subgroup
 * unchanged and are counted for the next gf_generate status. */
int gf_wilson_update(gf_ctx *ctx, int mu, int parity, double beta, int mode, uint64_t seed, uint32_t sweep);

/* n_sweeps compound sweeps on a canonical field U (host or device, in/out):
 * each one heatbath sweep (directions 0..3, parities 0, 1; counter sweep0 +
 * k) followed by n_or overrelaxation sweeps.  12-real storage is
 * reunitarised every 4 compound sweeps.  Returns GF_EREJECT if some draws hit
 * the rejection cap.  Stats: "sweeps", "or_sweeps", "sa_rejects",
 * "ms_total". */
int gf_generate(gf_ctx *ctx, double *U, double beta, int n_sweeps, int n_or, uint64_t seed, uint32_t sweep0);

/* --------------------------------------------------- learned warm start */

/* The learned warm start predicts, from the FP64 field at the FP32 -> FP64
 * switch of GF_MIXED, the gauge transformation that the remaining FP64
 * sweeps would apply, and applies it before they start; overrelaxation then
 * finishes as usual and decides convergence.
 *
 * Network inputs, per site (channels last, BF16): the 72 reals of the four
 * forward links U_mu(x), then tr(lambda_a Delta(x)) / s, a = 1..8, with
 * Delta(x) the gauge-fixing violation of eq. theta and s = sqrt(theta).
 * Output: 8 coefficients c_a(x); the applied transformation is
 * g(x) = exp(i s sum_a c_a(x) lambda_a / 2), an exact FP64 gauge
 * transformation of the field.  Sites are in lexicographic order.
 *
 * Network: four periodic 4D convolutions with 3^4 taps, channels
 * 80 -> 32 -> 32 -> 32 -> 8, ReLU between layers, BF16 weights and
 * activations, FP32 accumulation.  Parameters (FP32 master copy) are the
 * concatenation W1 b1 W2 b2 W3 b3 W4 b4 with W_l[81][C_out][C_in], tap
 * k = (dx+1) + 3(dy+1) + 9(dz+1) + 27(dt+1), Y[s][o] = b[o] +
 * sum_k sum_i W[k][o][i] X[s + d(k)][i].  Loss: mean squared error over all
 * sites and outputs.  Training uses Adam (beta 0.9 / 0.999, eps 1e-8). */
#define GF_NET_CIN 80
#define GF_NET_COUT 8
typedef struct gf_net gf_net;

size_t gf_net_param_count(void);
/* A network sized for lattices of extents dims (activations are kept). */
int gf_net_create(const int dims[4], gf_net **out);
int gf_net_destroy(gf_net *n);
const char *gf_net_last_error(const gf_net *n);
int gf_net_set_stream(gf_net *n, void *stream);
/* Copy gf_net_param_count() FP32 parameters in (host or device); resets Adam. */
int gf_net_set_params(gf_net *n, const float *params);
int gf_net_get_params(gf_net *n, float *params);
/* features: device BF16 [V][80]; out: device FP32 [V][8]. */
int gf_net_forward(gf_net *n, const void *features, float *out);
/* Loss and gradient w.r.t. the parameters (grad host or device, may be NULL). */
int gf_net_gradient(gf_net *n, const void *features, const float *target, float *grad, double *loss);
/* Options: "tensor_cores" (default 1): forward, backward-data and
 * weight-gradient convolutions as implicit GEMMs on the tcgen05 tensor cores
 * (BF16 in, FP32 accumulators in tensor memory); 0 = the CUDA-core kernels.
 * "conv_halo" (default 1): forward and backward-data convolutions stage a
 * tile's periodic halo once per 16 input channels and read every tap's operand
 * from it.  1 = x-line tiles (whole x lines, 128 / Lx lines of y, two z
 * planes; lattices with Lx = 8, 16 or 32, Ly % (128 / Lx) == 0 and
 * Lz % 2 == 0), else 8 x 16 x 2 site tiles (Lx % 8 == 0, Ly % 16 == 0,
 * Lz % 2 == 0); 2 = the 8 x 16 x 2 tiles only; lattices that fit neither, and
 * 0, use the per-tap gather kernel.  Other values: GF_EINVAL.  With 1 and
 * Lx = 8, 16 or 32, Ly % (128 / Lx) == 0, the weight and bias gradients are
 * GEMMs over the site sum with both operands staged by TMA from ghost-padded
 * copies (otherwise a gather kernel); where the x-line tiles apply, each
 * layer's input exists only as such a copy, written by the previous layer's
 * epilogue (the features are copied into theirs), and so does the output
 * gradient of each layer in the backward pass (extra device memory:
 * Lx (Ly+2) (Lz+2) (Lt+2) x 176 BF16 values, allocated on the first forward,
 * gradient or train call, beside two dY copies of (Lx+2) (Ly+2) (Lz+2) (Lt+2)
 * x 32 BF16 values allocated at creation).  Forward, gradient
 * and train calls synchronise the stream and return GF_ETIMEOUT if a bounded
 * wait in a tensor-core kernel expired. */
int gf_net_set_option(gf_net *n, const char *key, double value);
/* One Adam step on (features, target); loss before the step in *loss. */
int gf_net_train_step(gf_net *n, const void *features, const float *target, float lr, double *loss);

/* Gauge tracking on the resident field: reset the tracked g(x) to 1; with
 * option "track" = 1, gf_or_half_sweep / gf_or_sweeps / gf_converge also
 * rotate g(x) (stored as FP32, 12 reals per site). */
int gf_gauge_reset(gf_ctx *ctx);
/* The tracked g as a canonical site field double g[V][3][3][2] (host or
 * device), reprojected onto SU(3) in FP64. */
int gf_get_gauge(gf_ctx *ctx, double *g);
/* Alg. 1 convergence loop on the resident field (no upload/download);
 * FP32 fields are reunitarised at each check. */
int gf_converge(gf_ctx *ctx, double omega, double theta_target, int max_iter, int *iters_out, double *F_out,
                double *theta_out);
/* Resident FP64 field := g(x) U_mu(x) g(x+mu)^dagger for the caller's field
 * U (host or device) and the tracked g: the FP32 -> FP64 switch of GF_MIXED. */
int gf_apply_tracked_gauge(gf_ctx *ctx, const double *U);
/* Network inputs of the resident FP64 field with scale s (device BF16 [V][80]). */
int gf_features(gf_ctx *ctx, double scale, void *features);
/* Training labels: tr(lambda_a (g - g^dagger)/(2i)) / s of the tracked g
 * (the algebra coefficients of log g to first order), device FP32 [V][8]. */
int gf_gauge_algebra(gf_ctx *ctx, double scale, float *c);
/* Apply g(x) = exp(i s sum_a c_a(x) lambda_a / 2) to the resident FP64 field. */
int gf_apply_algebra(gf_ctx *ctx, const float *c, double scale);
/* Attach a trained network (NULL detaches): GF_MIXED then applies its
 * prediction at the switch before the FP64 sweeps.  The context does not own it.
 * Landau-gauge contexts only (the inputs carry the Landau violation); other
 * gauges return GF_EINVAL. */
int gf_set_net(gf_ctx *ctx, gf_net *net);

/* ------------------------------------ many lattices in one persistent launch */

/* A batch of n independent lattices (uneven volumes allowed) gauge-fixed
 * together: all fields share one device arena, their tiles form one work
 * list, and each precision phase of Alg. 1 -- theta checks (Sec. 4.1),
 * convergence decisions per lattice and the RED/BLACK half-sweeps -- runs
 * as ONE persistent cooperative kernel whose blocks meet at grid-wide
 * barriers; converged lattices drop out of the work list.  The whole call is
 * captured once as a CUDA graph and replayed while its inputs stay the same.
 * dims: n x 4 extents (each as for gf_create); gauge for all lattices. */
typedef struct gf_batch gf_batch;
int gf_batch_create(int n, const int *dims, int gauge, gf_batch **out);
int gf_batch_destroy(gf_batch *b);
const char *gf_batch_last_error(const gf_batch *b);
int gf_batch_set_stream(gf_batch *b, void *stream);

/* Options: "precision" (default GF_MIXED), "storage32", "storage64",
 * "check_every" (default 25), "theta_switch" (default 1e-6),
 * "threads_per_site", "block" (0 = autotuned or default), "use_graphs",
 * "barrier_timeout_ms" (bounded grid-barrier wait, default 2000; on expiry
 * the call returns GF_ETIMEOUT and the batch stays usable),
 * "barrier_extra_blocks" (test hook: 1 makes every barrier wait for a block
 * that does not exist, so the bounded wait expires), "fp64_arith" (default
 * 0; 1 = the FP64 phase runs as double-float sweeps on copies of the FP64
 * fields, one thread per site, with E = g - 1 tracked in double-float, then
 * g = 1 + E is applied to each FP64 field in FP64 and native FP64 sweeps
 * finish any lattice not yet below the target: the results stay gauge
 * transforms of the inputs to FP64 rounding, as in gf_overrelax). */
int gf_batch_set_option(gf_batch *b, const char *key, double value);

/* Stats of the last call: "site_updates", "ms_fp32", "ms_fp64" (the whole
 * FP64-class phase), "ms_total", "grid_fp32", "grid_fp64", "grid_df64",
 * "threads_per_site", "block", "tiles". */
int gf_batch_get_stat(const gf_batch *b, const char *key, double *value);

/* Gauge-fix every U[i] (device pointers, canonical layout, in place) by
 * overrelaxation with the batch's precision policy; per lattice: iters[i]
 * sweeps, final F[i] and theta[i] (arrays of n, may be NULL).  Returns
 * GF_OK if every lattice converged, GF_ENOTCONVERGED otherwise. */
int gf_batch_overrelax(gf_batch *b, double *const *U, double omega, double theta_target, int max_iter,
                       int *iters, double *F, double *theta);

/* The batched solve in one call (Alg. 1 for each of n Landau-gauge lattices,
 * theta checked every 25 sweeps on the device, Sec. 4.1): a batch with the
 * default options (GF_MIXED, FP32 12-real then FP64 18-real storage, switch
 * at theta < 1e-6, threads per site and block from the autotuner's cache of
 * this process or the defaults) is created, run once on the legacy default
 * stream and destroyed.  dims: n rows of {Lx, Ly, Lz, Lt}; U: n device
 * pointers (canonical layout, in place); iters, F, theta: arrays of n (may
 * be NULL).  Returns GF_OK if every lattice converged, GF_ENOTCONVERGED
 * otherwise, or the error of the first failing step (the message is not
 * kept: callers that need it, other options, another gauge, a stream or
 * repeated solves use gf_batch_create / gf_batch_overrelax, which also keep
 * the device arena and replay the captured graph). */
int gf_overrelax_batched(int n, const int (*dims)[4], double **U, double omega, double theta_target, int max_iter,
                         int *iters, double *F, double *theta);

/* Choose threads per site and block size for both storage formats by timing
 * every candidate on the fields U (left unchanged); cached per set of
 * extents for the process.  Outputs (FP32 phase choice) may be NULL. */
int gf_batch_autotune(gf_batch *b, double *const *U, int *threads_per_site, int *block);

/* ------------------------------------------------ measured arithmetic peak */

/* The arithmetic rate this GPU sustains, for the roofline of the sweeps that
 * are bound by an arithmetic unit rather than by HBM (the FP64 sweeps are
 * bound by the FP64 unit).  Launches, on the legacy default stream of the
 * current device, 8 blocks per SM of 256 threads, each thread running eight
 * independent chains of iters fused multiply-adds (fp64 = 1: double, 0:
 * float); one warm-up launch, then three timed with CUDA events.  The paper
 * has no counterpart (it quotes Fermi's nominal figures); this is a
 * measurement helper.  Outputs (may be NULL): *tflops = 2 x FMAs / time in
 * 10^12 flop/s, *ms_per_launch.  Synchronises the device's default stream.
 * GF_EINVAL for fp64 outside {0, 1} or iters < 1; GF_ECUDA on a CUDA error. */
int gf_fma_peak(int fp64, int iters, double *tflops, double *ms_per_launch);

/* ------------------------------------------------- allocation-free measure */

/* Largest lattice volume gf_measure_noalloc accepts. */
#define GF_NOALLOC_MAX_SITES (1 << 21)

/* F and theta of a canonical field U held in device memory, computed without
 * allocating anything: no cudaMalloc, no context, no library pool.  It is for
 * callers that cannot allocate device memory at the point of the call -- for
 * example code that runs while another thread captures a CUDA graph, code
 * inside a framework that owns all device memory through its own allocator,
 * or a service that forbids allocation after start-up.  (This entry point has
 * no counterpart in the paper; it is a deployment convenience beside
 * gf_functional / gf_theta, which allocate their scratch on first use.)
 *
 * dims, gauge: as for gf_create.  U: device pointer, canonical layout,
 * 16-byte aligned, read only.  out: device pointer to 2 doubles, written with
 * {F, theta} in stream order (read them after synchronising stream).
 * stream: cudaStream_t (NULL = legacy default stream).
 * Scratch: a fixed file-scope device array of 2 * GF_NOALLOC_MAX_SITES / 256
 * doubles (128 KiB), present on every GPU that loads the library until the
 * process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls on a device share the array and
 * leave their partial sums in it; calls whose kernels overlap on the GPU race
 * and must be ordered by the caller.
 * Errors: GF_EINVAL for a NULL, host or misaligned pointer, a pointer to
 * memory of a device other than the current one, a bad gauge or extent, or a
 * volume above GF_NOALLOC_MAX_SITES; GF_ECUDA if a CUDA error from earlier
 * work of the calling thread is pending on entry (it is left in place for the
 * caller, nothing is launched), or if the launch or the address lookup fails. */
int gf_measure_noalloc(const int dims[4], int gauge, const double *U, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
