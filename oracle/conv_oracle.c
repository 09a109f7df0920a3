/*
 * conv_oracle.c -- plain FP64 CPU oracle of the learned warm-start network:
 * periodic 4D convolutions with 3^4 taps, ReLU between layers, a mean-squared
 * error loss, and the exact backward pass.
 *
 * TEST INFRASTRUCTURE ONLY (see gf_oracle.c): only the tests, the smoke check
 * and the benchmark's CPU legs load it; it shares nothing with the CUDA path.
 *
 * Conventions (shared with the library's network kernels, stated here in
 * full so that both follow the same definition):
 *   activations X[site][C], site = x + Lx (y + Ly (z + Lz t)), channels last;
 *   tap index k = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1), d in {-1,0,1};
 *   weights W[k][co][ci], bias b[co];
 *   conv:   Y[s][co] = b[co] + sum_k sum_ci W[k][co][ci] X[s + d(k)][ci]
 *           (periodic neighbour s + d(k));
 *   network: a1 = relu(conv1(f)), a2 = relu(conv2(a1)), a3 = relu(conv3(a2)),
 *            out = conv4(a3);
 *   loss:   L = (1 / (V C_out)) sum_s sum_c (out[s][c] - target[s][c])^2.
 * Backward:
 *   dX[s][ci]      = sum_k sum_co W[k][co][ci] dY[s - d(k)][co]
 *   dW[k][co][ci]  = sum_s dY[s][co] X[s + d(k)][ci]
 *   db[co]         = sum_s dY[s][co].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int L[4]; long V; } grid4;

static void grid_init(grid4 *g, const int dims[4])
{
    g->V = 1;
    for (int m = 0; m < 4; ++m) {
        g->L[m] = dims[m];
        g->V *= dims[m];
    }
}

/* site index of s shifted by tap k (periodic); sign = +1 or -1 */
static long shifted(const grid4 *g, long s, int k, int sign)
{
    int c[4];
    long r = s;
    for (int m = 0; m < 4; ++m) {
        c[m] = (int)(r % g->L[m]);
        r /= g->L[m];
    }
    int d[4] = { k % 3 - 1, (k / 3) % 3 - 1, (k / 9) % 3 - 1, (k / 27) % 3 - 1 };
    for (int m = 0; m < 4; ++m) c[m] = ((c[m] + sign * d[m]) % g->L[m] + g->L[m]) % g->L[m];
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

void oracle_conv_forward(const double *X, const double *W, const double *b, const int dims[4], int cin, int cout,
                         double *Y)
{
    grid4 g;
    grid_init(&g, dims);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long s = 0; s < g.V; ++s) {
        for (int co = 0; co < cout; ++co) Y[s * cout + co] = b ? b[co] : 0.0;
        for (int k = 0; k < 81; ++k) {
            const double *x = X + shifted(&g, s, k, +1) * cin;
            for (int co = 0; co < cout; ++co) {
                const double *w = W + ((long)k * cout + co) * cin;
                double acc = 0.0;
                for (int ci = 0; ci < cin; ++ci) acc += w[ci] * x[ci];
                Y[s * cout + co] += acc;
            }
        }
    }
}

void oracle_conv_backward_data(const double *dY, const double *W, const int dims[4], int cin, int cout, double *dX)
{
    grid4 g;
    grid_init(&g, dims);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long s = 0; s < g.V; ++s) {
        for (int ci = 0; ci < cin; ++ci) dX[s * cin + ci] = 0.0;
        for (int k = 0; k < 81; ++k) {
            const double *dy = dY + shifted(&g, s, k, -1) * cout;
            for (int co = 0; co < cout; ++co) {
                const double *w = W + ((long)k * cout + co) * cin;
                for (int ci = 0; ci < cin; ++ci) dX[s * cin + ci] += w[ci] * dy[co];
            }
        }
    }
}

void oracle_conv_backward_weights(const double *dY, const double *X, const int dims[4], int cin, int cout, double *dW,
                                  double *db)
{
    grid4 g;
    grid_init(&g, dims);
    memset(dW, 0, sizeof(double) * 81 * (size_t)cout * cin);
    if (db) memset(db, 0, sizeof(double) * cout);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int k = 0; k < 81; ++k) {
        for (long s = 0; s < g.V; ++s) {
            const double *x = X + shifted(&g, s, k, +1) * cin;
            for (int co = 0; co < cout; ++co) {
                double dy = dY[s * cout + co];
                double *w = dW + ((long)k * cout + co) * cin;
                for (int ci = 0; ci < cin; ++ci) w[ci] += dy * x[ci];
            }
        }
    }
    if (db)
        for (long s = 0; s < g.V; ++s)
            for (int co = 0; co < cout; ++co) db[co] += dY[s * cout + co];
}

/*
 * The four-layer network: channels c[0] -> c[1] -> c[2] -> c[3] -> c[4].
 * params: W1 b1 W2 b2 W3 b3 W4 b4 concatenated (W as [81][co][ci]).
 * Returns the loss; if grad != NULL it receives dL/dparams (same layout) and,
 * if out != NULL, the network output.
 */
double oracle_net_loss(const double *f, const double *target, const double *params, const int dims[4],
                       const int c[5], double *grad, double *out)
{
    grid4 g;
    grid_init(&g, dims);
    long V = g.V;
    const double *W[4], *b[4];
    long off = 0;
    for (int l = 0; l < 4; ++l) {
        W[l] = params + off;
        off += 81L * c[l + 1] * c[l];
        b[l] = params + off;
        off += c[l + 1];
    }
    double *act[5];
    act[0] = (double *)f;
    for (int l = 1; l <= 4; ++l) act[l] = (double *)malloc(sizeof(double) * V * c[l]);
    for (int l = 0; l < 4; ++l) {
        oracle_conv_forward(act[l], W[l], b[l], dims, c[l], c[l + 1], act[l + 1]);
        if (l < 3)
            for (long i = 0; i < V * c[l + 1]; ++i) act[l + 1][i] = act[l + 1][i] > 0.0 ? act[l + 1][i] : 0.0;
    }
    double loss = 0.0;
    long n = V * c[4];
    for (long i = 0; i < n; ++i) {
        double d = act[4][i] - target[i];
        loss += d * d;
    }
    loss /= (double)n;
    if (out) memcpy(out, act[4], sizeof(double) * n);
    if (grad) {
        double *dY = (double *)malloc(sizeof(double) * n);
        for (long i = 0; i < n; ++i) dY[i] = 2.0 * (act[4][i] - target[i]) / (double)n;
        long goff = off;
        for (int l = 3; l >= 0; --l) {
            goff -= c[l + 1];
            double *db = grad + goff;
            goff -= 81L * c[l + 1] * c[l];
            double *dW = grad + goff;
            oracle_conv_backward_weights(dY, act[l], dims, c[l], c[l + 1], dW, db);
            if (l > 0) {
                double *dX = (double *)malloc(sizeof(double) * V * c[l]);
                oracle_conv_backward_data(dY, W[l], dims, c[l], c[l + 1], dX);
                for (long i = 0; i < V * c[l]; ++i)
                    if (!(act[l][i] > 0.0)) dX[i] = 0.0; /* ReLU: act[l] = relu(z) */
                free(dY);
                dY = dX;
            }
        }
        free(dY);
    }
    for (int l = 1; l <= 4; ++l) free(act[l]);
    return loss;
}
