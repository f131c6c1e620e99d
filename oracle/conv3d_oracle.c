/*
 * Oracle for the warm-start surrogate's 3-D convolutions: plain FP64 loops.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite to check the GPU
 * convolution kernels (forward, backward-data, backward-weight).  Shares no
 * code with them.
 *
 * Layout: activations x[n][d][h][w][c] (channels last), weights
 * wt[co][kd][kh][kw][ci] with kernel size k (odd), "same" zero padding, stride
 * 1; bias b[co].  Definitions:
 *   y[n,p,co]  = b[co] + sum_{t,ci} wt[co,t,ci] x[n, p + t - r, ci]
 *   dx[n,q,ci] = sum_{t,co} wt[co,t,ci] dy[n, q - t + r, co]
 *   dw[co,t,ci] = sum_{n,p} dy[n,p,co] x[n, p + t - r, ci],  db[co] = sum dy
 * (r = k/2, out-of-range positions read zero).
 */
#include <stddef.h>
#include <string.h>

static long idx5(int n, int z, int y, int x, int c, int D, int H, int W, int C)
{
    return ((((long)n * D + z) * H + y) * W + x) * (long)C + c;
}

void oracle_conv3d_fwd(const double *x, const double *wt, const double *b, double *y, int N, int D, int H, int W,
                       int Ci, int Co, int k)
{
    int r = k / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < D; ++z)
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    for (int co = 0; co < Co; ++co) {
                        double s = b ? b[co] : 0.0;
                        for (int a = 0; a < k; ++a)
                            for (int bb = 0; bb < k; ++bb)
                                for (int c = 0; c < k; ++c) {
                                    int zi = z + a - r, yi = yy + bb - r, xi = xx + c - r;
                                    if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;
                                    const double *wp = wt + ((((long)co * k + a) * k + bb) * k + c) * Ci;
                                    const double *xp = x + idx5(n, zi, yi, xi, 0, D, H, W, Ci);
                                    for (int ci = 0; ci < Ci; ++ci) s += wp[ci] * xp[ci];
                                }
                        y[idx5(n, z, yy, xx, co, D, H, W, Co)] = s;
                    }
}

void oracle_conv3d_bwd_data(const double *dy, const double *wt, double *dx, int N, int D, int H, int W, int Ci,
                            int Co, int k)
{
    int r = k / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < D; ++z)
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    for (int ci = 0; ci < Ci; ++ci) {
                        double s = 0.0;
                        for (int a = 0; a < k; ++a)
                            for (int bb = 0; bb < k; ++bb)
                                for (int c = 0; c < k; ++c) {
                                    /* output position p with p + t - r = q */
                                    int zo = z - a + r, yo = yy - bb + r, xo = xx - c + r;
                                    if (zo < 0 || zo >= D || yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
                                    for (int co = 0; co < Co; ++co)
                                        s += wt[((((long)co * k + a) * k + bb) * k + c) * Ci + ci] *
                                             dy[idx5(n, zo, yo, xo, co, D, H, W, Co)];
                                }
                        dx[idx5(n, z, yy, xx, ci, D, H, W, Ci)] = s;
                    }
}

void oracle_conv3d_bwd_weight(const double *x, const double *dy, double *dw, double *db, int N, int D, int H, int W,
                              int Ci, int Co, int k)
{
    int r = k / 2;
#pragma omp parallel for schedule(static)
    for (int co = 0; co < Co; ++co) {
        for (int a = 0; a < k; ++a)
            for (int bb = 0; bb < k; ++bb)
                for (int c = 0; c < k; ++c)
                    for (int ci = 0; ci < Ci; ++ci) {
                        double s = 0.0;
                        for (int n = 0; n < N; ++n)
                            for (int z = 0; z < D; ++z)
                                for (int yy = 0; yy < H; ++yy)
                                    for (int xx = 0; xx < W; ++xx) {
                                        int zi = z + a - r, yi = yy + bb - r, xi = xx + c - r;
                                        if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;
                                        s += dy[idx5(n, z, yy, xx, co, D, H, W, Co)] *
                                             x[idx5(n, zi, yi, xi, ci, D, H, W, Ci)];
                                    }
                        dw[((((long)co * k + a) * k + bb) * k + c) * Ci + ci] = s;
                    }
        if (db) {
            double s = 0.0;
            long P = (long)N * D * H * W;
            for (long p = 0; p < P; ++p) s += dy[p * Co + co];
            db[co] = s;
        }
    }
}
