/*
 * FP64 oracle of the convolutional surrogate's layers -- TEST INFRASTRUCTURE ONLY
 * (see oracle.h for who may load this code).
 *
 * The surrogate is a stack of periodic 3x3x3 convolutions over the lattice; nothing
 * here comes from the paper (which defines no learned component): each function is
 * the plain definition of the operation, written as loops in double precision.
 *
 * Layout: activations x[n * C + c] (site-major, channels contiguous), site
 * n = (z*N + y)*N + x periodic in every direction; weights W[(t * cout + co) * cin + ci]
 * with tap t = (tz*3 + ty)*3 + tx and offset o(t) = (tx - 1, ty - 1, tz - 1).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "oracle.h"

/* site n shifted by (dx, dy, dz), periodic */
static int64_t site_shift(int N, int64_t n, int dx, int dy, int dz)
{
    const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((int64_t)N * N));
    const int xs = ((x + dx) % N + N) % N, ys = ((y + dy) % N + N) % N, zs = ((z + dz) % N + N) % N;
    return ((int64_t)zs * N + ys) * N + xs;
}

/* y[n][co] = b[co] + sum_t sum_ci W[t][co][ci] x[n + o(t)][ci]   (b may be NULL) */
void orc_conv3d_fwd(int N, int cin, int cout, const double* x, const double* W, const double* b, double* y)
{
    const int64_t V = (int64_t)N * N * N;
    for (int64_t n = 0; n < V; ++n)
        for (int co = 0; co < cout; ++co) {
            double s = b ? b[co] : 0.0;
            for (int t = 0; t < 27; ++t) {
                const int64_t m = site_shift(N, n, t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1);
                for (int ci = 0; ci < cin; ++ci) s += W[((int64_t)t * cout + co) * cin + ci] * x[m * cin + ci];
            }
            y[n * cout + co] = s;
        }
}

/* Adjoint of the linear part of orc_conv3d_fwd with respect to x:
 * dx[m][ci] = sum_t sum_co W[t][co][ci] dy[m - o(t)][co] */
void orc_conv3d_bwd_data(int N, int cin, int cout, const double* dy, const double* W, double* dx)
{
    const int64_t V = (int64_t)N * N * N;
    for (int64_t m = 0; m < V; ++m)
        for (int ci = 0; ci < cin; ++ci) {
            double s = 0.0;
            for (int t = 0; t < 27; ++t) {
                const int64_t n = site_shift(N, m, 1 - t % 3, 1 - (t / 3) % 3, 1 - t / 9);
                for (int co = 0; co < cout; ++co) s += W[((int64_t)t * cout + co) * cin + ci] * dy[n * cout + co];
            }
            dx[m * cin + ci] = s;
        }
}

/* Gradients of sum_n sum_co y[n][co] dy[n][co] with respect to W and b:
 * dW[t][co][ci] = sum_n dy[n][co] x[n + o(t)][ci],   db[co] = sum_n dy[n][co]   (db may be NULL) */
void orc_conv3d_bwd_weight(int N, int cin, int cout, const double* x, const double* dy, double* dW, double* db)
{
    const int64_t V = (int64_t)N * N * N;
    memset(dW, 0, sizeof(double) * 27 * (size_t)cout * cin);
    for (int t = 0; t < 27; ++t)
        for (int64_t n = 0; n < V; ++n) {
            const int64_t m = site_shift(N, n, t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1);
            for (int co = 0; co < cout; ++co) {
                const double g = dy[n * cout + co];
                for (int ci = 0; ci < cin; ++ci) dW[((int64_t)t * cout + co) * cin + ci] += g * x[m * cin + ci];
            }
        }
    if (db)
        for (int co = 0; co < cout; ++co) {
            double s = 0.0;
            for (int64_t n = 0; n < V; ++n) s += dy[n * cout + co];
            db[co] = s;
        }
}

/* Activations: 0 = ReLU, 1 = GELU in its tanh form,
 * gelu(u) = u/2 (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3))). */
double orc_act(int act, double u)
{
    if (act == 0) return u > 0.0 ? u : 0.0;
    const double c = sqrt(2.0 / 3.14159265358979323846);
    return 0.5 * u * (1.0 + tanh(c * (u + 0.044715 * u * u * u)));
}

double orc_act_grad(int act, double u)
{
    if (act == 0) return u > 0.0 ? 1.0 : 0.0;
    const double c = sqrt(2.0 / 3.14159265358979323846);
    const double th = tanh(c * (u + 0.044715 * u * u * u));
    return 0.5 * (1.0 + th) + 0.5 * u * (1.0 - th * th) * c * (1.0 + 3.0 * 0.044715 * u * u);
}

void orc_act_array(int act, int64_t n, const double* u, double* h)
{
    for (int64_t i = 0; i < n; ++i) h[i] = orc_act(act, u[i]);
}

/* du = dh * act'(u) */
void orc_act_bwd_array(int act, int64_t n, const double* u, const double* dh, double* du)
{
    for (int64_t i = 0; i < n; ++i) du[i] = dh[i] * orc_act_grad(act, u[i]);
}
