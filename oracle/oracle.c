/*
 * FP64 CPU oracle, C part. TEST INFRASTRUCTURE ONLY: tests, the smoke check and
 * the benchmark's CPU-baseline leg call this code; the product path never does.
 *
 * Plain loops, no blocking, no tricks. Every function states the formula it
 * follows (Wagner, Nestler, Stoll, "Fast Evaluation of Additive Kernels").
 *
 *  orc_direct   : the additive Gaussian kernel product K v and the length-scale
 *                 derivative products dK/d(ell_s) v, straight from their
 *                 definitions (Sec. 3.3, eq. "add_gauss_kernel" and the
 *                 dK_ij/d ell formula right after it), for a chosen set of rows.
 *  orc_spread   : the spreading step of the adjoint NFFT,
 *                 g_l = sum_j v_j phi~(x_j - l/n), l in I_n^D (Sec. 3.1, the
 *                 inner sum of eq. "approx fast sum" computed approximately).
 *  orc_gather   : the interpolation step of the NFFT,
 *                 f_i = sum_l h_l phi~(x_i - l/n) (Sec. 3.1, the outer sum).
 *  orc_direct_grad_x : the gradient of w^T K v with respect to the points, from
 *                 the kernel's definition.
 *  orc_gather_grad : the interpolation and its gradient in the target point
 *                 (the window differentiated).
 *
 * phi is the Kaiser-Bessel window (kind 0) with shape b and cutoff m on a grid
 * of n points per dimension:
 *   phi(x) = sinh(b*sqrt(m^2 - (n x)^2)) / (pi * sqrt(m^2 - (n x)^2)),  |n x| <= m,
 * or (kind 1, spreading and interpolation only) the exponential of semicircle
 * (Barnett, Magland, af Klinteberg 2019) with shape beta:
 *   phi(x) = exp(beta * (sqrt(1 - (n x / m)^2) - 1)),  |n x| <= m,
 * zero outside; phi~ is its 1-periodisation. Grid index l runs over
 * -n/2 .. n/2-1 and is stored at array position l + n/2 (wrapped mod n).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846;

/* Kaiser-Bessel window as a function of t = n*x (grid units). */
static double kb(double t, int m, double b)
{
    double s2 = (double)m * (double)m - t * t;
    if (s2 < 0.0) return 0.0;
    double s = sqrt(s2);
    if (s < 1e-8) return b / ORC_PI;           /* limit of sinh(b s)/s as s -> 0 */
    return sinh(b * s) / (ORC_PI * s);
}

/* Exponential-of-semicircle window as a function of t = n*x (grid units). */
static double es(double t, int m, double beta)
{
    double z = t / (double)m;
    double s2 = 1.0 - z * z;
    if (s2 < 0.0) return 0.0;
    return exp(beta * (sqrt(s2) - 1.0));
}

/* The window of the given kind (0 Kaiser-Bessel, 1 exponential of semicircle) with its shape. */
static double window_value(double t, int m, double shape, int kind)
{
    return kind == 1 ? es(t, m, shape) : kb(t, m, shape);
}

/* Threads of the OpenMP loops below (timing the baseline on one core or on all of them). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Direct sums for rows[0..nrows).
 *   Kv[r]          = sigma_f^2 sum_s sum_j exp(-|x_i^W - x_j^W|^2 / (2 ell_s^2)) v_j
 *   dK[s*nrows+r]  = sigma_f^2 sum_j |x_i^W - x_j^W|^2 / ell_s^3 * exp(...) v_j
 * X is N x d row-major float32 (the same numbers the GPU sees), promoted to double.
 * Windows are CSR: features of window s are win_feat[win_off[s] .. win_off[s+1]).
 */
void orc_direct(int64_t N, int d, const float *X, int P, const int *win_off, const int *win_feat,
                const double *ell, double sigma_f, const double *v, int64_t nrows,
                const int64_t *rows, double *Kv, double *dK)
{
    (void)d;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double ksum = 0.0;
        for (int s = 0; s < P; ++s) {
            double e2 = 2.0 * ell[s] * ell[s];
            double l3 = ell[s] * ell[s] * ell[s];
            double ks = 0.0, ds = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                double r2 = 0.0;
                for (int q = win_off[s]; q < win_off[s + 1]; ++q) {
                    int f = win_feat[q];
                    double diff = (double)X[i * d + f] - (double)X[j * d + f];
                    r2 += diff * diff;
                }
                double k = exp(-r2 / e2);
                ks += k * v[j];
                ds += r2 / l3 * k * v[j];
            }
            ksum += ks;
            dK[(int64_t)s * nrows + r] = sigma_f * sigma_f * ds;
        }
        Kv[r] = sigma_f * sigma_f * ksum;
    }
}

/* Support of phi~(x - l/n) along one axis: l = floor(n x) - m + 1 + t, t = 0..2m-1. */
static void support(double x, int n, int m, double b, int kind, int64_t *idx, double *w)
{
    double u = x * n;
    double fl = floor(u);
    for (int t = 0; t < 2 * m; ++t) {
        double l = fl - m + 1 + t;
        w[t] = window_value(u - l, m, b, kind);
        int64_t a = ((int64_t)l + n / 2) % n;
        if (a < 0) a += n;
        idx[t] = a;
    }
}

/*
 * Spreading (adjoint NFFT, first step): g[a] += v_j * prod_t phi~(x_{j,t} - l_t/n)
 * for the 2m^D grid points around x_j. x is N x D row-major double in [-1/2,1/2).
 * g has n^D entries, index ((a0*n)+a1)*n+a2 for D = 3 (last axis fastest).
 * Threads spread disjoint point ranges into private grids that are summed at the end.
 */
void orc_spread(int64_t N, int D, const double *x, const double *v, int n, int m, double b, int kind, double *g)
{
    int64_t G = 1;
    for (int t = 0; t < D; ++t) G *= n;
    memset(g, 0, sizeof(double) * (size_t)G);
    int nth = orc_num_threads();
    double *priv = (double *)calloc((size_t)nth * (size_t)G, sizeof(double));
    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = priv + (size_t)tid * (size_t)G;
        int64_t idx[3][64];
        double w[3][64];
        #pragma omp for schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            for (int t = 0; t < D; ++t) support(x[j * D + t], n, m, b, kind, idx[t], w[t]);
            int W = 2 * m;
            if (D == 1) {
                for (int a = 0; a < W; ++a) mine[idx[0][a]] += v[j] * w[0][a];
            } else if (D == 2) {
                for (int a = 0; a < W; ++a)
                    for (int c = 0; c < W; ++c)
                        mine[idx[0][a] * n + idx[1][c]] += v[j] * w[0][a] * w[1][c];
            } else {
                for (int a = 0; a < W; ++a)
                    for (int c = 0; c < W; ++c)
                        for (int e = 0; e < W; ++e)
                            mine[(idx[0][a] * n + idx[1][c]) * n + idx[2][e]] +=
                                v[j] * w[0][a] * w[1][c] * w[2][e];
            }
        }
    }
    for (int t = 0; t < nth; ++t)
        for (int64_t a = 0; a < G; ++a) g[a] += priv[(size_t)t * (size_t)G + a];
    free(priv);
}

/*
 * Interpolation (NFFT, last step): out[i] = sum over the 2m^D grid points around x_i
 * of h[a] * prod_t phi~(x_{i,t} - l_t/n). nh grids are read (h is nh x n^D).
 * out is nh x N.
 */
void orc_gather(int64_t N, int D, const double *x, int n, int m, double b, int kind, int nh, const double *h,
                double *out)
{
    int64_t G = 1;
    for (int t = 0; t < D; ++t) G *= n;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t idx[3][64];
        double w[3][64];
        for (int t = 0; t < D; ++t) support(x[i * D + t], n, m, b, kind, idx[t], w[t]);
        int W = 2 * m;
        for (int q = 0; q < nh; ++q) {
            const double *hq = h + (size_t)q * (size_t)G;
            double s = 0.0;
            if (D == 1) {
                for (int a = 0; a < W; ++a) s += hq[idx[0][a]] * w[0][a];
            } else if (D == 2) {
                for (int a = 0; a < W; ++a)
                    for (int c = 0; c < W; ++c)
                        s += hq[idx[0][a] * n + idx[1][c]] * w[0][a] * w[1][c];
            } else {
                for (int a = 0; a < W; ++a)
                    for (int c = 0; c < W; ++c)
                        for (int e = 0; e < W; ++e)
                            s += hq[(idx[0][a] * n + idx[1][c]) * n + idx[2][e]] * w[0][a] * w[1][c] * w[2][e];
            }
            out[(size_t)q * (size_t)N + i] = s;
        }
    }
}

/*
 * Gradient of f = w^T K v with respect to the points, straight from the definition (Sec. 3.3 kernel):
 *   df/dx_{k,f} = sigma_f^2 sum_{s: f in W_s} sum_j (w_k v_j + w_j v_k) * (-(x_{k,f} - x_{j,f}) / ell_s^2)
 *                 * exp(-|x_k^W - x_j^W|^2 / (2 ell_s^2))
 * for rows k in rows[0..nrows); out is nrows x d (zero for features in no window).
 */
void orc_direct_grad_x(int64_t N, int d, const float *X, int P, const int *win_off, const int *win_feat,
                       const double *ell, double sigma_f, const double *v, const double *w, int64_t nrows,
                       const int64_t *rows, double *out)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t k = rows[r];
        for (int f = 0; f < d; ++f) out[r * d + f] = 0.0;
        for (int s = 0; s < P; ++s) {
            double e2 = 2.0 * ell[s] * ell[s];
            double l2 = ell[s] * ell[s];
            for (int64_t j = 0; j < N; ++j) {
                double r2 = 0.0;
                for (int q = win_off[s]; q < win_off[s + 1]; ++q) {
                    int f = win_feat[q];
                    double diff = (double)X[k * d + f] - (double)X[j * d + f];
                    r2 += diff * diff;
                }
                double kv = exp(-r2 / e2) * (w[k] * v[j] + w[j] * v[k]);
                for (int q = win_off[s]; q < win_off[s + 1]; ++q) {
                    int f = win_feat[q];
                    double diff = (double)X[k * d + f] - (double)X[j * d + f];
                    out[r * d + f] += sigma_f * sigma_f * (-diff / l2) * kv;
                }
            }
        }
    }
}

/* d/dt of the Kaiser-Bessel window kb(t) (t = n x), from kb = sinh(b s)/(pi s), s = sqrt(m^2 - t^2):
 *   dkb/dt = (-t/s) (b cosh(b s)/(pi s) - sinh(b s)/(pi s^2)),  -> -t b^3/(3 pi) as s -> 0. */
static double kb_dt(double t, int m, double b)
{
    double s2 = (double)m * (double)m - t * t;
    if (s2 < 0.0) return 0.0;
    double s = sqrt(s2);
    if (s < 1e-4) return -t * b * b * b / (3.0 * ORC_PI) * (1.0 + b * b * s2 / 10.0);
    return (-t / s) * (b * cosh(b * s) / (ORC_PI * s) - sinh(b * s) / (ORC_PI * s * s));
}

/*
 * Interpolation and its gradient (the NFFT's last step, differentiated in the target point):
 *   val[i]        = sum_l h_l prod_t phi~(x_{i,t} - l_t/n)
 *   grad[i*D + t] = sum_l h_l phi~'(x_{i,t} - l_t/n) prod_{u != t} phi~(x_{i,u} - l_u/n)
 * with phi' = n dkb/dt. One grid h (n^D values).
 */
void orc_gather_grad(int64_t N, int D, const double *x, int n, int m, double b, const double *h, double *val,
                     double *grad)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t idx[3][64];
        double w[3][64], dw[3][64];
        for (int t = 0; t < D; ++t) {
            double u = x[i * D + t] * n;
            double fl = floor(u);
            for (int q = 0; q < 2 * m; ++q) {
                double l = fl - m + 1 + q;
                w[t][q] = kb(u - l, m, b);
                dw[t][q] = n * kb_dt(u - l, m, b);
                int64_t a = ((int64_t)l + n / 2) % n;
                if (a < 0) a += n;
                idx[t][q] = a;
            }
        }
        int W = 2 * m;
        double s = 0.0, g[3] = {0.0, 0.0, 0.0};
        if (D == 1) {
            for (int a = 0; a < W; ++a) {
                double hv = h[idx[0][a]];
                s += hv * w[0][a];
                g[0] += hv * dw[0][a];
            }
        } else if (D == 2) {
            for (int a = 0; a < W; ++a)
                for (int c = 0; c < W; ++c) {
                    double hv = h[idx[0][a] * n + idx[1][c]];
                    s += hv * w[0][a] * w[1][c];
                    g[0] += hv * dw[0][a] * w[1][c];
                    g[1] += hv * w[0][a] * dw[1][c];
                }
        } else {
            for (int a = 0; a < W; ++a)
                for (int c = 0; c < W; ++c)
                    for (int e = 0; e < W; ++e) {
                        double hv = h[(idx[0][a] * n + idx[1][c]) * n + idx[2][e]];
                        s += hv * w[0][a] * w[1][c] * w[2][e];
                        g[0] += hv * dw[0][a] * w[1][c] * w[2][e];
                        g[1] += hv * w[0][a] * dw[1][c] * w[2][e];
                        g[2] += hv * w[0][a] * w[1][c] * dw[2][e];
                    }
        }
        val[i] = s;
        for (int t = 0; t < D; ++t) grad[i * D + t] = g[t];
    }
}
