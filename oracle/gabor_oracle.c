/*
 * Plain FP64 CPU oracle for the 2-D complex Gabor filter bank and the 2-D localized
 * sliding DFT of Um, Kim and Min, "Fast 2-D Complex Gabor Filter with Kernel
 * Decomposition" (arXiv 1704.05231).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * it (through oracle/__init__.py).  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every function evaluates a definition from the paper literally, as a direct sum, in
 * double precision, with no reuse, blocking or reordering:
 *
 *   oracle_gabor_direct  Eq. 1 with the kernel of Eq. 2: a direct 2-D sum over a square
 *                        (or caller-given rectangular) support of the Gaussian.
 *   oracle_gabor_rows    Eq. 3: the horizontal 1-D Gabor pass J on its own.
 *   oracle_gabor_cols    Eq. 4: the vertical 1-D Gabor pass applied to a complex J.
 *   oracle_sdft_direct   Eq. 17 with the basis of Eq. 18: a direct 2-D windowed DFT at
 *                        every requested pixel.
 *
 * Readings of points the paper leaves open (the same ones the library implements):
 *   - S_sigma(d) = exp(-d^2 / (2 sigma^2)) / (sqrt(2 pi) sigma), the sampled continuous
 *     density, not renormalised after truncation (the paper only says "Gaussian with zero
 *     mean and standard deviation sigma", Sec. II).
 *   - The image is zero outside [0,W) x [0,H) (boundary 0); boundary 1 extends it by
 *     repeating the edge pixel, boundary 2 by mirroring about the pixel edges (f(-1) = f(0),
 *     f(W) = f(W-1), period 2W).  The output has the input's size.
 *   - Gabor support: |x-k| <= R and |y-l| <= R with R = ceil(rf * sigma - 1e-9), rf = 3
 *     by default (the cut-off of Sec. III applied to the Gabor filter as well).
 *   - SDFT support: the M_x x M_y window, m - xhat in [0, M_x), n - yhat in [0, M_y), with
 *     xhat = x - M_x/2 and M even (Eq. 17).  The caller may widen or narrow it.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off gabor_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* The 1-D Gaussian S_sigma of Sec. II (G_sigma(x,y) = S_sigma(x) S_sigma(y)). */
double oracle_gauss(double d, double sigma)
{
    return exp(-(d * d) / (2.0 * sigma * sigma)) / (sqrt(2.0 * M_PI) * sigma);
}

/* Truncation radius R = ceil(rf*sigma) (the -1e-9 keeps 3*4 = 12 from becoming 13). */
int oracle_radius(double sigma, double rf)
{
    return (int)ceil(rf * sigma - 1e-9);
}

/* Index of the image sample that position i (of n) reads under the boundary rule, or -1 for
 * a zero sample. */
static int ext_index(int i, int n, int boundary)
{
    if (i >= 0 && i < n) return i;
    if (boundary == 1) return i < 0 ? 0 : n - 1;
    if (boundary == 2) {
        int m = i % (2 * n);
        if (m < 0) m += 2 * n;
        return m < n ? m : 2 * n - 1 - m;
    }
    return -1;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * Eq. 1: F(x,y) = sum_{k,l} f(k,l) C(x-k, y-l) G(x-k, y-l), with
 * C(x,y) = exp(i omega (x cos theta + y sin theta)) (Eq. 2) and G = S(x) S(y).
 * Writing dx = x-k, dy = y-l the sum runs over dx in [dx_lo, dx_hi], dy in [dy_lo, dy_hi]
 * and over image pixels only (zero outside).
 *
 * f_re: H*W row-major doubles, f_im: the same or NULL for a real image.
 * px/py: npts output pixel coordinates, or NULL for all H*W pixels in row-major order.
 * out:   2*n doubles, (re, im) interleaved.
 */
int oracle_gabor_direct_b(const double *f_re, const double *f_im, int H, int W,
                          double omega, double theta, double sigma,
                          int dx_lo, int dx_hi, int dy_lo, int dy_hi,
                          const int *px, const int *py, long npts,
                          double *out, int nthreads, int boundary)
{
    if (H <= 0 || W <= 0 || sigma <= 0.0 || dx_hi < dx_lo || dy_hi < dy_lo) return -1;
    if (boundary < 0 || boundary > 2) return -1;
    const int nx = dx_hi - dx_lo + 1, ny = dy_hi - dy_lo + 1;
    double *kr = (double *)malloc(sizeof(double) * (size_t)nx * ny);
    double *ki = (double *)malloc(sizeof(double) * (size_t)nx * ny);
    if (!kr || !ki) { free(kr); free(ki); return -2; }
    const double c = cos(theta), s = sin(theta);
    for (int j = 0; j < ny; ++j) {
        const int dy = dy_lo + j;
        for (int i = 0; i < nx; ++i) {
            const int dx = dx_lo + i;
            const double phase = omega * ((double)dx * c + (double)dy * s);
            const double g = oracle_gauss((double)dx, sigma) * oracle_gauss((double)dy, sigma);
            kr[(size_t)j * nx + i] = cos(phase) * g;
            ki[(size_t)j * nx + i] = sin(phase) * g;
        }
    }
    const long n = px ? npts : (long)H * W;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < n; ++p) {
        const int x = px ? px[p] : (int)(p % W);
        const int y = px ? py[p] : (int)(p / W);
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < ny; ++j) {
            const int l = ext_index(y - (dy_lo + j), H, boundary);
            if (l < 0) continue;
            for (int i = 0; i < nx; ++i) {
                const int k = ext_index(x - (dx_lo + i), W, boundary);
                if (k < 0) continue;
                const double a = f_re[(size_t)l * W + k];
                const double b = f_im ? f_im[(size_t)l * W + k] : 0.0;
                const double cr = kr[(size_t)j * nx + i], ci = ki[(size_t)j * nx + i];
                sr += a * cr - b * ci;
                si += a * ci + b * cr;
            }
        }
        out[2 * p] = sr;
        out[2 * p + 1] = si;
    }
    free(kr);
    free(ki);
    return 0;
}

int oracle_gabor_direct(const double *f_re, const double *f_im, int H, int W,
                        double omega, double theta, double sigma,
                        int dx_lo, int dx_hi, int dy_lo, int dy_hi,
                        const int *px, const int *py, long npts,
                        double *out, int nthreads)
{
    return oracle_gabor_direct_b(f_re, f_im, H, W, omega, theta, sigma, dx_lo, dx_hi, dy_lo, dy_hi,
                                 px, py, npts, out, nthreads, 0);
}

/*
 * Eq. 3: J(x,y) = sum_k f(k,y) H(x-k) S(x-k), H(x) = exp(i omega x cos theta),
 * over |x-k| <= R and 0 <= k < W.  Output 2*H*W doubles (re, im).
 */
int oracle_gabor_rows(const double *f_re, const double *f_im, int H, int W,
                      double omega, double theta, double sigma, int R,
                      double *out, int nthreads)
{
    if (H <= 0 || W <= 0 || sigma <= 0.0 || R < 0) return -1;
    const double wc = omega * cos(theta);
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double sr = 0.0, si = 0.0;
            for (int d = -R; d <= R; ++d) {
                const int k = x - d;
                if (k < 0 || k >= W) continue;
                const double g = oracle_gauss((double)d, sigma);
                const double hr = cos(wc * d) * g, hi = sin(wc * d) * g;
                const double a = f_re[(size_t)y * W + k];
                const double b = f_im ? f_im[(size_t)y * W + k] : 0.0;
                sr += a * hr - b * hi;
                si += a * hi + b * hr;
            }
            out[2 * ((size_t)y * W + x)] = sr;
            out[2 * ((size_t)y * W + x) + 1] = si;
        }
    }
    return 0;
}

/*
 * Eq. 4: F(x,y) = sum_l J(x,l) V(y-l) S(y-l), V(y) = exp(i omega y sin theta),
 * over |y-l| <= R and 0 <= l < H.  J and out are 2*H*W doubles (re, im).
 */
int oracle_gabor_cols(const double *J, int H, int W,
                      double omega, double theta, double sigma, int R,
                      double *out, int nthreads)
{
    if (H <= 0 || W <= 0 || sigma <= 0.0 || R < 0) return -1;
    const double ws = omega * sin(theta);
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double sr = 0.0, si = 0.0;
            for (int d = -R; d <= R; ++d) {
                const int l = y - d;
                if (l < 0 || l >= H) continue;
                const double g = oracle_gauss((double)d, sigma);
                const double vr = cos(ws * d) * g, vi = sin(ws * d) * g;
                const double a = J[2 * ((size_t)l * W + x)], b = J[2 * ((size_t)l * W + x) + 1];
                sr += a * vr - b * vi;
                si += a * vi + b * vr;
            }
            out[2 * ((size_t)y * W + x)] = sr;
            out[2 * ((size_t)y * W + x) + 1] = si;
        }
    }
    return 0;
}

/*
 * Eq. 17-18: F_{u,v}(x,y) = sum_{m,n} f(m,n) C_{u,v}(xhat-m, yhat-n) G(x-m, y-n),
 * C_{u,v}(p,q) = exp(i (2 pi u p / Mx + 2 pi v q / My)), xhat = x - Mx/2, yhat = y - My/2.
 * With m = xhat + a and n = yhat + b the sum runs over a in [a_lo, a_hi],
 * b in [b_lo, b_hi] (the window [0,Mx) x [0,My) by default) and over image pixels only.
 * The phase u*a is reduced exactly modulo Mx in integers before the cosine.
 *
 * out: [My][Mx][n][2] doubles, n = npts or H*W.
 */
int oracle_sdft_direct_b(const double *f_re, const double *f_im, int H, int W,
                         double sigma, int My, int Mx,
                         int a_lo, int a_hi, int b_lo, int b_hi,
                         const int *px, const int *py, long npts,
                         double *out, int nthreads, int boundary)
{
    if (H <= 0 || W <= 0 || sigma <= 0.0 || Mx <= 0 || My <= 0 || (Mx & 1) || (My & 1)
        || a_hi < a_lo || b_hi < b_lo || boundary < 0 || boundary > 2)
        return -1;
    const int na = a_hi - a_lo + 1, nb = b_hi - b_lo + 1;
    const size_t nw = (size_t)na * nb;
    /* w[v][u][j][i] = exp(-i 2 pi (u a / Mx + v b / My)) S(Mx/2 - a) S(My/2 - b). */
    double *wr = (double *)malloc(sizeof(double) * nw * Mx * My);
    double *wi = (double *)malloc(sizeof(double) * nw * Mx * My);
    if (!wr || !wi) { free(wr); free(wi); return -2; }
    for (int v = 0; v < My; ++v)
        for (int u = 0; u < Mx; ++u)
            for (int j = 0; j < nb; ++j)
                for (int i = 0; i < na; ++i) {
                    const int a = a_lo + i, b = b_lo + j;
                    const int ra = ((u * a) % Mx + Mx) % Mx;
                    const int rb = ((v * b) % My + My) % My;
                    const double phase = -2.0 * M_PI * ((double)ra / Mx + (double)rb / My);
                    const double g = oracle_gauss((double)(Mx / 2 - a), sigma)
                                   * oracle_gauss((double)(My / 2 - b), sigma);
                    const size_t idx = (((size_t)v * Mx + u) * nb + j) * na + i;
                    wr[idx] = cos(phase) * g;
                    wi[idx] = sin(phase) * g;
                }
    const long n = px ? npts : (long)H * W;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < n; ++p) {
        const int x = px ? px[p] : (int)(p % W);
        const int y = px ? py[p] : (int)(p / W);
        const int xh = x - Mx / 2, yh = y - My / 2;
        for (int v = 0; v < My; ++v)
            for (int u = 0; u < Mx; ++u) {
                double sr = 0.0, si = 0.0;
                const size_t base = ((size_t)v * Mx + u) * nw;
                for (int j = 0; j < nb; ++j) {
                    const int yy = ext_index(yh + b_lo + j, H, boundary);
                    if (yy < 0) continue;
                    for (int i = 0; i < na; ++i) {
                        const int xx = ext_index(xh + a_lo + i, W, boundary);
                        if (xx < 0) continue;
                        const double a = f_re[(size_t)yy * W + xx];
                        const double b = f_im ? f_im[(size_t)yy * W + xx] : 0.0;
                        const double cr = wr[base + (size_t)j * na + i];
                        const double ci = wi[base + (size_t)j * na + i];
                        sr += a * cr - b * ci;
                        si += a * ci + b * cr;
                    }
                }
                const size_t o = (((size_t)v * Mx + u) * n + p) * 2;
                out[o] = sr;
                out[o + 1] = si;
            }
    }
    free(wr);
    free(wi);
    return 0;
}

int oracle_sdft_direct(const double *f_re, const double *f_im, int H, int W,
                       double sigma, int My, int Mx,
                       int a_lo, int a_hi, int b_lo, int b_hi,
                       const int *px, const int *py, long npts,
                       double *out, int nthreads)
{
    return oracle_sdft_direct_b(f_re, f_im, H, W, sigma, My, Mx, a_lo, a_hi, b_lo, b_hi, px, py, npts,
                                out, nthreads, 0);
}

/*
 * ---------------------------------------------------------------------------------------
 * Recursive (IIR) Gaussian variant of Algorithm 1 (Sec. II adopts the recursive Gaussian of
 * Young and van Vliet; approximate, assessed by SER against the FIR result, Sec. IV-C).
 *
 * The smoother is the third-order forward / backward recursion of Young and van Vliet,
 * "Recursive implementation of the Gaussian filter", Signal Processing 44 (1995): with
 *   q  = 0.98711 sigma - 0.96330                    (sigma >= 2.5)
 *   q  = 3.97156 - 4.14554 sqrt(1 - 0.26891 sigma)  (0.5 <= sigma < 2.5)
 *   b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3
 *   b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3
 *   b2 = -(1.4281 q^2 + 1.26661 q^3),  b3 = 0.422205 q^3,  B = 1 - (b1 + b2 + b3) / b0
 * forward  w[n] = B x[n] + (b1 w[n-1] + b2 w[n-2] + b3 w[n-3]) / b0
 * backward y[n] = B w[n] + (b1 y[n+1] + b2 y[n+2] + b3 y[n+3]) / b0.
 * A signal of n samples is extended by P = ceil(12 sigma) + 32 samples on each side (zeros for
 * boundary 0, the extension rule otherwise); the recursions start from zero state at the
 * ends of the extended range.
 */
void oracle_iir_coeffs(double sigma, double c[4])
{
    const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330
                                  : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    const double q2 = q * q, q3 = q2 * q;
    const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    const double b2 = -(1.4281 * q2 + 1.26661 * q3);
    const double b3 = 0.422205 * q3;
    c[0] = 1.0 - (b1 + b2 + b3) / b0;
    c[1] = b1 / b0;
    c[2] = b2 / b0;
    c[3] = b3 / b0;
}

int oracle_iir_pad(double sigma) { return (int)ceil(12.0 * sigma) + 32; }

/* In place: the forward then backward recursion over x[0 .. n-1] (zero state outside). */
static void iir_smooth(double *x, long n, const double c[4])
{
    double w1 = 0.0, w2 = 0.0, w3 = 0.0;
    for (long i = 0; i < n; ++i) {
        const double w = c[0] * x[i] + c[1] * w1 + c[2] * w2 + c[3] * w3;
        w3 = w2;
        w2 = w1;
        w1 = w;
        x[i] = w;
    }
    w1 = w2 = w3 = 0.0;
    for (long i = n - 1; i >= 0; --i) {
        const double y = c[0] * x[i] + c[1] * w1 + c[2] * w2 + c[3] * w3;
        w3 = w2;
        w2 = w1;
        w1 = y;
        x[i] = y;
    }
}

/* The recursive smoother alone on a real signal x[0 .. n-1] (extended per `boundary`): out[n]. */
int oracle_iir_smooth(const double *x, int n, double sigma, int boundary, double *out)
{
    if (n <= 0 || sigma < 0.5 || boundary < 0 || boundary > 2) return -1;
    const int P = oracle_iir_pad(sigma);
    const long m = (long)n + 2 * P;
    double *t = (double *)malloc(sizeof(double) * (size_t)m);
    if (!t) return -2;
    double c[4];
    oracle_iir_coeffs(sigma, c);
    for (long i = 0; i < m; ++i) {
        const int k = ext_index((int)(i - P), n, boundary);
        t[i] = k >= 0 ? x[k] : 0.0;
    }
    iir_smooth(t, m, c);
    for (int i = 0; i < n; ++i) out[i] = t[i + P];
    free(t);
    return 0;
}

/*
 * Algorithm 1 with the recursive smoother, in the paper's steps and notation, for one
 * (omega, theta, sigma): f_c, f_s (Eq. 5) are smoothed along x, J = e^{i w^c x} (S*f_c -
 * i S*f_s) (Eq. 5-6); then along y the complex signal J(x, l) e^{-i w^s l} is smoothed and
 * remodulated, F(x, y) = e^{i w^s y} [S * (J e^{-i w^s .})](y) (Eq. 7-10 written in complex
 * form).  Rows and columns are processed over the extended range [-P, n + P).
 * out: 2*H*W doubles (re, im).
 */
int oracle_iir_gabor(const double *f, int H, int W, double omega, double theta, double sigma,
                     int boundary, double *out, int nthreads)
{
    if (H <= 0 || W <= 0 || sigma < 0.5 || boundary < 0 || boundary > 2) return -1;
    const int P = oracle_iir_pad(sigma);
    const long He = (long)H + 2 * P, We = (long)W + 2 * P;
    double c[4];
    oracle_iir_coeffs(sigma, c);
    const double wc = omega * cos(theta), ws = omega * sin(theta);
    /* J over every extended row y in [-P, H + P) and the image columns x in [0, W) */
    double *J = (double *)malloc(sizeof(double) * 2 * (size_t)He * W);
    if (!J) return -2;
    set_threads(nthreads);
    int fail = 0;
#pragma omp parallel
    {
        double *tc = (double *)malloc(sizeof(double) * (size_t)We);
        double *ts = (double *)malloc(sizeof(double) * (size_t)We);
        if (!tc || !ts) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (long r = 0; r < He; ++r) {
                const int yy = ext_index((int)(r - P), H, boundary);
                for (long i = 0; i < We; ++i) {
                    const long x = i - P;
                    const int xx = ext_index((int)x, W, boundary);
                    const double v = (yy >= 0 && xx >= 0) ? f[(size_t)yy * W + xx] : 0.0;
                    tc[i] = v * cos(wc * (double)x);
                    ts[i] = v * sin(wc * (double)x);
                }
                iir_smooth(tc, We, c);
                iir_smooth(ts, We, c);
                for (int x = 0; x < W; ++x) {
                    const double A = tc[x + P], Bs = ts[x + P];
                    const double co = cos(wc * x), si = sin(wc * x);
                    /* J = e^{i wc x} (A - i B) */
                    J[2 * ((size_t)r * W + x)] = co * A + si * Bs;
                    J[2 * ((size_t)r * W + x) + 1] = si * A - co * Bs;
                }
            }
        }
        free(tc);
        free(ts);
    }
    if (fail) { free(J); return -2; }
#pragma omp parallel
    {
        double *tr = (double *)malloc(sizeof(double) * (size_t)He);
        double *ti = (double *)malloc(sizeof(double) * (size_t)He);
        if (tr && ti) {
#pragma omp for schedule(static)
            for (int x = 0; x < W; ++x) {
                for (long r = 0; r < He; ++r) {
                    const double y = (double)(r - P);
                    const double a = J[2 * ((size_t)r * W + x)], b = J[2 * ((size_t)r * W + x) + 1];
                    const double co = cos(ws * y), si = sin(ws * y);
                    /* J e^{-i ws y} */
                    tr[r] = a * co + b * si;
                    ti[r] = b * co - a * si;
                }
                iir_smooth(tr, He, c);
                iir_smooth(ti, He, c);
                for (int y = 0; y < H; ++y) {
                    const double a = tr[y + P], b = ti[y + P];
                    const double co = cos(ws * y), si = sin(ws * y);
                    out[2 * ((size_t)y * W + x)] = a * co - b * si;
                    out[2 * ((size_t)y * W + x) + 1] = a * si + b * co;
                }
            }
        }
        free(tr);
        free(ti);
    }
    free(J);
    return 0;
}
