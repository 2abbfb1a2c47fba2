/*
 * FP64 CPU oracle for the analytic ball-union correlation of Behandish & Ilies,
 * "Analytic methods for geometric modeling via spherical decomposition".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Two layers, both in double precision and written as plain loops:
 *
 *  (a) exact:  g(R,t) = sum_{i in A, j in B} V(r_i, r_j, |c_i - R c_j - t|),
 *      the pairwise form of Eq. (convgP) (Sec. 3.1) with indicator balls (the
 *      alpha -> infinity limit of Eq. (psi), Sec. 2.2), where the primitive
 *      obstacle f_B1 * f_B2 evaluated at distance d is the volume V of the
 *      intersection of two balls.  Periodised with period P per axis.
 *
 *  (b) band-limited: the Fourier form the method computes.
 *      S_{X,l}(m) = sum_{j in X, level l} exp(-2 pi i m.x_j / P)   Eq. (rhoPhat), Sec. 2.5
 *      f^_X(m)    = sum_l h^(rho_l, 2 pi |m| / P) S_{X,l}(m)        Eq. (fballhat), Sec. 2.5
 *      g^(m)      = f^_A(m) conj(f^_{RB}(m))                         Eq. (ccghat), Sec. 3.2
 *      g(t)       = P^-3 sum_m g^(m) exp(+2 pi i m.t / P)            App. C (CFT, Fourier series)
 *      with modes m in [-N/2, N/2)^3, every mode with a component equal to
 *      -N/2 set to zero (so g^ is exactly Hermitian and g exactly real), and
 *      the translation grid t_k = -P/2 + k P / N.
 *
 * The lifted (4D) nonequiradius correlation of Sec. 3.2 has its own exact
 * layer at the end of this file (bco_lifted_exact); its band-limited layer is
 * a direct 4D NDFT written with numpy in oracle/__init__.py.
 *
 * Conventions: knots are (x, y, z) triples; B is rotated by the unit quaternion
 * q = (w, x, y, z) about its own origin and then translated by t (App. B, the
 * action (R, t)x = Rx + t).  Spectra are stored as the Hermitian half
 * [ix][iy][iz], ix, iy in FFT order (index i <-> m = i for i < N/2, i - N
 * otherwise), iz = m_z in [0, N/2], complex numbers as interleaved (re, im).
 * The output translation grid is [kx][ky][kz] with kz fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ lens V */
/* Volume of the intersection of two balls with radii r1, r2 whose centres are
 * d apart: the value of f_B1 * f_B2 (Sec. 3.1, primitive obstacle B_O of radius
 * r1 + r2) for indicator kernels.  Elementary geometry: the lens is the union
 * of two spherical caps cut by the radical plane. */
double bco_lens_volume(double r1, double r2, double d)
{
    if (d < 0) d = -d;
    if (d >= r1 + r2) return 0.0;
    double rmin = r1 < r2 ? r1 : r2;
    if (d <= fabs(r1 - r2)) return 4.0 / 3.0 * M_PI * rmin * rmin * rmin;
    double s = r1 + r2 - d;
    return M_PI * s * s * (d * d + 2.0 * d * (r1 + r2) - 3.0 * (r1 - r2) * (r1 - r2)) / (12.0 * d);
}

void bco_lens_volume_many(int n, const double *r1, const double *r2, const double *d, double *out)
{
    for (int i = 0; i < n; i++) out[i] = bco_lens_volume(r1[i], r2[i], d[i]);
}

/* ------------------------------------------------------------- ball FT h^ */
/* Fourier transform of the indicator of a ball of radius r at angular
 * wavenumber k = 2 pi |omega| under F{f}(omega) = int f(x) exp(-2 pi i omega.x) dx
 * (Eq. (CFT_int), App. C):  h^(r,k) = 4 pi (sin kr - kr cos kr) / k^3.
 * For x = kr < 0.5 the Maclaurin series of sin x - x cos x is summed instead:
 * sin x - x cos x = sum_{k>=1} (-1)^(k+1) 2k x^(2k+1) / (2k+1)!, which avoids
 * the cancellation of the closed form near k = 0; h^(r,0) = 4 pi r^3 / 3. */
double bco_ball_ft(double r, double k)
{
    double x = k * r;
    if (x < 0.5) {
        /* h^ = 4 pi r^3 * sum_{k>=1} (-1)^(k+1) 2k x^(2k-2) / (2k+1)! */
        double sum = 0.0, xp = 1.0, fact = 6.0; /* (2k+1)! for k = 1 */
        for (int kk = 1; kk <= 12; kk++) {
            double term = 2.0 * kk * xp / fact;
            sum += (kk & 1) ? term : -term;
            xp *= x * x;
            fact *= (double)(2 * kk + 2) * (double)(2 * kk + 3);
        }
        return 4.0 * M_PI * r * r * r * sum;
    }
    return 4.0 * M_PI * (sin(x) - x * cos(x)) / (k * k * k);
}

void bco_ball_ft_many(int n, const double *r, const double *k, double *out)
{
    for (int i = 0; i < n; i++) out[i] = bco_ball_ft(r[i], k[i]);
}

/* ------------------------------------------------------------- rotations */
/* Rotation matrix (row major) of the unit quaternion q = (w, x, y, z), after
 * normalisation (App. B: R in SO(3)).  q and -q give the same matrix. */
int bco_quat_to_matrix(const double *q, double *R)
{
    double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(n2 > 0.0)) return -1;
    double s = 1.0 / sqrt(n2);
    double w = q[0] * s, x = q[1] * s, y = q[2] * s, z = q[3] * s;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    return 0;
}

/* out_j = R c_j (Eq. (Mink0), Sec. 2.4: a rigid motion only moves the centres). */
int bco_rotate(int n, const double *xyz, const double *q, double *out)
{
    double R[9];
    if (bco_quat_to_matrix(q, R)) return -1;
    for (int j = 0; j < n; j++) {
        const double *c = xyz + 3 * j;
        for (int a = 0; a < 3; a++)
            out[3 * j + a] = R[3 * a] * c[0] + R[3 * a + 1] * c[1] + R[3 * a + 2] * c[2];
    }
    return 0;
}

/* --------------------------------------------------------- layer (a) exact */
/* Wrap one coordinate difference into [-P/2, P/2) (nearest periodic image). */
static double min_image(double v, double P)
{
    return v - P * floor(v / P + 0.5);
}

/* g_per(t) = sum_i sum_j V(r_i, r_j, |c_i - R c_j - t| taken at the nearest
 * periodic image), for each of the nt translations t.  Every pair of balls
 * overlaps through at most one periodic image when r_i + r_j < P/2, which the
 * caller guarantees (returns -2 otherwise); then the nearest image is the only
 * nonzero term of the periodic sum sum_n g(t + n P).  q may be NULL (no rotation). */
int bco_exact_corr(int na, const double *xa, const double *ra,
                   int nb, const double *xb, const double *rb,
                   const double *q, double P, int nt, const double *t, double *out)
{
    double rmax_a = 0, rmax_b = 0;
    for (int i = 0; i < na; i++) if (ra[i] > rmax_a) rmax_a = ra[i];
    for (int j = 0; j < nb; j++) if (rb[j] > rmax_b) rmax_b = rb[j];
    if (rmax_a + rmax_b >= 0.5 * P) return -2;
    double *yb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    if (q) {
        if (bco_rotate(nb, xb, q, yb)) { free(yb); return -1; }
    } else {
        memcpy(yb, xb, sizeof(double) * 3 * (size_t)nb);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < nt; k++) {
        double acc = 0.0;
        for (int i = 0; i < na; i++) {
            for (int j = 0; j < nb; j++) {
                double dx = min_image(xa[3 * i] - yb[3 * j] - t[3 * k], P);
                double dy = min_image(xa[3 * i + 1] - yb[3 * j + 1] - t[3 * k + 1], P);
                double dz = min_image(xa[3 * i + 2] - yb[3 * j + 2] - t[3 * k + 2], P);
                double d2 = dx * dx + dy * dy + dz * dz;
                double rs = ra[i] + rb[j];
                if (d2 < rs * rs) acc += bco_lens_volume(ra[i], rb[j], sqrt(d2));
            }
        }
        out[k] = acc;
    }
    free(yb);
    return 0;
}

/* --------------------------------------------------- layer (b) band-limited */
static int mode_of(int i, int N) { return i < N / 2 ? i : i - N; }

/* Level-summed shape spectrum on the Hermitian half of the mode box:
 *   f^(m) = sum_l h^(rho_l, 2 pi |m| / P) * sum_{j: level_j = l} exp(-2 pi i m . x_j / P)
 * with x_j = R c_j when q is given.  The phase of a knot factors over the axes,
 * exp(-2 pi i m.x/P) = prod_d exp(-2 pi i m_d x_d / P); the per-axis factors
 * of each knot are tabulated once (one cos/sin each) and multiplied out for
 * every mode.  Output: N*N*(N/2+1) complex as interleaved doubles.
 * Returns 0, -1 for a zero quaternion, -3 for a level out of range. */
int bco_shape_spectrum(int n, const double *xyz, const int *level, int L, const double *radii,
                       const double *q, double P, int N, double *out)
{
    const int H = N / 2 + 1;
    for (int j = 0; j < n; j++)
        if (level[j] < 0 || level[j] >= L) return -3;
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (q) {
        if (bco_rotate(n, xyz, q, x)) { free(x); return -1; }
    } else {
        memcpy(x, xyz, sizeof(double) * 3 * (size_t)n);
    }
    /* per-knot axis factors: e_d[j][i] = exp(-2 pi i m(i) x_{j,d} / P) */
    double *eyr = (double *)malloc(sizeof(double) * (size_t)n * N + 8);
    double *eyi = (double *)malloc(sizeof(double) * (size_t)n * N + 8);
    double *ezr = (double *)malloc(sizeof(double) * (size_t)n * H + 8);
    double *ezi = (double *)malloc(sizeof(double) * (size_t)n * H + 8);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < N; i++) {
            double a = -2.0 * M_PI * mode_of(i, N) * x[3 * j + 1] / P;
            eyr[(size_t)j * N + i] = cos(a);
            eyi[(size_t)j * N + i] = sin(a);
        }
        for (int i = 0; i < H; i++) {
            double a = -2.0 * M_PI * i * x[3 * j + 2] / P;
            ezr[(size_t)j * H + i] = cos(a);
            ezi[(size_t)j * H + i] = sin(a);
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int ix = 0; ix < N; ix++) {
        const int mx = mode_of(ix, N);
        /* S_l(mx, :, :) accumulated per level */
        double *Sr = (double *)calloc((size_t)L * N * H, sizeof(double));
        double *Si = (double *)calloc((size_t)L * N * H, sizeof(double));
        for (int j = 0; j < n; j++) {
            double a = -2.0 * M_PI * mx * x[3 * j] / P;
            double exr = cos(a), exi = sin(a);
            const double *yr = eyr + (size_t)j * N, *yi = eyi + (size_t)j * N;
            const double *zr = ezr + (size_t)j * H, *zi = ezi + (size_t)j * H;
            double *sr = Sr + (size_t)level[j] * N * H, *si = Si + (size_t)level[j] * N * H;
            for (int iy = 0; iy < N; iy++) {
                double pr = exr * yr[iy] - exi * yi[iy];
                double pi = exr * yi[iy] + exi * yr[iy];
                double *rr = sr + (size_t)iy * H, *ri = si + (size_t)iy * H;
                for (int iz = 0; iz < H; iz++) {
                    rr[iz] += pr * zr[iz] - pi * zi[iz];
                    ri[iz] += pr * zi[iz] + pi * zr[iz];
                }
            }
        }
        for (int iy = 0; iy < N; iy++) {
            const int my = mode_of(iy, N);
            for (int iz = 0; iz < H; iz++) {
                double k = 2.0 * M_PI * sqrt((double)mx * mx + (double)my * my + (double)iz * iz) / P;
                double fr = 0.0, fi = 0.0;
                for (int l = 0; l < L; l++) {
                    double h = bco_ball_ft(radii[l], k);
                    fr += h * Sr[((size_t)l * N + iy) * H + iz];
                    fi += h * Si[((size_t)l * N + iy) * H + iz];
                }
                size_t o = (((size_t)ix * N + iy) * H + iz) * 2;
                out[o] = fr;
                out[o + 1] = fi;
            }
        }
        free(Sr);
        free(Si);
    }
    free(x); free(eyr); free(eyi); free(ezr); free(ezi);
    return 0;
}

/* g^(m) = f^_A(m) conj(f^_B(m)); modes with a component equal to -N/2 (and the
 * m_z = N/2 column of the half spectrum, its Hermitian image) are set to 0. */
void bco_corr_spectrum(int N, const double *fa, const double *fb, double *g)
{
    const int H = N / 2 + 1;
    for (int ix = 0; ix < N; ix++)
        for (int iy = 0; iy < N; iy++)
            for (int iz = 0; iz < H; iz++) {
                size_t o = (((size_t)ix * N + iy) * H + iz) * 2;
                int nyq = (ix == N / 2) || (iy == N / 2) || (iz == N / 2);
                double ar = fa[o], ai = fa[o + 1], br = fb[o], bi = fb[o + 1];
                g[o] = nyq ? 0.0 : ar * br + ai * bi;
                g[o + 1] = nyq ? 0.0 : ai * br - ar * bi;
            }
}

/* g(t) = P^-3 sum_m g^(m) exp(+2 pi i m.t / P) at arbitrary t.  The sum runs
 * over the full mode box; the half with m_z < 0 is the complex conjugate of the
 * stored half (Hermitian symmetry of the transform of a real function, App. C),
 * so the full sum equals Re[ sum_{m_z = 0} + 2 sum_{0 < m_z < N/2} ]. */
void bco_inverse_at(int N, double P, const double *g, int nt, const double *t, double *out)
{
    const int H = N / 2 + 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nt; k++) {
        double *exr = (double *)malloc(sizeof(double) * (4 * (size_t)N + 2 * (size_t)H));
        double *exi = exr + N, *eyr = exi + N, *eyi = eyr + N; /* N each */
        double *ezr = eyi + N, *ezi = ezr + H;                  /* H each */
        for (int i = 0; i < N; i++) {
            double a = 2.0 * M_PI * mode_of(i, N) * t[3 * k] / P;
            exr[i] = cos(a); exi[i] = sin(a);
            double b = 2.0 * M_PI * mode_of(i, N) * t[3 * k + 1] / P;
            eyr[i] = cos(b); eyi[i] = sin(b);
        }
        for (int i = 0; i < H; i++) {
            double w = (i == 0) ? 1.0 : 2.0;
            double a = 2.0 * M_PI * i * t[3 * k + 2] / P;
            ezr[i] = w * cos(a); ezi[i] = w * sin(a);
        }
        double acc = 0.0;
        for (int ix = 0; ix < N; ix++) {
            for (int iy = 0; iy < N; iy++) {
                double pr = exr[ix] * eyr[iy] - exi[ix] * eyi[iy];
                double pi = exr[ix] * eyi[iy] + exi[ix] * eyr[iy];
                const double *gg = g + (((size_t)ix * N + iy) * H) * 2;
                double sr = 0.0, si = 0.0;
                for (int iz = 0; iz < H; iz++) {
                    sr += gg[2 * iz] * ezr[iz] - gg[2 * iz + 1] * ezi[iz];
                    si += gg[2 * iz] * ezi[iz] + gg[2 * iz + 1] * ezr[iz];
                }
                acc += pr * sr - pi * si; /* real part of (p * s) */
            }
        }
        out[k] = acc / (P * P * P);
        free(exr);
    }
}

/* The same sum on the whole translation grid t_k = -P/2 + k P / N, done as
 * three direct (not fast) one-dimensional sums, z then y then x, since the
 * exponential factors over the axes.  out: N^3 doubles, [kx][ky][kz]. */
void bco_inverse_grid(int N, double P, const double *g, double *out)
{
    const int H = N / 2 + 1;
    const size_t NN = (size_t)N * N;
    double *er = (double *)malloc(sizeof(double) * NN), *ei = (double *)malloc(sizeof(double) * NN);
    for (int i = 0; i < N; i++)
        for (int k = 0; k < N; k++) {
            double tk = -0.5 * P + k * P / N;
            double a = 2.0 * M_PI * mode_of(i, N) * tk / P;
            er[(size_t)i * N + k] = cos(a);
            ei[(size_t)i * N + k] = sin(a);
        }
    /* z: B[ix][iy][kz] = sum_{iz} w(iz) g[ix][iy][iz] exp(2 pi i iz t_kz / P) */
    double *Br = (double *)malloc(sizeof(double) * NN * N), *Bi = (double *)malloc(sizeof(double) * NN * N);
#pragma omp parallel for schedule(static)
    for (int ix = 0; ix < N; ix++)
        for (int iy = 0; iy < N; iy++) {
            const double *gg = g + (((size_t)ix * N + iy) * H) * 2;
            for (int kz = 0; kz < N; kz++) {
                double sr = 0.0, si = 0.0;
                for (int iz = 0; iz < H; iz++) {
                    double w = (iz == 0) ? 1.0 : 2.0;
                    double cr = w * er[(size_t)iz * N + kz], ci = w * ei[(size_t)iz * N + kz];
                    sr += gg[2 * iz] * cr - gg[2 * iz + 1] * ci;
                    si += gg[2 * iz] * ci + gg[2 * iz + 1] * cr;
                }
                Br[((size_t)ix * N + iy) * N + kz] = sr;
                Bi[((size_t)ix * N + iy) * N + kz] = si;
            }
        }
    /* y: C[ix][ky][kz] = sum_{iy} B[ix][iy][kz] exp(2 pi i m(iy) t_ky / P) */
    double *Cr = (double *)malloc(sizeof(double) * NN * N), *Ci = (double *)malloc(sizeof(double) * NN * N);
#pragma omp parallel for schedule(static)
    for (int ix = 0; ix < N; ix++)
        for (int ky = 0; ky < N; ky++)
            for (int kz = 0; kz < N; kz++) {
                double sr = 0.0, si = 0.0;
                for (int iy = 0; iy < N; iy++) {
                    double cr = er[(size_t)iy * N + ky], ci = ei[(size_t)iy * N + ky];
                    double br = Br[((size_t)ix * N + iy) * N + kz], bi = Bi[((size_t)ix * N + iy) * N + kz];
                    sr += br * cr - bi * ci;
                    si += br * ci + bi * cr;
                }
                Cr[((size_t)ix * N + ky) * N + kz] = sr;
                Ci[((size_t)ix * N + ky) * N + kz] = si;
            }
    /* x: g[kx][ky][kz] = P^-3 Re sum_{ix} C[ix][ky][kz] exp(2 pi i m(ix) t_kx / P) */
#pragma omp parallel for schedule(static)
    for (int kx = 0; kx < N; kx++)
        for (int ky = 0; ky < N; ky++)
            for (int kz = 0; kz < N; kz++) {
                double sr = 0.0;
                for (int ix = 0; ix < N; ix++) {
                    double cr = er[(size_t)ix * N + kx], ci = ei[(size_t)ix * N + kx];
                    sr += Cr[((size_t)ix * N + ky) * N + kz] * cr - Ci[((size_t)ix * N + ky) * N + kz] * ci;
                }
                out[((size_t)kx * N + ky) * N + kz] = sr / (P * P * P);
            }
    free(er); free(ei); free(Br); free(Bi); free(Cr); free(Ci);
}

/* ------------------------------------------- lifted (4D) correlation, layer (a) */
/* Nonequiradius correlation of Sec. 3.2 (Eq. (convgA), Lemma 2): knot (x, r) of
 * A lifts to the trimmed half-cone D(x, r) = {(y, s) : |y - x| <= r - s,
 * r - L <= s <= r}; B is rotated and mirrored in r (its knot (c, r') lifts to
 * {(y, s) : |y - R c| <= s + r', -r' <= s <= L - r'}).  The correlation of the
 * two lifted indicator sums at the lifted translation (t, r_s) is the 4D volume
 * of overlap, summed over knot pairs.  At height s the two sections are balls
 * of radii rho1 = r_i - s and rho2 = s + r_j - r_s whose sum S = r_i + r_j - r_s
 * does not depend on s, at centre distance d = |x_i - R c_j - t| (nearest
 * periodic image); so the lens volume is a polynomial in s on each of three
 * pieces (ball 2 inside ball 1, lens, ball 1 inside ball 2) and the integral
 * over s is taken in closed form.  Nonzero only when d < S (Lemma 2 at r_s = 0:
 * the balls intersect).  Requires r_i + r_j + |r_s| < P/2. */
static double lifted_pair(double ri, double rj, double rs, double d, double L)
{
    const double S = ri + rj - rs;
    if (S <= 0.0 || d >= S) return 0.0;
    double lo = ri - L > rs - rj ? ri - L : rs - rj;
    double hi = ri < rs - rj + L ? ri : rs - rj + L;
    if (hi <= lo) return 0.0;
    const double c = ri - rj + rs; /* delta(s) = rho1 - rho2 = c - 2 s */
    const double b1 = 0.5 * (c - d), b2 = 0.5 * (c + d);
    double v = 0.0;
    /* s < b1: delta > d, ball 2 inside ball 1: (4/3) pi rho2^3, d rho2 / ds = 1 */
    {
        double a = lo, b = hi < b1 ? hi : b1;
        if (b > a) {
            double p = a + rj - rs, q = b + rj - rs;
            v += M_PI / 3.0 * (q * q * q * q - p * p * p * p);
        }
    }
    /* b1 < s < b2: the lens pi (S - d)^2 (d^2 + 2 d S - 3 delta^2) / (12 d) */
    if (d > 0.0) {
        double a = lo > b1 ? lo : b1, b = hi < b2 ? hi : b2;
        if (b > a) {
            double da = c - 2.0 * a, db = c - 2.0 * b;
            double int_delta2 = (da * da * da - db * db * db) / 6.0;
            v += M_PI * (S - d) * (S - d) / (12.0 * d) * ((d * d + 2.0 * d * S) * (b - a) - 3.0 * int_delta2);
        }
    }
    /* s > b2: delta < -d, ball 1 inside ball 2: (4/3) pi rho1^3, d rho1 / ds = -1 */
    {
        double a = lo > b2 ? lo : b2, b = hi;
        if (b > a) {
            double p = ri - a, q = ri - b;
            v += M_PI / 3.0 * (p * p * p * p - q * q * q * q);
        }
    }
    return v;
}

double bco_lifted_pair(double ri, double rj, double rs, double d, double L) { return lifted_pair(ri, rj, rs, d, L); }

int bco_lifted_exact(int na, const double *xa, const double *ra, int nb, const double *xb, const double *rb,
                     const double *q, double L, double P, double rs, int nt, const double *t, double *out)
{
    double rmax_a = 0, rmax_b = 0;
    for (int i = 0; i < na; i++) if (ra[i] > rmax_a) rmax_a = ra[i];
    for (int j = 0; j < nb; j++) if (rb[j] > rmax_b) rmax_b = rb[j];
    if (rmax_a + rmax_b + fabs(rs) >= 0.5 * P) return -2;
    double *yb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    if (q) {
        if (bco_rotate(nb, xb, q, yb)) { free(yb); return -1; }
    } else {
        memcpy(yb, xb, sizeof(double) * 3 * (size_t)nb);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < nt; k++) {
        double acc = 0.0;
        for (int i = 0; i < na; i++) {
            for (int j = 0; j < nb; j++) {
                double dx = min_image(xa[3 * i] - yb[3 * j] - t[3 * k], P);
                double dy = min_image(xa[3 * i + 1] - yb[3 * j + 1] - t[3 * k + 1], P);
                double dz = min_image(xa[3 * i + 2] - yb[3 * j + 2] - t[3 * k + 2], P);
                acc += lifted_pair(ra[i], rb[j], rs, sqrt(dx * dx + dy * dy + dz * dz), L);
            }
        }
        out[k] = acc;
    }
    free(yb);
    return 0;
}
