// Lifted (4D) nonequiradius correlation of Sec. 3.2 (Eqs. (rhoA), (rhoAhat),
// (fconehat), (convgA); Lemma 2), computed as a direct 4D NDFT.
//
// Knot (x, r) of a shape lifts to the trimmed half-cone D(x, r) (Eq. (L2cone))
// whose r = 0 section is the ball of radius r; B is rotated and mirrored in r
// (the pre-reflection of Sec. 3.2).  In the Fourier domain
//     rho^_X(xi, eta) = sum_i exp(-2 pi i (xi . x_i / P + eta r_i / P_r))     (Eq. (rhoAhat))
//     g^(xi, eta)     = rho^_A conj(rho^_{R B mirrored}) f^_D0(xi, eta)^2       (Eq. (convgA) in Fourier form)
//     f^_D0(xi, eta)  = int_0^L h^(s, 2 pi |xi| / P) exp(+2 pi i eta s / P_r) ds
//     g(t, r_s)       = P^-3 P_r^-1 sum g^ exp(2 pi i (xi . t / P + eta r_s / P_r))
// with xi in [-N/2, N/2)^3, eta in [-N_r/2, N_r/2), lower-edge modes zero.
// The r = 0 section of g is the 4D overlap volume of the two cone unions,
// positive exactly where the two ball unions meet (Lemma 2); other sections
// are the obstacles of offset shapes.
//
//   k_lift_gauss      Gauss-Legendre nodes on [-1, 1] (Newton on the Legendre
//                     three-term recurrence; Golub & Welsch 1969 give the same
//                     nodes) for the cone transform, FP64;
//   k_lift_cone       f^_D0 per (|xi|^2, eta) by that quadrature, FP64, rounded once;
//   k_lift_twiddles   exp(-2 pi i k / N), FP64, rounded once;
//   k_lift_phases     per knot and axis the factors exp(-2 pi i m x_a / P) and
//                     exp(-2 pi i eta r / P_r) (FP64 arguments, rounded once),
//                     knot-major, after rotating and mirroring B;
//   k_lift_ndft       rho^ as a contraction over the knots of the separable
//                     factors: rows (xi_x, xi_y), columns (xi_z, eta), 64 x 64
//                     output tiles, knots split across blocks (FP32 on the
//                     CUDA cores, partial sums added with vector atomics);
//   k_lift_scale      each knot's coordinates over the periods, rotated and
//                     mirrored (FP64, and as 32-bit fixed-point fractions);
//   k_lift_operands,  the default contraction (bc_lift_umma.cuh): the phase matrices
//   k_lift_gemm_umma  written as split-TF32 operand blocks in the tensor core's
//                     shared-memory layout, then their complex product with
//                     tcgen05.mma, accumulators in tensor memory;
//   k_lift_planes,    the legacy tensor-core contraction: real / imaginary
//   k_lift_gemm_tc    planes, then mma.sync in 3-pass split TF32 with cp.async
//                     double buffering;
//   k_lift_collapse   per translation mode and section r_s the sum over eta of
//                     rho^_A conj(rho^_B) f^_D0^2 exp(2 pi i eta r_s / P_r), with
//                     the P^-3 P_r^-1 scale and the grid-origin sign;
//   k_lift_ifft_x     inverse transform along x; the inverse along y and the
//                     complex-to-real inverse along z are the correlation's own
//                     passes (k_ifft_y, k_ifft_z).
// Contraction 3 computes both spectra by the 4D type-1 NUFFT and forms the
// collapse from them in bc_lift_nufft.cu (lift4_pair), in place of the direct
// contractions and k_lift_collapse.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ballcorr.h"
#include "bc_device.cuh"
#include "bc_lift4.h"
#include "bc_lift_umma.cuh"

namespace bc {

constexpr int LIFT_GAUSS = 48;   // quadrature nodes of the cone transform
constexpr int LIFT_TILE = 64;    // output tile of the contraction (rows and columns)
constexpr int LIFT_KC = 32;      // knots staged per step
constexpr int LIFT_MAX_SLICES = 16;
constexpr int LIFT_CHUNK = 32768; // knots per pass of the tensor-core contractions (bounds their operand memory)

__device__ __forceinline__ int lift_mode(int j, int n) { return j < n / 2 ? j : j - n; }

// Node k of the n-point Gauss-Legendre rule and its weight.
__global__ void k_lift_gauss(int n, double *x, double *w)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double pi = 3.14159265358979323846;
    double z = cos(pi * (k + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = z;
        for (int j = 1; j < n; j++) {
            const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    x[k] = z;
    w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// cone[q * Nr + e] = f^_D0 at |xi|^2 = q and eta = mode(e).
__global__ void k_lift_cone(int qmax, int Nr, double L, double period, double period_r, const double *__restrict__ gx,
                            const double *__restrict__ gw, float2 *cone)
{
    const double pi = 3.14159265358979323846;
    const int total = (qmax + 1) * Nr;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        const int q = u / Nr, e = u - q * Nr;
        const double k = 2.0 * pi * sqrt((double)q) / period;
        const double alpha = 2.0 * pi * lift_mode(e, Nr) / period_r;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < LIFT_GAUSS; j++) {
            const double s = 0.5 * L * (gx[j] + 1.0);
            const double h = 0.5 * L * gw[j] * ball_ft64(s, k);
            double sn, cs;
            sincos(alpha * s, &sn, &cs);
            re += h * cs;
            im += h * sn;
        }
        cone[u] = make_float2((float)re, (float)im);
    }
}

__global__ void k_lift_twiddles(int N, float2 *tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double sn, cs;
    sincospi(2.0 * k / N, &sn, &cs);
    tw[k] = make_float2((float)cs, (float)-sn);
}

// Per knot: E[i * T + m] for the T = N + N + N/2 + Nr factors of knot i
// (x modes, y modes in FFT order; z modes 0 .. N/2 - 1; eta modes in FFT order).
__global__ void k_lift_phases(const float4 *__restrict__ knots, int n, double qw, double qx, double qy, double qz,
                              int mirror, int N, int Nr, double period, double period_r, float2 *E)
{
    const int T = 2 * N + N / 2 + Nr;
    const int i = blockIdx.x;
    if (i >= n) return;
    const float4 c = knots[i];
    // R from the unit quaternion (w, x, y, z)
    const double R00 = 1 - 2 * (qy * qy + qz * qz), R01 = 2 * (qx * qy - qw * qz), R02 = 2 * (qx * qz + qw * qy);
    const double R10 = 2 * (qx * qy + qw * qz), R11 = 1 - 2 * (qx * qx + qz * qz), R12 = 2 * (qy * qz - qw * qx);
    const double R20 = 2 * (qx * qz - qw * qy), R21 = 2 * (qy * qz + qw * qx), R22 = 1 - 2 * (qx * qx + qy * qy);
    const double x = R00 * c.x + R01 * c.y + R02 * c.z;
    const double y = R10 * c.x + R11 * c.y + R12 * c.z;
    const double z = R20 * c.x + R21 * c.y + R22 * c.z;
    const double r = mirror ? -(double)c.w : (double)c.w;
    for (int m = threadIdx.x; m < T; m += blockDim.x) {
        double v, arg;
        if (m < N) {
            v = x / period;
            arg = lift_mode(m, N) * v;
        } else if (m < 2 * N) {
            v = y / period;
            arg = lift_mode(m - N, N) * v;
        } else if (m < 2 * N + N / 2) {
            v = z / period;
            arg = (m - 2 * N) * v;
        } else {
            v = r / period_r;
            arg = lift_mode(m - 2 * N - N / 2, Nr) * v;
        }
        arg -= rint(arg); // exp(-2 pi i arg) depends on arg mod 1 only
        double sn, cs;
        sincospi(2.0 * arg, &sn, &cs);
        E[(long long)i * T + m] = make_float2((float)cs, (float)-sn);
    }
}

// out[a][b] += sum_{i in this block's knot range} E1[a][i] E2[b][i], a = (xi_x, xi_y)
// (rows, N * N), b = (xi_z, eta) (columns, N/2 * Nr), E1 = Ex Ey, E2 = Ez Er.
// Thread t owns the 4 x 4 outputs rows 4 (t / 16) .., columns 4 (t % 16) ...
__global__ void __launch_bounds__(256)
k_lift_ndft(const float2 *__restrict__ E, int n, int N, int Nr, int kper, float2 *out)
{
    __shared__ float2 E1s[LIFT_KC][LIFT_TILE], E2s[LIFT_KC][LIFT_TILE];
    const int T = 2 * N + N / 2 + Nr;
    const int C = (N / 2) * Nr;
    const int a0 = blockIdx.y * LIFT_TILE, b0 = blockIdx.x * LIFT_TILE;
    const int k_begin = blockIdx.z * kper, k_end = min(n, k_begin + kper);
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = make_float2(0.f, 0.f);
    for (int k0 = k_begin; k0 < k_end; k0 += LIFT_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < LIFT_KC * LIFT_TILE; e += blockDim.x) {
            const int kk = e / LIFT_TILE, j = e - kk * LIFT_TILE;
            const int i = k0 + kk;
            float2 v1 = make_float2(0.f, 0.f), v2 = make_float2(0.f, 0.f);
            if (i < k_end) {
                const float2 *Ei = E + (long long)i * T;
                const int a = a0 + j, ax = a / N, ay = a - ax * N;
                v1 = cmul(Ei[ax], Ei[N + ay]);
                const int b = b0 + j, bz = b / Nr, be = b - bz * Nr;
                v2 = cmul(Ei[2 * N + bz], Ei[2 * N + N / 2 + be]);
            }
            E1s[kk][j] = v1;
            E2s[kk][j] = v2;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < LIFT_KC; kk++) {
            float2 x[4], y[4];
#pragma unroll
            for (int r = 0; r < 4; r++) x[r] = E1s[kk][4 * tr + r];
#pragma unroll
            for (int c = 0; c < 4; c++) y[c] = E2s[kk][4 * tc + c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    acc[r][c].x = fmaf(x[r].x, y[c].x, fmaf(-x[r].y, y[c].y, acc[r][c].x));
                    acc[r][c].y = fmaf(x[r].x, y[c].y, fmaf(x[r].y, y[c].x, acc[r][c].y));
                }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++)
            atomicAdd(out + (long long)(a0 + 4 * tr + r) * C + b0 + 4 * tc + c, acc[r][c]);
}

// Split TF32 on the tensor cores: each FP32 factor is split into TF32 parts
// x = x_hi + x_lo (x_hi = tf32(x), x_lo = tf32(x - x_hi)) and each real
// product formed as a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation
// (mma.sync m16n8k8 .tf32; the a_lo b_lo term, 2^-22 relative, is dropped).
struct LiftU { // a knot's coordinates over the periods: x / P, y / P, z / P, r / P_r
    double x, y, z, w;
};

__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a b in split TF32 (three products)
__device__ __forceinline__ void mma3(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4], unsigned bh0,
                                     unsigned bh1, unsigned bl0, unsigned bl1)
{
    mma_tf32(d, ah, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, al, bh0, bh1);
}

// Phase matrices as real / imaginary planes, knots contiguous (leading
// dimension ld >= n, columns n .. ld - 1 zero): rows a < M = N^2 of P1 hold
// exp(-2 pi i (m_x x + m_y y) / P) for a = (j_x, j_y); rows b < C = N/2 Nr of
// P2 hold exp(-2 pi i (m_z z / P + eta r / P_r)) for b = (m_z, j_eta).  The
// argument is formed and reduced mod 1 in FP64 from the knot's scaled
// coordinates (u = x / P etc., rotated and mirrored for B), then sincospi runs
// in FP32 on the reduced value.
__global__ void k_lift_scale(const float4 *__restrict__ knots, int n, double qw, double qx, double qy, double qz,
                             int mirror, double period, double period_r, LiftU *u, LiftQ *fq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 c = knots[i];
    const double R00 = 1 - 2 * (qy * qy + qz * qz), R01 = 2 * (qx * qy - qw * qz), R02 = 2 * (qx * qz + qw * qy);
    const double R10 = 2 * (qx * qy + qw * qz), R11 = 1 - 2 * (qx * qx + qz * qz), R12 = 2 * (qy * qz - qw * qx);
    const double R20 = 2 * (qx * qz - qw * qy), R21 = 2 * (qy * qz + qw * qx), R22 = 1 - 2 * (qx * qx + qy * qy);
    const LiftU v{(R00 * c.x + R01 * c.y + R02 * c.z) / period, (R10 * c.x + R11 * c.y + R12 * c.z) / period,
                  (R20 * c.x + R21 * c.y + R22 * c.z) / period, (mirror ? -(double)c.w : (double)c.w) / period_r};
    if (u) u[i] = v;
    if (fq) fq[i] = LiftQ{lift_fixed(v.x), lift_fixed(v.y), lift_fixed(v.z), lift_fixed(v.w)};
}

__global__ void k_lift_planes(const LiftU *__restrict__ u, int n, int ld, int N, int Nr, float *p1re, float *p1im,
                              float *p2re, float *p2im)
{
    const int M = N * N;
    const int row = blockIdx.y; // < M + C
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ld) return;
    float re = 0.f, im = 0.f;
    if (i < n) {
        const LiftU v = u[i];
        double arg;
        if (row < M) {
            const int jx = row / N, jy = row - jx * N;
            arg = lift_mode(jx, N) * v.x + lift_mode(jy, N) * v.y;
        } else {
            const int b = row - M, mz = b / Nr, je = b - mz * Nr;
            arg = mz * v.z + lift_mode(je, Nr) * v.w;
        }
        const float r = (float)(arg - rint(arg));
        float sn, cs;
        sincospif(2.0f * r, &sn, &cs);
        re = cs;
        im = -sn;
    }
    if (row < M) {
        p1re[(long long)row * ld + i] = re;
        p1im[(long long)row * ld + i] = im;
    } else {
        p2re[(long long)(row - M) * ld + i] = re;
        p2im[(long long)(row - M) * ld + i] = im;
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K)); }

// out[a][b] += sum_{i in this block's knot range} P1[a][i] P2[b][i] (complex) on
// the tensor cores.  64 x 64 output tile; the four planes' 64 x 32 tiles of a
// knot chunk are copied with cp.async into a two-stage shared ring (row stride
// LIFT_TS = 36 floats: 16-byte aligned rows, and fragment loads -- lanes
// (g, t) reading row g, column t -- fall on banks 4 g + t, all distinct).
constexpr int LIFT_TS = 36;
constexpr int LIFT_STAGE = 4 * LIFT_TILE * LIFT_TS; // floats per stage (four planes)

__global__ void __launch_bounds__(256)
k_lift_gemm_tc(const float *__restrict__ p1re, const float *__restrict__ p1im, const float *__restrict__ p2re,
               const float *__restrict__ p2im, int ld, int C, int kper, float2 *out)
{
    extern __shared__ float4 lift_sm[];
    float *ring = reinterpret_cast<float *>(lift_sm);
    const int a0 = blockIdx.y * LIFT_TILE, b0 = blockIdx.x * LIFT_TILE;
    const int k_begin = blockIdx.z * kper, k_end = min(ld, k_begin + kper);
    const int nchunk = (k_end - k_begin + LIFT_KC - 1) / LIFT_KC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int g = lane >> 2, t = lane & 3;
    // one chunk = 4 planes x 64 rows x 32 floats = 2048 16-byte pieces, 8 per
    // thread: piece q of thread t is plane q / 2, row ((q mod 2) 256 + t) / 8
    auto issue = [&](int c, int stage) {
        float *dst = ring + stage * LIFT_STAGE;
        const int k0 = k_begin + c * LIFT_KC;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int plane = q >> 1, rem = ((q & 1) << 8) + (int)threadIdx.x, row = rem >> 3, piece = rem & 7;
            const float *src = plane == 0 ? p1re + (long long)(a0 + row) * ld
                             : plane == 1 ? p1im + (long long)(a0 + row) * ld
                             : plane == 2 ? p2re + (long long)(b0 + row) * ld
                                          : p2im + (long long)(b0 + row) * ld;
            cp_async16(dst + plane * LIFT_TILE * LIFT_TS + row * LIFT_TS + piece * 4, src + k0 + piece * 4);
        }
        cp_async_commit();
    };
    float cre[4][4], cim[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) cre[j][q] = cim[j][q] = 0.f;
    if (nchunk > 0) issue(0, 0);
    for (int c = 0; c < nchunk; c++) {
        if (c + 1 < nchunk) {
            issue(c + 1, (c + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *st = ring + (c & 1) * LIFT_STAGE;
        const float *Are = st, *Aim = st + LIFT_TILE * LIFT_TS, *Bre = st + 2 * LIFT_TILE * LIFT_TS,
                    *Bim = st + 3 * LIFT_TILE * LIFT_TS;
#pragma unroll
        for (int ks = 0; ks < LIFT_KC; ks += 8) {
            const int r0 = 16 * wm + g;
            unsigned arh[4], arl[4], aih[4], ail[4];
            split_tf32(Are[r0 * LIFT_TS + ks + t], arh[0], arl[0]);
            split_tf32(Are[(r0 + 8) * LIFT_TS + ks + t], arh[1], arl[1]);
            split_tf32(Are[r0 * LIFT_TS + ks + t + 4], arh[2], arl[2]);
            split_tf32(Are[(r0 + 8) * LIFT_TS + ks + t + 4], arh[3], arl[3]);
            split_tf32(Aim[r0 * LIFT_TS + ks + t], aih[0], ail[0]);
            split_tf32(Aim[(r0 + 8) * LIFT_TS + ks + t], aih[1], ail[1]);
            split_tf32(Aim[r0 * LIFT_TS + ks + t + 4], aih[2], ail[2]);
            split_tf32(Aim[(r0 + 8) * LIFT_TS + ks + t + 4], aih[3], ail[3]);
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const int col = 32 * wn + 8 * nt + g;
                unsigned brh0, brl0, brh1, brl1, bih0, bil0, bih1, bil1;
                split_tf32(Bre[col * LIFT_TS + ks + t], brh0, brl0);
                split_tf32(Bre[col * LIFT_TS + ks + t + 4], brh1, brl1);
                split_tf32(Bim[col * LIFT_TS + ks + t], bih0, bil0);
                split_tf32(Bim[col * LIFT_TS + ks + t + 4], bih1, bil1);
                const unsigned nih0 = bih0 ^ 0x80000000u, nil0 = bil0 ^ 0x80000000u; // -B_im (exact)
                const unsigned nih1 = bih1 ^ 0x80000000u, nil1 = bil1 ^ 0x80000000u;
                // a fresh accumulator per 8-knot step, added to the running sum with
                // round-to-nearest adds (the tensor cores truncate when they accumulate)
                float dre[4] = {0.f, 0.f, 0.f, 0.f}, dim[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(dre, arh, arl, brh0, brh1, brl0, brl1);
                mma3(dre, aih, ail, nih0, nih1, nil0, nil1);
                mma3(dim, arh, arl, bih0, bih1, bil0, bil1);
                mma3(dim, aih, ail, brh0, brh1, brl0, brl1);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    cre[nt][q] += dre[q];
                    cim[nt][q] += dim[q];
                }
            }
        }
        __syncthreads(); // the stage is refilled two chunks later
    }
    const int row = a0 + 16 * wm + g;
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const int col = b0 + 32 * wn + 8 * nt + 2 * t;
        atomicAdd(out + (long long)row * C + col, make_float2(cre[nt][0], cim[nt][0]));
        atomicAdd(out + (long long)row * C + col + 1, make_float2(cre[nt][1], cim[nt][1]));
        atomicAdd(out + (long long)(row + 8) * C + col, make_float2(cre[nt][2], cim[nt][2]));
        atomicAdd(out + (long long)(row + 8) * C + col + 1, make_float2(cre[nt][3], cim[nt][3]));
    }
}

// h[s][jx][jy][mz] = sign scale sum_eta rho^_A conj(rho^_B) cone^2 exp(2 pi i eta r_s / P_r),
// zero on the lower-edge modes; scale = P^-3 P_r^-1, sign = (-1)^(m_x + m_y + m_z).
// NS >= nslices sections are accumulated in registers (the phases of the
// sections beyond nslices are zero, and those sums are not written).
template <int NS>
__global__ void k_lift_collapse(const float2 *__restrict__ ra, const float2 *__restrict__ rb,
                                const float2 *__restrict__ cone, int N, int Nr, const float *__restrict__ slices,
                                int nslices, double period_r, float scale, float2 *h)
{
    __shared__ float2 ph[NS][64];
    for (int e = threadIdx.x; e < NS * Nr; e += blockDim.x) {
        const int s = e / Nr, k = e - s * Nr;
        float2 v = make_float2(0.f, 0.f);
        if (s < nslices) {
            double arg = lift_mode(k, Nr) * (double)slices[s] / period_r;
            arg -= rint(arg);
            double sn, cs;
            sincospi(2.0 * arg, &sn, &cs);
            v = make_float2((float)cs, (float)sn);
        }
        ph[s][k] = v;
    }
    __syncthreads();
    const int H = N / 2;
    const int total = N * N * H;
    const long long plane = (long long)N * N * H;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        const int jx = u / (N * H), rem = u - jx * (N * H);
        const int jy = rem / H, mz = rem - jy * H;
        float2 acc[NS];
#pragma unroll
        for (int s = 0; s < NS; s++) acc[s] = make_float2(0.f, 0.f);
        if (jx != N / 2 && jy != N / 2) {
            const int mx = lift_mode(jx, N), my = lift_mode(jy, N);
            const int q = mx * mx + my * my + mz * mz;
            const long long base = (long long)(jx * N + jy) * (H * Nr) + (long long)mz * Nr;
            // two modes eta per 16-byte load (each thread's N_r values are contiguous, so
            // every sector a warp fetches is used whole)
            const float4 *a4 = reinterpret_cast<const float4 *>(ra + base), *b4 = reinterpret_cast<const float4 *>(rb + base),
                         *c4 = reinterpret_cast<const float4 *>(cone + (long long)q * Nr);
            for (int k2 = 0; k2 < Nr / 2; k2++) {
                const float4 av = a4[k2], bv = b4[k2], fv = c4[k2];
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    const int k = 2 * k2 + hh;
                    if (k == Nr / 2) continue;
                    const float2 a = hh ? make_float2(av.z, av.w) : make_float2(av.x, av.y);
                    const float2 b = hh ? make_float2(bv.z, bv.w) : make_float2(bv.x, bv.y);
                    const float2 f = hh ? make_float2(fv.z, fv.w) : make_float2(fv.x, fv.y);
                    const float2 p = cmul(cmulc(a, b), cmul(f, f));
#pragma unroll
                    for (int s = 0; s < NS; s++) acc[s] = cadd(acc[s], cmul(p, ph[s][k]));
                }
            }
            const float sg = ((mx + my + mz) & 1) ? -scale : scale;
#pragma unroll
            for (int s = 0; s < NS; s++) acc[s] = cscale(acc[s], sg);
        }
#pragma unroll
        for (int s = 0; s < NS; s++)
            if (s < nslices) h[s * plane + u] = acc[s];
    }
}

static cudaError_t launch_lift_collapse(const float2 *ra, const float2 *rb, const float2 *cone, int N, int Nr,
                                        const float *slices, int nslices, double period_r, float scale, float2 *h,
                                        cudaStream_t st)
{
    const int blocks = (int)(((long long)N * N * (N / 2) + 255) / 256);
    if (nslices <= 1) k_lift_collapse<1><<<blocks, 256, 0, st>>>(ra, rb, cone, N, Nr, slices, nslices, period_r, scale, h);
    else if (nslices <= 2) k_lift_collapse<2><<<blocks, 256, 0, st>>>(ra, rb, cone, N, Nr, slices, nslices, period_r, scale, h);
    else if (nslices <= 4) k_lift_collapse<4><<<blocks, 256, 0, st>>>(ra, rb, cone, N, Nr, slices, nslices, period_r, scale, h);
    else if (nslices <= 8) k_lift_collapse<8><<<blocks, 256, 0, st>>>(ra, rb, cone, N, Nr, slices, nslices, period_r, scale, h);
    else k_lift_collapse<16><<<blocks, 256, 0, st>>>(ra, rb, cone, N, Nr, slices, nslices, period_r, scale, h);
    return cudaGetLastError();
}

// Inverse along x, in place: item (slice, jy, chunk of 16 z-modes); 16 lines
// of N values at stride N H.
template <int NI>
__global__ void __launch_bounds__(TB) k_lift_ifft_x(float2 *h, int nslices, const float2 *__restrict__ twg)
{
    __shared__ float2 tw[NI], A[NI * CL], B[NI * CL];
    constexpr int H = NI / 2, nch = H / CL;
    for (int k = threadIdx.x; k < NI; k += blockDim.x) tw[k] = twg[k];
    const int items = nslices * NI * nch;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = it / (NI * nch), rem = it - s * (NI * nch);
        const int jy = rem / nch, ch = rem - jy * nch;
        float2 *base = h + (long long)s * NI * NI * H + (long long)jy * H + ch * CL;
        __syncthreads();
        for (int e = threadIdx.x; e < NI * CL; e += blockDim.x) {
            const int jx = e / CL, c = e - jx * CL;
            A[jx * CL + c] = base[(long long)jx * NI * H + c];
        }
        __syncthreads();
        const float2 *res = il_fft<NI, true, CL, TB>(A, B, tw);
        for (int e = threadIdx.x; e < NI * CL; e += blockDim.x) {
            const int kx = e / CL, c = e - kx * CL;
            base[(long long)kx * NI * H + c] = res[kx * CL + c];
        }
    }
}

} // namespace bc

using namespace bc;

// ------------------------------------------------------------------ C ABI
struct bc_lift_s {
    int device = 0, nsm = 1;
    cudaStream_t stream = nullptr;
    int N = 0, Nr = 0, qmax = 0;
    int contraction = 2;
    double L = 0, period = 2, period_r = 0;
    float2 *cone = nullptr, *tw = nullptr;
    Lift4Tables t4;            // contraction 3 (4D NUFFT): window and transform tables
    void *t4_mem = nullptr;    // their storage
    void *ws = nullptr; // rho^_A, rho^_B, phase tables, h planes, slices, pair descriptors, staging
    size_t ws_bytes = 0;
    char *pin = nullptr; // pinned host staging: sections, pair descriptors, the error word
};

constexpr size_t LIFT_PIN_BYTES = 4096;

static bc_status lift_fail(bc_status s, const std::string &msg)
{
    set_last_error(msg);
    return s;
}

static bc_status lift_cuda(cudaError_t e, const char *where)
{
    set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA;
}

extern "C" {

bc_status bc_lift_create(const bc_lift_params *p, void *cuda_stream, bc_lift_t *out)
{
    if (!p || !out) return lift_fail(BC_ERR_ARG, "bc_lift_create: null pointer");
    *out = nullptr;
    if (p->N != 32 && p->N != 64 && p->N != 96 && p->N != 128)
        return lift_fail(BC_ERR_UNSUPPORTED, "bc_lift_create: N must be 32, 64, 96 or 128");
    if (p->Nr != 8 && p->Nr != 16 && p->Nr != 32 && p->Nr != 64)
        return lift_fail(BC_ERR_UNSUPPORTED, "bc_lift_create: Nr must be 8, 16, 32 or 64");
    if (!(p->L > 0) || !std::isfinite(p->L)) return lift_fail(BC_ERR_ARG, "bc_lift_create: L must be > 0");
    if (!(p->period > 0) || !std::isfinite(p->period)) return lift_fail(BC_ERR_ARG, "bc_lift_create: period must be > 0");
    if (!(p->period_r > 0) || !std::isfinite(p->period_r)) return lift_fail(BC_ERR_ARG, "bc_lift_create: period_r must be > 0");
    if (p->contraction < 0 || p->contraction > 3)
        return lift_fail(BC_ERR_ARG, "bc_lift_create: contraction must be 0, 1, 2 or 3");
    if (p->contraction == 3 && p->Nr < 16)
        return lift_fail(BC_ERR_UNSUPPORTED, "bc_lift_create: the 4D NUFFT (contraction 3) needs Nr >= 16");
    bc_lift_s *lf = new (std::nothrow) bc_lift_s();
    if (!lf) return lift_fail(BC_ERR_OOM, "bc_lift_create: host allocation");
    lf->stream = (cudaStream_t)cuda_stream;
    lf->N = p->N;
    lf->Nr = p->Nr;
    lf->L = p->L;
    lf->period = p->period;
    lf->period_r = p->period_r;
    lf->contraction = p->contraction;
    lf->qmax = 3 * (p->N / 2) * (p->N / 2);
    cudaError_t e;
    double *g = nullptr;
    auto bail = [&](cudaError_t err, const char *w) {
        if (g) cudaFree(g);
        bc_lift_destroy(lf);
        return lift_cuda(err, w);
    };
    if ((e = cudaGetDevice(&lf->device)) != cudaSuccess) return bail(e, "bc_lift_create: device");
    if ((e = cudaDeviceGetAttribute(&lf->nsm, cudaDevAttrMultiProcessorCount, lf->device)) != cudaSuccess)
        return bail(e, "bc_lift_create: device");
    if ((e = cudaMalloc(&lf->cone, sizeof(float2) * (lf->qmax + 1) * lf->Nr)) != cudaSuccess) return bail(e, "cudaMalloc cone");
    if ((e = cudaMalloc(&lf->tw, sizeof(float2) * lf->N)) != cudaSuccess) return bail(e, "cudaMalloc twiddles");
    if ((e = cudaMalloc(&g, sizeof(double) * 2 * LIFT_GAUSS)) != cudaSuccess) return bail(e, "cudaMalloc nodes");
    if ((e = cudaMallocHost(&lf->pin, LIFT_PIN_BYTES)) != cudaSuccess) return bail(e, "cudaMallocHost staging");
    if ((e = cudaFuncSetAttribute(k_lift_gemm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_lift_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float) * 2 * LIFT_STAGE))) != cudaSuccess)
        return bail(e, "bc_lift_create: shared memory");
    k_lift_gauss<<<1, 64, 0, lf->stream>>>(LIFT_GAUSS, g, g + LIFT_GAUSS);
    const int total = (lf->qmax + 1) * lf->Nr;
    k_lift_cone<<<(total + 255) / 256, 256, 0, lf->stream>>>(lf->qmax, lf->Nr, lf->L, lf->period, lf->period_r, g,
                                                             g + LIFT_GAUSS, lf->cone);
    k_lift_twiddles<<<(lf->N + 63) / 64, 64, 0, lf->stream>>>(lf->N, lf->tw);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "bc_lift_create: tables");
    if (lf->contraction == 3) {
        // window (width 8, the default shape for oversampling 2, FP32-representable
        // beta) and transform tables of the spatial and lifted axes
        const int N = lf->N, Nr = lf->Nr, W = 8;
        const double a = W / 2.0 * 1.5;
        const double beta = (double)(float)(M_PI * std::sqrt(a * a - 0.8));
        const size_t fl = (size_t)N + Nr + CONSTS_FLOATS + 2 * (size_t)N + 2 * (size_t)Nr + 8;
        const size_t bytes = sizeof(float) * fl + sizeof(float2) * (2 * (size_t)N + 2 * (size_t)Nr + N + Nr) + 256;
        if ((e = cudaMalloc(&lf->t4_mem, bytes)) != cudaSuccess) return bail(e, "cudaMalloc NUFFT tables");
        float2 *tw = (float2 *)lf->t4_mem; // n + n_r twiddles, then N + N_r scratch ones
        lf->t4.tw_s = tw;
        lf->t4.tw_r = tw + 2 * N;
        float2 *twN = tw + 2 * N + 2 * Nr, *twNr = twN + N;
        float *f = (float *)(twNr + Nr);
        lf->t4.deconv_s = f;
        lf->t4.deconv_r = f + N;
        lf->t4.consts = f + N + Nr;
        lf->t4.dbox = (int *)(lf->t4.consts + CONSTS_FLOATS);
        if ((e = cudaMallocHost(&lf->t4.hbox, 8 * sizeof(int))) != cudaSuccess) return bail(e, "cudaMallocHost box");
        Geometry gs{}, gr{};
        gs.N = N, gs.n = 2 * N, gs.W = W, gs.L = 0;
        gr.N = Nr, gr.n = 2 * Nr, gr.W = W, gr.L = 0;
        if ((e = launch_build_tables(gs, beta, lf->period, nullptr, lf->t4.deconv_s, nullptr, lf->t4.tw_s, twN,
                                     lf->t4.consts, lf->stream)) != cudaSuccess ||
            (e = launch_build_tables(gr, beta, lf->period_r, nullptr, lf->t4.deconv_r, nullptr, lf->t4.tw_r, twNr,
                                     lf->t4.consts, lf->stream)) != cudaSuccess)
            return bail(e, "bc_lift_create: NUFFT tables");
    }
    if ((e = cudaStreamSynchronize(lf->stream)) != cudaSuccess) return bail(e, "bc_lift_create: sync");
    cudaFree(g);
    g = nullptr;
    *out = lf;
    return BC_OK;
}

bc_status bc_lift_destroy(bc_lift_t lf)
{
    if (!lf) return BC_OK;
    cudaStreamSynchronize(lf->stream);
    if (lf->cone) cudaFree(lf->cone);
    if (lf->tw) cudaFree(lf->tw);
    if (lf->t4_mem) cudaFree(lf->t4_mem);
    if (lf->t4.hbox) cudaFreeHost(lf->t4.hbox);
    if (lf->ws) cudaFree(lf->ws);
    if (lf->pin) cudaFreeHost(lf->pin);
    delete lf;
    return BC_OK;
}

bc_status bc_lift_correlate(bc_lift_t lf, const float *A, int nA, const float *B, int nB, const float *quat,
                            const float *slices, int nslices, float *out, int on_device)
{
    if (!lf || !quat || !slices || !out || (nA > 0 && !A) || (nB > 0 && !B))
        return lift_fail(BC_ERR_ARG, "bc_lift_correlate: null argument");
    if (nA < 0 || nB < 0 || nA > (1 << 22) || nB > (1 << 22))
        return lift_fail(BC_ERR_ARG, "bc_lift_correlate: knot counts must be in [0, 2^22]");
    if (nslices < 1 || nslices > LIFT_MAX_SLICES)
        return lift_fail(BC_ERR_ARG, "bc_lift_correlate: nslices must be in [1, 16]");
    double qn = 0;
    for (int k = 0; k < 4; k++) qn += (double)quat[k] * quat[k];
    if (!(qn > 1e-30) || !std::isfinite(qn)) return lift_fail(BC_ERR_ARG, "bc_lift_correlate: zero or non-finite quaternion");
    for (int s = 0; s < nslices; s++)
        if (!std::isfinite(slices[s])) return lift_fail(BC_ERR_ARG, "bc_lift_correlate: non-finite section");
    const double inv = 1.0 / std::sqrt(qn);
    const int N = lf->N, Nr = lf->Nr, H = N / 2;
    const int T = 2 * N + H + Nr;
    const size_t M = (size_t)N * N, C = (size_t)H * Nr;
    const size_t rho_bytes = lf->contraction == 3 ? 0 : sizeof(float2) * M * C; // the NUFFT keeps no rho^
    const size_t nmax = (size_t)(nA > nB ? nA : nB);
    // the tensor-core contractions take the knots in passes of at most LIFT_CHUNK
    // (their operands cost 16 M + 32 C, resp. 8 (M + C), bytes per knot); each
    // pass adds its partial spectrum into rho^ with atomics
    const size_t nchunk = nmax < (size_t)LIFT_CHUNK ? nmax : (size_t)LIFT_CHUNK;
    const int ld = nchunk > 0 ? (int)((nchunk + LIFT_KC - 1) / LIFT_KC) * LIFT_KC : LIFT_KC; // padded pass length
    // contraction 2: A blocks (hi, lo) 16 M ld bytes, B blocks 32 C ld bytes, fixed-point knots
    const size_t e_bytes = lf->contraction == 3 ? lift4_ws_bytes(N, Nr)
                         : lf->contraction == 2 ? (16 * M + 32 * C) * (size_t)ld + sizeof(LiftQ) * (nchunk + 1)
                         : lf->contraction == 1 ? sizeof(float) * 2 * (M + C) * (size_t)ld + sizeof(LiftU) * (nchunk + 1)
                                                : sizeof(float2) * (size_t)T * (nmax > 0 ? nmax : 1);
    const size_t plane = (size_t)N * N * H;
    const size_t h_bytes = sizeof(float2) * plane * nslices;
    const size_t knot_bytes = on_device ? 0 : sizeof(float4) * (size_t)(nA + nB);
    const size_t out_bytes = on_device ? 0 : sizeof(float) * (size_t)N * N * N * nslices;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al(rho_bytes) * 2 + al(e_bytes) + al(h_bytes) + al(sizeof(float) * LIFT_MAX_SLICES) +
                        al(sizeof(PairDesc) * LIFT_MAX_SLICES) + al(sizeof(int)) + al(knot_bytes) + al(out_bytes);
    cudaStream_t st = lf->stream;
    cudaError_t e;
    if (need > lf->ws_bytes) {
        if (lf->ws) {
            cudaStreamSynchronize(st);
            cudaFree(lf->ws);
            lf->ws = nullptr;
            lf->ws_bytes = 0;
        }
        if ((e = cudaMalloc(&lf->ws, need)) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: workspace");
        lf->ws_bytes = need;
    }
    char *w = (char *)lf->ws;
    float2 *rhoA = (float2 *)w;
    w += al(rho_bytes);
    float2 *rhoB = (float2 *)w;
    w += al(rho_bytes);
    float2 *E = (float2 *)w;
    w += al(e_bytes);
    float2 *h = (float2 *)w;
    w += al(h_bytes);
    float *dsl = (float *)w;
    w += al(sizeof(float) * LIFT_MAX_SLICES);
    PairDesc *dpairs = (PairDesc *)w;
    w += al(sizeof(PairDesc) * LIFT_MAX_SLICES);
    int *derr = (int *)w;
    w += al(sizeof(int));
    const float4 *kA = (const float4 *)A, *kB = (const float4 *)B;
    if (!on_device) {
        float4 *stage = (float4 *)w;
        if (nA > 0 && (e = cudaMemcpyAsync(stage, A, sizeof(float4) * nA, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return lift_cuda(e, "bc_lift_correlate: copy A");
        if (nB > 0 && (e = cudaMemcpyAsync(stage + nA, B, sizeof(float4) * nB, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return lift_cuda(e, "bc_lift_correlate: copy B");
        kA = stage;
        kB = stage + nA;
        w += al(knot_bytes);
    }
    float *dout = on_device ? out : (float *)w;
    // descriptors through pinned staging (the previous call has synchronised, so it is free)
    float *psl = (float *)lf->pin;
    PairDesc *ppairs = (PairDesc *)(lf->pin + 256);
    int *perr = (int *)(lf->pin + 256 + sizeof(PairDesc) * LIFT_MAX_SLICES);
    for (int s = 0; s < nslices; s++) {
        psl[s] = slices[s];
        ppairs[s] = PairDesc{0, 0, (long long)(s * plane), (long long)s * N * N * N, 0};
    }
    *perr = 0;
    if ((e = cudaMemcpyAsync(dsl, psl, sizeof(float) * nslices, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dpairs, ppairs, sizeof(PairDesc) * nslices, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return lift_cuda(e, "bc_lift_correlate: descriptors");
    if ((e = cudaMemsetAsync(derr, 0, sizeof(int), st)) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: error word");
    const float scale = (float)(1.0 / (lf->period * lf->period * lf->period * lf->period_r));
    if (lf->contraction == 3) {
        // both spectra by the 4D NUFFT, their r transforms fused with the collapse
        const double qw = quat[0] * inv, qx = quat[1] * inv, qy = quat[2] * inv, qz = quat[3] * inv;
        const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                             2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                             2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
        if ((e = lift4_pair(lf->t4, N, Nr, kA, nA, kB, nB, R, lf->period, lf->period_r, lf->cone, dsl, nslices, scale, E,
                            h, lf->nsm, st)) != cudaSuccess)
            return lift_cuda(e, "bc_lift_correlate: 4D NUFFT");
    } else {
    // both spectra are accumulated with atomics: one clear for the pair
    if ((e = cudaMemsetAsync(rhoA, 0, 2 * al(rho_bytes), st)) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: clear");
    // the two lifted spectra
    const dim3 tiles((unsigned)(C / LIFT_TILE), (unsigned)(M / LIFT_TILE));
    for (int side = 0; side < 2; side++) {
        const float4 *kn = side ? kB : kA;
        const int n = side ? nB : nA;
        float2 *rho = side ? rhoB : rhoA;
        if (n == 0) continue;
        const double qw = side ? quat[0] * inv : 1.0, qx = side ? quat[1] * inv : 0.0, qy = side ? quat[2] * inv : 0.0,
                     qz = side ? quat[3] * inv : 0.0;
        const int ntile = (int)(tiles.x * tiles.y);
        // knots split across blocks so that about four blocks per SM run
        auto split_of = [&](int len, int &kper) {
            int split = (4 * lf->nsm + ntile - 1) / ntile;
            kper = (len + split - 1) / split;
            kper = ((kper + LIFT_KC - 1) / LIFT_KC) * LIFT_KC;
            return (len + kper - 1) / kper;
        };
        if (lf->contraction == 2) {
            const int mt = (int)(M / 128), ctn = (int)(C / 128);
            // A hi / lo: mt x nkb x 2 blocks of 128 x 32 floats = 2 M ld floats each;
            // B hi / lo: ctn x nkb x 2 blocks of 256 x 32 floats = 4 C ld floats each
            float *ahi = (float *)E, *alo = ahi + 2 * M * (size_t)ld, *bhi = alo + 2 * M * (size_t)ld,
                  *blo = bhi + 4 * C * (size_t)ld;
            LiftQ *fq = (LiftQ *)(blo + 4 * C * (size_t)ld);
            for (int k0 = 0; k0 < n; k0 += LIFT_CHUNK) {
                const int nc = n - k0 < LIFT_CHUNK ? n - k0 : LIFT_CHUNK;
                const int nkb = (nc + LIFT_KC - 1) / LIFT_KC;
                k_lift_scale<<<(nc + 255) / 256, 256, 0, st>>>(kn + k0, nc, qw, qx, qy, qz, side, lf->period, lf->period_r,
                                                               nullptr, fq);
                k_lift_operands<<<dim3((nkb * LIFT_KC + 255) / 256, (unsigned)(M + C)), 256, 0, st>>>(fq, nc, nkb, N, Nr, ahi,
                                                                                                   alo, bhi, blo);
                const int ns = umma_nsplit(mt * ctn, nkb, lf->nsm), units = mt * ctn * ns;
                k_lift_gemm_umma<<<units < lf->nsm ? units : lf->nsm, UMMA_THREADS, UMMA_SMEM, st>>>(
                    ahi, alo, bhi, blo, nkb, mt, ctn, ns, (int)C, rho, derr);
            }
        } else if (lf->contraction == 1) {
            float *p1re = (float *)E, *p1im = p1re + M * (size_t)ld, *p2re = p1im + M * (size_t)ld,
                  *p2im = p2re + C * (size_t)ld;
            LiftU *u = (LiftU *)(p2im + C * (size_t)ld);
            const size_t smem = sizeof(float) * 2 * LIFT_STAGE;
            for (int k0 = 0; k0 < n; k0 += LIFT_CHUNK) {
                const int nc = n - k0 < LIFT_CHUNK ? n - k0 : LIFT_CHUNK;
                const int ldc = ((nc + LIFT_KC - 1) / LIFT_KC) * LIFT_KC; // this pass's plane stride
                int kper;
                const int split = split_of(ldc, kper);
                k_lift_scale<<<(nc + 255) / 256, 256, 0, st>>>(kn + k0, nc, qw, qx, qy, qz, side, lf->period, lf->period_r,
                                                               u, nullptr);
                k_lift_planes<<<dim3((ldc + 255) / 256, (unsigned)(M + C)), 256, 0, st>>>(u, nc, ldc, N, Nr, p1re, p1im,
                                                                                        p2re, p2im);
                k_lift_gemm_tc<<<dim3(tiles.x, tiles.y, split), 256, smem, st>>>(p1re, p1im, p2re, p2im, ldc, (int)C, kper,
                                                                                 rho);
            }
        } else {
            int kper;
            const int split = split_of(n, kper);
            k_lift_phases<<<n, 64, 0, st>>>(kn, n, qw, qx, qy, qz, side, N, Nr, lf->period, lf->period_r, E);
            k_lift_ndft<<<dim3(tiles.x, tiles.y, split), 256, 0, st>>>(E, n, N, Nr, kper, rho);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: spectrum");
    }
    if ((e = launch_lift_collapse(rhoA, rhoB, lf->cone, N, Nr, dsl, nslices, lf->period_r, scale, h, st)) != cudaSuccess)
        return lift_cuda(e, "bc_lift_correlate: collapse");
    }
    switch (N) {
    case 32: k_lift_ifft_x<32><<<lf->nsm, TB, 0, st>>>(h, nslices, lf->tw); break;
    case 64: k_lift_ifft_x<64><<<lf->nsm, TB, 0, st>>>(h, nslices, lf->tw); break;
    case 96: k_lift_ifft_x<96><<<lf->nsm, TB, 0, st>>>(h, nslices, lf->tw); break;
    default: k_lift_ifft_x<128><<<lf->nsm, TB, 0, st>>>(h, nslices, lf->tw); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: collapse");
    Geometry g{};
    g.N = N;
    g.n = 2 * N;
    g.H = H;
    Tables t{};
    t.tw_N = lf->tw;
    if ((e = launch_ifft_y(g, t, dpairs, nslices, h, lf->nsm, st)) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: ifft y");
    if ((e = launch_ifft_z(g, t, dpairs, nslices, h, dout, nullptr, lf->nsm, st)) != cudaSuccess)
        return lift_cuda(e, "bc_lift_correlate: ifft z");
    if (!on_device) {
        if ((e = cudaMemcpyAsync(out, dout, sizeof(float) * (size_t)N * N * N * nslices, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return lift_cuda(e, "bc_lift_correlate: copy out");
    }
    if ((e = cudaMemcpyAsync(perr, derr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return lift_cuda(e, "bc_lift_correlate: error word");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return lift_cuda(e, "bc_lift_correlate: sync");
    const int herr = *perr;
    if (herr) return lift_fail(BC_ERR_TIMEOUT, "bc_lift_correlate: tensor-core contraction stalled (waits " +
                                                   std::to_string(herr) + ": 1 copy, 2 accumulator, 4 stage, 8 drain); "
                                                   "the spectrum is incomplete");
    return BC_OK;
}

} // extern "C"
