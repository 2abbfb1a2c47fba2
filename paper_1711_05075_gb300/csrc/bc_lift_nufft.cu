// The lifted spectrum rho^_X(xi, eta) of Eq. (rhoAhat) (Sec. 3.2) as a 4D
// type-1 nonuniform FFT over (x, r), the alternative to the direct 4D NDFT
// contractions of bc_lift.cu (contraction 3 of bc_lift_params).
//
// Knot i of a shape, rotated (B) and mirrored in r (B), sits at the fine-grid
// coordinates u_a = frac(x_a / P) n (a = x, y, z; n = 2N) and u_r = frac(r / P_r)
// n_r (n_r = 2 N_r).  With the Kaiser-Bessel window phi of width W = 8 (the
// window of the correlation's spreading, its piecewise-polynomial evaluation
// and its deconvolution table),
//     G[g]     = sum_i prod_{a in x,y,z,r} phi(u_{i,a} - g_a)      (periodic in every axis)
//     G^(k)    = sum_g G[g] exp(-2 pi i k . g / n)                  (4D DFT of the grid)
//     rho^(xi, eta) = G^(xi, eta) / (phi^(xi_x/n) phi^(xi_y/n) phi^(xi_z/n) phi^(eta/n_r)),
// which equals the direct sum of Eq. (rhoAhat) up to the window's aliasing
// error, since exp(-2 pi i k u / n) = exp(-2 pi i k x / P).  Kept modes: xi_x,
// xi_y in [-N/2, N/2) and eta in [-N_r/2, N_r/2) in FFT order, xi_z in [0, N/2)
// (the density is real: the collapse uses the half space), in the layout of
// the direct contractions, rho[(j_x N + j_y) (N/2 N_r) + m_z N_r + k].
//
//   k_l4_spread   one warp per knot: the 4W window weights by the lanes, then
//                 the W^4 stencil cells with atomic adds into the real grid
//                 [g_r][g_x][g_y][g_z];
//   k_l4_z        transform along z (real lines, 16 per tile), keep m_z < N/2;
//   k_l4_mid      transform along y, then along x (16 adjacent lines per tile,
//                 one 128-byte row per position), keep N modes each;
//   k_l4_r        transform along r, keep N_r modes, deconvolve, write rho^.
// Transforms: the library's shared-memory Stockham FFT (bc_fft.cuh) on tiles of
// 16 interleaved lines.  The grid and the z planes share the workspace with
// the y and x planes (each pass's output fits in the space its input left).
#include <cmath>

#include "bc_device.cuh"
#include "bc_lift4.h"

namespace bc {

constexpr int L4_W = 8; // window width of the lifted NUFFT

// 4W window weights of one knot per warp, then the W^4 stencil.
__global__ void __launch_bounds__(256)
k_l4_spread(const float4 *__restrict__ knots, int n, double R00, double R01, double R02, double R10, double R11,
            double R12, double R20, double R21, double R22, int mirror, int ns, int nr, double inv_p, double inv_pr,
            const float *__restrict__ consts, float *G)
{
    constexpr int W = L4_W;
    __shared__ float wts[8][4][W];
    __shared__ int g0s[8][4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = lane / W, t = lane - a * W; // lanes 0 .. 4W - 1: axis a, stencil offset t
    float kc[KB_NC];
    kb_load(consts, t, kc);
    for (int i = blockIdx.x * 8 + wib; i < n; i += gridDim.x * 8) {
        const float4 c = knots[i];
        if (lane < 4 * W) {
            double v;
            if (a == 0) v = (R00 * c.x + R01 * c.y + R02 * c.z) * inv_p;
            else if (a == 1) v = (R10 * c.x + R11 * c.y + R12 * c.z) * inv_p;
            else if (a == 2) v = (R20 * c.x + R21 * c.y + R22 * c.z) * inv_p;
            else v = (mirror ? -(double)c.w : (double)c.w) * inv_pr;
            const int na = a < 3 ? ns : nr;
            const double u = (v - floor(v)) * na; // in [0, na]
            const int g0 = (int)ceil(u - 0.5 * W);
            // offset t's weight is phi(x + W/2 - 1 - t), x = u - g0 - (W/2 - 1) in (0, 1]
            wts[wib][a][t] = kb_poly(kc, (float)(u - g0 - (0.5 * W - 1.0)));
            if (t == 0) g0s[wib][a] = g0;
        }
        __syncwarp();
        const int gr0 = g0s[wib][3], gx0 = g0s[wib][0], gy0 = g0s[wib][1], gz0 = g0s[wib][2];
        for (int e = lane; e < W * W * W * W; e += 32) {
            const int tz = e % W, ty = (e / W) % W, tx = (e / (W * W)) % W, tr = e / (W * W * W);
            int gr = gr0 + tr, gx = gx0 + tx, gy = gy0 + ty, gz = gz0 + tz;
            gr = gr < 0 ? gr + nr : (gr >= nr ? gr - nr : gr);
            gx = gx < 0 ? gx + ns : (gx >= ns ? gx - ns : gx);
            gy = gy < 0 ? gy + ns : (gy >= ns ? gy - ns : gy);
            gz = gz < 0 ? gz + ns : (gz >= ns ? gz - ns : gz);
            const float w = wts[wib][3][tr] * wts[wib][0][tx] * wts[wib][1][ty] * wts[wib][2][tz];
            atomicAdd(G + (((long long)gr * ns + gx) * ns + gy) * ns + gz, w);
        }
        __syncwarp();
    }
}

// Transform along z of the real grid's lines (16 adjacent lines per tile),
// Z1[line][m_z] for m_z < NF/4 (N/2).
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_z(const float *__restrict__ G, float2 *Z1, long long nlines,
                                             const float2 *__restrict__ twg)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *A = tw + NF, *B = A + NF * CL;
    constexpr int H = NF / 4;
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    const long long tiles = nlines / CL;
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        __syncthreads();
        const float *src = G + tt * CL * NF;
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int c = e / NF, pos = e - c * NF;
            A[pos * CL + c] = make_float2(src[e], 0.f);
        }
        __syncthreads();
        const float2 *res = il_fft<NF, false, CL, TB>(A, B, tw);
        float2 *dst = Z1 + tt * CL * H;
        for (int e = threadIdx.x; e < CL * H; e += TB) {
            const int c = e / H, mz = e - c * H;
            dst[e] = res[mz * CL + c];
        }
    }
}

// Transform of 16 adjacent lines per tile along a strided axis of length NF,
// keeping the NF/2 modes in FFT order.  Tile t = (outer o, chunk ch): line c
// of the tile has its element at position p at in[(o / n2) s1i + (o % n2) s2i
// + 16 ch + c + p pi], its kept mode j at out[(o / n2) s1o + (o % n2) s2o +
// 16 ch + c + j po].
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_mid(const float2 *__restrict__ in, float2 *out, long long nouter, int n2,
                                               int nch, long long s1i, long long s2i, long long pi, long long s1o,
                                               long long s2o, long long po, const float2 *__restrict__ twg)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *A = tw + NF, *B = A + NF * CL;
    constexpr int KEEP = NF / 2;
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    const long long tiles = nouter * nch;
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        const long long o = tt / nch;
        const int ch = (int)(tt - o * nch);
        const long long o1 = o / n2, o2 = o - o1 * n2;
        const float2 *src = in + o1 * s1i + o2 * s2i + CL * ch;
        float2 *dst = out + o1 * s1o + o2 * s2o + CL * ch;
        __syncthreads();
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int pos = e / CL, c = e - pos * CL;
            A[e] = src[pos * pi + c];
        }
        __syncthreads();
        const float2 *res = il_fft<NF, false, CL, TB>(A, B, tw);
        for (int e = threadIdx.x; e < CL * KEEP; e += TB) {
            const int j = e / CL, c = e - j * CL;
            const int pos = j < KEEP / 2 ? j : NF - KEEP + j;
            dst[j * po + c] = res[pos * CL + c];
        }
    }
}

// Transform along r (length NF = n_r), keep N_r = NF/2 modes, deconvolve in all
// four axes and write rho^ in the contraction layout.  X1[g_r][j_x][j_y][m_z].
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_r(const float2 *__restrict__ X1, float2 *rho, int N,
                                             const float *__restrict__ dxs, const float *__restrict__ drr,
                                             const float2 *__restrict__ twg)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *A = tw + NF, *B = A + NF * CL;
    constexpr int KEEP = NF / 2;
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    const int H = N / 2, nch = H / CL;
    const long long plane = (long long)N * N * H;
    const long long tiles = (long long)N * N * nch;
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        const int o = (int)(tt / nch), ch = (int)(tt - (long long)o * nch);
        const int jx = o / N, jy = o - jx * N;
        const float2 *src = X1 + (long long)o * H + CL * ch;
        __syncthreads();
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int pos = e / CL, c = e - pos * CL;
            A[e] = src[pos * plane + c];
        }
        __syncthreads();
        const float2 *res = il_fft<NF, false, CL, TB>(A, B, tw);
        const float dxy = dxs[jx] * dxs[jy];
        float2 *dst = rho + (long long)o * H * KEEP + (long long)CL * ch * KEEP;
        for (int e = threadIdx.x; e < CL * KEEP; e += TB) {
            const int c = e / KEEP, k = e - c * KEEP;
            const int pos = k < KEEP / 2 ? k : NF - KEEP + k;
            dst[e] = cscale(res[pos * CL + c], dxy * dxs[CL * ch + c] * drr[k]);
        }
    }
}

size_t lift4_ws_bytes(int N, int Nr)
{
    // the real grid (n_r (2N)^3 floats) and the z planes (n_r (2N)^2 N/2 complex);
    // the y planes reuse the grid's space, the x planes the z planes'
    const size_t nr = 2 * (size_t)Nr, n = 2 * (size_t)N;
    const size_t g = sizeof(float) * nr * n * n * n, z = sizeof(float2) * nr * n * n * (N / 2);
    return ((g + 255) & ~(size_t)255) + z;
}

template <int NF>
static cudaError_t l4_z(const float *G, float2 *Z1, long long nlines, const float2 *tw, int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_z<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_z<NF><<<resident_blocks(k_l4_z<NF>, smem, nsm), TB, smem, s>>>(G, Z1, nlines, tw);
    return cudaGetLastError();
}

template <int NF>
static cudaError_t l4_mid(const float2 *in, float2 *out, long long nouter, int n2, int nch, long long s1i, long long s2i,
                          long long pi, long long s1o, long long s2o, long long po, const float2 *tw, int nsm,
                          cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_mid<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_mid<NF><<<resident_blocks(k_l4_mid<NF>, smem, nsm), TB, smem, s>>>(in, out, nouter, n2, nch, s1i, s2i, pi,
                                                                             s1o, s2o, po, tw);
    return cudaGetLastError();
}

template <int NF>
static cudaError_t l4_r(const float2 *X1, float2 *rho, int N, const float *dxs, const float *drr, const float2 *tw,
                        int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_r<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_r<NF><<<resident_blocks(k_l4_r<NF>, smem, nsm), TB, smem, s>>>(X1, rho, N, dxs, drr, tw);
    return cudaGetLastError();
}

// rho (N^2 x N/2 x N_r complex, overwritten) = the lifted spectrum of n knots.
cudaError_t lift4_spectrum(const Lift4Tables &t, int N, int Nr, const float4 *knots, int n, const double (&R)[9],
                           int mirror, double period, double period_r, void *ws, float2 *rho, int nsm, cudaStream_t s)
{
    const int ns = 2 * N, nr = 2 * Nr, H = N / 2;
    const size_t gbytes = sizeof(float) * (size_t)nr * ns * ns * ns;
    float *G = (float *)ws;
    float2 *Z1 = (float2 *)((char *)ws + ((gbytes + 255) & ~(size_t)255));
    float2 *Y1 = (float2 *)G, *X1 = Z1;
    cudaError_t e = cudaMemsetAsync(G, 0, gbytes, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int blocks = (n + 7) / 8 < 65535 ? (n + 7) / 8 : 65535;
        k_l4_spread<<<blocks, 256, 0, s>>>(knots, n, R[0], R[1], R[2], R[3], R[4], R[5], R[6], R[7], R[8], mirror, ns, nr,
                                           1.0 / period, 1.0 / period_r, t.consts, G);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // z: lines (g_r, g_x, g_y) of ns reals -> Z1[g_r][g_x][g_y][m_z]
    const long long zlines = (long long)nr * ns * ns;
    switch (ns) {
    case 64: e = l4_z<64>(G, Z1, zlines, t.tw_s, nsm, s); break;
    case 128: e = l4_z<128>(G, Z1, zlines, t.tw_s, nsm, s); break;
    case 192: e = l4_z<192>(G, Z1, zlines, t.tw_s, nsm, s); break;
    case 256: e = l4_z<256>(G, Z1, zlines, t.tw_s, nsm, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int nch = H / CL;
    // y: outer (g_r, g_x), Z1[o][g_y][m_z] -> Y1[o][j_y][m_z]
    // x: outer (g_r, j_y), Y1[g_r][g_x][j_y][m_z] -> X1[g_r][j_x][j_y][m_z]
    auto mid = [&](const float2 *in, float2 *out, long long nouter, int n2, long long s1i, long long s2i, long long pi,
                   long long s1o, long long s2o, long long po) {
        switch (ns) {
        case 64: return l4_mid<64>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, t.tw_s, nsm, s);
        case 128: return l4_mid<128>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, t.tw_s, nsm, s);
        case 192: return l4_mid<192>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, t.tw_s, nsm, s);
        case 256: return l4_mid<256>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, t.tw_s, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    };
    if ((e = mid(Z1, Y1, (long long)nr * ns, 1, (long long)ns * H, 0, H, (long long)N * H, 0, H)) != cudaSuccess) return e;
    if ((e = mid(Y1, X1, (long long)nr * N, N, (long long)ns * N * H, H, (long long)N * H, (long long)N * N * H, H,
                 (long long)N * H)) != cudaSuccess)
        return e;
    // r: X1[g_r][j_x][j_y][m_z] -> rho[(j_x N + j_y)][m_z][k], deconvolved
    switch (nr) {
    case 32: return l4_r<32>(X1, rho, N, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    case 64: return l4_r<64>(X1, rho, N, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    case 128: return l4_r<128>(X1, rho, N, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
