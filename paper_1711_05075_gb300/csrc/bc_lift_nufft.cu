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
//   k_l4_z        transform along z (two real lines per complex line, 32 per
//                 tile), keep m_z < N/2;
//   k_l4_mid      transform along y, then along x (16 adjacent lines per tile,
//                 one 128-byte row per position), keep N modes each;
//   k_l4_r        transform along r, keep N_r modes, deconvolve, write rho^.
// Support box: the coordinates are taken half a period on, u_a = frac(x_a / P +
// 1/2) n and u_r = frac(r / P_r + 1/2) n_r, so that a shape around the origin
// (and a lifted axis of radii in (0, L), mirrored for B) occupies one
// contiguous range of cells per axis; k_l4_box finds the range the stencils
// cover, and the grid, the spreading and every transform pass are restricted
// to it (a range wider than the axis falls back to the whole axis).  The
// half-period shift multiplies the spectrum by (-1)^(m_x + m_y + m_z + m_r),
// undone with the deconvolution.  Box element i of an axis sits at line
// position (lo + i) mod n; positions outside the box are zero.
// Transforms: the library's shared-memory Stockham FFT (bc_fft.cuh) on tiles of
// 16 interleaved lines.  The grid and the z planes share the workspace with
// the y and x planes (each pass's output fits in the space its input left).
#include <cmath>

#include "bc_device.cuh"
#include "bc_lift4.h"

namespace bc {

constexpr int L4_W = 8; // window width of the lifted NUFFT

// Fine-grid coordinate of knot c on axis a (0, 1, 2: rotated x, y, z; 3: r,
// mirrored for B), half a period on.
__device__ __forceinline__ double l4_coord(const float4 &c, int a, const double (&R)[9], int mirror, int ns, int nr,
                                           double inv_p, double inv_pr)
{
    double v;
    if (a < 3) v = (R[3 * a] * c.x + R[3 * a + 1] * c.y + R[3 * a + 2] * c.z) * inv_p + 0.5;
    else v = (mirror ? -(double)c.w : (double)c.w) * inv_pr + 0.5;
    return (v - floor(v)) * (a < 3 ? ns : nr);
}

struct L4Rot {
    double R[9];
};

// box[a] = min, box[4 + a] = max over the knots of the first stencil cell
// ceil(u_a - W/2) (box preset to INT_MAX / INT_MIN).
__global__ void k_l4_box(const float4 *__restrict__ knots, int n, L4Rot rot, int mirror, int ns, int nr, double inv_p,
                         double inv_pr, int *box)
{
    int lo[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX}, hi[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 c = knots[i];
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int g0 = (int)ceil(l4_coord(c, a, rot.R, mirror, ns, nr, inv_p, inv_pr) - 0.5 * L4_W);
            lo[a] = min(lo[a], g0);
            hi[a] = max(hi[a], g0);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
        if ((threadIdx.x & 31) == 0 && lo[a] != INT_MAX) {
            atomicMin(box + a, lo[a]);
            atomicMax(box + 4 + a, hi[a]);
        }
    }
}

// Box of the grid: per axis (x, y, z, r) the first cell lo and the extent b;
// cell g of the axis is box element (g - lo) mod n.
struct L4Box {
    int lo[4], b[4];
};

// 4W window weights of one knot per warp, then the W^4 stencil into the box
// grid G[i_r][i_x][i_y][i_z].
__global__ void __launch_bounds__(256)
k_l4_spread(const float4 *__restrict__ knots, int n, L4Rot rot, int mirror, int ns, int nr, double inv_p,
            double inv_pr, L4Box bx, const float *__restrict__ consts, float *G)
{
    constexpr int W = L4_W;
    __shared__ float wts[8][4][W];
    __shared__ int g0s[8][4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = lane / W, t = lane - a * W; // lanes 0 .. 4W - 1: axis a, stencil offset t
    float kc[KB_NC];
    kb_load(consts, t, kc);
    const int bX = bx.b[0], bY = bx.b[1], bZ = bx.b[2];
    for (int i = blockIdx.x * 8 + wib; i < n; i += gridDim.x * 8) {
        const float4 c = knots[i];
        if (lane < 4 * W) {
            const double u = l4_coord(c, a, rot.R, mirror, ns, nr, inv_p, inv_pr);
            const int g0 = (int)ceil(u - 0.5 * W);
            // offset t's weight is phi(x + W/2 - 1 - t), x = u - g0 - (W/2 - 1) in (0, 1]
            wts[wib][a][t] = kb_poly(kc, (float)(u - g0 - (0.5 * W - 1.0)));
            if (t == 0) {
                const int na = a < 3 ? ns : nr;
                int e0 = (g0 - bx.lo[a]) % na; // box element of the first stencil cell
                g0s[wib][a] = e0 < 0 ? e0 + na : e0;
            }
        }
        __syncwarp();
        const int er0 = g0s[wib][3], ex0 = g0s[wib][0], ey0 = g0s[wib][1], ez0 = g0s[wib][2];
        for (int e = lane; e < W * W * W * W; e += 32) {
            const int tz = e % W, ty = (e / W) % W, tx = (e / (W * W)) % W, tr = e / (W * W * W);
            // within a box narrower than its axis the stencil never wraps; a whole-axis box wraps
            int ir = er0 + tr, ix = ex0 + tx, iy = ey0 + ty, iz = ez0 + tz;
            ir = ir >= nr ? ir - nr : ir;
            ix = ix >= ns ? ix - ns : ix;
            iy = iy >= ns ? iy - ns : iy;
            iz = iz >= ns ? iz - ns : iz;
            const float w = wts[wib][3][tr] * wts[wib][0][tx] * wts[wib][1][ty] * wts[wib][2][tz];
            atomicAdd(G + (((long long)ir * bX + ix) * bY + iy) * bZ + iz, w);
        }
        __syncwarp();
    }
}

// Transform along z of the box grid's lines (b_r b_x b_y real lines of b_z
// cells), two real lines per complex line (32 consecutive lines per tile): with
// Z = FFT(a + i b), A_k = (Z_k + conj Z_{n-k}) / 2 and B_k = (Z_k - conj
// Z_{n-k}) / (2i).  Z1[line][m_z] for m_z < NF/4 (N/2).
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_z(const float *__restrict__ G, float2 *Z1, long long nlines, int bz, int loz,
                                             const float2 *__restrict__ twg)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *A = tw + NF, *B = A + NF * CL;
    constexpr int H = NF / 4;
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    const long long tiles = (nlines + 2 * CL - 1) / (2 * CL);
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        __syncthreads();
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int q = e / NF, pos = e - q * NF;
            int iz = (pos - loz) % NF;
            iz = iz < 0 ? iz + NF : iz;
            const long long l0 = tt * 2 * CL + 2 * q;
            const bool in = iz < bz;
            const float a = in && l0 < nlines ? G[l0 * bz + iz] : 0.f;
            const float b = in && l0 + 1 < nlines ? G[(l0 + 1) * bz + iz] : 0.f;
            A[pos * CL + q] = make_float2(a, b);
        }
        __syncthreads();
        const float2 *res = il_fft<NF, false, CL, TB>(A, B, tw);
        float2 *dst = Z1 + tt * 2 * CL * H;
        for (int e = threadIdx.x; e < 2 * CL * H; e += TB) {
            const int r = e / H, mz = e - r * H, q = r >> 1;
            const float2 zk = res[mz * CL + q], zn = res[(mz == 0 ? 0 : NF - mz) * CL + q];
            dst[e] = (r & 1) ? make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x))
                             : make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        }
    }
}

// Transform of 16 adjacent lines per tile along a strided axis of length NF,
// keeping the NF/2 modes in FFT order.  Tile t = (outer o, chunk ch): line c
// of the tile has box element i (line position (lo + i) mod NF, i < b) at
// in[(o / n2) s1i + (o % n2) s2i + 16 ch + c + i pi], its kept mode j at
// out[(o / n2) s1o + (o % n2) s2o + 16 ch + c + j po].
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_mid(const float2 *__restrict__ in, float2 *out, long long nouter, int n2,
                                               int nch, long long s1i, long long s2i, long long pi, long long s1o,
                                               long long s2o, long long po, int lo, int b,
                                               const float2 *__restrict__ twg)
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
            int i = (pos - lo) % NF;
            i = i < 0 ? i + NF : i;
            A[e] = i < b ? src[i * pi + c] : make_float2(0.f, 0.f);
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
// four axes, undo the half-period shift and write rho^ in the contraction
// layout.  X1[j_x][j_y][i_r][m_z] (the b box planes of a mode row are 512-byte
// neighbours), box element i_r at position (lo + i_r) mod NF.
template <int NF>
__global__ void __launch_bounds__(TB) k_l4_r(const float2 *__restrict__ X1, float2 *rho, int N, int lo, int b,
                                             const float *__restrict__ dxs, const float *__restrict__ drr,
                                             const float2 *__restrict__ twg)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *A = tw + NF, *B = A + NF * CL;
    constexpr int KEEP = NF / 2;
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    const int H = N / 2, nch = H / CL;
    const long long tiles = (long long)N * N * nch;
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        const int o = (int)(tt / nch), ch = (int)(tt - (long long)o * nch);
        const int jx = o / N, jy = o - jx * N;
        const float2 *src = X1 + (long long)o * b * H + CL * ch;
        __syncthreads();
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int pos = e / CL, c = e - pos * CL;
            int i = (pos - lo) % NF;
            i = i < 0 ? i + NF : i;
            A[e] = i < b ? src[(long long)i * H + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 *res = il_fft<NF, false, CL, TB>(A, B, tw);
        const float dxy = dxs[jx] * dxs[jy];
        float2 *dst = rho + (long long)o * H * KEEP + (long long)CL * ch * KEEP;
        for (int e = threadIdx.x; e < CL * KEEP; e += TB) {
            const int c = e / KEEP, k = e - c * KEEP;
            const int pos = k < KEEP / 2 ? k : NF - KEEP + k;
            const int mz = CL * ch + c;
            // (-1)^m of each axis: the parity of the FFT index (N and N_r are even)
            const float sg = ((jx + jy + mz + k) & 1) ? -1.f : 1.f;
            dst[e] = cscale(res[pos * CL + c], sg * dxy * dxs[mz] * drr[k]);
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
static cudaError_t l4_z(const float *G, float2 *Z1, long long nlines, int bz, int loz, const float2 *tw, int nsm,
                        cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_z<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_z<NF><<<resident_blocks(k_l4_z<NF>, smem, nsm), TB, smem, s>>>(G, Z1, nlines, bz, loz, tw);
    return cudaGetLastError();
}

template <int NF>
static cudaError_t l4_mid(const float2 *in, float2 *out, long long nouter, int n2, int nch, long long s1i, long long s2i,
                          long long pi, long long s1o, long long s2o, long long po, int lo, int b, const float2 *tw,
                          int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_mid<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_mid<NF><<<resident_blocks(k_l4_mid<NF>, smem, nsm), TB, smem, s>>>(in, out, nouter, n2, nch, s1i, s2i, pi,
                                                                             s1o, s2o, po, lo, b, tw);
    return cudaGetLastError();
}

template <int NF>
static cudaError_t l4_r(const float2 *X1, float2 *rho, int N, int lo, int b, const float *dxs, const float *drr,
                        const float2 *tw, int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 2 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_r<NF>, smem);
    if (e != cudaSuccess) return e;
    k_l4_r<NF><<<resident_blocks(k_l4_r<NF>, smem, nsm), TB, smem, s>>>(X1, rho, N, lo, b, dxs, drr, tw);
    return cudaGetLastError();
}

// rho (N^2 x N/2 x N_r complex, overwritten) = the lifted spectrum of n knots.
// Synchronises s once (the support box comes back to the host through the
// page-locked words hbox).
cudaError_t lift4_spectrum(const Lift4Tables &t, int N, int Nr, const float4 *knots, int n, const double (&R)[9],
                           int mirror, double period, double period_r, void *ws, float2 *rho, int nsm, cudaStream_t s)
{
    const int ns = 2 * N, nr = 2 * Nr, H = N / 2;
    L4Rot rot;
    for (int k = 0; k < 9; k++) rot.R[k] = R[k];
    const double ip = 1.0 / period, ipr = 1.0 / period_r;
    // the support box
    cudaError_t e;
    if ((e = cudaMemsetAsync(t.dbox, 0x7f, 4 * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(t.dbox + 4, 0x80, 4 * sizeof(int), s)) != cudaSuccess)
        return e;
    if (n > 0) {
        const int blocks = (n + 255) / 256 < 4 * nsm ? (n + 255) / 256 : 4 * nsm;
        k_l4_box<<<blocks, 256, 0, s>>>(knots, n, rot, mirror, ns, nr, ip, ipr, t.dbox);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(t.hbox, t.dbox, 8 * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    L4Box bx;
    for (int a = 0; a < 4; a++) {
        const int na = a < 3 ? ns : nr;
        const long long lo = t.hbox[a], hi = (long long)t.hbox[4 + a] + L4_W - 1;
        if (n == 0 || hi - lo + 1 >= na) {
            bx.lo[a] = 0;
            bx.b[a] = na;
        } else {
            bx.lo[a] = (int)lo;
            bx.b[a] = (int)(hi - lo + 1);
        }
    }
    const int bX = bx.b[0], bY = bx.b[1], bZ = bx.b[2], bR = bx.b[3];
    const size_t gfl = (size_t)bR * bX * bY * bZ;
    float *G = (float *)ws;
    float2 *Z1 = (float2 *)((char *)ws + ((sizeof(float) * (size_t)nr * ns * ns * ns + 255) & ~(size_t)255));
    float2 *Y1 = (float2 *)G, *X1 = Z1;
    if ((e = cudaMemsetAsync(G, 0, sizeof(float) * gfl, s)) != cudaSuccess) return e;
    if (n > 0) {
        const int blocks = (n + 7) / 8 < 65535 ? (n + 7) / 8 : 65535;
        k_l4_spread<<<blocks, 256, 0, s>>>(knots, n, rot, mirror, ns, nr, ip, ipr, bx, t.consts, G);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // z: lines (i_r, i_x, i_y) of b_z cells -> Z1[line][m_z]
    const long long zlines = (long long)bR * bX * bY;
    switch (ns) {
    case 64: e = l4_z<64>(G, Z1, zlines, bZ, bx.lo[2], t.tw_s, nsm, s); break;
    case 128: e = l4_z<128>(G, Z1, zlines, bZ, bx.lo[2], t.tw_s, nsm, s); break;
    case 192: e = l4_z<192>(G, Z1, zlines, bZ, bx.lo[2], t.tw_s, nsm, s); break;
    case 256: e = l4_z<256>(G, Z1, zlines, bZ, bx.lo[2], t.tw_s, nsm, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int nch = H / CL;
    auto mid = [&](const float2 *in, float2 *out, long long nouter, int n2, long long s1i, long long s2i, long long pi,
                   long long s1o, long long s2o, long long po, int lo, int b) {
        switch (ns) {
        case 64: return l4_mid<64>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, lo, b, t.tw_s, nsm, s);
        case 128: return l4_mid<128>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, lo, b, t.tw_s, nsm, s);
        case 192: return l4_mid<192>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, lo, b, t.tw_s, nsm, s);
        case 256: return l4_mid<256>(in, out, nouter, n2, nch, s1i, s2i, pi, s1o, s2o, po, lo, b, t.tw_s, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    };
    // y: outer (i_r, i_x), Z1[o][i_y][m_z] -> Y1[o][j_y][m_z]
    if ((e = mid(Z1, Y1, (long long)bR * bX, 1, (long long)bY * H, 0, H, (long long)N * H, 0, H, bx.lo[1], bY)) !=
        cudaSuccess)
        return e;
    // x: outer (i_r, j_y), Y1[i_r][i_x][j_y][m_z] -> X1[j_x][j_y][i_r][m_z]
    if ((e = mid(Y1, X1, (long long)bR * N, N, (long long)bX * N * H, H, (long long)N * H, H, (long long)bR * H,
                 (long long)N * bR * H, bx.lo[0], bX)) != cudaSuccess)
        return e;
    // r: X1[j_x][j_y][i_r][m_z] -> rho[(j_x N + j_y)][m_z][k], deconvolved
    switch (nr) {
    case 32: return l4_r<32>(X1, rho, N, bx.lo[3], bR, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    case 64: return l4_r<64>(X1, rho, N, bx.lo[3], bR, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    case 128: return l4_r<128>(X1, rho, N, bx.lo[3], bR, t.deconv_s, t.deconv_r, t.tw_r, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
