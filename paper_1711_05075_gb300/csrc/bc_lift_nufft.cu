// The lifted spectra rho^_X(xi, eta) of Eq. (rhoAhat) (Sec. 3.2) as 4D type-1
// nonuniform FFTs over (x, r), the alternative to the direct 4D NDFT
// contractions of bc_lift.cu (contraction 3 of bc_lift_params), with the
// collapse of the lifted correlation formed from them directly.
//
// Knot i of a shape, rotated (B) and mirrored in r (B), sits at the fine-grid
// coordinates u_a = frac(x_a / P) n (a = x, y, z; n = 2N) and u_r = frac(r / P_r)
// n_r (n_r = 2 N_r) (half a period on, see the support box below).  With the Kaiser-Bessel window phi of width W = 8 (the
// window of the correlation's spreading, its piecewise-polynomial evaluation
// and its deconvolution table),
//     G[g]     = sum_i prod_{a in x,y,z,r} phi(u_{i,a} - g_a)      (periodic in every axis)
//     G^(k)    = sum_g G[g] exp(-2 pi i k . g / n)                  (4D DFT of the grid)
//     rho^(xi, eta) = G^(xi, eta) / (phi^(xi_x/n) phi^(xi_y/n) phi^(xi_z/n) phi^(eta/n_r)),
// which equals the direct sum of Eq. (rhoAhat) up to the window's aliasing
// error, since exp(-2 pi i k u / n) = exp(-2 pi i k x / P).  Kept modes: xi_x,
// xi_y in [-N/2, N/2) and eta in [-N_r/2, N_r/2) in FFT order, xi_z in [0, N/2)
// (the density is real: the collapse uses the half space); they are formed
// tile by tile inside k_l4_rc and never stored.
//
//   k_l4_spread   one warp per knot: the 4W window weights by the lanes, then
//                 the W^4 stencil cells with atomic adds into the real grid
//                 [g_r][g_x][g_y][g_z];
//   k_l4_z        transform along z (two real lines per complex line, 32 per
//                 tile), keep m_z < N/2;
//   k_l4_mid      transform along y, then along x (16 adjacent lines per tile,
//                 one 128-byte row per position), keep N modes each;
//   k_l4_rc       transform along r of both shapes' x planes, keep N_r modes,
//                 deconvolve, and form the collapse of the lifted correlation
//                 (the sum over eta per section, as k_lift_collapse forms it
//                 from rho^_A and rho^_B) without writing the spectra.
// Support box: the coordinates are taken half a period on, u_a = frac(x_a / P +
// 1/2) n and u_r = frac(r / P_r + 1/2) n_r, so that a shape around the origin
// (and a lifted axis of radii in (0, L), mirrored for B) occupies one
// contiguous range of cells per axis; k_l4_box finds the range the stencils
// cover, and the grid, the spreading and every transform pass are restricted
// to it (a range wider than the axis falls back to the whole axis).  The
// half-period shift multiplies each spectrum by (-1)^(m_x + m_y + m_z + m_r),
// which cancels in the product of the two spectra.  Box element i of an axis
// sits at line position (lo + i) mod n; positions outside the box are zero.
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

// The r transforms of both spectra and the collapse of the lifted correlation
// in one pass, without rho^ in memory: per tile (j_x, j_y, 16 z-modes) the box
// planes of A and of B (X1[j_x][j_y][i_r][m_z], box element i_r at line position
// (lo + i_r) mod n_r) are transformed along r, and for each section s
//     h[s][j_x][j_y][m_z] = sign scale sum_{eta != -N_r/2} G^_A conj(G^_B)
//                           (D_x D_y D_z D_r)^2 cone(|m|^2, eta)^2 exp(2 pi i eta r_s / P_r),
// zero on the lower-edge modes (j_x or j_y = N/2); scale = P^-3 P_r^-1, sign =
// (-1)^(m_x + m_y + m_z).  The half-period shifts of the two spectra cancel in
// the product.  Thread (line c, eta group g) sums every 16th eta; the 16 groups
// of a line are then added by shuffles within 16 lanes.
template <int NF, int NS>
__global__ void __launch_bounds__(TB) k_l4_rc(const float2 *__restrict__ XA, const float2 *__restrict__ XB, int N,
                                              int loA, int bA, int loB, int bB, const float *__restrict__ dxs,
                                              const float *__restrict__ drr, const float2 *__restrict__ cone,
                                              const float *__restrict__ slices, int nslices, double period_r,
                                              float scale, const float2 *__restrict__ twg, float2 *h)
{
    extern __shared__ float2 l4sm[];
    float2 *tw = l4sm, *TA = tw + NF, *SA = TA + NF * CL, *TBt = SA + NF * CL, *SB = TBt + NF * CL;
    __shared__ float2 ph[NS][64];
    constexpr int KEEP = NF / 2; // N_r
    for (int k = threadIdx.x; k < NF; k += TB) tw[k] = twg[k];
    for (int e = threadIdx.x; e < NS * KEEP; e += TB) {
        const int sec = e / KEEP, k = e - sec * KEEP;
        float2 v = make_float2(0.f, 0.f);
        if (sec < nslices) {
            const int m = k < KEEP / 2 ? k : k - KEEP;
            double arg = m * (double)slices[sec] / period_r;
            arg -= rint(arg);
            double sn, cs;
            sincospi(2.0 * arg, &sn, &cs);
            v = make_float2((float)cs, (float)sn);
        }
        ph[sec][k] = v;
    }
    const int H = N / 2, nch = H / CL;
    const long long plane = (long long)N * N * H;
    const long long tiles = (long long)N * N * nch;
    const int c = threadIdx.x >> 4, g = threadIdx.x & 15;
    for (long long tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        const int o = (int)(tt / nch), ch = (int)(tt - (long long)o * nch);
        const int jx = o / N, jy = o - jx * N;
        const float2 *srcA = XA + (long long)o * bA * H + CL * ch, *srcB = XB + (long long)o * bB * H + CL * ch;
        __syncthreads();
        for (int e = threadIdx.x; e < CL * NF; e += TB) {
            const int pos = e / CL, cc = e - pos * CL;
            int ia = (pos - loA) % NF, ib = (pos - loB) % NF;
            ia = ia < 0 ? ia + NF : ia;
            ib = ib < 0 ? ib + NF : ib;
            TA[e] = ia < bA ? srcA[(long long)ia * H + cc] : make_float2(0.f, 0.f);
            TBt[e] = ib < bB ? srcB[(long long)ib * H + cc] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 *ra = il_fft<NF, false, CL, TB>(TA, SA, tw);
        const float2 *rb = il_fft<NF, false, CL, TB>(TBt, SB, tw);
        const int mz = CL * ch + c;
        const int mx = jx < N / 2 ? jx : jx - N, my = jy < N / 2 ? jy : jy - N;
        const int q = mx * mx + my * my + mz * mz;
        const float dxyz = dxs[jx] * dxs[jy] * dxs[mz];
        float2 acc[NS];
#pragma unroll
        for (int sec = 0; sec < NS; sec++) acc[sec] = make_float2(0.f, 0.f);
        for (int k = g; k < KEEP; k += 16) {
            if (k == KEEP / 2) continue;
            const int pos = k < KEEP / 2 ? k : NF - KEEP + k;
            const float d = dxyz * drr[k];
            const float2 f = cone[(long long)q * KEEP + k];
            const float2 p = cscale(cmul(cmulc(ra[pos * CL + c], rb[pos * CL + c]), cmul(f, f)), d * d);
#pragma unroll
            for (int sec = 0; sec < NS; sec++) acc[sec] = cadd(acc[sec], cmul(p, ph[sec][k]));
        }
        const bool zero = jx == N / 2 || jy == N / 2;
        const float sg = ((mx + my + mz) & 1) ? -scale : scale;
#pragma unroll
        for (int sec = 0; sec < NS; sec++) {
            float2 v = acc[sec];
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
            }
            if (g == 0 && sec < nslices)
                h[sec * plane + (long long)o * H + mz] = zero ? make_float2(0.f, 0.f) : cscale(v, sg);
        }
    }
}

// Workspace: the real grid (n_r (2N)^3 floats), the z planes (n_r (2N)^2 N/2
// complex) and A's x planes (n_r N^2 N/2 complex); the y planes reuse the
// grid's space, B's x planes the z planes'.
static size_t l4_align(size_t b) { return (b + 255) & ~(size_t)255; }
size_t lift4_ws_bytes(int N, int Nr)
{
    const size_t nr = 2 * (size_t)Nr, n = 2 * (size_t)N;
    const size_t g = sizeof(float) * nr * n * n * n, z = sizeof(float2) * nr * n * n * (N / 2);
    const size_t x = sizeof(float2) * nr * (size_t)N * N * (N / 2);
    return l4_align(g) + l4_align(z) + x;
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

// The x planes X1[j_x][j_y][i_r][m_z] of n knots (box, spreading, z, y and x
// passes); lo_r and b_r receive the box along r.  Synchronises s once (the
// support box comes back to the host through the page-locked words hbox).
static cudaError_t l4_xplanes(const Lift4Tables &t, int N, int Nr, const float4 *knots, int n, const L4Rot &rot,
                              int mirror, double ip, double ipr, void *ws, float2 *X1, int &lo_r, int &b_r, int nsm,
                              cudaStream_t s)
{
    const int ns = 2 * N, nr = 2 * Nr, H = N / 2;
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
    float2 *Z1 = (float2 *)((char *)ws + l4_align(sizeof(float) * (size_t)nr * ns * ns * ns));
    float2 *Y1 = (float2 *)G;
    lo_r = bx.lo[3];
    b_r = bR;
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
    return mid(Y1, X1, (long long)bR * N, N, (long long)bX * N * H, H, (long long)N * H, H, (long long)bR * H,
               (long long)N * bR * H, bx.lo[0], bX);
}

template <int NF, int NS>
static cudaError_t l4_rc(const float2 *XA, const float2 *XB, int N, int loA, int bA, int loB, int bB,
                         const Lift4Tables &t, const float2 *cone, const float *slices, int nslices, double period_r,
                         float scale, float2 *h, int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NF + 4 * (size_t)NF * CL);
    cudaError_t e = set_smem(k_l4_rc<NF, NS>, smem);
    if (e != cudaSuccess) return e;
    k_l4_rc<NF, NS><<<resident_blocks(k_l4_rc<NF, NS>, smem, nsm), TB, smem, s>>>(
        XA, XB, N, loA, bA, loB, bB, t.deconv_s, t.deconv_r, cone, slices, nslices, period_r, scale, t.tw_r, h);
    return cudaGetLastError();
}

template <int NF>
static cudaError_t l4_rc_ns(const float2 *XA, const float2 *XB, int N, int loA, int bA, int loB, int bB,
                            const Lift4Tables &t, const float2 *cone, const float *slices, int nslices,
                            double period_r, float scale, float2 *h, int nsm, cudaStream_t s)
{
    if (nslices <= 1) return l4_rc<NF, 1>(XA, XB, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    if (nslices <= 2) return l4_rc<NF, 2>(XA, XB, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    if (nslices <= 4) return l4_rc<NF, 4>(XA, XB, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    if (nslices <= 8) return l4_rc<NF, 8>(XA, XB, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    return l4_rc<NF, 16>(XA, XB, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
}

cudaError_t lift4_pair(const Lift4Tables &t, int N, int Nr, const float4 *kA, int nA, const float4 *kB, int nB,
                       const double (&RB)[9], double period, double period_r, const float2 *cone, const float *slices,
                       int nslices, float scale, void *ws, float2 *h, int nsm, cudaStream_t s)
{
    const int ns = 2 * N, nr = 2 * Nr;
    if (nA == 0 || nB == 0) return cudaMemsetAsync(h, 0, sizeof(float2) * (size_t)N * N * (N / 2) * nslices, s);
    const double ip = 1.0 / period, ipr = 1.0 / period_r;
    float2 *Z1 = (float2 *)((char *)ws + l4_align(sizeof(float) * (size_t)nr * ns * ns * ns));
    float2 *XA = (float2 *)((char *)Z1 + l4_align(sizeof(float2) * (size_t)nr * ns * ns * (N / 2)));
    L4Rot ra, rb;
    for (int k = 0; k < 9; k++) {
        ra.R[k] = (k % 4 == 0) ? 1.0 : 0.0; // A unrotated
        rb.R[k] = RB[k];
    }
    int loA = 0, bA = nr, loB = 0, bB = nr;
    cudaError_t e;
    if ((e = l4_xplanes(t, N, Nr, kA, nA, ra, 0, ip, ipr, ws, XA, loA, bA, nsm, s)) != cudaSuccess) return e;
    if ((e = l4_xplanes(t, N, Nr, kB, nB, rb, 1, ip, ipr, ws, Z1, loB, bB, nsm, s)) != cudaSuccess) return e;
    switch (nr) {
    case 32: return l4_rc_ns<32>(XA, Z1, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    case 64: return l4_rc_ns<64>(XA, Z1, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    case 128: return l4_rc_ns<128>(XA, Z1, N, loA, bA, loB, bB, t, cone, slices, nslices, period_r, scale, h, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
