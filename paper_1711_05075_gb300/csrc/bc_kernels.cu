// CUDA kernels of the ball-union correlation (sm_103a, FP32 data path).
//
// Pipeline for one batch of "instances" (shape A, and shape B under each
// rotation) and "pairs" (A with one rotated B):
//
//   k_prepare   rotate the knots (Eq. (Mink0), Sec. 2.4: a rigid motion only
//               moves the centres), map them to fine-grid coordinates and find
//               each instance's support box (the cells its spreading touches).
//   k_spread    type-1 NUFFT step 1 for the impulse densities of Eq. (rhoP):
//               Kaiser-Bessel spreading of every knot onto its level's grid,
//               restricted to the support box (cells outside it stay zero).
//   k_fft_z     step 2, first axis: real-to-complex transform of every grid
//               row along z; only m_z in [0, N/2) is kept (output pruning).
//   k_fft_y     step 2, second axis, over the rows inside the support box only
//               (input pruning); keeps m_y in (-N/2, N/2).
//   k_fft_x     step 2, third axis, fused with step 3 and the correlation:
//               window deconvolution, the ball transform of each level and the
//               level sum (Eq. (fballhat)), the conjugate product of Eq. (ccghat)
//               with the P^-3 scale and the grid-origin sign, and the inverse
//               transform along x.
//   k_ifft_y    inverse transform along y.
//   k_ifft_z    complex-to-real inverse along z (two rows per complex transform)
//               giving g on the N^3 translation grid.
//
// The support-box pruning computes exactly the transforms of the full
// oversampled grids: the cells it skips hold zeros.
#include <climits>
#include <cstdint>

#include "bc_fft.cuh"
#include "bc_internal.h"

namespace bc {

bool supported_N(int N)
{
    return N == 32 || N == 64 || N == 96 || N == 128 || N == 256;
}

__device__ __forceinline__ int mode_of(int j, int N) { return j < N / 2 ? j : j - N; }

// ------------------------------------------------------------------ tables
// FP64 construction of the window-deconvolution, ball-transform and twiddle
// tables, each rounded once to FP32.
//
// Window: phi(v) = I0(beta sqrt(1 - (2v/W)^2)) / I0(beta) on |v| <= W/2 (fine-grid
// cells).  Its transform is phi^(xi) = W sinh(sqrt(beta^2 - (pi W xi)^2)) /
// sqrt(beta^2 - (pi W xi)^2) / I0(beta) (sin form when the radicand is negative;
// Kaiser-Bessel pair, Jackson et al., IEEE TMI 1991).  deconv[j] = 1/phi^(m/n).
//
// Ball transform (Sec. 2.5, indicator kernel of Eq. (L2ball)):
// h^(r, k) = 4 pi (sin kr - kr cos kr) / k^3 with k = 2 pi sqrt(q) / P, and for
// x = kr < 0.5 the Maclaurin series 4 pi r^3 (1/3 - x^2/30 + x^4/840 -
// x^6/45360 + x^8/3991680), indexed by the integer q = |m|^2.
__global__ void k_build_tables(int N, int n, int W, int L, int qmax, double beta, double period,
                               const double *__restrict__ radii, float *deconv, float *ballft, float2 *tw_n,
                               float2 *tw_N, float *consts)
{
    const double pi = 3.14159265358979323846;
    if (blockIdx.x == 0 && threadIdx.x == 0) consts[0] = (float)(exp(beta) / cyl_bessel_i0(beta));
    const int total = N + L * (qmax + 1) + n + N;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        if (t < N) {
            int m = t < N / 2 ? t : t - N;
            double xi = (double)m / (double)n;
            double a = beta * beta - (pi * W * xi) * (pi * W * xi);
            double s = sqrt(fabs(a));
            double ph;
            if (a > 0) ph = W * sinh(s) / s;
            else if (a < 0) ph = W * sin(s) / s;
            else ph = W;
            ph /= cyl_bessel_i0(beta);
            deconv[t] = (float)(1.0 / ph);
        } else if (t < N + L * (qmax + 1)) {
            int u = t - N;
            int l = u / (qmax + 1), q = u - l * (qmax + 1);
            double r = radii[l];
            double k = 2.0 * pi * sqrt((double)q) / period;
            double x = k * r, v;
            if (x < 0.5) {
                double x2 = x * x;
                v = 4.0 * pi * r * r * r *
                    (1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0 - x2 * x2 * x2 / 45360.0 +
                     x2 * x2 * x2 * x2 / 3991680.0);
            } else {
                v = 4.0 * pi * (sin(x) - x * cos(x)) / (k * k * k);
            }
            ballft[u] = (float)v;
        } else if (t < N + L * (qmax + 1) + n) {
            int k = t - N - L * (qmax + 1);
            double a = 2.0 * pi * k / n;
            tw_n[k] = make_float2((float)cos(a), (float)(-sin(a)));
        } else {
            int k = t - N - L * (qmax + 1) - n;
            double a = 2.0 * pi * k / N;
            tw_N[k] = make_float2((float)cos(a), (float)(-sin(a)));
        }
    }
}

cudaError_t launch_build_tables(const Geometry &g, double beta, double period, const double *radii_dev,
                                float *deconv, float *ballft, float2 *tw_n, float2 *tw_N, float *consts,
                                cudaStream_t s)
{
    const int qmax = 3 * (g.N / 2) * (g.N / 2);
    const int total = g.N + g.L * (qmax + 1) + g.n + g.N;
    k_build_tables<<<(total + 255) / 256, 256, 0, s>>>(g.N, g.n, g.W, g.L, qmax, beta, period, radii_dev, deconv,
                                                        ballft, tw_n, tw_N, consts);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ knots
// (x, y, z) + level id -> float4 (x, y, z, level bits).  stats[0]: max |c|^2
// (float bits), stats[1]: flags (1 = level out of range, 2 = non-finite).
__global__ void k_pack_knots(const float *__restrict__ xyz, const int *__restrict__ level, int n, int L,
                             float4 *knots, unsigned int *stats)
{
    float r2max = 0.f;
    unsigned int flags = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        float x = xyz[3 * j], y = xyz[3 * j + 1], z = xyz[3 * j + 2];
        int l = level[j];
        if (l < 0 || l >= L) flags |= 1u;
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) flags |= 2u;
        float r2 = x * x + y * y + z * z;
        if (isfinite(r2)) r2max = fmaxf(r2max, r2);
        knots[j] = make_float4(x, y, z, __int_as_float(l));
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2max = fmaxf(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
        flags |= __shfl_xor_sync(0xffffffffu, flags, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats[0], __float_as_uint(r2max));
        if (flags) atomicOr(&stats[1], flags);
    }
}

cudaError_t launch_pack_knots(const float *xyz, const int *level, int n, int L, float4 *knots,
                              unsigned int *stats, cudaStream_t s)
{
    int blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    k_pack_knots<<<blocks, 256, 0, s>>>(xyz, level, n, L, knots, stats);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ prepare
// One block per instance.  Knot j of instance i becomes
// ku = (u_x, u_y, u_z, level | i << 4) with u = (R c) n / P wrapped into
// [-n/2, n/2) (fine-grid cells; the period P spans n cells).  The spreading
// stencil of a knot covers cells g0 .. g0 + W - 1 per axis, g0 = ceil(u - W/2).
__global__ void k_prepare(Geometry g, const InstDesc *__restrict__ inst, float4 *ku, InstPlan *plan, int *err)
{
    const int i = blockIdx.x;
    const InstDesc d = inst[i];
    // rotation matrix of the normalised quaternion (w, x, y, z)
    float qw = d.q[0], qx = d.q[1], qy = d.q[2], qz = d.q[3];
    float s = 1.0f / sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= s; qx *= s; qy *= s; qz *= s;
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    const float nf = (float)g.n, halfW = 0.5f * (float)g.W;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int j = threadIdx.x; j < d.nknots; j += blockDim.x) {
        float4 c = d.knots[d.src_off + j];
        float p[3];
        p[0] = fmaf(R00, c.x, fmaf(R01, c.y, R02 * c.z));
        p[1] = fmaf(R10, c.x, fmaf(R11, c.y, R12 * c.z));
        p[2] = fmaf(R20, c.x, fmaf(R21, c.y, R22 * c.z));
        float u[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float v = p[a] * g.n_over_P;
            v -= nf * floorf(v / nf + 0.5f);
            u[a] = v;
            int g0 = (int)ceilf(v - halfW);
            lo[a] = min(lo[a], g0);
            hi[a] = max(hi[a], g0 + g.W - 1);
        }
        int tag = __float_as_int(c.w) | (i << 4);
        ku[d.knot_off + j] = make_float4(u[0], u[1], u[2], __int_as_float(tag));
    }
    __shared__ int red[6][32];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        for (int a = 0; a < 3; a++) {
            red[a][w] = lo[a];
            red[3 + a][w] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int L0[3], H0[3];
        for (int a = 0; a < 3; a++) {
            L0[a] = INT_MAX;
            H0[a] = INT_MIN;
            for (int k = 0; k < nw; k++) {
                L0[a] = min(L0[a], red[a][k]);
                H0[a] = max(H0[a], red[3 + a][k]);
            }
        }
        InstPlan pl;
        bool empty = d.nknots <= 0;
        for (int a = 0; a < 3; a++) {
            int b = empty ? 0 : min(H0[a] - L0[a] + 1, g.n);
            if (b > d.cap_e) {
                atomicOr(err, 1);
                empty = true;
            }
            pl.lo[a] = empty ? 0 : L0[a];
            pl.b[a] = b;
            pl.pos0[a] = empty ? 0 : ((L0[a] % g.n) + g.n) % g.n;
        }
        if (empty) pl.b[0] = pl.b[1] = pl.b[2] = 0;
        pl.bzp = (pl.b[2] + 3) & ~3;
        plan[i] = pl;
    }
}

cudaError_t launch_prepare(const Geometry &g, const InstDesc *inst, int ninst, float4 *ku, InstPlan *plan,
                           int *err, cudaStream_t s)
{
    if (ninst <= 0) return cudaSuccess;
    k_prepare<<<ninst, 1024, 0, s>>>(g, inst, ku, plan, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ spread
// One warp per knot.  Lanes 0..3W-1 evaluate the separable window weights
// phi(u_a - g) for the W cells of each axis; the W^3 products are then added
// into the knot's level grid (compact support-box layout
// [level][ix][iy][iz], iz padded to bzp), z fastest across lanes.
constexpr int SPREAD_WARPS = 8;

__global__ void __launch_bounds__(SPREAD_WARPS * 32)
k_spread(Geometry g, const float *__restrict__ consts, const InstDesc *__restrict__ inst,
         const float4 *__restrict__ ku, const InstPlan *__restrict__ plan, float *grid, int total)
{
    const float inv_scaled_i0beta = consts[0];
    __shared__ float wts[SPREAD_WARPS][3][16];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = g.W, W2 = W * W, W3 = W2 * W;
    const float halfW = 0.5f * (float)W, twoOverW = 2.0f / (float)W;
    for (int k = blockIdx.x * SPREAD_WARPS + wib; k < total; k += gridDim.x * SPREAD_WARPS) {
        const float4 v = ku[k];
        const int tag = __float_as_int(v.w);
        const int level = tag & 15, i = tag >> 4;
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const float u[3] = {v.x, v.y, v.z};
        int g0[3];
#pragma unroll
        for (int a = 0; a < 3; a++) g0[a] = (int)ceilf(u[a] - halfW);
        if (lane < 3 * W) {
            // phi = I0(beta sq) / I0(beta), sq = sqrt(1 - s^2), evaluated as
            // exp(beta (sq - 1)) * [exp(-x) I0(x)] / [exp(-beta) I0(beta)], x = beta sq.
            // I0 grows like e^x, so I0(x) alone carries the FP32 rounding of x as a
            // relative error of about x * 2^-24; exp(-x) I0(x) varies slowly and
            // the exponent beta (sq - 1) = -beta s^2 / (1 + sq) is small where
            // phi is large.
            const int a = lane / W, t = lane - a * W;
            const float s = (u[a] - (float)(g0[a] + t)) * twoOverW;
            const float s2 = fminf(s * s, 1.f);
            const float sq = sqrtf(1.f - s2);
            const float x = g.beta * sq;
            const float scaled_i0 = cyl_bessel_i0f(x) * expf(-x);
            wts[wib][a][t] = expf(-g.beta * s2 / (1.f + sq)) * scaled_i0 * inv_scaled_i0beta;
        }
        __syncwarp();
        const long long boxsz = (long long)p.b[0] * p.b[1] * p.bzp;
        float *G = grid + inst[i].grid_off + (long long)level * boxsz;
        for (int e = lane; e < W3; e += 32) {
            const int dx = e / W2, dy = (e / W) % W, dz = e % W;
            int ix = g0[0] + dx - p.lo[0];
            int iy = g0[1] + dy - p.lo[1];
            int iz = g0[2] + dz - p.lo[2];
            if (ix >= g.n) ix -= g.n;
            if (iy >= g.n) iy -= g.n;
            if (iz >= g.n) iz -= g.n;
            const float val = wts[wib][0][dx] * wts[wib][1][dy] * wts[wib][2][dz];
            atomicAdd(&G[((long long)ix * p.b[1] + iy) * p.bzp + iz], val);
        }
        __syncwarp();
    }
}

cudaError_t launch_spread(const Geometry &g, const Tables &t, const InstDesc *inst, int total_knots,
                          const float4 *ku, const InstPlan *plan, float *grid, cudaStream_t s)
{
    if (total_knots <= 0) return cudaSuccess;
    int blocks = (total_knots + SPREAD_WARPS - 1) / SPREAD_WARPS;
    if (blocks > 65535) blocks = 65535;
    k_spread<<<blocks, SPREAD_WARPS * 32, 0, s>>>(g, t.consts, inst, ku, plan, grid, total_knots);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ helpers
// Block loop over the work blocks of a sequence of instances, giving each
// block of the grid an even share across instances.
struct RotStart {
    int rot = 0;
    __device__ __forceinline__ int first() const
    {
        int st = rot % (int)gridDim.x;
        return ((int)blockIdx.x - st + (int)gridDim.x) % (int)gridDim.x;
    }
};

template <int NF>
__device__ __forceinline__ void load_twiddles(float2 *dst, const float2 *__restrict__ src)
{
    for (int k = threadIdx.x; k < NF; k += blockDim.x) dst[k] = src[k];
}

// ------------------------------------------------------------------ fft z
// Real rows of the level grids -> m_z in [0, N/2), two rows per complex
// transform: with Z = FFT(a + i b), A_k = (Z_k + conj Z_{n-k}) / 2 and
// B_k = (Z_k - conj Z_{n-k}) / (2i).  Compact index iz lands at position
// (pos0_z + iz) mod n of the length-n row, the rest of the row is zero.
// Every grid cell read is reset to zero, so the spreading buffer is clean for
// the next launch without a separate memset pass.
template <int NF>
__global__ void __launch_bounds__(256)
k_fft_z(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
        float *grid, float2 *z1)
{
    constexpr int LINES = (4096 / NF) < 4 ? 4 : (4096 / NF);
    constexpr int LS = NF + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + NF, *B = A + LINES * LS;
    load_twiddles<NF>(tw, tb.tw_n);
    const int H = g.H, L = g.L;
    RotStart rs;
    for (int i = 0; i < ninst; i++) {
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const int b0 = p.b[0], b1 = p.b[1], bz = p.b[2], bzp = p.bzp, by2 = (b1 + 1) >> 1;
        const int items = L * b0 * by2;
        const int nblk = (items + LINES - 1) / LINES;
        const InstDesc d = inst[i];
        for (int blk = rs.first(); blk < nblk; blk += gridDim.x) {
            for (int e = threadIdx.x; e < LINES * NF; e += blockDim.x) A[(e / NF) * LS + (e % NF)] = make_float2(0.f, 0.f);
            __syncthreads();
            for (int e = threadIdx.x; e < LINES * bz; e += blockDim.x) {
                const int q = e / bz, iz = e - q * bz;
                const int item = blk * LINES + q;
                if (item >= items) continue;
                const int l = item / (b0 * by2), rem = item - l * (b0 * by2);
                const int ix = rem / by2, iy0 = 2 * (rem - ix * by2);
                float *G = grid + d.grid_off + (long long)l * b0 * b1 * bzp + ((long long)ix * b1 + iy0) * bzp;
                float a = G[iz];
                G[iz] = 0.f;
                float b = 0.f;
                if (iy0 + 1 < b1) {
                    b = G[bzp + iz];
                    G[bzp + iz] = 0.f;
                }
                int pos = p.pos0[2] + iz;
                if (pos >= NF) pos -= NF;
                A[q * LS + pos] = make_float2(a, b);
            }
            __syncthreads();
            float2 *res = fft_lines<NF, false>(A, B, LINES, LS, tw);
            for (int e = threadIdx.x; e < LINES * H; e += blockDim.x) {
                const int q = e / H, k = e - q * H;
                const int item = blk * LINES + q;
                if (item >= items) continue;
                const int l = item / (b0 * by2), rem = item - l * (b0 * by2);
                const int ix = rem / by2, iy0 = 2 * (rem - ix * by2);
                const float2 zk = res[q * LS + k];
                const float2 zn = res[q * LS + (k == 0 ? 0 : NF - k)];
                const float2 ak = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
                const float2 bk = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
                float2 *Z = z1 + d.z1_off + (((long long)l * b0 + ix) * b1 + iy0) * H;
                Z[k] = ak;
                if (iy0 + 1 < b1) Z[H + k] = bk;
            }
            __syncthreads();
        }
        rs.rot += nblk;
    }
}

// ------------------------------------------------------------------ fft y
// For each (level, ix) plane and a chunk of C z-modes: transform along y over
// the support rows only; keep m_y in (-N/2, N/2) at FFT index j (m_y = -N/2,
// j = N/2, is stored as zero).
template <int NF>
__global__ void __launch_bounds__(256)
k_fft_y(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
        const float2 *__restrict__ z1, float2 *y1)
{
    constexpr int C = 16;
    constexpr int LS = NF + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + NF, *B = A + C * LS;
    load_twiddles<NF>(tw, tb.tw_n);
    const int H = g.H, L = g.L, N = g.N;
    const int Cc = H < C ? H : C;
    const int nch = H / Cc;
    RotStart rs;
    for (int i = 0; i < ninst; i++) {
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const int b0 = p.b[0], b1 = p.b[1];
        const int items = L * b0 * nch;
        const InstDesc d = inst[i];
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int l = it / (b0 * nch), rem = it - l * (b0 * nch);
            const int ix = rem / nch, ch = rem - ix * nch;
            for (int e = threadIdx.x; e < Cc * NF; e += blockDim.x) A[(e / NF) * LS + (e % NF)] = make_float2(0.f, 0.f);
            __syncthreads();
            const float2 *Z = z1 + d.z1_off + ((long long)l * b0 + ix) * b1 * H + ch * Cc;
            for (int e = threadIdx.x; e < b1 * Cc; e += blockDim.x) {
                const int iy = e / Cc, c = e - iy * Cc;
                int pos = p.pos0[1] + iy;
                if (pos >= NF) pos -= NF;
                A[c * LS + pos] = Z[(long long)iy * H + c];
            }
            __syncthreads();
            float2 *res = fft_lines<NF, false>(A, B, Cc, LS, tw);
            float2 *Y = y1 + d.y1_off + ((long long)l * b0 + ix) * N * H + ch * Cc;
            for (int e = threadIdx.x; e < N * Cc; e += blockDim.x) {
                const int j = e / Cc, c = e - j * Cc;
                const int m = mode_of(j, N);
                float2 v = make_float2(0.f, 0.f);
                if (j != N / 2) v = res[c * LS + (m < 0 ? m + NF : m)];
                Y[(long long)j * H + c] = v;
            }
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ fft x + combine
// For each pair and each (j_y, chunk of C z-modes):
//   F_s(m) = sum_l T_l(|m|^2) D(m) FFT_x[Y1_{s,l}](m)    (s = A, B)
//   g'(m)  = P^-3 (-1)^(m_x+m_y+m_z) F_A(m) conj(F_B(m)), zero on the Nyquist planes
//   H(k_x, j_y, m_z) = sum_{j_x} g'(m) exp(+2 pi i j_x k_x / N)
// D(m) = deconv[j_x] deconv[j_y] deconv[m_z].  The sign moves the origin of the
// translation grid to t = -P/2: exp(2 pi i m (-P/2) / P) = (-1)^m.
// With pair.a < 0, F_A comes from the cached spectrum; with pair.b < 0, F_A is
// written to `fa_out` and nothing else happens.
template <int NF, int NI>
__global__ void __launch_bounds__(256)
k_fft_x(Geometry g, Tables tb, const InstDesc *__restrict__ inst, const InstPlan *__restrict__ plan,
        const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ y1,
        const float2 *__restrict__ fa_cache, float2 *fa_out, float2 *h)
{
    constexpr int C = 16;
    constexpr int LSF = NF + 1, LSI = NI + 1;
    extern __shared__ float2 sm[];
    float2 *twF = sm, *twI = twF + NF, *A = twI + NI, *B = A + C * LSF, *FA = B + C * LSF, *FB = FA + C * NI;
    load_twiddles<NF>(twF, tb.tw_n);
    load_twiddles<NI>(twI, tb.tw_N);
    const int H = g.H, L = g.L, N = NI;
    const int Cc = H < C ? H : C;
    const int nch = H / Cc;
    const int items = N * nch;
    const int Q = tb.qmax + 1;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int jy = it / nch, ch = it - jy * nch;
            const int my = mode_of(jy, N);
            const float djy = tb.deconv[jy];
            for (int side = 0; side < 2; side++) {
                float2 *acc = side ? FB : FA;
                const int si = side ? pr.b : pr.a;
                if (side == 1 && si < 0) break;
                if (si < 0) {
                    for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) {
                        const int c = e / NI, jx = e - c * NI;
                        acc[e] = fa_cache[((long long)jx * N + jy) * H + ch * Cc + c];
                    }
                    continue;
                }
                for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
                const InstPlan p = plan[si];
                if (p.b[0] == 0) continue;
                const InstDesc d = inst[si];
                const int b0 = p.b[0];
                for (int l = 0; l < L; l++) {
                    for (int e = threadIdx.x; e < Cc * NF; e += blockDim.x) A[(e / NF) * LSF + (e % NF)] = make_float2(0.f, 0.f);
                    __syncthreads();
                    const float2 *Y = y1 + d.y1_off + (long long)l * b0 * N * H + (long long)jy * H + ch * Cc;
                    for (int e = threadIdx.x; e < b0 * Cc; e += blockDim.x) {
                        const int ix = e / Cc, c = e - ix * Cc;
                        int pos = p.pos0[0] + ix;
                        if (pos >= NF) pos -= NF;
                        A[c * LSF + pos] = Y[(long long)ix * N * H + c];
                    }
                    __syncthreads();
                    float2 *res = fft_lines<NF, false>(A, B, Cc, LSF, twF);
                    const float *T = tb.ballft + (long long)l * Q;
                    for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) {
                        const int c = e / NI, jx = e - c * NI;
                        if (jx == N / 2) continue;
                        const int mx = mode_of(jx, N), mz = ch * Cc + c;
                        const float Mv = T[mx * mx + my * my + mz * mz] * tb.deconv[jx] * djy * tb.deconv[mz];
                        const float2 v = res[c * LSF + (mx < 0 ? mx + NF : mx)];
                        acc[e] = make_float2(fmaf(Mv, v.x, acc[e].x), fmaf(Mv, v.y, acc[e].y));
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            if (pr.b < 0) {
                for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) {
                    const int jx = e / Cc, c = e - jx * Cc;
                    fa_out[((long long)jx * N + jy) * H + ch * Cc + c] = FA[c * NI + jx];
                }
                __syncthreads();
                continue;
            }
            for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) {
                const int c = e / NI, jx = e - c * NI;
                const int mx = mode_of(jx, N), mz = ch * Cc + c;
                float2 v = make_float2(0.f, 0.f);
                if (jx != N / 2 && jy != N / 2) {
                    v = cmulc(FA[e], FB[e]);
                    const float sg = ((mx + my + mz) & 1) ? -g.inv_P3 : g.inv_P3;
                    v = cscale(v, sg);
                }
                A[c * LSI + jx] = v;
            }
            __syncthreads();
            float2 *res = fft_lines<NI, true>(A, B, Cc, LSI, twI);
            float2 *Hp = h + pr.h_off + (long long)jy * H + ch * Cc;
            for (int e = threadIdx.x; e < Cc * NI; e += blockDim.x) {
                const int kx = e / Cc, c = e - kx * Cc;
                Hp[(long long)kx * N * H + c] = res[c * LSI + kx];
            }
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ inverse y
template <int NI>
__global__ void __launch_bounds__(256)
k_ifft_y(Geometry g, Tables tb, const PairDesc *__restrict__ pairs, int npairs, float2 *h)
{
    constexpr int C = 16;
    constexpr int LS = NI + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + NI, *B = A + C * LS;
    load_twiddles<NI>(tw, tb.tw_N);
    const int H = g.H, N = NI;
    const int Cc = H < C ? H : C;
    const int nch = H / Cc;
    const int items = N * nch;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        if (pr.b < 0) continue;
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int kx = it / nch, ch = it - kx * nch;
            float2 *Hp = h + pr.h_off + (long long)kx * N * H + ch * Cc;
            for (int e = threadIdx.x; e < N * Cc; e += blockDim.x) {
                const int jy = e / Cc, c = e - jy * Cc;
                A[c * LS + jy] = Hp[(long long)jy * H + c];
            }
            __syncthreads();
            float2 *res = fft_lines<NI, true>(A, B, Cc, LS, tw);
            for (int e = threadIdx.x; e < N * Cc; e += blockDim.x) {
                const int ky = e / Cc, c = e - ky * Cc;
                Hp[(long long)ky * H + c] = res[c * LS + ky];
            }
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ inverse z (c2r)
// Rows a (k_y even) and b (k_y + 1) of the half spectrum are packed as
// Z_k = A_k + i B_k over the full range (A_{N-k} = conj A_k, A_0 taken real,
// the m_z = N/2 term zero); the inverse transform of Z is a + i b.
template <int NI>
__global__ void __launch_bounds__(256)
k_ifft_z(Geometry g, Tables tb, const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ h,
         float *out)
{
    constexpr int LINES = (4096 / NI) < 4 ? 4 : (4096 / NI);
    constexpr int LS = NI + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + NI, *B = A + LINES * LS;
    load_twiddles<NI>(tw, tb.tw_N);
    const int H = g.H, N = NI;
    const int items = N * (N / 2);
    const int nblk = (items + LINES - 1) / LINES;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        if (pr.b < 0) continue;
        for (int blk = rs.first(); blk < nblk; blk += gridDim.x) {
            for (int e = threadIdx.x; e < LINES * NI; e += blockDim.x) {
                const int q = e / NI, k = e - q * NI;
                const int item = blk * LINES + q;
                float2 z = make_float2(0.f, 0.f);
                if (item < items) {
                    const int kx = item / (N / 2), ky0 = 2 * (item - kx * (N / 2));
                    const float2 *r0 = h + pr.h_off + ((long long)kx * N + ky0) * H;
                    const float2 *r1 = r0 + H;
                    if (k == 0) {
                        z = make_float2(r0[0].x, r1[0].x);
                    } else if (k < H) {
                        const float2 a = r0[k], b = r1[k];
                        z = make_float2(a.x - b.y, a.y + b.x);
                    } else if (k > H) {
                        const float2 a = r0[NI - k], b = r1[NI - k];
                        z = make_float2(a.x + b.y, b.x - a.y);
                    }
                }
                A[q * LS + k] = z;
            }
            __syncthreads();
            float2 *res = fft_lines<NI, true>(A, B, LINES, LS, tw);
            for (int e = threadIdx.x; e < LINES * NI; e += blockDim.x) {
                const int q = e / NI, kz = e - q * NI;
                const int item = blk * LINES + q;
                if (item >= items) continue;
                const int kx = item / (N / 2), ky0 = 2 * (item - kx * (N / 2));
                float *o = out + pr.out_off + ((long long)kx * N + ky0) * N;
                const float2 v = res[q * LS + kz];
                o[kz] = v.x;
                o[N + kz] = v.y;
            }
            __syncthreads();
        }
        rs.rot += nblk;
    }
}

// ------------------------------------------------------------------ launchers
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

template <int NF>
static cudaError_t fft_z_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                           float *grid, float2 *z1, int nsm, cudaStream_t s)
{
    constexpr int LINES = (4096 / NF) < 4 ? 4 : (4096 / NF);
    size_t smem = sizeof(float2) * (NF + 2 * LINES * (NF + 1));
    cudaError_t e = set_smem(k_fft_z<NF>, smem);
    if (e != cudaSuccess) return e;
    k_fft_z<NF><<<2 * nsm, 256, smem, s>>>(g, t, inst, ninst, plan, grid, z1);
    return cudaGetLastError();
}

cudaError_t launch_fft_z(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                         float *grid, float2 *z1, int nsm, cudaStream_t s)
{
    switch (g.n) {
    case 64: return fft_z_t<64>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 128: return fft_z_t<128>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 192: return fft_z_t<192>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 256: return fft_z_t<256>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 512: return fft_z_t<512>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NF>
static cudaError_t fft_y_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                           const float2 *z1, float2 *y1, int nsm, cudaStream_t s)
{
    size_t smem = sizeof(float2) * (NF + 2 * 16 * (NF + 1));
    cudaError_t e = set_smem(k_fft_y<NF>, smem);
    if (e != cudaSuccess) return e;
    k_fft_y<NF><<<2 * nsm, 256, smem, s>>>(g, t, inst, ninst, plan, z1, y1);
    return cudaGetLastError();
}

cudaError_t launch_fft_y(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                         const float2 *z1, float2 *y1, int nsm, cudaStream_t s)
{
    switch (g.n) {
    case 64: return fft_y_t<64>(g, t, inst, ninst, plan, z1, y1, nsm, s);
    case 128: return fft_y_t<128>(g, t, inst, ninst, plan, z1, y1, nsm, s);
    case 192: return fft_y_t<192>(g, t, inst, ninst, plan, z1, y1, nsm, s);
    case 256: return fft_y_t<256>(g, t, inst, ninst, plan, z1, y1, nsm, s);
    case 512: return fft_y_t<512>(g, t, inst, ninst, plan, z1, y1, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NF, int NI>
static cudaError_t fft_x_t(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                           const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *fa_out,
                           float2 *h, int nsm, cudaStream_t s)
{
    size_t smem = sizeof(float2) * (NF + NI + 2 * 16 * (NF + 1) + 2 * 16 * NI);
    cudaError_t e = set_smem(k_fft_x<NF, NI>, smem);
    if (e != cudaSuccess) return e;
    k_fft_x<NF, NI><<<2 * nsm, 256, smem, s>>>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h);
    return cudaGetLastError();
}

cudaError_t launch_fft_x(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                         const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *fa_out,
                         float2 *h, int nsm, cudaStream_t s)
{
    switch (g.N) {
    case 32: return fft_x_t<64, 32>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    case 64: return fft_x_t<128, 64>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    case 96: return fft_x_t<192, 96>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    case 128: return fft_x_t<256, 128>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    case 256: return fft_x_t<512, 256>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NI>
static cudaError_t ifft_y_t(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, float2 *h, int nsm,
                            cudaStream_t s)
{
    size_t smem = sizeof(float2) * (NI + 2 * 16 * (NI + 1));
    cudaError_t e = set_smem(k_ifft_y<NI>, smem);
    if (e != cudaSuccess) return e;
    k_ifft_y<NI><<<2 * nsm, 256, smem, s>>>(g, t, pairs, npairs, h);
    return cudaGetLastError();
}

cudaError_t launch_ifft_y(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, float2 *h, int nsm,
                          cudaStream_t s)
{
    switch (g.N) {
    case 32: return ifft_y_t<32>(g, t, pairs, npairs, h, nsm, s);
    case 64: return ifft_y_t<64>(g, t, pairs, npairs, h, nsm, s);
    case 96: return ifft_y_t<96>(g, t, pairs, npairs, h, nsm, s);
    case 128: return ifft_y_t<128>(g, t, pairs, npairs, h, nsm, s);
    case 256: return ifft_y_t<256>(g, t, pairs, npairs, h, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NI>
static cudaError_t ifft_z_t(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                            float *out, int nsm, cudaStream_t s)
{
    constexpr int LINES = (4096 / NI) < 4 ? 4 : (4096 / NI);
    size_t smem = sizeof(float2) * (NI + 2 * LINES * (NI + 1));
    cudaError_t e = set_smem(k_ifft_z<NI>, smem);
    if (e != cudaSuccess) return e;
    k_ifft_z<NI><<<2 * nsm, 256, smem, s>>>(g, t, pairs, npairs, h, out);
    return cudaGetLastError();
}

cudaError_t launch_ifft_z(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                          float *out, int nsm, cudaStream_t s)
{
    switch (g.N) {
    case 32: return ifft_z_t<32>(g, t, pairs, npairs, h, out, nsm, s);
    case 64: return ifft_z_t<64>(g, t, pairs, npairs, h, out, nsm, s);
    case 96: return ifft_z_t<96>(g, t, pairs, npairs, h, out, nsm, s);
    case 128: return ifft_z_t<128>(g, t, pairs, npairs, h, out, nsm, s);
    case 256: return ifft_z_t<256>(g, t, pairs, npairs, h, out, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
