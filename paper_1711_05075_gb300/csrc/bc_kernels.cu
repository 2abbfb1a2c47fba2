// CUDA kernels of the ball-union correlation (sm_103a, FP32 data path).
//
// Pipeline for one batch of "instances" (shape A, and shape B under each
// rotation) and "pairs" (A with one rotated B):
//
//   k_prepare   rotate the knots (Eq. (Mink0), Sec. 2.4: a rigid motion only
//               moves the centres), map them to fine-grid coordinates and find
//               each instance's support box (the cells its spreading touches);
//               The last block to finish turns the boxes into
//               per-instance plans.
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
// The transform passes work on shared-memory tiles of 16 interleaved lines
// (bc_fft.cuh) loaded and stored with 16-byte accesses.
//
// The support-box pruning computes exactly the transforms of the full
// oversampled grids: the cells it skips hold zeros.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "bc_passes.cuh"

namespace bc {

bool supported_split(int N) { return N == 32 || N == 64 || N == 96 || N == 128 || N == 256; }

bool supported_N(int N)
{
    return N == 32 || N == 64 || N == 96 || N == 128 || N == 256;
}

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
    if (blockIdx.x == 0 && threadIdx.x < W) {
        // window piece t (kb_poly): interpolate f(y) = phi(y + 1/2 + W/2 - 1 - t),
        // y in [-1/2, 1/2], at the Chebyshev nodes y_k = cos(pi (k + 1/2) / KB_NC) / 2
        // as sum_j a_j T_j(2y), then expand in powers of y
        const int t = threadIdx.x;
        const double i0b = cyl_bessel_i0(beta);
        double f[KB_NC], a[KB_NC];
        for (int k = 0; k < KB_NC; k++) {
            const double v = 0.5 * cos(pi * (k + 0.5) / KB_NC) + 0.5 + 0.5 * W - 1.0 - t;
            const double s2 = (2.0 * v / W) * (2.0 * v / W);
            f[k] = s2 <= 1.0 ? cyl_bessel_i0(beta * sqrt(1.0 - s2)) / i0b : 0.0;
        }
        for (int j = 0; j < KB_NC; j++) {
            double acc = 0.0;
            for (int k = 0; k < KB_NC; k++) acc += f[k] * cos(pi * j * (k + 0.5) / KB_NC);
            a[j] = (j == 0 ? 1.0 : 2.0) * acc / KB_NC;
        }
        // power coefficients in z = 2y: T_0 = 1, T_1 = z, T_{j+1} = 2 z T_j - T_{j-1}
        double tm[KB_NC] = {}, tc[KB_NC] = {}, b[KB_NC] = {};
        tm[0] = 1.0;
        tc[1] = 1.0;
        b[0] = a[0];
        b[1] = a[1];
        for (int j = 2; j < KB_NC; j++) {
            double tn[KB_NC];
            for (int m = 0; m < KB_NC; m++) tn[m] = (m > 0 ? 2.0 * tc[m - 1] : 0.0) - tm[m];
            for (int m = 0; m < KB_NC; m++) {
                b[m] += a[j] * tn[m];
                tm[m] = tc[m];
                tc[m] = tn[m];
            }
        }
        double scale = 1.0;
        for (int m = 0; m < KB_NC; m++, scale *= 2.0) consts[KB_OFF + t * KB_NC + m] = (float)(b[m] * scale);
    }
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
            ballft[u] = (float)ball_ft64(radii[l], 2.0 * pi * sqrt((double)q) / period);
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

// Shape-complementarity weights (Sec. 4.2): the offset S + B0 of a union of
// balls is the union of the balls grown by r0, so the affinity function's
// real part f_{S+B0} - lambda f_S has, per level, the transform
// [h^(rho_l + r0, k) - lambda h^(rho_l, k)] S_l(m).  out[l][q], built in FP64
// and rounded once, replaces the ball transform table for a score.
__global__ void k_build_score_table(int L, int qmax, double period, const double *__restrict__ radii, double r0,
                                    double lambda, float *out)
{
    const double pi = 3.14159265358979323846;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < L * (qmax + 1); u += gridDim.x * blockDim.x) {
        const int l = u / (qmax + 1), q = u - l * (qmax + 1);
        const double k = 2.0 * pi * sqrt((double)q) / period;
        out[u] = (float)(ball_ft64(radii[l] + r0, k) - lambda * ball_ft64(radii[l], k));
    }
}

cudaError_t launch_build_score_table(const Geometry &g, double period, const double *radii_dev, double r0,
                                     double lambda, float *out, cudaStream_t s)
{
    const int qmax = 3 * (g.N / 2) * (g.N / 2);
    const int total = g.L * (qmax + 1);
    k_build_score_table<<<(total + 255) / 256, 256, 0, s>>>(g.L, qmax, period, radii_dev, r0, lambda, out);
    return cudaGetLastError();
}

// The x pass's level weights as one table, laid out so that the weights of
// an x-pass item (row j_y, z-modes 16 ch .. 16 ch + 15) are one contiguous
// slice: xw[(((j_y nch + ch) L + l) (N/2 + 1) + a) 16 + c] =
// ballft_l(a^2 + m_y^2 + m_z^2) (D(a) D(m_y) D(m_z)), m_z = 16 ch + c, the same
// FP32 expression build_xweights evaluates inside the pass.
__global__ void k_build_xw(int N, int L, int qmax, const float *__restrict__ deconv, const float *__restrict__ ballft,
                           float *xw)
{
    const int A = N / 2 + 1, nch = N / 2 / CL;
    const long long total = (long long)N * nch * L * A * CL;
    const long long Q = qmax + 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % CL), a = (int)((e / CL) % A), l = (int)((e / ((long long)CL * A)) % L);
        const long long item = e / ((long long)CL * A * L);
        const int jy = (int)(item / nch), ch = (int)(item % nch);
        const int my = jy < N / 2 ? jy : jy - N, mz = ch * CL + c;
        xw[e] = ballft[l * Q + a * a + my * my + mz * mz] * (deconv[a] * deconv[jy] * deconv[mz]);
    }
}

size_t xw_floats(const Geometry &g) { return (size_t)g.N * (g.N / 2 / CL) * g.L * (g.N / 2 + 1) * CL; }

cudaError_t launch_build_xw(const Geometry &g, const float *deconv, const float *ballft, float *xw, cudaStream_t s)
{
    k_build_xw<<<1024, 256, 0, s>>>(g.N, g.L, 3 * (g.N / 2) * (g.N / 2), deconv, ballft, xw);
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
// Knot j of instance i becomes ku = (u_x, u_y, u_z, level | i << 4) with
// u = (R c) n / P wrapped into [-n/2, n/2) (fine-grid cells; the period P spans
// n cells).  The spreading stencil of a knot covers cells g0 .. g0 + W - 1 per
// axis, g0 = ceil(u - W/2); the support box of the instance is the union of
// the stencils, accumulated with atomics into bb (lo[3], hi[3] per instance).
// Grid: (blocks over knots, instance).
constexpr int PREP_THREADS = 256;

// With plan != null the last block to finish (counted on bb[6], which the
// reset leaves at 0 and that block puts back) turns every instance's support
// box into its plan and resets the box accumulators (plan_instance); a box
// larger than the instance's capacity raises the error word and the instance
// is treated as empty.
__global__ void __launch_bounds__(PREP_THREADS)
k_prepare(Geometry g, const InstDesc *__restrict__ inst, int ninst, float4 *ku, int *bb, int *cnt, InstPlan *plan,
          int *err)
{
    pdl_signal(); // the spreading pass may be launched (it waits for this grid)
    const int i = blockIdx.y;
    const InstDesc d = inst[i];
    const int j = blockIdx.x * PREP_THREADS + threadIdx.x;
    if (blockIdx.x * PREP_THREADS < d.nknots) { // else the whole block is beyond this instance's knots
    float qw = d.q[0], qx = d.q[1], qy = d.q[2], qz = d.q[3];
    if (d.qdev) {
        qw = d.qdev[0];
        qx = d.qdev[1];
        qy = d.qdev[2];
        qz = d.qdev[3];
    }
    const float s = 1.0f / sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= s; qx *= s; qy *= s; qz *= s;
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    const float nf = (float)g.n, halfW = 0.5f * (float)g.W;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (j < d.nknots) {
        const float4 c = d.knots[d.src_off + j];
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
            const int g0 = (int)ceilf(v - halfW);
            lo[a] = g0;
            hi[a] = g0 + g.W - 1;
        }
        const int tag = __float_as_int(c.w) | (i << 4);
        ku[d.knot_off + j] = make_float4(u[0], u[1], u[2], __int_as_float(tag));
        if (cnt) { // knot count per (instance, level, first stencil cell along x mod n)
            const int gx = lo[0] < 0 ? lo[0] + g.n : lo[0];
            atomicAdd(&cnt[((long long)i * g.L + __float_as_int(c.w)) * g.n + gx], 1);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    __shared__ int red[6][PREP_THREADS / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int a = 0; a < 3; a++) {
            red[a][w] = lo[a];
            red[3 + a][w] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        int v = a < 3 ? INT_MAX : INT_MIN;
        for (int k = 0; k < PREP_THREADS / 32; k++) v = a < 3 ? min(v, red[a][k]) : max(v, red[a][k]);
        if (a < 3) atomicMin(&bb[8 * i + a], v);
        else atomicMax(&bb[8 * i + a], v);
    }
    } // this block's knots
    if (!plan) return;
    __shared__ int last;
    __threadfence(); // this block's box updates precede its count
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&bb[6], 1) == (int)(gridDim.x * gridDim.y) - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int k = threadIdx.x; k < ninst; k += PREP_THREADS) plan_instance(g, inst, k, bb, plan, err);
    if (threadIdx.x == 0) bb[6] = 0;
}

__global__ void k_reset_boxes(int *bb, int ninst)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 8 * ninst) bb[t] = (t & 7) < 3 ? INT_MAX : (t & 7) < 6 ? INT_MIN : 0; // slots 6, 7: counters
}

cudaError_t launch_reset_boxes(int *bb, int ninst, cudaStream_t s)
{
    if (ninst <= 0) return cudaSuccess;
    k_reset_boxes<<<(8 * ninst + 255) / 256, 256, 0, s>>>(bb, ninst);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const Geometry &g, const InstDesc *inst, int ninst, int max_knots, float4 *ku, int *bb,
                           InstPlan *plan, int *err, int *cnt, int *cur, cudaStream_t s)
{
    if (ninst <= 0) return cudaSuccess;
    const int bx = max_knots > 0 ? (max_knots + PREP_THREADS - 1) / PREP_THREADS : 1;
    // binned spreading plans (and scans its bin counts) in its own kernel
    k_prepare<<<dim3(bx, ninst), PREP_THREADS, 0, s>>>(g, inst, ninst, ku, bb, cnt, cnt ? nullptr : plan, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cnt) return launch_plan_bins(g, inst, ninst, bb, plan, err, cnt, cur, s);
    return cudaSuccess;
}

// ------------------------------------------------------------------ spread
// Spreading boxes are stored block-transposed: per (instance, level)
// [ix][iy / 32][iz][iy mod 32], so that the 32 rows of a z-transform tile are
// one contiguous 128-byte run per z position.
//
// One warp per knot.  Lanes 0..3W-1 evaluate the separable window weights
// phi(u_a - g) for the W cells of each axis; the W y-cells of a stencil column
// (dx, dz) are then added with 16-byte vector atomics on 4-aligned groups
// (zero weights fill the unused slots of the first and last group; a group
// never crosses a 32-row block).  For W <= 9 a column has at most three groups
// and the lanes take (column, group) tasks, three per column with dz fastest:
// the lanes of one vector atomic cover the groups of about ten consecutive
// columns, which are adjacent 128-byte runs, so each run is updated by one
// coalesced request.  Wider windows give each lane whole columns.  A column
// that wraps around the period (only when the box spans all n cells) uses
// scalar atomics.
constexpr int SPREAD_WARPS = 8;

__device__ __forceinline__ long long level_box_floats(const InstPlan &p)
{
    return (long long)p.b[0] * ((p.b[1] + 31) >> 5) * p.b[2] * 32;
}

__global__ void __launch_bounds__(SPREAD_WARPS * 32)
k_spread(Geometry g, const float *__restrict__ consts, const InstDesc *__restrict__ inst,
         const float4 *__restrict__ ku, const InstPlan *__restrict__ plan, float *grid, int total)
{
    __shared__ float wts[SPREAD_WARPS][3][16];
    __shared__ float4 wy4[SPREAD_WARPS][3];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = g.W, W2 = W * W;
    const float halfW = 0.5f * (float)W, invW = 1.0f / (float)W, xoff = 0.5f * (float)W - 1.f;
    // lane 0 .. 3W - 1 evaluates the weight of stencil offset t on axis a for every knot
    const int wa = lane / W, wt = lane - wa * W;
    float kc[KB_NC];
    kb_load(consts, lane < 3 * W ? wt : 0, kc);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    for (int k = blockIdx.x * SPREAD_WARPS + wib; k < total; k += gridDim.x * SPREAD_WARPS) {
        const float4 v = ku[k];
        const int tag = __float_as_int(v.w);
        const int level = tag & 15, i = tag >> 4;
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const float u0 = v.x, u1 = v.y, u2 = v.z;
        const int g0[3] = {(int)ceilf(u0 - halfW), (int)ceilf(u1 - halfW), (int)ceilf(u2 - halfW)};
        if (lane < 3 * W) {
            const float ua = wa == 0 ? u0 : (wa == 1 ? u1 : u2);
            const int ga = wa == 0 ? g0[0] : (wa == 1 ? g0[1] : g0[2]);
            wts[wib][wa][wt] = kb_poly(kc, (ua - (float)ga) - xoff);
        }
        __syncwarp();
        const int nyb = (p.b[1] + 31) >> 5, bz = p.b[2];
        float *G = grid + inst[i].grid_off + (long long)level * level_box_floats(p);
        const int iy0 = g0[1] - p.lo[1];
        const bool ywrap = iy0 + W - 1 >= g.n;
        if (!ywrap && W <= 9) {
            // per knot: the y-group weight vectors and the address of stencil cell
            // (0, 0, group); a column's x and z offsets then add linearly unless
            // the stencil crosses the end of a full-period box
            const int a0 = iy0 & ~3;
            const int ng = ((iy0 + W - 1) >> 2) - (iy0 >> 2) + 1; // groups per column, at most 3
            const int ix0 = g0[0] - p.lo[0], iz0 = g0[2] - p.lo[2];
            const bool xzwrap = ix0 + W - 1 >= g.n || iz0 + W - 1 >= g.n;
            if (lane < 3) {
                const int e0 = a0 + 4 * lane - iy0;
                float4 gv;
                gv.x = (e0 >= 0 && e0 < W) ? wts[wib][1][e0] : 0.f;
                gv.y = (e0 + 1 >= 0 && e0 + 1 < W) ? wts[wib][1][e0 + 1] : 0.f;
                gv.z = (e0 + 2 >= 0 && e0 + 2 < W) ? wts[wib][1][e0 + 2] : 0.f;
                gv.w = (e0 + 3 >= 0 && e0 + 3 < W) ? wts[wib][1][e0 + 3] : 0.f;
                wy4[wib][lane] = gv;
            }
            __syncwarp();
            const long long xstride = (long long)nyb * bz * 32;
            float *G0 = G + (long long)ix0 * xstride + (long long)iz0 * 32;
            for (int t = lane; t < 3 * W2; t += 32) {
                const int colm = t / 3, grp = t - 3 * colm;
                if (grp >= ng) continue;
                const int dx = __float2int_rz(((float)colm + 0.5f) * invW), dz = colm - dx * W;
                const int a = a0 + 4 * grp;
                const long long yoff = (long long)(a >> 5) * bz * 32 + (a & 31);
                float *cell;
                if (!xzwrap) {
                    cell = G0 + dx * xstride + dz * 32 + yoff;
                } else {
                    int ix = ix0 + dx, iz = iz0 + dz;
                    if (ix >= g.n) ix -= g.n;
                    if (iz >= g.n) iz -= g.n;
                    cell = G + (long long)ix * xstride + (long long)iz * 32 + yoff;
                }
                const float cw = wts[wib][0][dx] * wts[wib][2][dz];
                const float4 gv = wy4[wib][grp];
                atomicAdd(reinterpret_cast<float4 *>(cell), make_float4(cw * gv.x, cw * gv.y, cw * gv.z, cw * gv.w));
            }
            __syncwarp();
            continue;
        }
        for (int r = lane; r < W2; r += 32) {
            const int dx = r / W, dz = r - dx * W;
            int ix = g0[0] + dx - p.lo[0];
            int iz = g0[2] + dz - p.lo[2];
            if (ix >= g.n) ix -= g.n;
            if (iz >= g.n) iz -= g.n;
            const float cw = wts[wib][0][dx] * wts[wib][2][dz];
            float *col = G + ((long long)ix * nyb * bz + iz) * 32;
            if (!ywrap) {
                for (int a = iy0 & ~3; a <= iy0 + W - 1; a += 4) {
                    const int e0 = a - iy0;
                    float4 val;
                    val.x = (e0 >= 0 && e0 < W) ? cw * wts[wib][1][e0] : 0.f;
                    val.y = (e0 + 1 >= 0 && e0 + 1 < W) ? cw * wts[wib][1][e0 + 1] : 0.f;
                    val.z = (e0 + 2 >= 0 && e0 + 2 < W) ? cw * wts[wib][1][e0 + 2] : 0.f;
                    val.w = (e0 + 3 >= 0 && e0 + 3 < W) ? cw * wts[wib][1][e0 + 3] : 0.f;
                    atomicAdd(reinterpret_cast<float4 *>(col + (long long)(a >> 5) * bz * 32 + (a & 31)), val);
                }
            } else {
                for (int dy = 0; dy < W; dy++) {
                    int iy = iy0 + dy;
                    if (iy >= g.n) iy -= g.n;
                    atomicAdd(col + (long long)(iy >> 5) * bz * 32 + (iy & 31), cw * wts[wib][1][dy]);
                }
            }
        }
        __syncwarp();
    }
}

cudaError_t launch_spread(const Geometry &g, const Tables &t, const InstDesc *inst, int total_knots,
                          const float4 *ku, const InstPlan *plan, float *grid, int nsm, cudaStream_t s)
{
    if (total_knots <= 0) return cudaSuccess;
    (void)nsm; // one warp per knot: measured faster than resident-sized grid-stride loops
    int blocks = (total_knots + SPREAD_WARPS - 1) / SPREAD_WARPS;
    if (blocks > 65535) blocks = 65535;
    return launch_k(k_spread, blocks, SPREAD_WARPS * 32, 0, s, g.pdl != 0, g, t.consts, inst, ku, plan, grid,
                    total_knots);
}

// ------------------------------------------------------------------ fft z
// Item: 32 real rows (iy0 .. iy0+31) of one (level, ix) plane, packed as 16
// complex lines (row 2q in the real part, row 2q+1 in the imaginary part of
// line q): in the block-transposed box layout, line q at z position iz is one
// float2 of a contiguous 128-byte run.  Compact index iz sits at position
// (pos0_z + iz) mod n of the length-n line; the rest of the line is zero.  The
// first transform stage reads its inputs straight from the box (and the next
// item's inputs are loaded while the current one finishes); once every thread
// has consumed them the item's box rows (one contiguous run) are reset to zero
// so the boxes are clean for the next launch.
// Output rows: with Z = FFT(a + i b), A_k = (Z_k + conj Z_{n-k}) / 2,
// B_k = (Z_k - conj Z_{n-k}) / (2i), for m_z = k in [0, N/2).
template <int NF, bool SP, int S>
__global__ void __launch_bounds__(TB, (NF <= 256 ? 2 : 1))
k_fft_z(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
        float *grid, float2 *z1)
{
    constexpr bool three = Radix<NF, S>::r2 > 1;
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *S0 = tw + NF, *S1 = S0 + NF * CL;
    float2 *OUT = three ? S0 : S1; // tile the last stage writes (not the one it reads)
    float2 *STG = three ? S1 : S0; // staging for the output rows
    load_twiddles<NF>(tw, tb.tw_n);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int H = NF / 4; // kept z modes (N/2, n = 2N)
    const int L = g.L;
    FirstInputs<NF, Radix<NF, S>::r0, CL, TB> in;
    RotStart rs;
    for (int i = 0; i < ninst; i++) {
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const int b0 = p.b[0], b1 = p.b[1], bz = p.b[2], pz = p.pos0[2];
        const int nyb = (b1 + 31) >> 5;
        const int items = L * b0 * nyb;
        const InstDesc d = inst[i];
        float2 *G2 = reinterpret_cast<float2 *>(grid + d.grid_off);
        auto src = [&](int it) {
            float2 *base = G2 + (long long)it * bz * 16;
            return [=](int c, int pos) {
                int iz = pos - pz;
                if (iz < 0) iz += NF;
                return iz < bz ? base[iz * 16 + c] : make_float2(0.f, 0.f);
            };
        };
        int it = rs.first();
        if (it < items) in.load(src(it));
        for (; it < items; it += gridDim.x) {
            const int l = it / (b0 * nyb), rem = it - l * (b0 * nyb);
            const int ix = rem / nyb, iy0 = (rem - ix * nyb) << 5;
            if constexpr (SP) in.scatter(S0);
            else rr_first<NF, Radix<NF, S>::r0, false, CL, TB>(in, S0);
            __syncthreads(); // every thread has consumed its loads of this item
            {
                // the item's box rows are one contiguous run of bz x 128 bytes
                float4 *run = reinterpret_cast<float4 *>(G2 + (long long)it * bz * 16);
                for (int e = threadIdx.x; e < bz * 8; e += TB) run[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (it + (int)gridDim.x < items) in.load(src(it + gridDim.x));
            auto sink = [&](int, int, int c, int pos, float2 v) { OUT[pos * CL + c] = v; };
            if constexpr (SP) sp_all<NF, false, CL, TB, S>(S0, S1, tw, sink);
            else rr_rest<NF, false, CL, TB, S>(S0, S1, tw, sink);
            __syncthreads();
            // unpack into a staging area [row][k] (row stride H + 1), then write
            // each 8H-byte row of z1 with consecutive threads on consecutive k
            for (int e = threadIdx.x; e < 32 * H; e += TB) {
                const int r = e & 31, kk = e >> 5;
                const int qq = r >> 1;
                const float2 zk = OUT[kk * CL + qq];
                const float2 zn = OUT[(kk == 0 ? 0 : NF - kk) * CL + qq];
                STG[r * (H + 1) + kk] = (r & 1) ? make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x))
                                                : make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            }
            __syncthreads();
            float2 *Z = z1 + d.z1_off + (((long long)l * b0 + ix) * b1 + iy0) * H;
            const int rows = min(32, b1 - iy0);
            for (int e = threadIdx.x; e < rows * H; e += TB) {
                const int r = e / H, kk = e - r * H;
                Z[(long long)r * H + kk] = STG[r * (H + 1) + kk];
            }
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ fft y
// Item: (level, ix) plane and a chunk of 16 z-modes.  Row iy of the chunk (16
// complex = 128 bytes) is position (pos0_y + iy) mod n of the lines; the
// transform runs along y; m_y in (-N/2, N/2) is kept at FFT index j (j = N/2,
// m_y = -N/2, stored as zero).  Last-stage outputs go straight to y1.  With a
// two-stage radix schedule (FP32) the item's rows are fetched into one of two
// shared-memory staging tiles with asynchronous 16-byte copies (zero-filled
// outside the support box) one whole item ahead; otherwise first-stage inputs
// come straight from z1 into registers and the next item is loaded while the
// current one finishes.
template <int NF, bool SP, int S>
struct YStaged {
    static constexpr bool on = !SP && Radix<NF, S>::r2 == 1;
};

template <int NF, bool SP, int S>
__global__ void __launch_bounds__(TB, (NF <= 256 ? 2 : 1))
k_fft_y(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
        const float2 *__restrict__ z1, float2 *y1)
{
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *S0 = tw + NF, *S1 = S0 + NF * CL;
    load_twiddles<NF>(tw, tb.tw_n);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int H = NF / 4, N = NF / 2;
    const int L = g.L;
    constexpr int nch = H / CL;
    RotStart rs;
    if constexpr (YStaged<NF, SP, S>::on) {
        // staging tiles: B(0) = S1 (unused by a two-stage schedule) and B(1) after it
        auto B = [&](int k) { return S1 + k * (NF * CL); };
        for (int i = 0; i < ninst; i++) {
            const InstPlan p = plan[i];
            if (p.b[0] == 0) continue;
            const int b0 = p.b[0], b1 = p.b[1], py = p.pos0[1];
            const int items = L * b0 * nch;
            const InstDesc d = inst[i];
            // rows of item `it` into tile dst: 16-byte chunks (position, two lines)
            auto fetch = [&](int it, float2 *dst) {
                const int lx = it / nch, ch = it - lx * nch;
                const float2 *base = z1 + d.z1_off + (long long)lx * b1 * H + ch * CL;
                for (int q = threadIdx.x; q < NF * CL / 2; q += TB) {
                    const int pos = q / (CL / 2), cc = (q % (CL / 2)) * 2;
                    int iy = pos - py;
                    if (iy < 0) iy += NF;
                    const bool ok = iy < b1;
                    cp_async16(dst + pos * CL + cc, ok ? base + (long long)iy * H + cc : base, ok);
                }
            };
            int it = rs.first();
            if (it < items) fetch(it, B(0));
            cp_async_commit();
            for (int k = 0; it < items; it += gridDim.x, k ^= 1) {
                // B(k ^ 1) was last read by the first stage of the previous item
                if (it + (int)gridDim.x < items) fetch(it + gridDim.x, B(k ^ 1));
                cp_async_commit();
                cp_async_wait_prev();
                __syncthreads();
                il_stage<NF, Radix<NF, S>::r0, 1, false, CL, TB>(B(k), S0, tw);
                __syncthreads();
                const int lx = it / nch, ch = it - lx * nch;
                float2 *Y = y1 + d.y1_off + (long long)lx * N * H + ch * CL;
                auto sink = [&](int, int, int c, int pos, float2 v) {
                    int jy;
                    if (pos < N / 2) jy = pos;
                    else if (pos >= NF - N / 2) jy = pos - NF + N;
                    else return;
                    Y[(long long)jy * H + c] = jy == N / 2 ? make_float2(0.f, 0.f) : v;
                };
                rr_rest<NF, false, CL, TB, S>(S0, S1, tw, sink);
                __syncthreads();
            }
            rs.rot += items;
        }
    } else {
        FirstInputs<NF, Radix<NF, S>::r0, CL, TB> in;
        for (int i = 0; i < ninst; i++) {
            const InstPlan p = plan[i];
            if (p.b[0] == 0) continue;
            const int b0 = p.b[0], b1 = p.b[1], py = p.pos0[1];
            const int items = L * b0 * nch;
            const InstDesc d = inst[i];
            auto src = [&](int it) {
                const int lx = it / nch, ch = it - lx * nch;
                const float2 *base = z1 + d.z1_off + (long long)lx * b1 * H + ch * CL;
                return [=](int c, int pos) {
                    int iy = pos - py;
                    if (iy < 0) iy += NF;
                    return iy < b1 ? base[(long long)iy * H + c] : make_float2(0.f, 0.f);
                };
            };
            int it = rs.first();
            if (it < items) in.load(src(it));
            for (; it < items; it += gridDim.x) {
                const int lx = it / nch, ch = it - lx * nch;
                if constexpr (SP) in.scatter(S0);
                else rr_first<NF, Radix<NF, S>::r0, false, CL, TB>(in, S0);
                __syncthreads();
                if (it + (int)gridDim.x < items) in.load(src(it + gridDim.x));
                float2 *Y = y1 + d.y1_off + (long long)lx * N * H + ch * CL;
                auto sink = [&](int, int, int c, int pos, float2 v) {
                    int jy;
                    if (pos < N / 2) jy = pos;
                    else if (pos >= NF - N / 2) jy = pos - NF + N;
                    else return;
                    Y[(long long)jy * H + c] = jy == N / 2 ? make_float2(0.f, 0.f) : v;
                };
                if constexpr (SP) sp_all<NF, false, CL, TB, S>(S0, S1, tw, sink);
                else rr_rest<NF, false, CL, TB, S>(S0, S1, tw, sink);
                __syncthreads();
            }
            rs.rot += items;
        }
    }
}

// The y pass with each item's rows staged at positions 0 .. b1 - 1 (compact
// index iy at position iy, zero beyond), for launches whose instances all have
// y boxes of at most YShift::MAXR cells (known on the host from their
// capacities): the first stage reads only the RN inputs per butterfly that can
// be nonzero, the staging tiles are MAXR rows instead of n, and three blocks
// fit on an SM.  The box origin comes back as exp(-2 pi i m_y pos0_y / n) on
// every kept output.  Same transform as k_fft_y, other rounding order.
template <int NF, int S>
struct YShift {
    static constexpr int R0 = Radix<NF, S>::r0, NB = NF / R0;
    static constexpr int MAXR = NF <= 128 ? NF : ((9 * NF / 16 + NB - 1) / NB) * NB;
    static constexpr bool on = Radix<NF, S>::r2 == 1 && NF <= 256;
    static constexpr size_t smem = sizeof(float2) * ((size_t)NF + (size_t)NF * CL + 2 * (size_t)MAXR * CL);
};

// First stage from a staging tile of YShift<NF, S>::MAXR rows.
template <int NF, int S>
__device__ __forceinline__ void ys_first(const float2 *__restrict__ stg, float2 *__restrict__ out)
{
    using YS = YShift<NF, S>;
    constexpr int R = YS::R0, NB = YS::NB, RN = YS::MAXR / NB, TOT = NB * CL, IT = (TOT + TB - 1) / TB;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = (int)threadIdx.x + it * TB;
        if ((TOT % TB) != 0 && idx >= TOT) break;
        const int c = idx % CL, j = idx / CL;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = r < RN ? stg[(j + r * NB) * CL + c] : make_float2(0.f, 0.f);
        dft_small<R, false>(v);
#pragma unroll
        for (int r = 0; r < R; r++) out[(j * R + r) * CL + c] = v[r];
    }
}

template <int NF, int S>
__global__ void __launch_bounds__(TB, 3)
k_fft_y_shift(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
              const float2 *__restrict__ z1, float2 *y1)
{
    using YS = YShift<NF, S>;
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *S0 = tw + NF;
    float2 *T0 = S0 + NF * CL, *T1 = T0 + YS::MAXR * CL; // staging tiles
    load_twiddles<NF>(tw, tb.tw_n);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int H = NF / 4, N = NF / 2;
    constexpr int nch = H / CL;
    const int L = g.L;
    RotStart rs;
    for (int i = 0; i < ninst; i++) {
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const int b0 = p.b[0], b1 = p.b[1], py = p.pos0[1];
        const int items = L * b0 * nch;
        const InstDesc d = inst[i];
        auto fetch = [&](int it, float2 *dst) {
            const int lx = it / nch, ch = it - lx * nch;
            const float2 *base = z1 + d.z1_off + (long long)lx * b1 * H + ch * CL;
            for (int q = threadIdx.x; q < YS::MAXR * (CL / 2); q += TB) {
                const int row = q / (CL / 2), cc = (q % (CL / 2)) * 2;
                const bool ok = row < b1;
                cp_async16(dst + row * CL + cc, ok ? base + (long long)row * H + cc : base, ok);
            }
        };
        int it = rs.first();
        if (it < items) fetch(it, T0);
        cp_async_commit();
        for (int k = 0; it < items; it += gridDim.x, k ^= 1) {
            // the other tile was last read by the previous item's first stage
            if (it + (int)gridDim.x < items) fetch(it + gridDim.x, k ? T0 : T1);
            cp_async_commit();
            cp_async_wait_prev();
            __syncthreads();
            ys_first<NF, S>(k ? T1 : T0, S0);
            __syncthreads();
            const int lx = it / nch, ch = it - lx * nch;
            float2 *Y = y1 + d.y1_off + (long long)lx * N * H + ch * CL;
            auto sink = [&](int, int, int c, int pos, float2 v) {
                int jy, my;
                if (pos < N / 2) jy = my = pos;
                else if (pos >= NF - N / 2) {
                    jy = pos - NF + N;
                    my = pos - NF;
                } else return;
                Y[(long long)jy * H + c] = jy == N / 2 ? make_float2(0.f, 0.f) : cmul(v, box_phase<NF>(tw, my, py));
            };
            rr_rest<NF, false, CL, TB, S>(S0, nullptr, tw, sink);
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ fft x + combine
// Every (j_y, chunk of 16 z-modes) item of every pair through x_item
// (bc_passes.cuh): forward x transform of both spectra with the level sum,
// conjugate product and inverse x transform.
template <int NF, int NI, bool SP, int S>
__global__ void __launch_bounds__(TB, (NF <= 256 ? 2 : 1))
k_fft_x(Geometry g, Tables tb, const InstDesc *__restrict__ inst, const InstPlan *__restrict__ plan,
        const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ y1,
        const float2 *__restrict__ fa_cache, float2 *fa_out, float2 *h, int G)
{
    extern __shared__ float4 sm4[];
    using XL = XSmem<NF, NI, SP, S>;
    const typename XL::Ptr sm = XL::carve(reinterpret_cast<float2 *>(sm4));
    load_twiddles<NF>(sm.twF, tb.tw_n);
    load_twiddles<NI>(sm.twI, tb.tw_N);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int nch = NI / 2 / CL;
    const int items = NI * nch;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int jy = it / nch, ch = it - jy * nch;
            x_item<NF, NI, SP, S>(g, tb, inst, plan, pr, jy, ch, y1, fa_cache, fa_out, h, G, sm);
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ inverse y
// Item: (k_x, chunk of 16 z-modes); in place on the half-spectrum planes: the
// first stage reads the item's rows into registers, the last stage writes them
// back; the next item is loaded while the current one finishes.
template <int NI>
__global__ void __launch_bounds__(TB, 2)
k_ifft_y(Geometry g, Tables tb, const PairDesc *__restrict__ pairs, int npairs, float2 *h)
{
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *S0 = tw + NI, *S1 = S0 + NI * CL;
    load_twiddles<NI>(tw, tb.tw_N);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int H = NI / 2, N = NI;
    constexpr int nch = H / CL;
    const int items = N * nch;
    FirstInputs<NI, Radix<NI>::r0, CL, TB> in;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        if (pr.b < 0) continue;
        auto base_of = [&](int it) {
            const int kx = it / nch, ch = it - kx * nch;
            return h + pr.h_off + (long long)kx * N * H + ch * CL;
        };
        auto src = [&](int it) {
            const float2 *base = base_of(it);
            return [=](int c, int pos) { return base[(long long)pos * H + c]; };
        };
        int it = rs.first();
        if (it < items) in.load(src(it));
        for (; it < items; it += gridDim.x) {
            rr_first<NI, Radix<NI>::r0, true, CL, TB>(in, S0);
            __syncthreads();
            if (it + (int)gridDim.x < items) in.load(src(it + gridDim.x));
            float2 *Hp = base_of(it);
            rr_rest<NI, true, CL, TB>(S0, S1, tw, [&](int, int, int c, int pos, float2 v) { Hp[(long long)pos * H + c] = v; });
            __syncthreads();
        }
        rs.rot += items;
    }
}

__global__ void k_decode_peaks(const unsigned long long *__restrict__ keys, int n, float *peak, int *argmax)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long key = keys[i];
    unsigned u = (unsigned)(key >> 32);
    u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    peak[i] = __uint_as_float(u);
    argmax[i] = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
}

cudaError_t launch_decode_peaks(const unsigned long long *keys, int n, float *peak, int *argmax, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_decode_peaks<<<(n + 255) / 256, 256, 0, s>>>(keys, n, peak, argmax);
    return cudaGetLastError();
}

// Item: 32 output rows (k_x, k_y0 .. k_y0+31) as 16 complex lines; lane l of a
// warp owns row k_y0 + l.  Rows a = 2q and b = 2q+1 of the half spectrum are
// packed as Z_k = A_k + i B_k over the full range (A_{N-k} = conj A_k, A_0
// taken real, the m_z = N/2 term zero); the inverse transform of Z is a + i b.
// The even lane of each pair writes Z_k, the odd lane Z_{N-k}.  With `keys`,
// the item's largest value (lowest index on ties) is folded into the pair's
// peak key with one 64-bit atomic max; with `out` null no grid is written.
template <int NI>
__global__ void __launch_bounds__(TB)
k_ifft_z(Geometry g, Tables tb, const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ h,
         float *out, unsigned long long *keys)
{
    __shared__ unsigned long long red[TB / 32];
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *A = tw + NI, *B = A + NI * CL;
    load_twiddles<NI>(tw, tb.tw_N);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    constexpr int H = NI / 2, N = NI;
    const int nyb = N / 32;
    const int items = N * nyb;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 1, odd = lane & 1;
    RotStart rs;
    for (int pi = 0; pi < npairs; pi++) {
        const PairDesc pr = pairs[pi];
        if (pr.b < 0) continue;
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int kx = it / nyb, ky0 = (it - kx * nyb) << 5;
            const float2 *row = h + pr.h_off + ((long long)kx * N + ky0 + lane) * H;
            if (threadIdx.x < CL) A[H * CL + threadIdx.x] = make_float2(0.f, 0.f); // m_z = N/2
            for (int k = 2 * w; k < H; k += 2 * (TB / 32)) {
                const float4 v = *reinterpret_cast<const float4 *>(row + k);
                const float4 o = make_float4(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1),
                                             __shfl_xor_sync(0xffffffffu, v.z, 1), __shfl_xor_sync(0xffffffffu, v.w, 1));
                const float4 a = odd ? o : v, b = odd ? v : o; // rows 2q and 2q+1 at modes k, k+1
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const float ax = u ? a.z : a.x, ay = u ? a.w : a.y, bx = u ? b.z : b.x, by = u ? b.w : b.y;
                    const int kk = k + u;
                    if (!odd) {
                        A[kk * CL + q] = kk == 0 ? make_float2(ax, bx) : make_float2(ax - by, ay + bx);
                    } else if (kk != 0) {
                        A[(N - kk) * CL + q] = make_float2(ax + by, bx - ay);
                    }
                }
            }
            __syncthreads();
            const float2 *res = il_fft<NI, true, CL, TB>(A, B, tw);
            // rows through a staging area [row][kz ^ row] (XOR swizzle: conflict-free
            // in both phases), then each 4N-byte output row written coalesced
            float *S = reinterpret_cast<float *>((res == A) ? B : A);
            for (int e = threadIdx.x; e < 32 * N; e += TB) {
                const int r = e & 31, kz = e >> 5;
                const float2 v = res[kz * CL + (r >> 1)];
                S[r * N + (kz ^ r)] = (r & 1) ? v.y : v.x;
            }
            __syncthreads();
            float *o = out ? out + pr.out_off + ((long long)kx * N + ky0) * N : nullptr;
            unsigned long long best = 0ull;
            for (int e = threadIdx.x; e < 32 * N; e += TB) {
                const int r = e / N, kz = e - r * N;
                const float v = S[r * N + (kz ^ r)];
                if (o) o[(long long)r * N + kz] = v;
                if (keys) {
                    const unsigned long long kk = peak_key(v, (unsigned)(((long long)kx * N + ky0 + r) * N + kz));
                    best = kk > best ? kk : best;
                }
            }
            if (keys) {
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, off);
                    best = other > best ? other : best;
                }
                if (lane == 0) red[w] = best;
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int i2 = 1; i2 < TB / 32; i2++) best = red[i2] > best ? red[i2] : best;
                    atomicMax(keys + pr.key, best);
                }
            }
            __syncthreads();
        }
        rs.rot += items;
    }
}

// ------------------------------------------------------------------ inverse y and z of whole planes
// One block per plane k_x of a pair (for batches of many pairs): the plane's
// N x N/2 half-spectrum values (one contiguous run in h) are copied into
// shared memory chunk-major ([chunk of 16 z-modes][k_y][16]), transformed along
// y chunk by chunk in place, and then along z as k_ifft_z does, 32 output rows
// at a time, from shared memory.  Same arithmetic as k_ifft_y followed by
// k_ifft_z; the plane never goes back to HBM between the two transforms.
template <int NI>
__global__ void __launch_bounds__(TB, 2)
k_ifft_yz(Geometry g, Tables tb, const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ h,
          float *out, unsigned long long *keys)
{
    __shared__ unsigned long long red[TB / 32];
    extern __shared__ float4 sm4[];
    constexpr int H = NI / 2, N = NI, nch = H / CL, nyb = N / 32;
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *P = tw + NI;           // [nch][N][CL]
    float2 *A = P + N * H;         // [N + 1][CL] scratch tiles
    float2 *B = A + NI * CL;
    load_twiddles<NI>(tw, tb.tw_N);
    pdl_signal();
    pdl_wait(); // earlier passes' outputs are read from here on
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 1, odd = lane & 1;
    const int units = npairs * N;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int pi = u / N, kx = u - pi * N;
        const PairDesc pr = pairs[pi];
        if (pr.b < 0) continue; // uniform per pair
        const float2 *src = h + pr.h_off + (long long)kx * N * H;
        for (int e = threadIdx.x; e < N * H / 2; e += TB) { // 16-byte pieces: row ky, modes 2e' .. 2e' + 1
            const int ky = e / (H / 2), m2 = (e - ky * (H / 2)) * 2;
            cp_async16(P + ((m2 / CL) * N + ky) * CL + (m2 % CL), src + (long long)ky * H + m2, true);
        }
        cp_async_commit();
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        for (int ch = 0; ch < nch; ch++) {
            float2 *T = P + ch * N * CL;
            const float2 *res = il_fft<NI, true, CL, TB>(T, A, tw);
            if (res != T) {
                for (int e = threadIdx.x; e < N * CL; e += TB) T[e] = res[e];
                __syncthreads();
            }
        }
        for (int kb = 0; kb < nyb; kb++) {
            const int ky0 = kb * 32;
            if (threadIdx.x < CL) A[H * CL + threadIdx.x] = make_float2(0.f, 0.f); // m_z = N/2
            for (int k = 2 * w; k < H; k += 2 * (TB / 32)) {
                // modes k, k + 1 of row ky0 + lane (both in the chunk of k: k is even and CL is even)
                const float2 *pr2 = P + ((k / CL) * N + ky0 + lane) * CL + (k % CL);
                const float4 v = *reinterpret_cast<const float4 *>(pr2);
                const float4 o = make_float4(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1),
                                             __shfl_xor_sync(0xffffffffu, v.z, 1), __shfl_xor_sync(0xffffffffu, v.w, 1));
                const float4 a = odd ? o : v, b = odd ? v : o; // rows 2q and 2q+1 at modes k, k+1
#pragma unroll
                for (int uu = 0; uu < 2; uu++) {
                    const float ax = uu ? a.z : a.x, ay = uu ? a.w : a.y, bx = uu ? b.z : b.x, by = uu ? b.w : b.y;
                    const int kk = k + uu;
                    if (!odd) {
                        A[kk * CL + q] = kk == 0 ? make_float2(ax, bx) : make_float2(ax - by, ay + bx);
                    } else if (kk != 0) {
                        A[(N - kk) * CL + q] = make_float2(ax + by, bx - ay);
                    }
                }
            }
            __syncthreads();
            const float2 *res = il_fft<NI, true, CL, TB>(A, B, tw);
            float *S = reinterpret_cast<float *>((res == A) ? B : A);
            for (int e = threadIdx.x; e < 32 * N; e += TB) {
                const int r = e & 31, kz = e >> 5;
                const float2 v = res[kz * CL + (r >> 1)];
                S[r * N + (kz ^ r)] = (r & 1) ? v.y : v.x;
            }
            __syncthreads();
            float *o = out ? out + pr.out_off + ((long long)kx * N + ky0) * N : nullptr;
            unsigned long long best = 0ull;
            for (int e = threadIdx.x; e < 32 * N; e += TB) {
                const int r = e / N, kz = e - r * N;
                const float v = S[r * N + (kz ^ r)];
                if (o) o[(long long)r * N + kz] = v;
                if (keys) {
                    const unsigned long long kk = peak_key(v, (unsigned)(((long long)kx * N + ky0 + r) * N + kz));
                    best = kk > best ? kk : best;
                }
            }
            if (keys) {
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, off);
                    best = other > best ? other : best;
                }
                if (lane == 0) red[w] = best;
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int i2 = 1; i2 < TB / 32; i2++) best = red[i2] > best ? red[i2] : best;
                    atomicMax(keys + pr.key, best);
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ launchers
template <int NF, bool SP = false, int S = 0>
static cudaError_t fft_z_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                           float *grid, float2 *z1, int nsm, cudaStream_t s)
{
    if (!SP && S == 0 && (g.sched & 1)) return fft_z_t<NF, false, 1>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    const size_t smem = sizeof(float2) * (NF + 2 * NF * CL);
    cudaError_t e = set_smem(k_fft_z<NF, SP, S>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_fft_z<NF, SP, S>, resident_blocks(k_fft_z<NF, SP, S>, smem, nsm), TB, smem, s, g.pdl != 0, g, t,
                    inst, ninst, plan, grid, z1);
}

cudaError_t launch_fft_z(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                         float *grid, float2 *z1, int nsm, cudaStream_t s)
{
    if (g.prec == 1) {
        switch (g.n) {
        case 64: return fft_z_t<64, true>(g, t, inst, ninst, plan, grid, z1, nsm, s);
        case 128: return fft_z_t<128, true>(g, t, inst, ninst, plan, grid, z1, nsm, s);
        case 192: return fft_z_t<192, true>(g, t, inst, ninst, plan, grid, z1, nsm, s);
        case 256: return fft_z_t<256, true, SplitSched<256>::S>(g, t, inst, ninst, plan, grid, z1, nsm, s);
        case 512: return fft_z_t<512, true>(g, t, inst, ninst, plan, grid, z1, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (g.n) {
    case 64: return fft_z_t<64>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 128: return fft_z_t<128>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 192: return fft_z_t<192>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 256: return fft_z_t<256>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    case 512: return fft_z_t<512>(g, t, inst, ninst, plan, grid, z1, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NF, bool SP = false, int S = 0>
static cudaError_t fft_y_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                           const float2 *z1, float2 *y1, int max_cap, int nsm, cudaStream_t s)
{
    if (!SP && S == 0 && (g.sched & 2)) return fft_y_t<NF, false, 1>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    if constexpr (!SP && YShift<NF, S>::on) {
        if (max_cap <= YShift<NF, S>::MAXR) {
            const size_t smem = YShift<NF, S>::smem;
            cudaError_t e = set_smem(k_fft_y_shift<NF, S>, smem);
            if (e != cudaSuccess) return e;
            return launch_k(k_fft_y_shift<NF, S>, resident_blocks(k_fft_y_shift<NF, S>, smem, nsm), TB, smem, s,
                            g.pdl != 0, g, t, inst, ninst, plan, z1, y1);
        }
    }
    const size_t smem = sizeof(float2) * (NF + (YStaged<NF, SP, S>::on ? 3 : 2) * NF * CL);
    cudaError_t e = set_smem(k_fft_y<NF, SP, S>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_fft_y<NF, SP, S>, resident_blocks(k_fft_y<NF, SP, S>, smem, nsm), TB, smem, s, g.pdl != 0, g, t,
                    inst, ninst, plan, z1, y1);
}

cudaError_t launch_fft_y(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst, const InstPlan *plan,
                         const float2 *z1, float2 *y1, int max_cap, int nsm, cudaStream_t s)
{
    if (g.prec == 1) {
        switch (g.n) {
        case 64: return fft_y_t<64, true>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
        case 128: return fft_y_t<128, true>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
        case 192: return fft_y_t<192, true>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
        case 256: return fft_y_t<256, true, SplitSched<256>::S>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
        case 512: return fft_y_t<512, true>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (g.n) {
    case 64: return fft_y_t<64>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    case 128: return fft_y_t<128>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    case 192: return fft_y_t<192>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    case 256: return fft_y_t<256>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    case 512: return fft_y_t<512>(g, t, inst, ninst, plan, z1, y1, max_cap, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NF, int NI, bool SP = false, int S = 0>
static cudaError_t fft_x_t(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                           const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *fa_out,
                           float2 *h, int nsm, cudaStream_t s)
{
    if (!SP && S == 0 && (g.sched & 4))
        return fft_x_t<NF, NI, false, 1>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
    // level weights for as many levels as fit beside the tiles at the kernel's
    // blocks per SM (two up to NF = 256, else one): all of them in the usual cases
    using XL = XSmem<NF, NI, SP, S>;
    const size_t room = (NF <= 256 ? 228 * 1024 / 2 : 228 * 1024) - 1024 - XL::bytes(0);
    const int G = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.L, room / XL::per_level));
    const size_t smem = XL::bytes(G);
    cudaError_t e = set_smem(k_fft_x<NF, NI, SP, S>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_fft_x<NF, NI, SP, S>, resident_blocks(k_fft_x<NF, NI, SP, S>, smem, nsm), TB, smem, s,
                    g.pdl != 0, g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, G);
}

cudaError_t launch_fft_x(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                         const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *fa_out,
                         float2 *h, int nsm, cudaStream_t s)
{
    if (g.prec == 1) {
        switch (g.N) {
        case 32: return fft_x_t<64, 32, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
        case 64: return fft_x_t<128, 64, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
        case 96: return fft_x_t<192, 96, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
        case 128:
            return fft_x_t<256, 128, true, SplitSched<256>::S>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out,
                                                                h, nsm, s);
        case 256: return fft_x_t<512, 256, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, fa_out, h, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    }
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
    const size_t smem = sizeof(float2) * (NI + 2 * NI * CL);
    cudaError_t e = set_smem(k_ifft_y<NI>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_ifft_y<NI>, resident_blocks(k_ifft_y<NI>, smem, nsm), TB, smem, s, g.pdl != 0, g, t, pairs,
                    npairs, h);
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
static cudaError_t ifft_yz_t(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                             float *out, unsigned long long *keys, int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NI + (size_t)NI * (NI / 2) + 2 * (size_t)NI * CL);
    cudaError_t e = set_smem(k_ifft_yz<NI>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_ifft_yz<NI>, resident_blocks(k_ifft_yz<NI>, smem, nsm), TB, smem, s, g.pdl != 0, g, t, pairs,
                    npairs, h, out, keys);
}

cudaError_t launch_ifft_yz(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                           float *out, unsigned long long *keys, int nsm, cudaStream_t s)
{
    switch (g.N) {
    case 32: return ifft_yz_t<32>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 64: return ifft_yz_t<64>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 96: return ifft_yz_t<96>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 128: return ifft_yz_t<128>(g, t, pairs, npairs, h, out, keys, nsm, s);
    default: return cudaErrorInvalidValue; // N = 256: a plane (256 KB) exceeds shared memory
    }
}

template <int NI>
static cudaError_t ifft_z_t(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                            float *out, unsigned long long *keys, int nsm, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (NI + 2 * NI * CL);
    cudaError_t e = set_smem(k_ifft_z<NI>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_ifft_z<NI>, resident_blocks(k_ifft_z<NI>, smem, nsm), TB, smem, s, g.pdl != 0, g, t, pairs,
                    npairs, h, out, keys);
}

cudaError_t launch_ifft_z(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                          float *out, unsigned long long *keys, int nsm, cudaStream_t s)
{
    switch (g.N) {
    case 32: return ifft_z_t<32>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 64: return ifft_z_t<64>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 96: return ifft_z_t<96>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 128: return ifft_z_t<128>(g, t, pairs, npairs, h, out, keys, nsm, s);
    case 256: return ifft_z_t<256>(g, t, pairs, npairs, h, out, keys, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
