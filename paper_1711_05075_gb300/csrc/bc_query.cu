// Single-configuration queries (Sec. 4.1, Eq. (single)): the correlation at
// arbitrary translations from a truncated set of modes of its spectrum,
//     g(R, t) = P^-3 sum_{m in M'} w_m Re( g^(m) exp(2 pi i m.t / P) ),
// with g^(m) = f^_A(m) conj(f^_RB(m)) (Eq. (ccghat)), M' the first m' modes of
// the canonical half space ordered outward from the origin, and w_m = 1 for
// m = 0, 2 otherwise (each mode stands for itself and its conjugate -m).
#include <cstdint>

#include "bc_device.cuh"

namespace bc {

// g^ at the listed modes from two half spectra F[jx][jy][mz] (jx, jy in FFT
// order, mz in [0, N/2)); mode i = (m_x, m_y, m_z, w).
__global__ void k_query_gather(const float2 *__restrict__ fa, const float2 *__restrict__ fb, const int4 *__restrict__ modes,
                               int count, int N, float2 *ghat)
{
    const int H = N / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int4 m = modes[i];
        const int jx = m.x < 0 ? m.x + N : m.x, jy = m.y < 0 ? m.y + N : m.y;
        const long long o = ((long long)jx * N + jy) * H + m.z;
        const float2 a = fa[o], b = fb[o];
        ghat[i] = cmulc(a, b);
    }
}

cudaError_t launch_query_gather(const float2 *fa, const float2 *fb, const int4 *modes, int count, int N, float2 *ghat,
                                cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    int blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_query_gather<<<blocks, 256, 0, s>>>(fa, fb, modes, count, N, ghat);
    return cudaGetLastError();
}

// One block per query point.  The block first tabulates exp(2 pi i k t_a / P)
// for k in (-N/2, N/2) on each axis: the argument k t_a / P is formed and
// reduced to [-1/2, 1/2] in FP64, then sincospi runs in FP32 on the reduced
// value (|error| ~ 1e-7, independent of k and t).  Each thread then sums its
// share of the modes, w Re(g^ E_x E_y E_z), and the block reduces.
constexpr int QUERY_THREADS = 256;

__global__ void __launch_bounds__(QUERY_THREADS)
k_query_eval(const float2 *__restrict__ ghat, const int4 *__restrict__ modes, int count, int N, double inv_period,
             float scale, const float *__restrict__ t, int npts, float *g)
{
    extern __shared__ float2 E[]; // [3][N], index k + N/2
    __shared__ float red[QUERY_THREADS / 32];
    const int half = N / 2;
    for (int p = blockIdx.x; p < npts; p += gridDim.x) {
        for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
            const int a = e / N, k = e - a * N - half;
            const double x = (double)k * (double)t[3 * p + a] * inv_period;
            const float r = (float)(x - rint(x));
            float sn, cs;
            sincospif(2.0f * r, &sn, &cs);
            E[e] = make_float2(cs, sn);
        }
        __syncthreads();
        float acc = 0.f;
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            const int4 m = modes[i];
            const float2 ph = cmul(cmul(E[m.x + half], E[N + m.y + half]), E[2 * N + m.z + half]);
            const float2 v = ghat[i];
            acc = fmaf((float)m.w, fmaf(v.x, ph.x, -v.y * ph.y), acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int w = 0; w < QUERY_THREADS / 32; w++) s += red[w];
            g[p] = s * scale;
        }
        __syncthreads();
    }
}

cudaError_t launch_query_eval(const float2 *ghat, const int4 *modes, int count, int N, double period, const float *t,
                              int npts, float *g, cudaStream_t s)
{
    if (npts <= 0) return cudaSuccess;
    const int blocks = npts < 65535 ? npts : 65535;
    const float scale = (float)(1.0 / (period * period * period));
    k_query_eval<<<blocks, QUERY_THREADS, sizeof(float2) * 3 * N, s>>>(ghat, modes, count, N, 1.0 / period, scale, t,
                                                                        npts, g);
    return cudaGetLastError();
}

} // namespace bc
