// Learned rotation proposal: a three-layer perceptron that maps a rotation and
// low-order Fourier-moment magnitudes of the two shapes to a predicted
// correlation peak, so that only the best-ranked rotations get full
// correlations.  The paper has no counterpart; the network follows the usual
// definitions (ReLU layers, mean squared error, Adam with bias correction --
// Kingma & Ba, 2015).
//
//   x  = [q (unit, w >= 0); f_A[0..63]; f_B[0..63]]          (132 features)
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3
//
// Precision: FP32 master weights and Adam moments; every product reads its
// operands rounded to BF16 (weights, inputs, hidden activations, hidden
// gradients) and accumulates in FP32 on the tensor cores (mma.sync m16n8k16
// BF16 -> FP32).  All reductions run in a fixed order, so training is
// deterministic for a fixed launch configuration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/ballcorr.h"
#include "bc_internal.h"

using namespace bc;

namespace {

constexpr int KIN = BC_MLP_IN;   // 132 input features
constexpr int KPAD = 144;        // padded to a multiple of 16 for the tensor-core K steps

struct Offsets {
    long long W1, b1, W2, b2, w3, b3, total;
};

Offsets offsets(int H)
{
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (long long)H * KIN;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (long long)H * H;
    o.w3 = o.b2 + H;
    o.b3 = o.w3 + H;
    o.total = o.b3 + 1;
    return o;
}

// ------------------------------------------------------------------ BF16 GEMM
// C[m][n] = sum_k A[m][k] B[k][n] (+ bias[n]) (relu), operands FP32 in global
// memory addressed through strides and rounded to BF16 when staged in shared
// memory; FP32 accumulation.  Block: 4 warps, tile 64 x 64, K step 32; each
// warp owns 32 x 32 as 2 x 4 mma tiles of 16 x 8.
struct GemmArgs {
    const float *A;
    long long sAm, sAk;
    const float *B;
    long long sBk, sBn;
    float *C;
    long long sCm, sCn;
    int M, N, K;
    const float *bias;
    int relu;
    int kchunk = 0;     // split K: slice z of the grid sums k in [z kchunk, (z + 1) kchunk) (0: all of K)
    long long sCz = 0;  // and writes its partial product at C + z sCz
};

constexpr int GT = 64, GK = 32, GKP = GK + 8; // smem row pitch in bf16 (80 bytes)

__device__ __forceinline__ unsigned pack2(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[GT][GKP]; // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[GT][GKP]; // [n][k]
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[i][j][r] = 0.f;

    const int kb = g.kchunk ? (int)blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    for (int k0 = kb; k0 < ke; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 128) {
            const int r = e / GK, kk = e - r * GK;
            const int m = m0 + r, n = n0 + r, k = k0 + kk;
            const float a = (m < g.M && k < ke) ? g.A[m * g.sAm + k * g.sAk] : 0.f;
            const float b = (n < g.N && k < ke) ? g.B[k * g.sBk + n * g.sBn] : 0.f;
            As[r][kk] = __float2bfloat16_rn(a);
            Bs[r][kk] = __float2bfloat16_rn(b);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = wm * 32 + i * 16 + gid;
                af[i][0] = pack2(&As[r][ks + 2 * tig]);
                af[i][1] = pack2(&As[r + 8][ks + 2 * tig]);
                af[i][2] = pack2(&As[r][ks + 2 * tig + 8]);
                af[i][3] = pack2(&As[r + 8][ks + 2 * tig + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = wn * 32 + j * 8 + gid;
                bfr[j][0] = pack2(&Bs[c][ks + 2 * tig]);
                bfr[j][1] = pack2(&Bs[c][ks + 2 * tig + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                                 : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                                 : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                                   "r"(bfr[j][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int m = m0 + wm * 32 + i * 16 + gid + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * tig + (r & 1);
                if (m < g.M && n < g.N) {
                    float v = acc[i][j][r];
                    if (g.bias) v += g.bias[n];
                    if (g.relu) v = fmaxf(v, 0.f);
                    g.C[blockIdx.z * g.sCz + m * g.sCm + n * g.sCn] = v;
                }
            }
}

cudaError_t gemm(const GemmArgs &a, cudaStream_t s)
{
    dim3 grid((a.N + GT - 1) / GT, (a.M + GT - 1) / GT);
    k_gemm_bf16<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// out[m][n] = sum_z part[z][m][n], z in increasing order (M x N dense partials)
__global__ void k_sum_partials(const float *__restrict__ part, int nz, int M, int N, float *out, long long sOm)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)M * N) return;
    float s = 0.f;
    for (int z = 0; z < nz; z++) s += part[z * (long long)M * N + e];
    out[(e / N) * sOm + e % N] = s;
}

// A weight gradient C = A B with a long K (the batch): K split into slices whose
// partial products land in `part` and are then summed in a fixed order, so the
// result does not depend on scheduling.  C is M x N with row stride sCm.
cudaError_t gemm_splitk(GemmArgs a, float *part, long long part_floats, cudaStream_t s)
{
    const int tiles = ((a.N + GT - 1) / GT) * ((a.M + GT - 1) / GT);
    int nz = std::max(1, std::min(32, 256 / std::max(tiles, 1)));
    nz = (int)std::min<long long>(nz, std::max(1LL, part_floats / ((long long)a.M * a.N)));
    nz = std::min(nz, (a.K + GK - 1) / GK);
    const int kchunk = ((a.K + nz - 1) / nz + GK - 1) / GK * GK;
    nz = (a.K + kchunk - 1) / kchunk;
    float *C = a.C;
    const long long sCm = a.sCm;
    a.C = part;
    a.sCm = a.N;
    a.sCn = 1;
    a.kchunk = kchunk;
    a.sCz = (long long)a.M * a.N;
    dim3 grid((a.N + GT - 1) / GT, (a.M + GT - 1) / GT, nz);
    k_gemm_bf16<<<grid, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long tot = (long long)a.M * a.N;
    k_sum_partials<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nz, a.M, a.N, C, sCm);
    return cudaGetLastError();
}

__device__ __forceinline__ float rbf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// y[b] = sum_j bf16(h2[b][j]) bf16(w3[j]) + b3 (one warp per row, fixed order)
__global__ void k_head(const float *__restrict__ h2, const float *__restrict__ w3, const float *__restrict__ b3, int n,
                       int H, float *y)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    float s = 0.f;
    for (int j = lane; j < H; j += 32) s = fmaf(rbf(h2[(long long)row * H + j]), rbf(w3[j]), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + b3[0];
}

// gy[b] = 2 (y[b] - t[b]) / n; dh2[b][j] = bf16(gy[b] bf16(w3[j])) if h2[b][j] > 0 else 0
__global__ void k_head_back(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ h2,
                            const float *__restrict__ w3, int n, int H, float *gy, float *dh2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * H) return;
    const int b = (int)(e / H), j = (int)(e - (long long)b * H);
    const float g = 2.f * (y[b] - t[b]) / (float)n;
    if (j == 0) gy[b] = g;
    dh2[e] = h2[e] > 0.f ? rbf(g * rbf(w3[j])) : 0.f;
}

// dh1 <- bf16(dh1) where h1 > 0, else 0 (in place)
__global__ void k_relu_back(float *dh, const float *__restrict__ h, long long total)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) dh[e] = h[e] > 0.f ? rbf(dh[e]) : 0.f;
}

// Column sums over the batch in two fixed-order stages: block c sums rows
// [c CS, (c + 1) CS) of every column into part[c][j], then the chunks are
// summed in order.  Terms: bf16(v[b][j]) (round_bf16), v[b][j], or, with w,
// w[b] bf16(v[b][j]).
constexpr int CS = 64;
__global__ void k_colsum_part(const float *__restrict__ v, const float *__restrict__ w, int n, int H, int round_bf16,
                              float *part)
{
    const int c = blockIdx.x, b0 = c * CS, b1 = min(n, b0 + CS);
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        float s = 0.f;
        for (int b = b0; b < b1; b++) {
            const float x = v[(long long)b * H + j];
            if (w) s = fmaf(w[b], rbf(x), s);
            else s += round_bf16 ? rbf(x) : x;
        }
        part[(long long)c * H + j] = s;
    }
}

__global__ void k_colsum_fin(const float *__restrict__ part, int nc, int H, float *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= H) return;
    float s = 0.f;
    for (int c = 0; c < nc; c++) s += part[(long long)c * H + j];
    out[j] = s;
}

cudaError_t colsum(const float *v, const float *w, int n, int H, int round_bf16, float *part, float *out, cudaStream_t s)
{
    const int nc = (n + CS - 1) / CS;
    k_colsum_part<<<nc, H >= 128 ? 128 : 32, 0, s>>>(v, w, n, H, round_bf16, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colsum_fin<<<(H + 127) / 128, 128, 0, s>>>(part, nc, H, out);
    return cudaGetLastError();
}

// batch row k = row perm(b0 + k) of X (KPAD floats) and t, perm(i) = (a i + c) mod n
__global__ void k_gather_batch(const float *__restrict__ X, const float *__restrict__ t, int n, long long a,
                               long long c, int b0, int nb, float *Xb, float *tb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nb * KPAD) return;
    const int k = (int)(e / KPAD), col = (int)(e - (long long)k * KPAD);
    const long long src = (a * (long long)(b0 + k) + c) % n;
    Xb[e] = X[src * KPAD + col];
    if (col == 0) tb[k] = t[src];
}

// mean of d[b]^2 with d = y - t, one block, fixed order
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, int n, float *loss)
{
    __shared__ float part[256];
    float s = 0.f;
    for (int b = threadIdx.x; b < n; b += 256) {
        const float d = y[b] - t[b];
        s = fmaf(d, d, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)n;
}

// Adam with bias correction on every parameter
__global__ void k_adam(float *p, float *m, float *v, const float *__restrict__ g, long long total, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// x[r] = [q_r / |q_r| with w >= 0; fa; fb; zeros to KPAD]; err |= 4 on a zero quaternion
__global__ void k_features(const float *__restrict__ q, int n, const float *__restrict__ fa,
                           const float *__restrict__ fb, float *X, int *err)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * KPAD) return;
    const int r = (int)(e / KPAD), c = (int)(e - (long long)r * KPAD);
    float v = 0.f;
    if (c < 4) {
        const float w = q[4 * r], x = q[4 * r + 1], y = q[4 * r + 2], z = q[4 * r + 3];
        const float n2 = w * w + x * x + y * y + z * z;
        if (!(n2 > 0.f)) {
            if (c == 0) atomicOr(err, 4);
            v = 0.f;
        } else {
            const float s = (w < 0.f ? -1.f : 1.f) / sqrtf(n2);
            v = q[4 * r + c] * s;
        }
    } else if (c < 68) {
        v = fa[c - 4];
    } else if (c < KIN) {
        v = fb[c - 68];
    }
    X[e] = v;
}

// ------------------------------------------------------------------ top-k
// One block sorts up to 16384 keys (score mapped to an order-preserving
// integer in the high half, the complement of the index in the low half) with
// a bitonic network in shared memory, descending; the first k indices are the
// k best scores, ties to the lowest index.

__global__ void __launch_bounds__(1024) k_topk(const float *__restrict__ s, int n, int P, int k, int *idx)
{
    extern __shared__ unsigned long long key[];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long v = 0ull;
        if (i < n) {
            unsigned u = __float_as_uint(s[i]);
            u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            v = ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)i);
        }
        key[i] = v;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool desc = ((lo & size) == 0);
                const unsigned long long a = key[lo], b = key[hi];
                if ((a < b) == desc) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) idx[i] = (int)(0xFFFFFFFFu - (unsigned)(key[i] & 0xFFFFFFFFull));
}

__global__ void k_gather_quats(const float *__restrict__ q, const int *__restrict__ idx, int k, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 * k) out[i] = q[4 * (long long)idx[i >> 2] + (i & 3)];
}

// out_i = s * q_i (Hamilton product: rotation by q_i, then by s), quaternions (w, x, y, z)
__global__ void k_compose_quats(float4 sq, const float *__restrict__ q, int n, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float w2 = q[4 * (long long)i], x2 = q[4 * (long long)i + 1], y2 = q[4 * (long long)i + 2],
                z2 = q[4 * (long long)i + 3];
    const float w1 = sq.x, x1 = sq.y, y1 = sq.z, z1 = sq.w;
    float *o = out + 4 * (long long)i;
    o[0] = w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2;
    o[1] = w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2;
    o[2] = w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2;
    o[3] = w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2;
}

// y = alpha y + beta x
__global__ void k_axpby(float *y, const float *__restrict__ x, int n, float alpha, float beta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = alpha * y[i] + beta * x[i];
}

} // namespace

// ------------------------------------------------------------------ network object
struct bc_mlp_s {
    bc_ctx_t ctx = nullptr;
    int H = 0;
    Offsets off{};
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr; // params, Adam moments, gradients
    long long step = 0;
    // activations for the current batch capacity
    int cap = 0;
    float *h1 = nullptr, *h2 = nullptr, *y = nullptr, *gy = nullptr, *dh2 = nullptr, *dh1 = nullptr;
    float *part = nullptr;        // split-K and column-sum partials
    long long part_floats = 0;
    float *xb = nullptr, *tb = nullptr; // a gathered training batch (bc_mlp_train)
    int xb_cap = 0;
    float *loss = nullptr;
};

namespace {

bc_status mfail(bc_status s, const std::string &msg)
{
    set_last_error(msg);
    return s;
}

bc_status mcuda(cudaError_t e, const char *where)
{
    set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA;
}

#define MCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return mcuda(e_, #call);                                                  \
    } while (0)

bc_status ensure_batch(bc_mlp_t net, int n)
{
    if (n <= net->cap) return BC_OK;
    float *bufs[] = {net->h1, net->h2, net->y, net->gy, net->dh2, net->dh1};
    for (float *b : bufs)
        if (b) cudaFree(b);
    const int cap = n + n / 4 + 64;
    const size_t H = net->H;
    MCK(cudaMalloc(&net->h1, sizeof(float) * cap * H));
    MCK(cudaMalloc(&net->h2, sizeof(float) * cap * H));
    MCK(cudaMalloc(&net->dh2, sizeof(float) * cap * H));
    MCK(cudaMalloc(&net->dh1, sizeof(float) * cap * H));
    MCK(cudaMalloc(&net->y, sizeof(float) * cap));
    MCK(cudaMalloc(&net->gy, sizeof(float) * cap));
    if (net->part) cudaFree(net->part);
    // up to 32 split-K slices of the largest weight gradient (H x H or H x 132), and
    // the column-sum partials (one row of H per CS batch rows)
    net->part_floats = std::max(32LL * (long long)H * std::max<long long>((long long)H, KIN),
                                (long long)((cap + CS - 1) / CS) * (long long)H);
    MCK(cudaMalloc(&net->part, sizeof(float) * net->part_floats));
    net->cap = cap;
    return BC_OK;
}

// forward pass into net->h1, net->h2, y
bc_status forward(bc_mlp_t net, const float *X, int n, float *y, cudaStream_t s)
{
    const int H = net->H;
    const Offsets &o = net->off;
    GemmArgs a1{X, KPAD, 1, net->p + o.W1, 1, KIN, net->h1, H, 1, n, H, KPAD, net->p + o.b1, 1};
    // W1 is stored [H][132]; rows of X are padded to 144 with zeros, so K runs to 144 and
    // B(k, n) = W1[n][k] must be zero for k >= 132: bound K by 132 instead.
    a1.K = KIN;
    MCK(gemm(a1, s));
    GemmArgs a2{net->h1, H, 1, net->p + o.W2, 1, H, net->h2, H, 1, n, H, H, net->p + o.b2, 1};
    MCK(gemm(a2, s));
    k_head<<<(n + 7) / 8, 256, 0, s>>>(net->h2, net->p + o.w3, net->p + o.b3, n, H, y);
    MCK(cudaGetLastError());
    return BC_OK;
}

// gradients of the mean squared error into net->g
bc_status backward(bc_mlp_t net, const float *X, const float *t, int n, cudaStream_t s)
{
    const int H = net->H;
    const Offsets &o = net->off;
    const long long nh = (long long)n * H;
    k_head_back<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(net->y, t, net->h2, net->p + o.w3, n, H, net->gy, net->dh2);
    MCK(cudaGetLastError());
    MCK(colsum(net->h2, net->gy, n, H, 1, net->part, net->g + o.w3, s)); // dw3[j] = sum_b gy[b] bf16(h2[b][j])
    MCK(colsum(net->gy, nullptr, n, 1, 0, net->part, net->g + o.b3, s));
    // dW2 = dh2^T h1  (M = H out, N = H in, K = n)
    GemmArgs w2{net->dh2, 1, H, net->h1, H, 1, net->g + o.W2, H, 1, H, H, n, nullptr, 0};
    MCK(gemm_splitk(w2, net->part, net->part_floats, s));
    MCK(colsum(net->dh2, nullptr, n, H, 1, net->part, net->g + o.b2, s));
    // dh1 = (dh2 W2) masked by h1 > 0  (M = n, N = H in, K = H out)
    GemmArgs d1{net->dh2, H, 1, net->p + o.W2, H, 1, net->dh1, H, 1, n, H, H, nullptr, 0};
    MCK(gemm(d1, s));
    k_relu_back<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(net->dh1, net->h1, nh);
    // dW1 = dh1^T X  (M = H, N = 132, K = n)
    GemmArgs w1{net->dh1, 1, H, X, KPAD, 1, net->g + o.W1, KIN, 1, H, KIN, n, nullptr, 0};
    MCK(gemm_splitk(w1, net->part, net->part_floats, s));
    MCK(colsum(net->dh1, nullptr, n, H, 1, net->part, net->g + o.b1, s));
    MCK(cudaGetLastError());
    return BC_OK;
}

} // namespace

cudaError_t bc::launch_topk(const float *scores, int n, int k, int *idx, cudaStream_t s)
{
    int P = 1;
    while (P < n) P <<= 1;
    if (P < 2) P = 2;
    const size_t smem = sizeof(unsigned long long) * P;
    cudaError_t e = cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_topk<<<1, 1024, smem, s>>>(scores, n, P, k, idx);
    return cudaGetLastError();
}

__global__ void k_moments(const float2 *__restrict__ F, const int *__restrict__ modes, int count, int N, int H, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int mx = modes[3 * i], my = modes[3 * i + 1], mz = modes[3 * i + 2];
    const int jx = mx < 0 ? mx + N : mx, jy = my < 0 ? my + N : my;
    const float2 v = F[((long long)jx * N + jy) * H + mz];
    out[i] = sqrtf(v.x * v.x + v.y * v.y) / F[0].x;
}

cudaError_t bc::launch_moments(const float2 *F, const int *modes, int count, int N, int H, float *out, cudaStream_t s)
{
    k_moments<<<(count + 63) / 64, 64, 0, s>>>(F, modes, count, N, H, out);
    return cudaGetLastError();
}

cudaError_t bc::launch_gather_quats(const float *q, const int *idx, int k, float *out, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_gather_quats<<<(4 * k + 255) / 256, 256, 0, s>>>(q, idx, k, out);
    return cudaGetLastError();
}

cudaError_t bc::launch_compose_quats(const float *sq, const float *q, int n, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_compose_quats<<<(n + 255) / 256, 256, 0, s>>>(make_float4(sq[0], sq[1], sq[2], sq[3]), q, n, out);
    return cudaGetLastError();
}

cudaError_t bc::launch_axpby(float *y, const float *x, int n, float alpha, float beta, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_axpby<<<(n + 255) / 256, 256, 0, s>>>(y, x, n, alpha, beta);
    return cudaGetLastError();
}

void bc::mlp_orphan(bc_mlp_s *net)
{
    float *bufs[] = {net->p,  net->m,   net->v,    net->g,  net->h1, net->h2,  net->y,
                     net->gy, net->dh2, net->dh1, net->loss, net->part, net->xb, net->tb};
    for (float *b : bufs)
        if (b) cudaFree(b);
    net->p = net->m = net->v = net->g = net->h1 = net->h2 = net->y = net->gy = net->dh2 = net->dh1 = net->loss = nullptr;
    net->part = net->xb = net->tb = nullptr;
    net->cap = net->xb_cap = 0;
    net->part_floats = 0;
    net->ctx = nullptr;
}

extern "C" {

bc_status bc_mlp_create(bc_ctx_t ctx, int hidden, const float *init, bc_mlp_t *out)
{
    try {
        if (!ctx || !init || !out) return mfail(BC_ERR_ARG, "bc_mlp_create: null argument");
        *out = nullptr;
        if (hidden < 16 || hidden > 1024 || hidden % 16) return mfail(BC_ERR_ARG, "bc_mlp_create: hidden must be a multiple of 16 in [16, 1024]");
        bc_mlp_t net = new (std::nothrow) bc_mlp_s();
        if (!net) return mfail(BC_ERR_OOM, "bc_mlp_create: host allocation failed");
        net->ctx = ctx;
        net->H = hidden;
        net->off = offsets(hidden);
        const size_t bytes = sizeof(float) * (size_t)net->off.total;
        cudaStream_t s = ctx_stream(ctx);
        cudaError_t e;
        if ((e = cudaMalloc(&net->p, bytes)) != cudaSuccess || (e = cudaMalloc(&net->m, bytes)) != cudaSuccess ||
            (e = cudaMalloc(&net->v, bytes)) != cudaSuccess || (e = cudaMalloc(&net->g, bytes)) != cudaSuccess ||
            (e = cudaMalloc(&net->loss, sizeof(float))) != cudaSuccess) {
            bc_mlp_destroy(net);
            return mcuda(e, "bc_mlp_create: cudaMalloc");
        }
        if ((e = cudaMemcpyAsync(net->p, init, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(net->m, 0, bytes, s)) != cudaSuccess || (e = cudaMemsetAsync(net->v, 0, bytes, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            bc_mlp_destroy(net);
            return mcuda(e, "bc_mlp_create: upload");
        }
        ctx_register_mlp(ctx, net);
        *out = net;
        return BC_OK;
    } catch (...) {
        return mfail(BC_ERR_INTERNAL, "bc_mlp_create: unexpected exception");
    }
}

bc_status bc_mlp_destroy(bc_mlp_t net)
{
    if (!net) return BC_OK;
    if (net->ctx) {
        cudaStreamSynchronize(ctx_stream(net->ctx));
        ctx_unregister_mlp(net->ctx, net);
        mlp_orphan(net);
    }
    delete net;
    return BC_OK;
}

long long bc_mlp_param_count(int hidden) { return offsets(hidden).total; }

bc_status bc_mlp_features(bc_mlp_t net, const float *quats, int n, const float *fa, const float *fb, float *X)
{
    if (!net || !quats || !fa || !fb || !X || n < 1) return mfail(BC_ERR_ARG, "bc_mlp_features: bad arguments");
    if (!net->ctx) return mfail(BC_ERR_ARG, "bc_mlp_features: the network's context was destroyed");
    const long long total = (long long)n * KPAD;
    k_features<<<(unsigned)((total + 255) / 256), 256, 0, ctx_stream(net->ctx)>>>(quats, n, fa, fb, X, ctx_err(net->ctx));
    MCK(cudaGetLastError());
    return BC_OK;
}

bc_status bc_mlp_predict(bc_mlp_t net, const float *X, int n, float *y)
{
    try {
        if (!net || !X || !y || n < 1) return mfail(BC_ERR_ARG, "bc_mlp_predict: bad arguments");
        if (!net->ctx) return mfail(BC_ERR_ARG, "bc_mlp_predict: the network's context was destroyed");
        if (bc_status st = ensure_batch(net, n)) return st;
        return forward(net, X, n, y, ctx_stream(net->ctx));
    } catch (...) {
        return mfail(BC_ERR_INTERNAL, "bc_mlp_predict: unexpected exception");
    }
}

bc_status bc_mlp_grads(bc_mlp_t net, const float *X, const float *t, int n, float *grads, float *loss)
{
    try {
        if (!net || !X || !t || n < 1) return mfail(BC_ERR_ARG, "bc_mlp_grads: bad arguments");
        if (!net->ctx) return mfail(BC_ERR_ARG, "bc_mlp_grads: the network's context was destroyed");
        if (bc_status st = ensure_batch(net, n)) return st;
        cudaStream_t s = ctx_stream(net->ctx);
        if (bc_status st = forward(net, X, n, net->y, s)) return st;
        if (bc_status st = backward(net, X, t, n, s)) return st;
        if (loss) {
            k_loss<<<1, 256, 0, s>>>(net->y, t, n, loss);
            MCK(cudaGetLastError());
        }
        if (grads) MCK(cudaMemcpyAsync(grads, net->g, sizeof(float) * (size_t)net->off.total, cudaMemcpyDeviceToDevice, s));
        return BC_OK;
    } catch (...) {
        return mfail(BC_ERR_INTERNAL, "bc_mlp_grads: unexpected exception");
    }
}

bc_status bc_mlp_train_step(bc_mlp_t net, const float *X, const float *t, int n, float lr, float *loss)
{
    try {
        if (!net || !X || !t || n < 1 || !(lr > 0.f)) return mfail(BC_ERR_ARG, "bc_mlp_train_step: bad arguments");
        if (bc_status st = bc_mlp_grads(net, X, t, n, nullptr, loss)) return st;
        net->step++;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
        const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
        const long long total = net->off.total;
        k_adam<<<(unsigned)((total + 255) / 256), 256, 0, ctx_stream(net->ctx)>>>(net->p, net->m, net->v, net->g, total, lr,
                                                                                 b1, b2, eps, c1, c2);
        MCK(cudaGetLastError());
        return BC_OK;
    } catch (...) {
        return mfail(BC_ERR_INTERNAL, "bc_mlp_train_step: unexpected exception");
    }
}

// Pseudo-random order of epoch `e`: perm(i) = (a i + c) mod n with a coprime
// to n, both drawn from splitmix64 of (seed, e) -- a bijection of [0, n).
static void epoch_order(unsigned long long seed, int e, int n, long long *a, long long *c)
{
    auto mix = [](unsigned long long z) {
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto gcd = [](long long x, long long y) {
        while (y) {
            const long long t = x % y;
            x = y;
            y = t;
        }
        return x;
    };
    long long aa = (long long)(mix(seed * 0x100000001B3ull + 2ull * (unsigned)e) % (unsigned long long)n);
    if (aa == 0) aa = 1;
    while (gcd(aa, n) != 1) aa = aa + 1 < n ? aa + 1 : 1;
    *a = aa;
    *c = (long long)(mix(seed * 0x100000001B3ull + 2ull * (unsigned)e + 1ull) % (unsigned long long)n);
}

bc_status bc_mlp_train(bc_mlp_t net, const float *X, const float *t, int n, int batch, int epochs, float lr,
                       unsigned long long seed, float *loss)
{
    try {
        if (!net || !X || !t || n < 1 || batch < 1 || batch > n || epochs < 1 || !(lr > 0.f))
            return mfail(BC_ERR_ARG, "bc_mlp_train: bad arguments");
        if (!net->ctx) return mfail(BC_ERR_ARG, "bc_mlp_train: the network's context was destroyed");
        if (bc_status st = ensure_batch(net, batch)) return st;
        cudaStream_t s = ctx_stream(net->ctx);
        if (batch > net->xb_cap) {
            if (net->xb) cudaFree(net->xb);
            if (net->tb) cudaFree(net->tb);
            net->xb = net->tb = nullptr;
            net->xb_cap = 0;
            MCK(cudaMalloc(&net->xb, sizeof(float) * (size_t)batch * KPAD));
            MCK(cudaMalloc(&net->tb, sizeof(float) * (size_t)batch));
            net->xb_cap = batch;
        }
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const long long total = net->off.total;
        const int steps = n / batch;
        for (int e = 0; e < epochs; e++) {
            long long a = 1, c = 0;
            epoch_order(seed, e, n, &a, &c);
            const float lr_e = (float)(lr * 0.5 * (1.0 + std::cos(M_PI * e / epochs)));
            for (int st = 0; st < steps; st++) {
                const long long tot = (long long)batch * KPAD;
                k_gather_batch<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, t, n, a, c, st * batch, batch, net->xb,
                                                                             net->tb);
                MCK(cudaGetLastError());
                if (bc_status r = forward(net, net->xb, batch, net->y, s)) return r;
                if (bc_status r = backward(net, net->xb, net->tb, batch, s)) return r;
                net->step++;
                const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
                const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
                k_adam<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(net->p, net->m, net->v, net->g, total, lr_e, b1,
                                                                      b2, eps, c1, c2);
                MCK(cudaGetLastError());
            }
        }
        if (loss) {
            // the loss of the last batch at the parameters it was taken with
            k_loss<<<1, 256, 0, s>>>(net->y, net->tb, batch, loss);
            MCK(cudaGetLastError());
        }
        return BC_OK;
    } catch (...) {
        return mfail(BC_ERR_INTERNAL, "bc_mlp_train: unexpected exception");
    }
}

bc_status bc_mlp_state(bc_mlp_t net, float *params, float *m, float *v, long long *step, int get)
{
    if (!net || !net->ctx) return mfail(BC_ERR_ARG, "bc_mlp_state: null network or destroyed context");
    cudaStream_t s = ctx_stream(net->ctx);
    const size_t bytes = sizeof(float) * (size_t)net->off.total;
    float *host[3] = {params, m, v};
    float *dev[3] = {net->p, net->m, net->v};
    for (int i = 0; i < 3; i++) {
        if (!host[i]) continue;
        if (get) MCK(cudaMemcpyAsync(host[i], dev[i], bytes, cudaMemcpyDeviceToHost, s));
        else MCK(cudaMemcpyAsync(dev[i], host[i], bytes, cudaMemcpyHostToDevice, s));
    }
    MCK(cudaStreamSynchronize(s));
    if (step) {
        if (get) *step = net->step;
        else net->step = *step;
    }
    return BC_OK;
}

} // extern "C"
