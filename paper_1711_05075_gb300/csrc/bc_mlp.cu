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
// gradients) and accumulates in FP32 on the tensor cores (tcgen05.mma
// kind::f16, BF16 x BF16 -> FP32 in tensor memory).  All reductions run in a fixed order, so training is
// deterministic for a fixed launch configuration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/ballcorr.h"
#include "bc_internal.h"
#include "bc_umma.cuh"

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
// memory addressed through strides, rounded to BF16 when staged in shared
// memory, products on the 5th-generation tensor cores
// (tcgen05.mma.cta_group::1.kind::f16: A and B BF16, D FP32 in tensor memory;
// M = 128, N = the tile width, K = 16 per instruction).
//
// One block of 256 threads computes a 128 x nt tile of C (nt = 64, 128 or 256
// columns, chosen per call so that the grid covers the SMs).  Per K step of 64
// the threads round the A (128 x 64) and B (nt x 64) tiles to BF16 and store
// them K-major in the 128-byte-swizzled layout (row r's 16-byte chunk j at
// chunk j xor (r mod 8), 8-row groups 1024 bytes apart); one thread issues the
// step's four MMAs and commits them to the buffer's barrier while the block
// converts the next step into the other buffer.  After the last step the warps
// drain the accumulator (warp w reads lanes 32 (w mod 4) .. + 31, every other
// 16-column chunk), add the bias, apply the ReLU and store.  Every wait is
// bounded (bit 32 of the context's error word on expiry).
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
    int *err = nullptr; // status word for an expired tensor-core wait (required)
    int nt = 256;       // tile width (64, 128 or 256; set by the launchers)
    int bone = -1;      // >= 0: B's row bone is 1 for every k (C's column bone = the row sums of A); B has rows [0, bone)
    const float *mask = nullptr; // C = bf16(x) where mask > 0, else 0 (mask addressed like C; no bias, ReLU or split K)
};

constexpr int GU_THREADS = 256, GU_K = 64;
constexpr int GU_A_BYTES = 128 * 128; // 128 rows of 64 BF16
constexpr int GU_ERR = 32;

int gu_smem(int nt) { return 1024 + 2 * (GU_A_BYTES + nt * 128) + 64; }

__host__ __device__ constexpr uint32_t umma_idesc_bf16(int n)
{
    // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major,
    // N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// the 16-byte chunk j (values 8 j .. 8 j + 7 along k) of row r of a swizzled tile
__device__ __forceinline__ void st_chunk(uint8_t *dst, int r, int j, float a0, float a1, float a2, float a3, float a4,
                                         float a5, float a6, float a7)
{
    *reinterpret_cast<uint4 *>(dst + r * 128 + ((j ^ (r & 7)) << 4)) =
        make_uint4(bf2(a0, a1), bf2(a2, a3), bf2(a4, a5), bf2(a6, a7));
}

// rows x 64 values of a strided FP32 matrix, rounded to BF16 into the swizzled
// tile at `dst`: element (r, k) = src[(r0 + r) sR + (k0 + k) sK], zero unless
// r0 + r < rlim and k0 + k < klim, except row r0 + r = rone (if any), which is
// 1 for every k0 + k < klim.  The global loads stay coalesced, with
// several in flight per thread:
//  - rows contiguous (sR = 1, 16-byte aligned groups of 4 rows): a thread takes
//    4 rows x 8 k as eight float4 loads, neighbouring threads neighbouring rows;
//  - otherwise pieces of 8 consecutive k of one row (two float4 loads when k is
//    contiguous and aligned, else 8 scalar loads), neighbouring threads
//    neighbouring pieces of a row.
__device__ __forceinline__ void gu_tile(uint8_t *dst, const float *__restrict__ src, long long sR, long long sK, int r0,
                                        int rows, int rlim, int k0, int klim, int rone)
{
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    if (sR == 1 && aligned && (sK & 3) == 0 && (r0 & 3) == 0) {
        const int groups = rows >> 2, items = groups * 8;
        for (int c = threadIdx.x; c < items; c += GU_THREADS) {
            const int gi = c % groups, j = c / groups;
            const int gr = r0 + 4 * gi;
            float4 w[8];
#pragma unroll
            for (int kk = 0; kk < 8; kk++) {
                const int k = k0 + 8 * j + kk;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < klim) {
                    const float *p = src + gr + (long long)k * sK;
                    if (gr + 3 < rlim) {
                        x = __ldg(reinterpret_cast<const float4 *>(p));
                    } else {
                        x.x = gr < rlim ? p[0] : (gr == rone ? 1.f : 0.f);
                        x.y = gr + 1 < rlim ? p[1] : (gr + 1 == rone ? 1.f : 0.f);
                        x.z = gr + 2 < rlim ? p[2] : (gr + 2 == rone ? 1.f : 0.f);
                        x.w = gr + 3 == rone ? 1.f : 0.f;
                    }
                }
                w[kk] = x;
            }
            st_chunk(dst, 4 * gi, j, w[0].x, w[1].x, w[2].x, w[3].x, w[4].x, w[5].x, w[6].x, w[7].x);
            st_chunk(dst, 4 * gi + 1, j, w[0].y, w[1].y, w[2].y, w[3].y, w[4].y, w[5].y, w[6].y, w[7].y);
            st_chunk(dst, 4 * gi + 2, j, w[0].z, w[1].z, w[2].z, w[3].z, w[4].z, w[5].z, w[6].z, w[7].z);
            st_chunk(dst, 4 * gi + 3, j, w[0].w, w[1].w, w[2].w, w[3].w, w[4].w, w[5].w, w[6].w, w[7].w);
        }
        return;
    }
    const bool kvec = aligned && sK == 1 && (sR & 3) == 0;
    const int items = rows * 8;
    for (int c0 = threadIdx.x; c0 < items; c0 += 4 * GU_THREADS) {
        float x[4][8];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int c = c0 + u * GU_THREADS;
            const int gr = r0 + (c >> 3), k = k0 + 8 * (c & 7);
            const float *p = src + (long long)gr * sR + (long long)k * sK;
            if (c < items && gr < rlim && kvec && k + 8 <= klim) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
                const float4 b = __ldg(reinterpret_cast<const float4 *>(p + 4));
                x[u][0] = a.x, x[u][1] = a.y, x[u][2] = a.z, x[u][3] = a.w;
                x[u][4] = b.x, x[u][5] = b.y, x[u][6] = b.z, x[u][7] = b.w;
            } else {
#pragma unroll
                for (int kk = 0; kk < 8; kk++)
                    x[u][kk] = (c < items && k + kk < klim) ? (gr < rlim ? p[kk * sK] : (gr == rone ? 1.f : 0.f)) : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int c = c0 + u * GU_THREADS;
            if (c < items)
                st_chunk(dst, c >> 3, c & 7, x[u][0], x[u][1], x[u][2], x[u][3], x[u][4], x[u][5], x[u][6], x[u][7]);
        }
    }
}

__global__ void __launch_bounds__(GU_THREADS, 3) k_gemm_umma(GemmArgs g, int err_bit)
{
    int *err = g.err;
    const int nt = g.nt, buf = GU_A_BYTES + nt * 128;
    extern __shared__ uint8_t gu_raw[];
    const uint32_t raw = smem_addr(gu_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gb = gu_raw + (base - raw);
    // [A 0 | B 0 | A 1 | B 1] [barriers: done[0], done[1]] [tensor-memory slot] [stop]
    uint64_t *bars = reinterpret_cast<uint64_t *>(gb + 2 * buf);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 2);
    volatile int *stop = reinterpret_cast<volatile int *>(slot + 1);
    const uint32_t bar0 = smem_addr(bars);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * nt;
    const int ncols = min(nt, g.N - n0);
    const int NT = (ncols + 15) & ~15;
    const uint32_t idesc = umma_idesc_bf16(NT);
    const int kb = g.kchunk ? (int)blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    const int steps = ke > kb ? (ke - kb + GU_K - 1) / GU_K : 0;
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(nt)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    bool ok = true;
    int issued = 0; // steps whose MMAs were issued (the same count in every thread)
    for (int st = 0; st < steps && ok; st++) {
        const int b = st & 1;
        // buffer b was last read by the MMAs of step st - 2
        if (st >= 2) ok = umma_wait(bar0 + 8 * b, ((st - 2) >> 1) & 1, stop, err, err_bit);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        uint8_t *ta = gb + b * buf, *tbt = ta + GU_A_BYTES;
        const int k0 = kb + st * GU_K;
        gu_tile(ta, g.A, g.sAm, g.sAk, m0, 128, g.M, k0, ke, -1);
        gu_tile(tbt, g.B, g.sBn, g.sBk, n0, NT, g.bone >= 0 ? g.bone : g.N, k0, ke, g.bone);
        fence_proxy_async_smem(); // the tile stores are visible to the tensor core's reads
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a = base + b * buf, bb = a + GU_A_BYTES;
#pragma unroll
            for (int k = 0; k < GU_K / 16; k++) // K = 16 BF16 (32 bytes) per MMA
                umma_bf16(tmem, umma_desc_sw128(a + 32 * k), umma_desc_sw128(bb + 32 * k), idesc,
                          (st > 0 || k > 0) ? 1 : 0);
            umma_commit(bar0 + 8 * b);
        }
        issued = st + 1;
    }
    // the last step's MMAs (all earlier ones complete before it)
    if (ok && steps > 0) ok = umma_wait(bar0 + 8 * ((steps - 1) & 1), ((steps - 1) >> 1) & 1, stop, err, err_bit);
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok) {
        const int qd = warp & 3, half = warp >> 2;
        const int row = m0 + 32 * qd + lane;
        float *cz = g.C + blockIdx.z * g.sCz;
        const bool vec = g.sCn == 1 && (g.sCm & 3) == 0 && (reinterpret_cast<uintptr_t>(cz) & 15) == 0;
        float *crow = cz + (long long)row * g.sCm;
        for (int c0 = 16 * half; c0 < NT; c0 += 32) {
            uint32_t v[16];
            if (steps > 0) {
                tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = 0u;
            }
            if (row < g.M) {
                float x[16], mk[16];
                if (g.mask) {
                    const float *mr = g.mask + (long long)row * g.sCm;
                    if (vec && c0 + 16 <= ncols) {
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const float4 m4 = __ldg(reinterpret_cast<const float4 *>(mr + n0 + c0) + q);
                            mk[4 * q] = m4.x, mk[4 * q + 1] = m4.y, mk[4 * q + 2] = m4.z, mk[4 * q + 3] = m4.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) mk[j] = c0 + j < ncols ? mr[(long long)(n0 + c0 + j) * g.sCn] : 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    x[j] = __uint_as_float(v[j]);
                    if (g.bias && c0 + j < ncols) x[j] += g.bias[n0 + c0 + j];
                    if (g.relu) x[j] = fmaxf(x[j], 0.f);
                    if (g.mask) x[j] = mk[j] > 0.f ? __bfloat162float(__float2bfloat16_rn(x[j])) : 0.f;
                }
                if (vec && c0 + 16 <= ncols) {
                    float4 *o = reinterpret_cast<float4 *>(crow + n0 + c0);
#pragma unroll
                    for (int q = 0; q < 4; q++) o[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        if (c0 + j < ncols) crow[(long long)(n0 + c0 + j) * g.sCn] = x[j];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        // a wait expired: let the MMAs already issued finish (bounded) before the memory goes;
        // the last commit to buffer b was step s (s < issued, s = b mod 2), phase s >> 1
        for (int b = 0; b < 2; b++) {
            const int s = ((issued - 1) & 1) == b ? issued - 1 : issued - 2;
            if (s < 0) continue;
            const uint64_t t0 = global_ns();
            while (!mbar_test(bar0 + 8 * b, (s >> 1) & 1) && global_ns() - t0 < UMMA_WAIT_NS) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nt) : "memory");
    }
}

int gu_nsm()
{
    static int n = 0;
    if (n <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n <= 0)
            n = 152;
    }
    return n;
}

// the widest tile whose grid (with nz slices of K) still gives every SM a block
int gu_pick_nt(int M, int N, int nz)
{
    const long long mt = (M + 127) / 128;
    for (int nt = 256; nt > 64; nt >>= 1)
        if ((long long)((N + nt - 1) / nt) * mt * nz >= gu_nsm()) return nt;
    return 64;
}

cudaError_t gu_launch(const GemmArgs &a, int nz, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, gu_smem(256));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.N + a.nt - 1) / a.nt, (a.M + 127) / 128, nz);
    k_gemm_umma<<<grid, GU_THREADS, gu_smem(a.nt), s>>>(a, GU_ERR);
    return cudaGetLastError();
}

cudaError_t gemm(GemmArgs a, cudaStream_t s)
{
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    a.nt = gu_pick_nt(a.M, a.N, 1);
    return gu_launch(a, 1, s);
}

// out[m][n] = sum_z part[z][m][n], z in increasing order (M x N partials, rows
// `ld` floats apart); with `ocol`, column N - 1 goes to ocol[m] instead
__global__ void k_sum_partials(const float *__restrict__ part, int nz, int M, int N, int ld, float *out,
                               long long sOm, float *ocol)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)M * N) return;
    const long long m = e / N, nn = e - m * N;
    float s = 0.f;
    for (int z = 0; z < nz; z++) s += part[(z * (long long)M + m) * ld + nn];
    if (ocol && nn == N - 1) ocol[m] = s;
    else out[m * sOm + nn] = s;
}

// A weight gradient C = A B with a long K (the batch): K split into slices whose
// partial products land in `part` and are then summed in a fixed order, so the
// result does not depend on scheduling.  C is M x N with row stride sCm; with
// `ocol` (and a.bone = N - 1), C's last column -- the row sums of A -- goes to
// ocol instead.
cudaError_t gemm_splitk(GemmArgs a, float *part, long long part_floats, cudaStream_t s, float *ocol = nullptr)
{
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    const int ld = (a.N + 3) & ~3; // partial rows padded to 16 bytes (vector stores)
    const long long mn = (long long)a.M * ld;
    const long long nzmax = std::max(1LL, std::min({32LL, part_floats / mn, (long long)(a.K + GU_K - 1) / GU_K}));
    a.nt = gu_pick_nt(a.M, a.N, (int)nzmax);
    const long long tiles = (long long)((a.N + a.nt - 1) / a.nt) * ((a.M + 127) / 128);
    int nz = (int)std::max(1LL, std::min(nzmax, (2LL * gu_nsm() + tiles - 1) / tiles)); // about two blocks per SM
    int kchunk = 0;
    if (a.K > 0) {
        kchunk = ((a.K + nz - 1) / nz + GU_K - 1) / GU_K * GU_K;
        nz = (a.K + kchunk - 1) / kchunk;
    } else {
        nz = 1;
    }
    float *C = a.C;
    const long long sCm = a.sCm;
    a.C = part;
    a.sCm = ld;
    a.sCn = 1;
    a.kchunk = kchunk;
    a.sCz = mn;
    cudaError_t e = gu_launch(a, nz, s);
    if (e != cudaSuccess) return e;
    const long long tot = (long long)a.M * a.N;
    k_sum_partials<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nz, a.M, a.N, ld, C, sCm, ocol);
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

// The training head, for a batch of n rows:
//   y[b]   = sum_j bf16(h2[b][j]) bf16(w3[j]) + b3            (the sum of k_head, same order)
//   gy[b]  = 2 (y[b] - t[b]) / n                              (d loss / d y, mean squared error)
//   dh2[b][j] = bf16(gy[b] bf16(w3[j])) where h2[b][j] > 0, else 0
// and the sums over the batch dw3[j] = sum_b gy[b] bf16(h2[b][j]), db2[j] =
// sum_b dh2[b][j], db3 = sum_b gy[b].  k_head_train: one warp per row (lane l
// holds columns l + 32 i, the next row's loads issued before the current row's
// arithmetic); block c sums its rows, warp by warp in order, into
// part[c][0, 2H].  k_head_sums: one warp per entry adds the blocks' rows in a
// fixed order (lane l the blocks l, l + 32, ..., then a fixed shuffle tree).
constexpr int HT_THREADS = 256;

template <int NC>
__global__ void __launch_bounds__(HT_THREADS) k_head_train(const float *__restrict__ h2, const float *__restrict__ w3,
                                                           const float *__restrict__ b3, const float *__restrict__ t,
                                                           int n, int H, int rows_per_block, float *y, float *gy,
                                                           float *dh2, float *part)
{
    extern __shared__ float ht_s[]; // 2H + 1 block sums
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = HT_THREADS / 32;
    const int r0 = blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
    float w3r[NC], aw[NC], ab[NC], v[NC], a3 = 0.f;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const int j = lane + 32 * i;
        w3r[i] = j < H ? rbf(w3[j]) : 0.f;
        aw[i] = ab[i] = 0.f;
    }
    int r = r0 + warp;
    if (r < r1) {
#pragma unroll
        for (int i = 0; i < NC; i++) v[i] = lane + 32 * i < H ? h2[(long long)r * H + lane + 32 * i] : 0.f;
    }
    for (; r < r1; r += nw) {
        float vn[NC];
        const int rn = r + nw;
#pragma unroll
        for (int i = 0; i < NC; i++) vn[i] = (rn < r1 && lane + 32 * i < H) ? h2[(long long)rn * H + lane + 32 * i] : 0.f;
        float sum = 0.f;
#pragma unroll
        for (int i = 0; i < NC; i++)
            if (lane + 32 * i < H) sum = fmaf(rbf(v[i]), w3r[i], sum);
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const float yr = sum + b3[0];
        const float g = 2.f * (yr - t[r]) / (float)n;
        if (lane == 0) {
            y[r] = yr;
            gy[r] = g;
        }
        float *dr = dh2 + (long long)r * H;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            const int j = lane + 32 * i;
            if (j < H) {
                const float d = v[i] > 0.f ? rbf(g * w3r[i]) : 0.f;
                dr[j] = d;
                aw[i] = fmaf(g, rbf(v[i]), aw[i]);
                ab[i] += d;
            }
            v[i] = vn[i];
        }
        a3 += g;
    }
    // block sums, warp 0 first
    for (int w = 0; w < nw; w++) {
        if (warp == w) {
#pragma unroll
            for (int i = 0; i < NC; i++) {
                const int j = lane + 32 * i;
                if (j < H) {
                    ht_s[j] = w ? ht_s[j] + aw[i] : aw[i];
                    ht_s[H + j] = w ? ht_s[H + j] + ab[i] : ab[i];
                }
            }
            if (lane == 0) ht_s[2 * H] = w ? ht_s[2 * H] + a3 : a3;
        }
        __syncthreads();
    }
    const int W = 2 * H + 1;
    for (int e = threadIdx.x; e < W; e += HT_THREADS) part[(long long)blockIdx.x * W + e] = ht_s[e];
}

__global__ void k_head_sums(const float *__restrict__ part, int nb, int H, float *dw3, float *db2, float *db3)
{
    const int W = 2 * H + 1;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= W) return;
    float sum = 0.f;
    for (int c = lane; c < nb; c += 32) sum += part[(long long)c * W + e];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        if (e < H) dw3[e] = sum;
        else if (e < 2 * H) db2[e - H] = sum;
        else db3[0] = sum;
    }
}

constexpr int HT_MAX_BLOCKS = 1024;

cudaError_t head_train(const float *h2, const float *w3, const float *b3, const float *t, int n, int H, float *y,
                       float *gy, float *dh2, float *part, long long part_floats, float *dw3, float *db2, float *db3,
                       cudaStream_t s)
{
    const long long W = 2LL * H + 1;
    // about four rows per warp
    int blocks = (int)std::min<long long>({(long long)(n + 31) / 32, (long long)HT_MAX_BLOCKS, part_floats / W});
    blocks = std::max(blocks, 1);
    const int rpb = (n + blocks - 1) / blocks;
    blocks = (n + rpb - 1) / rpb;
    const size_t smem = sizeof(float) * (size_t)W;
    const int nc = (H + 31) / 32;
#define HT_LAUNCH(NC) k_head_train<NC><<<blocks, HT_THREADS, smem, s>>>(h2, w3, b3, t, n, H, rpb, y, gy, dh2, part)
    if (nc <= 1) HT_LAUNCH(1);
    else if (nc <= 2) HT_LAUNCH(2);
    else if (nc <= 4) HT_LAUNCH(4);
    else if (nc <= 8) HT_LAUNCH(8);
    else if (nc <= 16) HT_LAUNCH(16);
    else HT_LAUNCH(32);
#undef HT_LAUNCH
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_head_sums<<<(unsigned)((W + 7) / 8), 256, 0, s>>>(part, blocks, H, dw3, db2, db3);
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

// the same with one float4 per thread (X 16-byte aligned; rows are KPAD = 36 float4)
__global__ void k_gather_batch4(const float4 *__restrict__ X, const float *__restrict__ t, int n, long long a,
                                long long c, int b0, int nb, float4 *Xb, float *tb)
{
    constexpr int R4 = KPAD / 4;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nb * R4) return;
    const int k = (int)(e / R4), col = (int)(e - (long long)k * R4);
    const long long src = (a * (long long)(b0 + k) + c) % n;
    Xb[e] = X[src * R4 + col];
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
// Row r: [q_r / |q_r| (w >= 0); fa; fb + r ldb] (ldb = 0: the same fb for every row).
__global__ void k_features(const float *__restrict__ q, int n, const float *__restrict__ fa,
                           const float *__restrict__ fb, long long ldb, float *X, int *err)
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
        v = fb[r * ldb + c - 68];
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
    int rotated_moments = 0;      // the ligand features are the moments of the rotated ligand (bc_mlp_set_features)
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
    // up to 32 split-K slices of the largest weight gradient (H x (H + 1) or H x 133,
    // the last column the bias gradient), and the training head's block sums
    net->part_floats = std::max(32LL * (long long)H * (std::max<long long>((long long)H, KIN) + 1),
                                (long long)HT_MAX_BLOCKS * (2LL * (long long)H + 1));
    MCK(cudaMalloc(&net->part, sizeof(float) * net->part_floats));
    net->cap = cap;
    return BC_OK;
}

// the hidden layers into net->h1, net->h2
bc_status hidden_layers(bc_mlp_t net, const float *X, int n, cudaStream_t s)
{
    const int H = net->H;
    const Offsets &o = net->off;
    GemmArgs a1{X, KPAD, 1, net->p + o.W1, 1, KIN, net->h1, H, 1, n, H, KPAD, net->p + o.b1, 1};
    // W1 is stored [H][132]; rows of X are padded to 144 with zeros, so K runs to 144 and
    // B(k, n) = W1[n][k] must be zero for k >= 132: bound K by 132 instead.
    a1.K = KIN;
    a1.err = ctx_err(net->ctx);
    MCK(gemm(a1, s));
    GemmArgs a2{net->h1, H, 1, net->p + o.W2, 1, H, net->h2, H, 1, n, H, H, net->p + o.b2, 1};
    a2.err = ctx_err(net->ctx);
    MCK(gemm(a2, s));
    return BC_OK;
}

// forward pass into net->h1, net->h2, y
bc_status forward(bc_mlp_t net, const float *X, int n, float *y, cudaStream_t s)
{
    if (bc_status st = hidden_layers(net, X, n, s)) return st;
    const Offsets &o = net->off;
    k_head<<<(n + 7) / 8, 256, 0, s>>>(net->h2, net->p + o.w3, net->p + o.b3, n, net->H, y);
    MCK(cudaGetLastError());
    return BC_OK;
}

// forward pass (net->y) and the gradients of the mean squared error into net->g
bc_status forward_backward(bc_mlp_t net, const float *X, const float *t, int n, cudaStream_t s)
{
    if (bc_status st = hidden_layers(net, X, n, s)) return st;
    const int H = net->H;
    const Offsets &o = net->off;
    // y, gy, dh2 and the sums over the batch: dw3, db2, db3
    MCK(head_train(net->h2, net->p + o.w3, net->p + o.b3, t, n, H, net->y, net->gy, net->dh2, net->part,
                   net->part_floats, net->g + o.w3, net->g + o.b2, net->g + o.b3, s));
    // dW2 = dh2^T h1  (M = H out, N = H in, K = n)
    GemmArgs w2{net->dh2, 1, H, net->h1, H, 1, net->g + o.W2, H, 1, H, H, n, nullptr, 0};
    w2.err = ctx_err(net->ctx);
    MCK(gemm_splitk(w2, net->part, net->part_floats, s));
    // dh1 = bf16(dh2 W2) where h1 > 0, else 0  (M = n, N = H in, K = H out)
    GemmArgs d1{net->dh2, H, 1, net->p + o.W2, H, 1, net->dh1, H, 1, n, H, H, nullptr, 0};
    d1.err = ctx_err(net->ctx);
    d1.mask = net->h1;
    MCK(gemm(d1, s));
    // [dW1 | db1] = dh1^T [X | 1]  (M = H, N = 132 + 1, K = n): the column of ones gives db1 = sum_b dh1[b]
    GemmArgs w1{net->dh1, 1, H, X, KPAD, 1, net->g + o.W1, KIN, 1, H, KIN + 1, n, nullptr, 0};
    w1.err = ctx_err(net->ctx);
    w1.bone = KIN;
    MCK(gemm_splitk(w1, net->part, net->part_floats, s, net->g + o.b1));
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

// ------------------------------------------------------------------ moments of a rotated shape
// m_{R S}[i] = |f^_S(R^T m_i)| / f^_S(0) (the moments of S turned by R) by direct
// sums over the knots, f^_S(k) = sum_i h^(rho_{l_i}, |k|) exp(-2 pi i k . c_i / P)
// (Eq. (fballhat) without spreading: the band-limited spectrum at off-grid
// frequencies), for many rotations.  exp(-2 pi i m . R c / P) is the product of
// u_a^{m_a}, u_a = exp(-i pi (2 / P) (R c)_a): three sincospif per knot, then two
// complex products per mode.  The mode table is compiled in (the 64 lowest modes
// are the same for every N >= 8: no component exceeds 3); the context checks it
// against the one it builds.  One block per rotation: two groups of 128 threads
// take 32 modes each over all knots (thread j of a group the knots j, j + 128,
// ...), then warp shuffles and a fixed-order combine of the four warps.
constexpr int MR_THREADS = 256, MR_GROUP = 32;

// components of mode i offset by 'D' ('A' = -3 .. 'G' = +3), in the order of the table
__host__ __device__ constexpr int mr_mode(int i, int a)
{
    return "CDDDCDDDEDEDEDDCCDCDECEDDCEDEEECDEDEEEDCCECEEECEEEEBDDDBDDDFDFDFDDBCDBDEBEDCBDCDFCFDDBEDCFDEFDFEEBDEDFEFDFCDFDEF"
           "EDBCEBEECBECCFCEFCFEEBEECFEEFEFEFCEFEEBBDBDFBFDDBFDFFFBDFDFFFDADDBBEBCFBEFBFECBF"[3 * i + a] -
           'D';
}

struct Cpx {
    float x, y;
};
__device__ __forceinline__ Cpx cmul(Cpx a, Cpx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// u^m for |m| <= 3 from p[0..3] = u^0 .. u^3 (u on the unit circle: u^-m = conj(u^m))
__device__ __forceinline__ Cpx cpow(const Cpx (&p)[4], int m)
{
    const Cpx v = p[m < 0 ? -m : m];
    return m < 0 ? Cpx{v.x, -v.y} : v;
}

// the earlier mode -m_i of the table, or -1 (|f^(-m)| = |f^(m)| for a real density,
// so such a mode is not summed but copied)
__host__ __device__ constexpr int mr_twin(int i)
{
    for (int j = 0; j < i; j++)
        if (mr_mode(j, 0) == -mr_mode(i, 0) && mr_mode(j, 1) == -mr_mode(i, 1) && mr_mode(j, 2) == -mr_mode(i, 2))
            return j;
    return -1;
}

constexpr int MR_SHELLS = 10; // |m|^2 <= 9 over the table

// exp(-2 pi i m . p / P) from the per-axis powers, skipping the zero components
template <int MX, int MY, int MZ>
__device__ __forceinline__ Cpx mr_phase(const Cpx (&u)[3][4])
{
    if constexpr (MX != 0 && MY != 0 && MZ != 0) return cmul(cmul(cpow(u[0], MX), cpow(u[1], MY)), cpow(u[2], MZ));
    else if constexpr (MX != 0 && MY != 0) return cmul(cpow(u[0], MX), cpow(u[1], MY));
    else if constexpr (MX != 0 && MZ != 0) return cmul(cpow(u[0], MX), cpow(u[2], MZ));
    else if constexpr (MY != 0 && MZ != 0) return cmul(cpow(u[1], MY), cpow(u[2], MZ));
    else if constexpr (MX != 0) return cpow(u[0], MX);
    else if constexpr (MY != 0) return cpow(u[1], MY);
    else return cpow(u[2], MZ);
}

// acc[2 j], acc[2 j + 1] += h^(rho_l, |m|) exp(-2 pi i m . p / P) for mode m = M (j = M mod 32)
template <int M>
__device__ __forceinline__ void mr_term(const Cpx (&u)[3][4], const float *wq, float (&acc)[2 * MR_GROUP])
{
    if constexpr (mr_twin(M) < 0) {
        constexpr int mx = mr_mode(M, 0), my = mr_mode(M, 1), mz = mr_mode(M, 2), j = M % MR_GROUP;
        const Cpx t = mr_phase<mx, my, mz>(u);
        const float w = wq[mx * mx + my * my + mz * mz];
        acc[2 * j] = fmaf(w, t.x, acc[2 * j]);
        acc[2 * j + 1] = fmaf(w, t.y, acc[2 * j + 1]);
    }
}

template <int G, int... J>
__device__ __forceinline__ void mr_terms(std::integer_sequence<int, J...>, const Cpx (&u)[3][4], const float *wq,
                                         float (&acc)[2 * MR_GROUP])
{
    (mr_term<G * MR_GROUP + J>(u, wq, acc), ...);
}

template <int G>
__device__ __forceinline__ void mr_sums(const float4 *__restrict__ kn, int nk, int j0, const float (&R)[9],
                                        float two_over_P, const float *wq_all, float (&acc)[2 * MR_GROUP], float &a0)
{
    for (int i = j0; i < nk; i += MR_THREADS / 2) {
        const float4 c = kn[i];
        const int l = __float_as_int(c.w);
        const float p[3] = {fmaf(R[0], c.x, fmaf(R[1], c.y, R[2] * c.z)), fmaf(R[3], c.x, fmaf(R[4], c.y, R[5] * c.z)),
                            fmaf(R[6], c.x, fmaf(R[7], c.y, R[8] * c.z))};
        Cpx u[3][4];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float s, co;
            sincospif(two_over_P * p[a], &s, &co);
            u[a][0] = {1.f, 0.f};
            u[a][1] = {co, -s};
            u[a][2] = cmul(u[a][1], u[a][1]);
            u[a][3] = cmul(u[a][2], u[a][1]);
        }
        const float *wq = wq_all + l * MR_SHELLS; // h^(rho_l, 2 pi sqrt(q) / P), q = |m|^2
        mr_terms<G>(std::make_integer_sequence<int, MR_GROUP>{}, u, wq, acc);
        if (G == 0) a0 += wq[0];
    }
}

__global__ void __launch_bounds__(MR_THREADS) k_moments_rot(const float4 *__restrict__ knots, int nk,
                                                            const float *__restrict__ quats,
                                                            const float *__restrict__ ballft, int qstride, int L,
                                                            float two_over_P, float *out, int *err)
{
    __shared__ float wq[BC_MAX_LEVELS * MR_SHELLS];
    __shared__ float red[MR_THREADS / 32][2 * MR_GROUP + 1];
    const int r = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < L * MR_SHELLS; e += MR_THREADS) {
        const int l = e / MR_SHELLS, q = e - l * MR_SHELLS;
        wq[e] = q < qstride ? ballft[(long long)l * qstride + q] : 0.f;
    }
    float qw = quats[4 * r], qx = quats[4 * r + 1], qy = quats[4 * r + 2], qz = quats[4 * r + 3];
    const float nq = qw * qw + qx * qx + qy * qy + qz * qz;
    if (!(nq > 0.f)) {
        if (threadIdx.x == 0) atomicOr(err, 4);
        qw = 1.f, qx = qy = qz = 0.f;
    } else {
        const float s = rsqrtf(nq);
        qw *= s, qx *= s, qy *= s, qz *= s;
    }
    const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    __syncthreads();
    float acc[2 * MR_GROUP], a0 = 0.f;
#pragma unroll
    for (int j = 0; j < 2 * MR_GROUP; j++) acc[j] = 0.f;
    const int G = threadIdx.x / (MR_THREADS / 2), j0 = threadIdx.x % (MR_THREADS / 2);
    if (G == 0) mr_sums<0>(knots, nk, j0, R, two_over_P, wq, acc, a0);
    else mr_sums<1>(knots, nk, j0, R, two_over_P, wq, acc, a0);
#pragma unroll
    for (int j = 0; j < 2 * MR_GROUP; j++)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    for (int o = 16; o > 0; o >>= 1) a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 2 * MR_GROUP; j++) red[warp][j] = acc[j];
        red[warp][2 * MR_GROUP] = a0;
    }
    __syncthreads();
    if (threadIdx.x < BC_MOMENTS) {
        int i = threadIdx.x;
        // a mode whose negation comes earlier takes that one's sum (|f^(-m)| = |f^(m)|)
        for (int t = 0; t < i; t++)
            if (mr_mode(t, 0) == -mr_mode(i, 0) && mr_mode(t, 1) == -mr_mode(i, 1) && mr_mode(t, 2) == -mr_mode(i, 2)) {
                i = t;
                break;
            }
        const int g = i / MR_GROUP, j = i - g * MR_GROUP, wpg = MR_THREADS / 64;
        float re = 0.f, im = 0.f, f0 = 0.f;
        for (int w = 0; w < wpg; w++) {
            re += red[g * wpg + w][2 * j];
            im += red[g * wpg + w][2 * j + 1];
            f0 += red[w][2 * MR_GROUP];
        }
        out[(long long)r * BC_MOMENTS + threadIdx.x] = sqrtf(re * re + im * im) / f0;
    }
}

cudaError_t bc::launch_moments_rot(const float4 *knots, int nk, const float *quats, int n, const float *ballft,
                                   int qstride, int L, float two_over_P, float *out, int *err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_moments_rot<<<n, MR_THREADS, 0, s>>>(knots, nk, quats, ballft, qstride, L, two_over_P, out, err);
    return cudaGetLastError();
}

bool bc::moments_rot_table_matches(const int *tab)
{
    for (int i = 0; i < BC_MOMENTS; i++)
        for (int a = 0; a < 3; a++)
            if (tab[3 * i + a] != mr_mode(i, a)) return false;
    return true;
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

static bc_status features_impl(bc_mlp_t net, const float *quats, int n, const float *fa, const float *fb,
                               long long ldb, float *X, const char *who)
{
    if (!net || !quats || !fa || !fb || !X || n < 1) return mfail(BC_ERR_ARG, std::string(who) + ": bad arguments");
    if (!net->ctx) return mfail(BC_ERR_ARG, std::string(who) + ": the network's context was destroyed");
    const long long total = (long long)n * KPAD;
    k_features<<<(unsigned)((total + 255) / 256), 256, 0, ctx_stream(net->ctx)>>>(quats, n, fa, fb, ldb, X,
                                                                                  ctx_err(net->ctx));
    MCK(cudaGetLastError());
    return BC_OK;
}

bc_status bc_mlp_features(bc_mlp_t net, const float *quats, int n, const float *fa, const float *fb, float *X)
{
    return features_impl(net, quats, n, fa, fb, 0, X, "bc_mlp_features");
}

bc_status bc_mlp_features_rows(bc_mlp_t net, const float *quats, int n, const float *fa, const float *fb_rows, float *X)
{
    return features_impl(net, quats, n, fa, fb_rows, BC_MOMENTS, X, "bc_mlp_features_rows");
}

bc_status bc_mlp_set_features(bc_mlp_t net, int rotated_moments)
{
    if (!net || (rotated_moments != 0 && rotated_moments != 1))
        return mfail(BC_ERR_ARG, "bc_mlp_set_features: null network, or rotated_moments not 0 or 1");
    net->rotated_moments = rotated_moments;
    return BC_OK;
}

int bc_mlp_rotated_moments(bc_mlp_t net) { return net ? net->rotated_moments : 0; }

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
        if (bc_status st = forward_backward(net, X, t, n, s)) return st;
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
        const bool x16 = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
        for (int e = 0; e < epochs; e++) {
            long long a = 1, c = 0;
            epoch_order(seed, e, n, &a, &c);
            const float lr_e = (float)(lr * 0.5 * (1.0 + std::cos(M_PI * e / epochs)));
            for (int st = 0; st < steps; st++) {
                if (x16) {
                    const long long tot = (long long)batch * (KPAD / 4);
                    k_gather_batch4<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
                        reinterpret_cast<const float4 *>(X), t, n, a, c, st * batch, batch,
                        reinterpret_cast<float4 *>(net->xb), net->tb);
                } else {
                    const long long tot = (long long)batch * KPAD;
                    k_gather_batch<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, t, n, a, c, st * batch, batch,
                                                                                 net->xb, net->tb);
                }
                MCK(cudaGetLastError());
                if (bc_status r = forward_backward(net, net->xb, net->tb, batch, s)) return r;
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
