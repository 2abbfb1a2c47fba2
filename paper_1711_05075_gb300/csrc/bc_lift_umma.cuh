// The lifted contraction (Sec. 3.2, Eq. (rhoAhat)) on the 5th-generation tensor
// cores: rho^[a][b] = sum_i P1[a][i] P2[b][i] (complex, no conjugate) with
// tcgen05.mma (kind::tf32, FP32 accumulation in tensor memory), operands staged
// in shared memory by the bulk-copy engine, in 3-pass split TF32.
//
// Real form.  Knot block kb (32 knots) gives two K-blocks h = 0, 1 of 32
// elements.  A (rows a of P1): h = 0 holds Re P1, h = 1 holds Im P1.  B (two
// rows per complex column b of P2, 2c and 2c + 1 of the column tile): h = 0
// holds (Re P2, Im P2), h = 1 holds (-Im P2, Re P2).  Then
//     D[a][2c]     = sum Re P1 Re P2 - Im P1 Im P2 = Re rho^,
//     D[a][2c + 1] = sum Re P1 Im P2 + Im P1 Re P2 = Im rho^,
// so each accumulator row is the complex row of rho^ in order.  Every value
// is split x = x_hi + x_lo (x_hi = x rounded to TF32, x_lo = x - x_hi) and each
// product formed as a_hi b_hi + a_hi b_lo + a_lo b_hi (the a_lo b_lo term is
// 2^-22 relative).
//
// Operand blocks in HBM are written by k_lift_operands in the order and layout
// the tensor core reads them from shared memory: one block per (row tile, kb, h),
// 128 rows (A, 16 KB) or 256 rows (B, 32 KB) of 128 bytes, K-major, with the
// 128-byte swizzle (16-byte chunk j of row r stored at chunk j xor (r mod 8)).
// A stage is then four contiguous bulk copies (A hi, A lo, B hi, B lo; 96 KB).
//
// Work unit: (knot range, row tile of 128, column tile of 128 complex columns);
// units are sized so that every block of the grid (one per SM) gets an equal
// share.  The tensor cores truncate when they add into the accumulator, so the
// accumulator is restarted for every stage (one K-block: 12 MMAs) and the
// epilogue adds each stage's partial tile into FP32 running sums in registers
// with round-to-nearest adds; a unit's sums go into rho^ with vector atomics.
//
// Roles (320 threads, one block per SM): warp 0 lane 0 issues the copies,
// warp 1 allocates tensor memory and its lane 0 issues the MMAs into two
// accumulator buffers of 256 columns (stage k uses buffer k mod 2), warps 2-9
// drain them (warp w reads tensor-memory lanes 32 (w mod 4) .. and column half
// (w - 2) / 4).  Every wait on an mbarrier gives up after about two seconds:
// the block then records the failure in *err, stops, waits (bounded) for its
// copies and MMAs in flight and frees its tensor memory.
//
// Phases: a knot's coordinate over its period, v, enters as the 32-bit
// fixed-point fraction round(v 2^32) mod 2^32 (lift_fixed, FP64); m v mod 1 is
// then exact in wrapping 32-bit integer arithmetic, and sincospi runs in FP32
// on the reduced value (|v 2^32 - round| <= 1/2, so the phase carries at most
// |m| 2^-33 + 2^-25 of argument error).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_umma.cuh"

namespace bc {

constexpr int UMMA_THREADS = 320;
constexpr int UMMA_A_BYTES = 128 * 128;                      // 128 rows x 32 TF32
constexpr int UMMA_B_BYTES = 256 * 128;                      // 256 rows x 32 TF32
constexpr int UMMA_STAGE = 2 * UMMA_A_BYTES + 2 * UMMA_B_BYTES; // A hi, A lo, B hi, B lo
constexpr int UMMA_SMEM = 2 * UMMA_STAGE + 1024 + 256;       // two stages, alignment, barriers
constexpr uint32_t UMMA_IDESC = umma_idesc_tf32(256);
static_assert(UMMA_IDESC == ((1u << 4) | (2u << 7) | (2u << 10) | (32u << 17) | (8u << 24)), "descriptor fields");

struct LiftQ { // a knot's x / P, y / P, z / P, r / P_r mod 1 in units of 2^-32
    unsigned x, y, z, w;
};

__host__ __device__ inline unsigned lift_fixed(double v)
{
    const double f = v - floor(v); // [0, 1)
    return (unsigned)(unsigned long long)llrint(f * 4294967296.0);
}

// Operand blocks for one shape from its fixed-point knots (rotated and
// mirrored already): row a < M = N^2 of P1 is (j_x, j_y), row b < C = N/2 Nr
// of P2 is (m_z, j_eta); knots i >= n are zero.
__global__ void k_lift_operands(const LiftQ *__restrict__ u, int n, int nkb, int N, int Nr, float *ahi, float *alo,
                                float *bhi, float *blo)
{
    const int M = N * N;
    const int row = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nkb * 32) return;
    float re = 0.f, im = 0.f;
    if (i < n) {
        const LiftQ v = u[i];
        unsigned ph;
        if (row < M) {
            const int jx = row / N, jy = row - jx * N;
            ph = (unsigned)(jx < N / 2 ? jx : jx - N) * v.x + (unsigned)(jy < N / 2 ? jy : jy - N) * v.y;
        } else {
            const int b = row - M, mz = b / Nr, je = b - mz * Nr;
            ph = (unsigned)mz * v.z + (unsigned)(je < Nr / 2 ? je : je - Nr) * v.w;
        }
        const float r = (float)(int)ph * 2.3283064365386963e-10f; // [-1/2, 1/2)
        float sn, cs;
        sincospif(2.0f * r, &sn, &cs);
        re = cs;
        im = -sn;
    }
    const float rh = tf32_round(re), rl = re - rh, ih = tf32_round(im), il = im - ih;
    const int kb = i >> 5, e = i & 31;
    if (row < M) {
        const long long blk = ((long long)(row >> 7) * nkb + kb) * 2; // h = 0; h = 1 is the next block
        const int o = umma_swz(row & 127, e);
        const long long o0 = blk * (UMMA_A_BYTES / 4) + o, o1 = o0 + UMMA_A_BYTES / 4;
        ahi[o0] = rh;
        alo[o0] = rl;
        ahi[o1] = ih;
        alo[o1] = il;
    } else {
        const int b = row - M, c = b & 127;
        const long long blk = ((long long)(b >> 7) * nkb + kb) * 2;
        const long long r0 = blk * (UMMA_B_BYTES / 4) + umma_swz(2 * c, e);
        const long long r1 = blk * (UMMA_B_BYTES / 4) + umma_swz(2 * c + 1, e);
        constexpr long long nx = UMMA_B_BYTES / 4;
        bhi[r0] = rh;
        blo[r0] = rl;
        bhi[r1] = ih;
        blo[r1] = il;
        bhi[r0 + nx] = -ih;
        blo[r0 + nx] = -il;
        bhi[r1 + nx] = rh;
        blo[r1 + nx] = rl;
    }
}

struct UmmaUnit {
    int rt, ct, kb0, kb1;
};

// unit u: column tile fastest, then row tile, then knot range (units running
// together share operand blocks in L2)
__device__ __forceinline__ UmmaUnit umma_unit(int u, int mt, int ctn, int nsplit, int nkb)
{
    const int tiles = mt * ctn;
    const int ks = u / tiles, rem = u - ks * tiles;
    UmmaUnit w;
    w.rt = rem / ctn;
    w.ct = rem - w.rt * ctn;
    w.kb0 = (int)((long long)ks * nkb / nsplit);
    w.kb1 = (int)((long long)(ks + 1) * nkb / nsplit);
    return w;
}

// out[a][b] += sum_i P1[a][i] P2[b][i]; out is M x C complex (row stride C);
// mt = M / 128 row tiles, ctn = C / 128 column tiles, nsplit knot ranges
// (nsplit <= nkb).
__global__ void __launch_bounds__(UMMA_THREADS, 1)
k_lift_gemm_umma(const float *__restrict__ ahi, const float *__restrict__ alo, const float *__restrict__ bhi,
                 const float *__restrict__ blo, int nkb, int mt, int ctn, int nsplit, int C, float2 *out, int *err)
{
    extern __shared__ uint8_t umma_raw[];
    const uint32_t raw = smem_addr(umma_raw);
    const uint32_t base = (raw + 1023u) & ~1023u; // the swizzle pattern repeats every 1024 bytes
    uint8_t *gbase = umma_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + 2 * UMMA_STAGE);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 9);
    volatile int *stop = reinterpret_cast<volatile int *>(slot + 1);
    const uint32_t b0 = smem_addr(bars);
    // full[s] = b0 + 8 s, empty[s] = b0 + 16 + 8 s (shared stages); acc_full[b] =
    // b0 + 32 + 8 b, acc_empty[b] = b0 + 48 + 8 b (accumulator buffers); drain = b0 + 64.
    // Stage k of the block's sequence uses shared stage k mod 2 and buffer k mod 2.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init(b0 + 8 * s, 1);
            mbar_init(b0 + 16 + 8 * s, 1);
            mbar_init(b0 + 32 + 8 * s, 1);
            mbar_init(b0 + 48 + 8 * s, UMMA_THREADS - 64);
        }
        mbar_init(b0 + 64, 1);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const int units = mt * ctn * nsplit;

    if (warp == 0) {
        if (lane == 0) { // copies
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                const UmmaUnit w = umma_unit(u, mt, ctn, nsplit, nkb);
                for (int kb = w.kb0; kb < w.kb1 && ok; kb++)
                    for (int h = 0; h < 2; h++, it++) {
                        const int s = it & 1;
                        if (!umma_wait(b0 + 16 + 8 * s, ((it >> 1) & 1) ^ 1, stop, err, 1)) {
                            ok = false;
                            break;
                        }
                        const uint32_t full = b0 + 8 * s;
                        mbar_expect_tx(full, UMMA_STAGE);
                        const uint32_t dst = base + s * UMMA_STAGE;
                        const long long ab = ((long long)w.rt * nkb + kb) * 2 + h;
                        const long long bb = ((long long)w.ct * nkb + kb) * 2 + h;
                        bulk_g2s(dst, ahi + ab * (UMMA_A_BYTES / 4), UMMA_A_BYTES, full);
                        bulk_g2s(dst + UMMA_A_BYTES, alo + ab * (UMMA_A_BYTES / 4), UMMA_A_BYTES, full);
                        bulk_g2s(dst + 2 * UMMA_A_BYTES, bhi + bb * (UMMA_B_BYTES / 4), UMMA_B_BYTES, full);
                        bulk_g2s(dst + 2 * UMMA_A_BYTES + UMMA_B_BYTES, blo + bb * (UMMA_B_BYTES / 4), UMMA_B_BYTES,
                                 full);
                    }
            }
            // copies still in flight land before the block exits (already
            // complete on the normal path)
            for (int k = it - 2 < 0 ? 0 : it - 2; k < it; k++) {
                const uint64_t t0 = global_ns();
                while (!mbar_test(b0 + 8 * (k & 1), (k >> 1) & 1) && global_ns() - t0 < UMMA_WAIT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) { // MMAs
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                const UmmaUnit w = umma_unit(u, mt, ctn, nsplit, nkb);
                for (int kb = w.kb0; kb < w.kb1 && ok; kb++)
                    for (int h = 0; h < 2; h++, it++) {
                        const int s = it & 1;
                        if (!umma_wait(b0 + 48 + 8 * s, ((it >> 1) & 1) ^ 1, stop, err, 2) ||
                            !umma_wait(b0 + 8 * s, (it >> 1) & 1, stop, err, 4)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = base + s * UMMA_STAGE;
                        const uint32_t d = tmem + (uint32_t)(s * 256);
#pragma unroll
                        for (int k = 0; k < 4; k++) { // K = 8 TF32 (32 bytes) per MMA
                            const uint64_t ah = umma_desc_sw128(a + 32 * k);
                            const uint64_t al = umma_desc_sw128(a + UMMA_A_BYTES + 32 * k);
                            const uint64_t bh = umma_desc_sw128(a + 2 * UMMA_A_BYTES + 32 * k);
                            const uint64_t bl = umma_desc_sw128(a + 2 * UMMA_A_BYTES + UMMA_B_BYTES + 32 * k);
                            umma_tf32(d, ah, bh, UMMA_IDESC, k > 0);
                            umma_tf32(d, ah, bl, UMMA_IDESC, 1);
                            umma_tf32(d, al, bh, UMMA_IDESC, 1);
                        }
                        umma_commit(b0 + 16 + 8 * s); // shared stage free once these MMAs complete
                        umma_commit(b0 + 32 + 8 * s); // accumulator ready
                    }
            }
            // every MMA this thread issued has completed before tensor memory is freed
            umma_commit(b0 + 64);
            const uint64_t t0 = global_ns();
            while (!mbar_test(b0 + 64, 0) && global_ns() - t0 < UMMA_WAIT_NS) {
            }
        }
    } else { // epilogue: warps 2-9
        const int q = warp & 3, half = (warp - 2) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
        float sum[128];
#pragma unroll
        for (int j = 0; j < 128; j++) sum[j] = 0.f;
        int it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const UmmaUnit w = umma_unit(u, mt, ctn, nsplit, nkb);
            for (int kb = w.kb0; kb < w.kb1 && ok; kb++)
                for (int h = 0; h < 2; h++, it++) {
                    const int s = it & 1;
                    ok = __all_sync(0xffffffffu, umma_wait(b0 + 32 + 8 * s, (it >> 1) & 1, stop, err, 8));
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) {
                        uint32_t r[32];
                        tmem_ld32(tl + (uint32_t)(s * 256 + 32 * cc), r);
#pragma unroll
                        for (int j = 0; j < 32; j++) sum[32 * cc + j] += __uint_as_float(r[j]);
                    }
                    tc_fence_before();
                    mbar_arrive(b0 + 48 + 8 * s);
                }
            if (!ok) break;
            // the unit's partial tile: row w.rt 128 + 32 q + lane, complex
            // columns w.ct 128 + 64 half .. + 63 (accumulator columns in re, im pairs)
            const int row = w.rt * 128 + q * 32 + lane;
            float4 *o = reinterpret_cast<float4 *>(out + (long long)row * C + w.ct * 128 + half * 64);
#pragma unroll
            for (int p = 0; p < 32; p++) {
                atomicAdd(o + p, make_float4(sum[4 * p], sum[4 * p + 1], sum[4 * p + 2], sum[4 * p + 3]));
                sum[4 * p] = sum[4 * p + 1] = sum[4 * p + 2] = sum[4 * p + 3] = 0.f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// Knot ranges per tile: the fewest that keep the grid (one block per SM) at
// least 90% busy, i.e. units / (waves x grid) >= 0.9, without exceeding the
// number of knot blocks.
inline int umma_nsplit(int tiles, int nkb, int nsm)
{
    if (nkb <= 0 || tiles <= 0) return 0;
    for (int ns = 1; ns < nkb; ns++) {
        const long long units = (long long)tiles * ns;
        const long long grid = units < nsm ? units : nsm;
        const long long waves = (units + grid - 1) / grid;
        if (units >= nsm && 10 * units >= 9 * waves * nsm) return ns;
    }
    return nkb;
}

} // namespace bc
