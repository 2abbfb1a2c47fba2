// Type-1 NUFFT step 2, first axis (the z transform of k_fft_z), as a pruned
// DFT on the 5th-generation tensor cores.
//
// Each z line of a support box holds at most bz nonzero cells, compact index
// iz at line position (pos0_z + iz) mod n, and only m_z in [0, N/2) is kept.
// Splitting iz = 32 j + e (chunks of 32 cells),
//     Z[m] = sum_j exp(-2 pi i m (pos0_z + 32 j) / n) D_j[m],
//     D_j[m] = sum_{e < 32} x[32 j + e] exp(-2 pi i m e / n),
// and D_j for 128 lines at once is a real matrix product: the lines' 32 cells
// (rows) times one fixed 32-cell DFT block B (row 2m: cos(2 pi m e / n), row
// 2m + 1: -sin), whose accumulator row is (Re D_j[m], Im D_j[m]),
// m = 0 .. N/2 - 1.  B stays resident in shared memory; each chunk's product
// is turned by its phase and summed in FP32 registers.  3-pass split TF32
// (x = x_hi + x_lo; a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32 accumulation of
// one chunk (the tensor cores truncate when they accumulate, so no
// accumulator spans more than one chunk's 12 MMAs).  The result is the z
// transform k_fft_z computes, in the same layout (z1 rows [level][ix][iy] of
// N/2 complex modes), and the boxes are left cleared as k_fft_z leaves them.
//
// Roles (448 threads, one block per SM; tiles of 4 box items = 128 lines):
//   warp 0, lane 0   the resident B block, then per chunk the tile's box cells
//                    (per item one contiguous run of up to 32 x 128 bytes)
//                    into a four-deep raw ring (bulk copies);
//   warp 1           allocates tensor memory; lane 0 issues tcgen05.mma
//                    (M = 128, N = N, K = 8; 12 per chunk) into one of two
//                    accumulators (chunk k of the block's sequence: operand
//                    stage k mod 3, accumulator k mod 2);
//   warps 2-5        one line per thread: split the raw cells to TF32 hi / lo
//                    into the 128-byte-swizzled K-major layout, then clear the
//                    copied cells in the box (coalesced 16-byte stores; bulk
//                    copies from a zeroed shared buffer, issued by the copy
//                    thread, measured slower: they delay the raw copies);
//   warps 6-13       one line and half of the modes each (tensor-memory lanes
//                    32 (w mod 4) .., columns of half (w - 6) / 4): add each
//                    chunk's accumulator, turned by its phase, into FP32 running
//                    sums; after the tile's last chunk the sums are parked in a
//                    third tensor-memory region and written out one 64-byte
//                    row piece per pass after each chunk of the next tile (the
//                    whole tile at once stalled the next tile's first chunk),
//                    through a shared-memory staging area: 8 lines x 64
//                    contiguous bytes per store instruction (a line per thread
//                    would scatter every store over 32 half-filled sectors).
// Every mbarrier wait is bounded (about 2 s); on expiry the block sets bit 8 of
// the context's error word, stops, waits (bounded) for its copies and MMAs in
// flight and frees its tensor memory.
#include <cstdint>

#include "bc_device.cuh"
#include "bc_umma.cuh"

namespace bc {

constexpr int ZU_THREADS = 448; // 14 warps
constexpr int ZU_ERR = 8; // error-word bit of a stalled tensor-core transform pass

template <int NF>
struct ZU {
    static constexpr int H = NF / 4;  // kept z modes (N / 2)
    static constexpr int NC = NF / 2; // accumulator columns: (re, im) per mode
    static constexpr int A_BYTES = 128 * 128;
    static constexpr int B_BYTES = NC * 128;
    static constexpr int OPD = 3, RAWD = 4;                   // operand and raw ring depths
    static constexpr int RAW = 4 * 32 * 128;                  // raw stage: 4 items x 32 cells x 32 lines
    static constexpr int STG = 32 * 80;                       // output staging per epilogue warp: 32 rows x 64 B (+16)
    static constexpr int SMEM = 2 * B_BYTES + OPD * 2 * A_BYTES + RAWD * RAW + 8 * STG + 1024 + 256 + NF * 8;
    static constexpr int TMEM_COLS = 3 * NC <= 128 ? 128 : 3 * NC <= 256 ? 256 : 512; // 2 accumulators + parked sums
    static constexpr uint32_t IDESC = umma_idesc_tf32(NC);
    static_assert(NC % 32 == 0 && NC <= 128, "accumulator width");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// The 32-cell DFT block: rows R < NF / 2, row 2m + c is cos (c = 0) or -sin
// (c = 1) of 2 pi m e / NF, e < 32; FP64 (the angle reduced exactly as m e mod
// NF), rounded once to FP32, split into TF32 hi and lo.
__global__ void k_build_zdft(int NF, float *bhi, float *blo)
{
    const int NC = NF / 2;
    const int total = NC * 32;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        const int R = u >> 5, e = u & 31, m = R >> 1;
        const int k = (m * e) % NF;
        double sn, cs;
        sincospi(2.0 * k / NF, &sn, &cs);
        const float v = (R & 1) ? (float)(-sn) : (float)cs;
        const float hi = tf32_round(v);
        const int o = umma_swz(R, e);
        bhi[o] = hi;
        blo[o] = v - hi;
    }
}

// The stage sequence every role walks: instances in order, each block's tiles
// of an instance (RotStart spreads them), each tile's K-blocks.
struct ZuWalk {
    int b0, b1, bz, pz, nyb, items, tiles, nkz;
    __device__ __forceinline__ bool load(const InstPlan &p, int L)
    {
        if (p.b[0] == 0) return false;
        b0 = p.b[0];
        b1 = p.b[1];
        bz = p.b[2];
        pz = p.pos0[2];
        nyb = (b1 + 31) >> 5;
        items = L * b0 * nyb;
        tiles = (items + 3) >> 2;
        nkz = (bz + 31) >> 5;
        return true;
    }
};

template <int NF>
__global__ void __launch_bounds__(ZU_THREADS, 1)
k_fft_z_umma(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
             float *grid, float2 *z1, const float *__restrict__ bhi, const float *__restrict__ blo, int *err)
{
    using Z = ZU<NF>;
    constexpr int H = Z::H, NC = Z::NC, OPD = Z::OPD, RAWD = Z::RAWD;
    extern __shared__ uint8_t zu_raw[];
    const uint32_t raw = smem_addr(zu_raw);
    const uint32_t base = (raw + 1023u) & ~1023u; // the swizzle pattern repeats every 1024 bytes
    uint8_t *gbase = zu_raw + (base - raw);
    // [B hi | B lo] [operand stages: A hi | A lo] x OPD [raw stages] x RAWD [barriers] [twiddles]
    const uint32_t bres = base, abase = base + 2 * Z::B_BYTES, rbase = abase + OPD * 2 * Z::A_BYTES;
    uint8_t *ga = gbase + 2 * Z::B_BYTES;
    const float *rawf = reinterpret_cast<const float *>(gbase + (rbase - base));
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (rbase - base) + RAWD * Z::RAW);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 20);
    volatile int *stop = reinterpret_cast<volatile int *>(slot + 1);
    float2 *tw = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(bars) + 256);
    uint8_t *stg_all = reinterpret_cast<uint8_t *>(bars) + 256 + NF * 8; // epilogue output staging
    const uint32_t bar0 = smem_addr(bars);
    // full[s], empty[s] (operand stages); rfull[k], rempty[k] (raw ring);
    // acc_full[b], acc_empty[b] (accumulators); B resident; drain
    const uint32_t FULL = bar0, EMPTY = bar0 + 24, RFULL = bar0 + 48, REMPTY = bar0 + 80, ACCF = bar0 + 112,
                   ACCE = bar0 + 128, BREADY = bar0 + 144, DRAIN = bar0 + 152;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < OPD; s++) {
            mbar_init(FULL + 8 * s, 128); // converter arrivals
            mbar_init(EMPTY + 8 * s, 1); // MMA commit
        }
        for (int k = 0; k < RAWD; k++) {
            mbar_init(RFULL + 8 * k, 1);   // the copy thread's arrival (+ the cells' bytes)
            mbar_init(REMPTY + 8 * k, 128); // converter arrivals
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(ACCF + 8 * b, 1);   // MMA commit
            mbar_init(ACCE + 8 * b, 256); // epilogue arrivals
        }
        mbar_init(BREADY, 1);
        mbar_init(DRAIN, 1);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = threadIdx.x; k < NF; k += blockDim.x) tw[k] = tb.tw_n[k];
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(Z::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    pdl_signal();
    pdl_wait(); // the spreading boxes and plans are read from here on
    const int L = g.L;
    ZuWalk w;

    if (warp == 0) {
        if (lane == 0) { // the B block, then box cells of each chunk into the raw ring
            mbar_expect_tx(BREADY, 2 * Z::B_BYTES);
            bulk_g2s(bres, bhi, Z::B_BYTES, BREADY);
            bulk_g2s(bres + Z::B_BYTES, blo, Z::B_BYTES, BREADY);
            int it = 0;
            bool ok = true;
            RotStart rs;
            for (int i = 0; i < ninst && ok; i++) {
                if (!w.load(plan[i], L)) continue;
                const float *G = grid + inst[i].grid_off;
                for (int t = rs.first(); t < w.tiles && ok; t += gridDim.x) {
                    const int nq = min(4, w.items - 4 * t);
                    for (int kz = 0; kz < w.nkz; kz++, it++) {
                        const int k = it % RAWD;
                        if (!umma_wait(REMPTY + 8 * k, ((it / RAWD) & 1) ^ 1, stop, err, ZU_ERR)) {
                            ok = false;
                            break;
                        }
                        const int len = min(32, w.bz - 32 * kz); // cells of this chunk
                        mbar_expect_tx(RFULL + 8 * k, (uint32_t)(nq * len * 128));
                        for (int q = 0; q < nq; q++)
                            bulk_g2s(rbase + k * Z::RAW + q * 4096,
                                     G + ((long long)(4 * t + q) * w.bz + 32 * kz) * 32, (uint32_t)(len * 128),
                                     RFULL + 8 * k);
                    }
                }
                rs.rot += w.tiles;
            }
            // copies still in flight land before the block exits (already
            // complete on the normal path)
            {
                const uint64_t t0 = global_ns();
                while (!mbar_test(BREADY, 0) && global_ns() - t0 < UMMA_WAIT_NS) {
                }
            }
            for (int k = it - RAWD < 0 ? 0 : it - RAWD; k < it; k++) {
                const uint64_t t0 = global_ns();
                while (!mbar_test(RFULL + 8 * (k % RAWD), (k / RAWD) & 1) && global_ns() - t0 < UMMA_WAIT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) { // MMAs
            int it = 0;
            bool ok = umma_wait(BREADY, 0, stop, err, ZU_ERR);
            const uint64_t bh0 = umma_desc_sw128(bres), bl0 = umma_desc_sw128(bres + Z::B_BYTES);
            RotStart rs;
            for (int i = 0; i < ninst && ok; i++) {
                if (!w.load(plan[i], L)) continue;
                for (int t = rs.first(); t < w.tiles && ok; t += gridDim.x)
                    for (int kz = 0; kz < w.nkz; kz++, it++) {
                        const int s = it % OPD, b = it & 1;
                        if (!umma_wait(ACCE + 8 * b, ((it >> 1) & 1) ^ 1, stop, err, ZU_ERR) ||
                            !umma_wait(FULL + 8 * s, (it / OPD) & 1, stop, err, ZU_ERR)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = abase + s * 2 * Z::A_BYTES;
                        const uint32_t d = tmem + (uint32_t)(b * NC);
#pragma unroll
                        for (int k = 0; k < 4; k++) { // K = 8 TF32 (32 bytes) per MMA; +2 in the descriptor
                            const uint64_t ah = umma_desc_sw128(a + 32 * k);
                            const uint64_t al = umma_desc_sw128(a + Z::A_BYTES + 32 * k);
                            umma_tf32(d, ah, bh0 + 2 * k, Z::IDESC, k > 0);
                            umma_tf32(d, ah, bl0 + 2 * k, Z::IDESC, 1);
                            umma_tf32(d, al, bh0 + 2 * k, Z::IDESC, 1);
                        }
                        umma_commit(EMPTY + 8 * s); // operand stage free once these MMAs complete
                        umma_commit(ACCF + 8 * b);  // accumulator ready
                    }
                rs.rot += w.tiles;
            }
            umma_commit(DRAIN); // every MMA issued has completed before tensor memory is freed
            const uint64_t t0 = global_ns();
            while (!mbar_test(DRAIN, 0) && global_ns() - t0 < UMMA_WAIT_NS) {
            }
        }
    } else if (warp < 6) { // converters: line r of the tile
        const int r = threadIdx.x - 64, q = r >> 5;
        int it = 0;
        bool ok = true;
        RotStart rs;
        for (int i = 0; i < ninst && ok; i++) {
            if (!w.load(plan[i], L)) continue;
            float *G = grid + inst[i].grid_off;
            for (int t = rs.first(); t < w.tiles && ok; t += gridDim.x) {
                const int nq = min(4, w.items - 4 * t);
                const bool valid = q < nq;
                for (int kz = 0; kz < w.nkz; kz++, it++) {
                    const int s = it % OPD, k = it % RAWD;
                    if (!umma_wait(RFULL + 8 * k, (it / RAWD) & 1, stop, err, ZU_ERR)) {
                        ok = false;
                        break;
                    }
                    const int len = min(32, w.bz - 32 * kz);
                    const float *src = rawf + (k * Z::RAW + q * 4096) / 4 + (r & 31);
                    float v[32];
#pragma unroll
                    for (int e = 0; e < 32; e++) v[e] = (valid && e < len) ? src[e * 32] : 0.f;
                    if (!umma_wait(EMPTY + 8 * s, ((it / OPD) & 1) ^ 1, stop, err, ZU_ERR)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = ga + s * 2 * Z::A_BYTES + r * 128;
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        float4 hi, lo;
                        hi.x = tf32_round(v[4 * j]);
                        hi.y = tf32_round(v[4 * j + 1]);
                        hi.z = tf32_round(v[4 * j + 2]);
                        hi.w = tf32_round(v[4 * j + 3]);
                        lo = make_float4(v[4 * j] - hi.x, v[4 * j + 1] - hi.y, v[4 * j + 2] - hi.z, v[4 * j + 3] - hi.w);
                        const int off = (j ^ (r & 7)) << 4;
                        *reinterpret_cast<float4 *>(sa + off) = hi;
                        *reinterpret_cast<float4 *>(sa + Z::A_BYTES + off) = lo;
                    }
                    fence_proxy_async_smem(); // the operand stores are visible to the tensor core's reads
                    mbar_arrive(FULL + 8 * s);
                    // the raw slot is released only after its values have been used (stored
                    // above): a release right after issuing the loads let the next bulk copy
                    // into the slot overtake loads still in flight
                    mbar_arrive(REMPTY + 8 * k);
                    // the copied cells are read: clear them in the box (boxes are left clear)
                    for (int qq = 0; qq < nq; qq++) {
                        float4 *dst = reinterpret_cast<float4 *>(G + ((long long)(4 * t + qq) * w.bz + 32 * kz) * 32);
                        for (int j = r; j < len * 8; j += 128) dst[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            rs.rot += w.tiles;
        }
    } else { // epilogue: line 32 (warp mod 4) + lane of the tile, modes of half (warp - 6) / 4
        constexpr int HC = NC / 2;   // accumulator columns per half
        constexpr int HM = H / 2;    // modes per half
        constexpr int PASSES = HM / 8; // 64-byte row pieces per half line
        const int q = warp & 3, half = (warp - 6) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * HC);
        const uint32_t tpark = tl + (uint32_t)(2 * NC); // parked sums of the previous tile
        float4 *stg = reinterpret_cast<float4 *>(stg_all + (warp - 6) * Z::STG); // [row][5] float4
        // the parked tile: its first z row for this warp's item (null: none), rows, passes written
        float4 *pk_out = nullptr;
        int pk_rows = 0, pk_done = PASSES;
        // writes pass p of the parked tile: 32 rows x 64 bytes through the staging area
        auto emit = [&](int p) {
            uint32_t v[16];
            tmem_ld16(tpark + (uint32_t)(16 * p), v);
#pragma unroll
            for (int c4 = 0; c4 < 4; c4++)
                stg[lane * 5 + c4] = make_float4(__uint_as_float(v[4 * c4]), __uint_as_float(v[4 * c4 + 1]),
                                                 __uint_as_float(v[4 * c4 + 2]), __uint_as_float(v[4 * c4 + 3]));
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int row = (lane >> 2) + 8 * k, c4 = lane & 3;
                if (row < pk_rows) pk_out[(long long)row * (H / 2) + 4 * p + c4] = stg[row * 5 + c4];
            }
            __syncwarp();
        };
        float sum[HC];
#pragma unroll
        for (int j = 0; j < HC; j++) sum[j] = 0.f;
        int it = 0;
        bool ok = true;
        RotStart rs;
        for (int i = 0; i < ninst && ok; i++) {
            if (!w.load(plan[i], L)) continue;
            const long long zoff = inst[i].z1_off;
            for (int t = rs.first(); t < w.tiles && ok; t += gridDim.x) {
                for (int kz = 0; kz < w.nkz; kz++, it++) {
                    const int b = it & 1;
                    ok = __all_sync(0xffffffffu, umma_wait(ACCF + 8 * b, (it >> 1) & 1, stop, err, ZU_ERR));
                    if (!ok) break;
                    tc_fence_after();
                    const int p0 = w.pz + 32 * kz; // the chunk's first line position
#pragma unroll
                    for (int cc = 0; cc < HC / 16; cc++) {
                        uint32_t v[16];
                        tmem_ld16(tl + (uint32_t)(b * NC + 16 * cc), v);
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const int mm = 8 * cc + j, m = half * HM + mm; // local and global mode
                            const float2 ph = tw[(m * p0) % NF];
                            const float re = __uint_as_float(v[2 * j]), im = __uint_as_float(v[2 * j + 1]);
                            sum[2 * mm] = fmaf(re, ph.x, fmaf(-im, ph.y, sum[2 * mm]));
                            sum[2 * mm + 1] = fmaf(re, ph.y, fmaf(im, ph.x, sum[2 * mm + 1]));
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(ACCE + 8 * b);
                    // part of the parked tile goes out after each chunk: all of it by this tile's last chunk
                    const int upto = kz == w.nkz - 1 ? PASSES : min(PASSES, pk_done + (PASSES + w.nkz - 1) / w.nkz);
                    if (pk_out)
                        for (; pk_done < upto; pk_done++) emit(pk_done);
                    pk_done = upto;
                }
                if (!ok) break;
                // park this tile's sums (the previous tile is fully written by now)
#pragma unroll
                for (int cc = 0; cc < HC / 16; cc++) {
                    uint32_t v[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = __float_as_uint(sum[16 * cc + j]);
                    tmem_st16(tpark + (uint32_t)(16 * cc), v);
                }
                tmem_wait_st();
                const int item = 4 * t + q; // the warp's 32 lines are the rows of one item
                pk_out = nullptr;
                pk_rows = 0;
                if (item < w.items) {
                    const int l = item / (w.b0 * w.nyb), rem = item - l * (w.b0 * w.nyb);
                    const int ix = rem / w.nyb, iy0 = (rem - ix * w.nyb) << 5;
                    pk_out = reinterpret_cast<float4 *>(z1 + zoff + ((long long)(l * w.b0 + ix) * w.b1 + iy0) * H +
                                                        half * HM);
                    pk_rows = min(32, w.b1 - iy0);
                }
                pk_done = 0;
#pragma unroll
                for (int j = 0; j < HC; j++) sum[j] = 0.f;
            }
            rs.rot += w.tiles;
        }
        if (ok && pk_out)
            for (; pk_done < PASSES; pk_done++) emit(pk_done); // the last parked tile
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Z::TMEM_COLS)
                     : "memory");
    }
}

template <int NF>
static cudaError_t fft_z_umma_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                                const InstPlan *plan, float *grid, float2 *z1, const float *bhi, const float *blo,
                                int *err, int nsm, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_fft_z_umma<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, ZU<NF>::SMEM);
    if (e != cudaSuccess) return e;
    return launch_k(k_fft_z_umma<NF>, nsm, ZU_THREADS, ZU<NF>::SMEM, s, g.pdl != 0, g, t, inst, ninst, plan, grid, z1,
                    bhi, blo, err);
}

// Self-test of the bounded wait the tensor-core kernels use: one thread waits
// on an mbarrier that nothing arrives at; the wait gives up after
// UMMA_WAIT_NS and sets bit ZU_ERR of *err, and the kernel returns.
__global__ void k_wait_selftest(int *err)
{
    __shared__ uint64_t bar;
    __shared__ int stop;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) umma_wait(smem_addr(&bar), 0, &stop, err, ZU_ERR);
}

cudaError_t launch_wait_selftest(int *err, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

bool supported_z_umma(int N) { return N == 32 || N == 64 || N == 96 || N == 128; }

cudaError_t launch_build_zdft(int n, float *bhi, float *blo, cudaStream_t s)
{
    const int total = (n / 2) * 32;
    k_build_zdft<<<(total + 255) / 256, 256, 0, s>>>(n, bhi, blo);
    return cudaGetLastError();
}

cudaError_t launch_fft_z_umma(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                              const InstPlan *plan, float *grid, float2 *z1, const float *bhi, const float *blo,
                              int *err, int nsm, cudaStream_t s)
{
    switch (g.n) {
    case 64: return fft_z_umma_t<64>(g, t, inst, ninst, plan, grid, z1, bhi, blo, err, nsm, s);
    case 128: return fft_z_umma_t<128>(g, t, inst, ninst, plan, grid, z1, bhi, blo, err, nsm, s);
    case 192: return fft_z_umma_t<192>(g, t, inst, ninst, plan, grid, z1, bhi, blo, err, nsm, s);
    case 256: return fft_z_umma_t<256>(g, t, inst, ninst, plan, grid, z1, bhi, blo, err, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
