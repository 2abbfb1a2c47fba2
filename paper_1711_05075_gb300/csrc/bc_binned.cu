// Binned spreading fused into the z transform (type-1 NUFFT steps 1 and 2,
// first axis), an alternative to k_spread + k_fft_z that keeps no spreading
// grid in HBM and adds no float atomics.
//
//   k_prepare (with counts)  counts the knots of every bin: (instance, level,
//                            g0_x mod n), g0 the first stencil cell per axis;
//   k_plan_bins              plans each instance (as k_prepare does without bins) and turns its
//                            counts into the first slot of every bin;
//   k_bin                    the 3W separable window weights phi(u_a - g)
//                            (Kaiser-Bessel, as in k_spread) and the stencil
//                            origin of every knot, written as one 128-byte
//                            record into the knot's bin;
//   k_fft_z_binned           per z-transform item (level, x-cell, 32 y-rows):
//                            the knots of the W bins that reach the x-cell are
//                            filtered by their y rows and their (y, z) stencil
//                            columns added into the item's shared-memory tile
//                            (fixed point, integer atomics); the tile is then
//                            transformed along z exactly as k_fft_z does.
//
// The tile holds the values k_spread would have left in the spreading box rows
// of the item, accumulated in fixed point (see k_fft_z_binned), so the
// z-transformed rows equal those of the grid path up to rounding.
#include <climits>
#include <cstdint>

#include "bc_device.cuh"

namespace bc {

// ------------------------------------------------------------------ plan + bin scan
// One block per instance: its plan (thread 0), and cur[b] = knot_off + the
// counts of the bins before b in the instance (bins ordered by level, then
// x-cell); cnt is cleared for the next launch.
constexpr int SCAN_THREADS = 256;

__global__ void __launch_bounds__(SCAN_THREADS)
k_plan_bins(Geometry g, const InstDesc *__restrict__ inst, int *bb, InstPlan *plan, int *err, int *cnt, int *cur)
{
    const int i = blockIdx.x;
    if (threadIdx.x == 0) plan_instance(g, inst, i, bb, plan, err);
    const int nb = g.L * g.n;
    const long long base = (long long)i * nb;
    const int per = (nb + SCAN_THREADS - 1) / SCAN_THREADS;
    const int t0 = threadIdx.x * per;
    int sum = 0;
    for (int k = 0; k < per; k++)
        if (t0 + k < nb) sum += cnt[base + t0 + k];
    __shared__ int wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; k++) before += wsum[k];
    int run = inst[i].knot_off + before + incl - sum;
    for (int k = 0; k < per; k++) {
        const int b = t0 + k;
        if (b >= nb) break;
        const int c = cnt[base + b];
        cur[base + b] = run;
        run += c;
        cnt[base + b] = 0;
    }
}

cudaError_t launch_plan_bins(const Geometry &g, const InstDesc *inst, int ninst, int *bb, InstPlan *plan, int *err,
                             int *cnt, int *cur, cudaStream_t s)
{
    if (ninst <= 0) return cudaSuccess;
    k_plan_bins<<<ninst, SCAN_THREADS, 0, s>>>(g, inst, bb, plan, err, cnt, cur);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ knot records
// Record of a knot (BIN_REC floats): [0] g0_y, [1] g0_z (int bits, the first
// stencil cell, g0 = ceil(u - W/2)), [2 + a W + t] = phi(u_a - (g0_a + t)) for
// axis a (x, y, z) and t < W.  Each warp takes 32 knots: lane j claims a slot
// for knot j, then the warp writes the 32 records one by one, lane l writing
// float l.
constexpr int BIN_WARPS = 8;

__global__ void __launch_bounds__(BIN_WARPS * 32)
k_bin(Geometry g, const float *__restrict__ consts, const float4 *__restrict__ ku, const InstPlan *__restrict__ plan,
      int *cur, float *rec, int total)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = g.W, L = g.L, n = g.n;
    const float halfW = 0.5f * (float)W, xoff = 0.5f * (float)W - 1.f;
    const int a = lane < 2 ? 0 : (lane - 2) / W, t = lane < 2 ? 0 : (lane - 2) - a * W; // this lane's weight
    float kc[KB_NC];
    kb_load(consts, lane >= 2 && lane - 2 < 3 * W ? t : 0, kc);
    for (int base = (blockIdx.x * BIN_WARPS + wib) * 32; base < total; base += gridDim.x * BIN_WARPS * 32) {
        const int k = base + lane;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        int slot = -1;
        if (k < total) {
            v = ku[k];
            const int tag = __float_as_int(v.w);
            const int level = tag & 15, i = tag >> 4;
            if (plan[i].b[0] != 0) { // instances dropped by their plan are skipped by the z pass too
                const int gx = (int)ceilf(v.x - halfW);
                slot = atomicAdd(&cur[((long long)i * L + level) * n + (gx < 0 ? gx + n : gx)], 1);
            }
        }
        for (int j = 0; j < 32; j++) {
            const int sj = __shfl_sync(0xffffffffu, slot, j);
            const float ux = __shfl_sync(0xffffffffu, v.x, j), uy = __shfl_sync(0xffffffffu, v.y, j),
                        uz = __shfl_sync(0xffffffffu, v.z, j);
            if (sj < 0) continue;
            const int gx = (int)ceilf(ux - halfW), gy = (int)ceilf(uy - halfW), gz = (int)ceilf(uz - halfW);
            float val = 0.f;
            if (lane == 0) {
                val = __int_as_float(gy);
            } else if (lane == 1) {
                val = __int_as_float(gz);
            } else if (lane - 2 < 3 * W) {
                const float ua = a == 0 ? ux : (a == 1 ? uy : uz);
                const int ga = a == 0 ? gx : (a == 1 ? gy : gz);
                val = kb_poly(kc, (ua - (float)ga) - xoff);
            }
            rec[(long long)sj * BIN_REC + lane] = val;
        }
    }
}

cudaError_t launch_bin(const Geometry &g, const Tables &t, const InstDesc *inst, int total_knots, const float4 *ku,
                       const InstPlan *plan, int *cur, float *rec, cudaStream_t s)
{
    (void)inst;
    if (total_knots <= 0) return cudaSuccess;
    int blocks = (total_knots + BIN_WARPS * 32 - 1) / (BIN_WARPS * 32);
    if (blocks > 65535) blocks = 65535;
    k_bin<<<blocks, BIN_WARPS * 32, 0, s>>>(g, t.consts, ku, plan, cur, rec, total_knots);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fused spread + fft z
// Item: (level l, compact x-cell ix, 32 compact y-rows iy0 ..), as in k_fft_z.
// Tile: 32 rows per z position (the interleaved complex layout [pos][16
// lines], rows 2q / 2q + 1 in the real / imaginary part of line q), z
// position = absolute cell mod n.
//
// The knots reaching x-cell xa = (lo_x + ix) mod n are those of bins xa - dx
// (mod n), dx < W, with x-weight index dx.  A knot adds
// phi_x[dx] phi_y[dy] phi_z[dz] at row (g0_y + dy - lo_y) mod n - iy0 (when in
// [0, 32)) and position (g0_z + dz) mod n.  The scanned knots go, in chunks of
// TB, through a shared hit list (appended with warp-aggregated atomics); each
// hit is spread by W threads, one per y offset, each adding its W z-cells.
//
// The tile accumulates in 32-bit fixed point with integer shared-memory
// atomics: every contribution lies in [0, 1] and a cell receives at most one
// contribution per scanned knot, so with 2^s = 2^30 / 2^ceil(log2(T + 1)) for
// T scanned knots no sum can overflow; each contribution is rounded to the
// nearest multiple of 2^-s (error <= 2^-(s+1), 2^-22 for T = 255) and the
// integer sums do not depend on the order of the additions.  The first
// transform stage reads the tile back as FP32 (value = sum 2^-s).
template <int NF, bool SP, int S>
__global__ void __launch_bounds__(TB, (NF <= 256 ? 2 : 1))
k_fft_z_binned(Geometry g, Tables tb, const InstDesc *__restrict__ inst, int ninst, const InstPlan *__restrict__ plan,
               const int *__restrict__ cur, const float *__restrict__ rec, float2 *z1)
{
    constexpr bool three = Radix<NF, S>::r2 > 1;
    constexpr int H = NF / 4; // kept z modes (N/2, n = 2N)
    extern __shared__ float4 sm4[];
    float2 *tw = reinterpret_cast<float2 *>(sm4);
    float2 *S0 = tw + NF, *S1 = S0 + NF * CL;
    float2 *OUT = three ? S0 : S1; // tile the last stage writes (not the one it reads)
    float2 *STG = three ? S1 : S0; // staging for the output rows
    int *X = reinterpret_cast<int *>(S1); // fixed-point tile [pos][32 rows]
    int *hslot = reinterpret_cast<int *>(S1 + NF * CL);
    int *hinfo = hslot + TB;
    __shared__ int bst[MAX_W], bpre[MAX_W + 1], nhit[2];
    load_twiddles<NF>(tw, tb.tw_n);
    if (threadIdx.x < 2) nhit[threadIdx.x] = 0;
    const int L = g.L, W = g.W;
    const unsigned magicW = 0xFFFFFFFFu / (unsigned)W + 1u; // e / W = umulhi(e, magicW) for e < 2^16
    const int lane = threadIdx.x & 31;
    FirstInputs<NF, Radix<NF, S>::r0, CL, TB> in;
    RotStart rs;
    int chunk = 0;
    for (int i = 0; i < ninst; i++) {
        const InstPlan p = plan[i];
        if (p.b[0] == 0) continue;
        const int b0 = p.b[0], b1 = p.b[1];
        const int nyb = (b1 + 31) >> 5;
        const int items = L * b0 * nyb;
        const int koff = inst[i].knot_off;
        float2 *zbase = z1 + inst[i].z1_off;
        for (int it = rs.first(); it < items; it += gridDim.x) {
            const int l = it / (b0 * nyb), rem = it - l * (b0 * nyb);
            const int ix = rem / nyb, iy0 = (rem - ix * nyb) << 5;
            for (int e = threadIdx.x; e < NF * 8; e += TB) reinterpret_cast<int4 *>(X)[e] = make_int4(0, 0, 0, 0);
            if (threadIdx.x < W) {
                int xa = p.lo[0] + ix;
                if (xa < 0) xa += NF;
                if (xa >= NF) xa -= NF;
                int b = xa - (int)threadIdx.x;
                if (b < 0) b += NF;
                const long long bin = ((long long)i * L + l) * NF + b;
                const int s0 = (l == 0 && b == 0) ? koff : cur[bin - 1];
                bst[threadIdx.x] = s0;
                bpre[threadIdx.x + 1] = cur[bin] - s0;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                bpre[0] = 0;
                for (int k = 1; k <= W; k++) bpre[k] += bpre[k - 1];
            }
            __syncthreads();
            const int total = bpre[W];
            const int sh = 30 - (32 - __clz(total)); // 2^sh * total < 2^30
            const float scale = ldexpf(1.f, sh);
            for (int base = 0; base < total; base += TB) {
                const int k = base + (int)threadIdx.x;
                bool hit = false;
                int slot = 0, info = 0;
                if (k < total) {
                    int dx = 0;
                    while (k >= bpre[dx + 1]) dx++;
                    slot = bst[dx] + (k - bpre[dx]);
                    int iy = __float_as_int(rec[(long long)slot * BIN_REC]) - p.lo[1];
                    if (iy >= NF) iy -= NF;
                    int rel = iy - iy0;
                    if (rel < 0) rel += NF;
                    hit = rel < 32 || rel > NF - W; // rows rel .. rel + W - 1 (mod n) meet [0, 32)
                    info = dx | (rel << 4);
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                int wbase = 0;
                if (lane == 0 && m) wbase = atomicAdd(&nhit[chunk & 1], __popc(m));
                wbase = __shfl_sync(0xffffffffu, wbase, 0);
                if (hit) {
                    const int q = wbase + __popc(m & ((1u << lane) - 1u));
                    hslot[q] = slot;
                    hinfo[q] = info;
                }
                __syncthreads();
                const int nh = nhit[chunk & 1];
                if (threadIdx.x == 0) nhit[(chunk + 1) & 1] = 0; // counter of the next chunk (its readers are done)
                for (int e = threadIdx.x; e < nh * W; e += TB) {
                    const int h = (int)__umulhi((unsigned)e, magicW);
                    const int dy = e - h * W;
                    const int inf = hinfo[h];
                    int row = (inf >> 4) + dy;
                    if (row >= NF) row -= NF;
                    if (row < 32) {
                        const float *R = rec + (long long)hslot[h] * BIN_REC;
                        const float cxy = R[2 + (inf & 15)] * R[2 + W + dy] * scale;
                        const float *wz = R + 2 + 2 * W;
                        int pos = __float_as_int(R[1]);
                        if (pos < 0) pos += NF;
                        for (int dz = 0; dz < W; dz++) {
                            atomicAdd(&X[pos * 32 + row], __float2int_rn(cxy * wz[dz]));
                            if (++pos == NF) pos = 0;
                        }
                    }
                }
                __syncthreads();
                chunk++;
            }
            __syncthreads();
            const float inv_scale = ldexpf(1.f, -sh);
            in.load([&](int c, int pos) {
                const int2 v = reinterpret_cast<const int2 *>(X)[pos * CL + c];
                return make_float2((float)v.x * inv_scale, (float)v.y * inv_scale);
            });
            __syncthreads(); // the tile is in registers; S1 is free for the transform
            if constexpr (SP) in.scatter(S0);
            else rr_first<NF, Radix<NF, S>::r0, false, CL, TB>(in, S0);
            __syncthreads();
            auto sink = [&](int, int, int c, int pos, float2 v) { OUT[pos * CL + c] = v; };
            if constexpr (SP) sp_all<NF, false, CL, TB, S>(S0, S1, tw, sink);
            else rr_rest<NF, false, CL, TB, S>(S0, S1, tw, sink);
            __syncthreads();
            // Z = FFT(a + i b) -> A_k = (Z_k + conj Z_{n-k}) / 2, B_k = (Z_k - conj Z_{n-k}) / (2i),
            // unpacked into a staging area [row][k] (row stride H + 1), then each
            // 8H-byte row of z1 written with consecutive threads on consecutive k
            for (int e = threadIdx.x; e < 32 * H; e += TB) {
                const int r = e & 31, kk = e >> 5;
                const int qq = r >> 1;
                const float2 zk = OUT[kk * CL + qq];
                const float2 zn = OUT[(kk == 0 ? 0 : NF - kk) * CL + qq];
                STG[r * (H + 1) + kk] = (r & 1) ? make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x))
                                                : make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            }
            __syncthreads();
            float2 *Z = zbase + (((long long)l * b0 + ix) * b1 + iy0) * H;
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

template <int NF, bool SP = false, int S = 0>
static cudaError_t fft_z_binned_t(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                                  const InstPlan *plan, const int *cur, const float *rec, float2 *z1, int nsm,
                                  cudaStream_t s)
{
    if (!SP && S == 0 && (g.sched & 1)) return fft_z_binned_t<NF, false, 1>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    const size_t smem = sizeof(float2) * (NF + 2 * NF * CL) + sizeof(int) * 2 * TB;
    cudaError_t e = set_smem(k_fft_z_binned<NF, SP, S>, smem);
    if (e != cudaSuccess) return e;
    k_fft_z_binned<NF, SP, S><<<resident_blocks(k_fft_z_binned<NF, SP, S>, smem, nsm), TB, smem, s>>>(
        g, t, inst, ninst, plan, cur, rec, z1);
    return cudaGetLastError();
}

cudaError_t launch_fft_z_binned(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                                const InstPlan *plan, const int *cur, const float *rec, float2 *z1, int nsm,
                                cudaStream_t s)
{
    if (g.W > MAX_W || 2 + 3 * g.W > BIN_REC) return cudaErrorInvalidValue;
    if (g.prec == 1) {
        switch (g.n) {
        case 64: return fft_z_binned_t<64, true>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
        case 128: return fft_z_binned_t<128, true>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
        case 192: return fft_z_binned_t<192, true>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
        case 256: return fft_z_binned_t<256, true, SplitSched<256>::S>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
        case 512: return fft_z_binned_t<512, true>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (g.n) {
    case 64: return fft_z_binned_t<64>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    case 128: return fft_z_binned_t<128>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    case 192: return fft_z_binned_t<192>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    case 256: return fft_z_binned_t<256>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    case 512: return fft_z_binned_t<512>(g, t, inst, ninst, plan, cur, rec, z1, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
