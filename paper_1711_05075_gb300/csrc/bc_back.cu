// The back half of a correlation pass in one persistent launch: the x pass
// (forward x transforms of both spectra with the window deconvolution, ball
// transforms and level sum of Eq. (fballhat), the conjugate product of
// Eq. (ccghat), the inverse x transform), the inverse y pass and the inverse z
// pass onto the translation grid, for every pair of the pass.
//
// Work units, in this order in one device queue:
//   X  (pair, chunk ch of 16 z-modes, row j_y)      npairs * N * N/32
//   IY (pair, chunk ch, plane k_x)                  npairs * N * N/32
//   IZ (pair, plane k_x, block of 32 rows k_y)      npairs * N * N/32
// Every block of the (resident-sized) grid claims units with one atomic
// counter, one unit ahead, and runs them.  Dependencies are counted per
// (pair, ch) for X -> IY (all N rows j_y of the chunk) and per (pair, k_x) for
// IY -> IZ (all chunks of the plane); a unit waits (bounded, by %globaltimer)
// for its count, then runs.  Units are claimed in increasing order and a unit
// only waits on units before it, each of which was claimed by a running block
// that does not wait on anything after it, so every wait ends.  A wait that
// still runs out after two seconds sets bit 4 of the status word (reported as
// BC_ERR_TIMEOUT) and the block goes on, so no block is left spinning.
//
// What this buys over three launches: the last wave of the x pass (512 units
// of a 128^3 pair over 304 resident blocks is 1.68 waves) is filled with the
// inverse-y units of the chunks already complete, and the launch gaps and
// ramp-ups between the three passes disappear.  Data produced inside the
// launch (the half-spectrum planes) is read through L2 (ld.global.cg).
#include <cstdint>

#include "bc_passes.cuh"

namespace bc {

namespace {

constexpr int BACK_ERR = 16;                          // status-word bit of an expired dependency wait
constexpr unsigned long long BACK_WAIT_NS = 2000000000ull; // two seconds

__device__ __forceinline__ unsigned long long back_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until *c reaches `target` (at most BACK_WAIT_NS, and a bounded
// number of polls); then the whole block proceeds.
__device__ __forceinline__ void wait_count(const unsigned *c, unsigned target, int *err)
{
    if (threadIdx.x == 0 && ld_acquire_u32(c) < target) {
        const unsigned long long t0 = back_ns();
        bool ok = false;
        for (long long it = 0; it < (1ll << 32); it++) {
            __nanosleep(128);
            if (ld_acquire_u32(c) >= target) {
                ok = true;
                break;
            }
            if (back_ns() - t0 > BACK_WAIT_NS) break;
        }
        if (!ok) atomicOr(err, BACK_ERR);
    }
    __syncthreads();
}

// The block's stores of the unit are visible (device scope) before the count moves.
__device__ __forceinline__ void signal_done(unsigned *c)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c, 1u);
    }
}

// Inverse y transform of plane k_x, chunk ch, in place on the half-spectrum planes.
template <int NI>
__device__ __forceinline__ void iy_unit(const PairDesc &pr, int kx, int ch, float2 *h, const float2 *tw, float2 *S0,
                                        float2 *S1)
{
    constexpr int H = NI / 2, N = NI;
    float2 *base = h + pr.h_off + (long long)kx * N * H + ch * CL;
    FirstInputs<NI, Radix<NI>::r0, CL, TB> in;
    in.load([=](int c, int pos) { return __ldcg(base + (long long)pos * H + c); });
    rr_first<NI, Radix<NI>::r0, true, CL, TB>(in, S0);
    __syncthreads();
    rr_rest<NI, true, CL, TB>(S0, S1, tw, [&](int, int, int c, int pos, float2 v) { base[(long long)pos * H + c] = v; });
}

// Complex-to-real inverse z transform of rows k_y0 .. k_y0 + 31 of plane k_x
// (the layout and packing of k_ifft_z), with the plane's output rows written
// to `out` and/or the block maximum folded into the pair's peak key.
template <int NI>
__device__ __forceinline__ void iz_unit(const PairDesc &pr, int kx, int ky0, const float2 *h, float *out,
                                        unsigned long long *keys, const float2 *tw, float2 *A, float2 *B,
                                        unsigned long long *red)
{
    constexpr int H = NI / 2, N = NI;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 1, odd = lane & 1;
    const float2 *row = h + pr.h_off + ((long long)kx * N + ky0 + lane) * H;
    if (threadIdx.x < CL) A[H * CL + threadIdx.x] = make_float2(0.f, 0.f); // m_z = N/2
    for (int k = 2 * w; k < H; k += 2 * (TB / 32)) {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(row + k));
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
}

// sync: [0] the unit counter, [1, 1 + npairs nch) the X counts per (pair, ch),
// then npairs N IY counts per (pair, k_x); all zero at launch.
template <int NF, int NI, bool SP, int S>
__global__ void __launch_bounds__(TB, (NF <= 256 ? 2 : 1))
k_back(Geometry g, Tables tb, const InstDesc *__restrict__ inst, const InstPlan *__restrict__ plan,
       const PairDesc *__restrict__ pairs, int npairs, const float2 *__restrict__ y1,
       const float2 *__restrict__ fa_cache, float2 *h, float *out, unsigned long long *keys, int G, unsigned *sync,
       int *err)
{
    extern __shared__ float4 sm4[];
    __shared__ unsigned long long red[TB / 32];
    __shared__ int s_unit;
    using XL = XSmem<NF, NI, SP, S>;
    const typename XL::Ptr sm = XL::carve(reinterpret_cast<float2 *>(sm4));
    load_twiddles<NF>(sm.twF, tb.tw_n);
    load_twiddles<NI>(sm.twI, tb.tw_N);
    constexpr int N = NI, nch = NI / 2 / CL, nyb = NI / 32;
    const int per = N * nch; // X and IY units per pair (N * nyb IZ units: the same count)
    const int nx = npairs * per, total = 3 * nx;
    unsigned *next = sync, *cx = sync + 1, *ciy = cx + npairs * nch;
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(next, 1u);
    __syncthreads();
    int u = s_unit;
    while (u < total) {
        __syncthreads(); // every thread has read s_unit
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(next, 1u); // claim the unit after this one
        if (u < nx) {
            const int p = u / per, r = u - p * per, ch = r / N, jy = r - ch * N;
            x_item<NF, NI, SP, S>(g, tb, inst, plan, pairs[p], jy, ch, y1, fa_cache, nullptr, h, G, sm);
            signal_done(cx + p * nch + ch);
        } else if (u < 2 * nx) {
            const int v = u - nx, p = v / per, r = v - p * per, ch = r / N, kx = r - ch * N;
            wait_count(cx + p * nch + ch, N, err);
            iy_unit<NI>(pairs[p], kx, ch, h, sm.twI, sm.S0, sm.S1);
            signal_done(ciy + p * N + kx);
        } else {
            const int v = u - 2 * nx, p = v / per, r = v - p * per, kx = r / nyb, kb = r - kx * nyb;
            wait_count(ciy + p * N + kx, nch, err);
            iz_unit<NI>(pairs[p], kx, kb * 32, h, out, keys, sm.twI, sm.S0, sm.S1, red);
            __syncthreads();
        }
        u = s_unit;
    }
}

template <int NF, int NI, bool SP = false, int S = 0>
cudaError_t back_t(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan, const PairDesc *pairs,
                   int npairs, const float2 *y1, const float2 *fa_cache, float2 *h, float *out,
                   unsigned long long *keys, unsigned *sync, int *err, int nsm, cudaStream_t s)
{
    if (!SP && S == 0 && (g.sched & 4))
        return back_t<NF, NI, false, 1>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    // the x pass's shared-memory layout (level weights for as many levels as fit
    // at the kernel's blocks per SM); the inverse units reuse its tiles
    using XL = XSmem<NF, NI, SP, S>;
    const size_t room = (NF <= 256 ? 228 * 1024 / 2 : 228 * 1024) - 1024 - 512 - XL::bytes(0);
    const int G = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.L, room / XL::per_level));
    const size_t smem = XL::bytes(G);
    cudaError_t e = set_smem(k_back<NF, NI, SP, S>, smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sync, 0, sizeof(unsigned) * back_sync_words(NI, npairs), s)) != cudaSuccess) return e;
    k_back<NF, NI, SP, S><<<resident_blocks(k_back<NF, NI, SP, S>, smem, nsm), TB, smem, s>>>(
        g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, G, sync, err);
    return cudaGetLastError();
}

// One block waits on a count nothing raises: the wait gives up after its two
// seconds and records the expiry (bit 4 of *err).
__global__ void k_queue_wait_selftest(const unsigned *c, int *err) { wait_count(c, 1u, err); }

} // namespace

cudaError_t launch_queue_wait_selftest(unsigned *zeroed, int *err, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(zeroed, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_queue_wait_selftest<<<1, 32, 0, s>>>(zeroed, err);
    return cudaGetLastError();
}

size_t back_sync_words(int N, int npairs) { return 1 + (size_t)npairs * (N / 32) + (size_t)npairs * N; }

cudaError_t launch_back(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                        const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *h,
                        float *out, unsigned long long *keys, unsigned *sync, int *err, int nsm, cudaStream_t s)
{
    if (npairs <= 0) return cudaSuccess;
    if (g.prec == 1) {
        switch (g.N) {
        case 32: return back_t<64, 32, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
        case 64: return back_t<128, 64, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
        case 96: return back_t<192, 96, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
        case 128:
            return back_t<256, 128, true, SplitSched<256>::S>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out,
                                                               keys, sync, err, nsm, s);
        case 256: return back_t<512, 256, true>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (g.N) {
    case 32: return back_t<64, 32>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    case 64: return back_t<128, 64>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    case 96: return back_t<192, 96>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    case 128: return back_t<256, 128>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    case 256: return back_t<512, 256>(g, t, inst, plan, pairs, npairs, y1, fa_cache, h, out, keys, sync, err, nsm, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace bc
