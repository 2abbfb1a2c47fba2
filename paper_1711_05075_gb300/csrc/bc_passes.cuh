// Device pieces of the transform passes shared by the separate-launch kernels
// (bc_kernels.cu) and the persistent back-half kernel (bc_back.cu).  Not part
// of the public interface.
#pragma once
#include <climits>

#include "bc_device.cuh"

namespace bc {

__device__ __forceinline__ int mode_of(int j, int N) { return j < N / 2 ? j : j - N; }

// Asynchronous 16-byte global-to-shared copies (zero-filled when !valid).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recently committed group have landed (for this thread)
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Level-summed spectrum of one instance for the modes owned by this thread
// after the last stage of the x transform: output position pos = j + r NS of
// butterfly (c, j) is kept when r < R/4 (m_x = pos) or r >= 3R/4
// (m_x = pos - n), i.e. exactly m_x in [-N/2, N/2); those slots of F hold
// sum_l T_l(|m|^2) D(m) FFT_x[Y_l](m) for m_y = mode(j_y), m_z = 16 ch + c.
// Level l + 1 is loaded while level l is transformed.
template <int NF, int S>
struct XModes {
    static constexpr int R = LastStage<NF, S>::R, NS = LastStage<NF, S>::NS;
    static constexpr int IT = (NS * CL + TB - 1) / TB;
    static __device__ __forceinline__ constexpr bool kept(int r) { return r < R / 4 || r >= 3 * R / 4; }
};

// Per-item table of the level weights the x pass applies: for the item's m_y
// and its 16 z-modes m_z = 16 ch + c, and a = |m_x| in [0, N/2],
//   Ts[(lg (N/2 + 1) + a) 16 + c] = T_{l0+lg}(a^2 + m_y^2 + m_z^2) D(a) D(m_y) D(m_z),
// lg < nl.  The window transform is even, so D(-a) = D(a) and one entry serves
// m_x = a and m_x = -a; the index a = N/2 addresses m_x = -N/2 in the
// deconvolution table's FFT order.  Built in shared memory by the whole block,
// it replaces the table gathers of every level of both spectra.
template <int NI>
__device__ __forceinline__ void build_xweights(float *Ts, const Tables &tb, int l0, int nl, int jy, int ch)
{
    constexpr int A = NI / 2 + 1;
    const int my = mode_of(jy, NI);
    const float dy = tb.deconv[jy];
    const long long Q = tb.qmax + 1;
    const int tot = nl * A * CL;
    for (int e = threadIdx.x; e < tot; e += TB) {
        const int c = e % CL, a = (e / CL) % A, lg = e / (CL * A);
        const int mz = ch * CL + c;
        Ts[e] = tb.ballft[(l0 + lg) * Q + a * a + my * my + mz * mz] * (tb.deconv[a] * dy * tb.deconv[mz]);
    }
}

// Ts holds the weights of levels [ts_base, ts_base + G) of the current item;
// a level outside that range rebuilds it (after the barrier that ends the
// previous level, before the one that publishes the level's first stage).
template <int NF, int NI, bool SP, int S>
__device__ __forceinline__ void spectrum_x(float2 (&F)[XModes<NF, S>::IT][XModes<NF, S>::R], const Geometry &g,
                                           const Tables &tb, const InstDesc *__restrict__ inst,
                                           const InstPlan *__restrict__ plan, int si, const float2 *__restrict__ y1,
                                           int jy, int ch, const float2 *tw, float2 *S0, float2 *S1, float *Ts, int G,
                                           int &ts_base)
{
    using XM = XModes<NF, S>;
    constexpr int H = NI / 2, N = NI, A = NI / 2 + 1;
    const int L = g.L;
#pragma unroll
    for (int it = 0; it < XM::IT; it++)
#pragma unroll
        for (int r = 0; r < XM::R; r++) F[it][r] = make_float2(0.f, 0.f);
    const InstPlan p = plan[si];
    if (p.b[0] == 0) return;
    const InstDesc d = inst[si];
    const int b0 = p.b[0], px = p.pos0[0];
    auto src = [&](int l) {
        const float2 *base = y1 + d.y1_off + (long long)l * b0 * N * H + (long long)jy * H + ch * CL;
        return [=](int c, int pos) {
            int ix = pos - px;
            if (ix < 0) ix += NF;
            return ix < b0 ? base[(long long)ix * N * H + c] : make_float2(0.f, 0.f);
        };
    };
    FirstInputs<NF, Radix<NF, S>::r0, CL, TB> in;
    in.load(src(0));
    for (int l = 0; l < L; l++) {
        if (l < ts_base || l >= ts_base + G) {
            ts_base = l;
            build_xweights<NI>(Ts, tb, l, min(G, L - l), jy, ch);
        }
        if constexpr (SP) in.scatter(S0);
        else rr_first<NF, Radix<NF, S>::r0, false, CL, TB>(in, S0);
        __syncthreads();
        if (l + 1 < L) in.load(src(l + 1));
        const float *Tl = Ts + (l - ts_base) * A * CL;
        auto sink = [&](int it, int r, int c, int pos, float2 v) {
            if (!XM::kept(r)) return;
            const int mx = r < XM::R / 4 ? pos : pos - NF;
            const float Mv = Tl[(mx < 0 ? -mx : mx) * CL + c];
            F[it][r] = make_float2(fmaf(Mv, v.x, F[it][r].x), fmaf(Mv, v.y, F[it][r].y));
        };
        if constexpr (SP) sp_all<NF, false, CL, TB, S>(S0, S1, tw, sink);
        else rr_rest<NF, false, CL, TB, S>(S0, S1, tw, sink);
        __syncthreads();
    }
}

// Calls f(it, r, c, jx) for every kept mode slot of the calling thread.
template <int NF, int NI, int S, class Fn>
__device__ __forceinline__ void for_kept(Fn f)
{
    using XM = XModes<NF, S>;
#pragma unroll
    for (int it = 0; it < XM::IT; it++) {
        const int idx = (int)threadIdx.x + it * TB;
        if ((XM::NS * CL) % TB != 0 && idx >= XM::NS * CL) break;
        const int c = idx % CL, j = idx / CL;
#pragma unroll
        for (int r = 0; r < XM::R; r++) {
            if (!XM::kept(r)) continue;
            const int pos = j + r * XM::NS;
            const int mx = r < XM::R / 4 ? pos : pos - NF;
            f(it, r, c, mx < 0 ? mx + NI : mx);
        }
    }
}

// ------------------------------------------------------------ staged x pass
// When both instances of a pair have x boxes of at most XStage::MAXR cells
// (the whole line up to n = 128; 5/8 of it, rounded up to whole first-stage
// strides, beyond: 128 of 192, 160 of 256, so that two blocks still fit on an
// SM), an item's rows
// are fetched into two shared-memory staging tiles with asynchronous 16-byte
// copies one (instance, level) phase ahead, so the global loads of the next
// phase overlap the transform of the current one without holding registers.
// Compact index ix sits at position ix of the length-n line (zero beyond the
// box), not at pos0 + ix: the transform then differs from the unshifted one
// by the factor exp(-2 pi i m_x pos0 / n), applied once to each level sum.
// The first stage reads only the XStage::RN inputs per butterfly that can be
// nonzero.
template <int NF, bool SP, int S>
struct XStage {
    static constexpr int R0 = Radix<NF, S>::r0, NB = NF / R0;
    static constexpr int MAXR = NF <= 128 ? NF : ((5 * NF / 8 + NB - 1) / NB) * NB;
    static constexpr int RN = MAXR / NB;
    // where the tiles, the staging tiles and four levels of weights fit two
    // blocks per SM (n = 256 with the 4.8.8 schedule stages 192 rows: too many)
    static constexpr int NI = NF / 2;
    static constexpr size_t bytes4 =
        sizeof(float2) * ((size_t)NF + NI + (size_t)NF * CL * (Radix<NF, S>::r2 == 1 ? 1 : 2) + (size_t)NI * CL +
                          2 * (size_t)MAXR * CL) +
        sizeof(float) * 4 * (NI / 2 + 1) * CL;
    static constexpr bool on = !SP && NF <= 256 && bytes4 <= 113 * 1024;
};

// Shared-memory layout of the x pass (float2 units unless stated):
// twF [NF], twI [NI], S0 [NF CL], S1 [NF CL] (two-stage staged schedules: S1
// is only the inverse transform's scratch and lives in FAt), FAt [NI CL],
// staging tiles 2 x [MAXR CL] (staged passes), then G levels of weights
// (floats, (NI/2 + 1) CL per level).
template <int NF, int NI, bool SP, int S>
struct XSmem {
    static constexpr bool staged = XStage<NF, SP, S>::on;
    static constexpr bool alias_s1 = staged && Radix<NF, S>::r2 == 1;
    static constexpr int MAXR = staged ? XStage<NF, SP, S>::MAXR : 0;
    static constexpr size_t f2 = (size_t)NF + NI + (size_t)NF * CL + (alias_s1 ? 0 : (size_t)NF * CL) +
                                 (size_t)NI * CL + 2 * (size_t)MAXR * CL;
    static constexpr size_t per_level = sizeof(float) * (NI / 2 + 1) * CL;
    static constexpr size_t bytes(int G) { return sizeof(float2) * f2 + per_level * (size_t)G; }
    struct Ptr {
        float2 *twF, *twI, *S0, *S1, *FAt, *stg0, *stg1;
        float *Ts;
    };
    static __device__ __forceinline__ Ptr carve(float2 *base)
    {
        Ptr p;
        p.twF = base;
        p.twI = p.twF + NF;
        p.S0 = p.twI + NI;
        p.FAt = p.S0 + (size_t)NF * CL + (alias_s1 ? 0 : (size_t)NF * CL);
        p.S1 = alias_s1 ? p.FAt : p.S0 + (size_t)NF * CL;
        p.stg0 = p.FAt + (size_t)NI * CL;
        p.stg1 = p.stg0 + (size_t)MAXR * CL;
        p.Ts = reinterpret_cast<float *>(p.stg1 + (size_t)MAXR * CL);
        return p;
    }
};

// First stage from a staging tile: butterfly (c, j) of the first radix-R0
// stage reads rows j + r NB; rows at or beyond MAXR are zero (r >= RN).
template <int NF, bool SP, int S>
__device__ __forceinline__ void xs_first(const float2 *__restrict__ stg, float2 *__restrict__ out)
{
    using XS = XStage<NF, SP, S>;
    constexpr int R = XS::R0, NB = XS::NB, TOT = NB * CL, IT = (TOT + TB - 1) / TB;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = (int)threadIdx.x + it * TB;
        if ((TOT % TB) != 0 && idx >= TOT) break;
        const int c = idx % CL, j = idx / CL;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = r < XS::RN ? stg[(j + r * NB) * CL + c] : make_float2(0.f, 0.f);
        dft_small<R, false>(v);
#pragma unroll
        for (int r = 0; r < R; r++) out[(j * R + r) * CL + c] = v[r];
    }
}

// exp(-2 pi i m px / NF) from the forward twiddle table (m may be negative).
template <int NF>
__device__ __forceinline__ float2 box_phase(const float2 *twF, int m, int px)
{
    const int k = ((m + NF) * px) % NF;
    return twF[k];
}

// The x-pass item of x_item (below) on staged rows; same result up to rounding.
template <int NF, int NI, bool SP, int S>
__device__ __forceinline__ void x_item_staged(const Geometry &g, const Tables &tb, const InstDesc *__restrict__ inst,
                                              const InstPlan *__restrict__ plan, const PairDesc &pr, int jy, int ch,
                                              const float2 *__restrict__ y1, const float2 *__restrict__ fa_cache,
                                              float2 *fa_out, float2 *h, int G, const typename XSmem<NF, NI, SP, S>::Ptr &sm)
{
    using XM = XModes<NF, S>;
    using XS = XStage<NF, SP, S>;
    constexpr int H = NI / 2, N = NI, A = NI / 2 + 1;
    const int L = g.L;
    const int part = threadIdx.x & 7, r8 = threadIdx.x >> 3;
    const int my = mode_of(jy, N);
    const bool hasA = pr.a >= 0, hasB = pr.b >= 0;
    const int nph = ((hasA ? 1 : 0) + (hasB ? 1 : 0)) * L;
    auto inst_of = [&](int ph) { return (hasA && ph < L) ? pr.a : pr.b; };
    // rows of phase ph (instance inst_of(ph), level ph mod L) into a staging tile
    auto fetch = [&](int ph, float2 *dst) {
        const int si = inst_of(ph), l = ph < L ? ph : ph - L;
        const int b0 = plan[si].b[0];
        const float2 *base = y1 + inst[si].y1_off + (long long)l * b0 * N * H + (long long)jy * H + ch * CL;
        for (int q = threadIdx.x; q < XS::MAXR * (CL / 2); q += TB) {
            const int row = q / (CL / 2), cc = (q % (CL / 2)) * 2;
            const bool ok = row < b0;
            cp_async16(dst + row * CL + cc, ok ? base + (long long)row * N * H + cc : base, ok);
        }
    };
    float2 F[XM::IT][XM::R];
    auto zero_f = [&]() {
#pragma unroll
        for (int it = 0; it < XM::IT; it++)
#pragma unroll
            for (int r = 0; r < XM::R; r++) F[it][r] = make_float2(0.f, 0.f);
    };
    zero_f();
    if (!hasA) { // F_A from the cached spectrum (already in place)
        for_kept<NF, NI, S>([&](int, int, int c, int jx) {
            sm.FAt[jx * CL + c] = fa_cache[((long long)jx * N + jy) * H + ch * CL + c];
        });
    }
    int ts_base = INT_MIN / 2; // no level weights built for this item yet
    if (tb.xw && G >= L) {     // the item's weight slice comes with the first rows
        constexpr int nch = NI / 2 / CL;
        const float *src = tb.xw + (long long)(jy * nch + ch) * L * A * CL;
        for (int q = threadIdx.x; q < L * A * CL / 4; q += TB) cp_async16(sm.Ts + 4 * q, src + 4 * q, true);
        ts_base = 0;
    }
    fetch(0, sm.stg0);
    cp_async_commit();
    for (int ph = 0; ph < nph; ph++) {
        const float2 *cur = (ph & 1) ? sm.stg1 : sm.stg0;
        // the other tile was last read by the previous phase's first stage
        if (ph + 1 < nph) fetch(ph + 1, (ph & 1) ? sm.stg0 : sm.stg1);
        cp_async_commit();
        cp_async_wait_prev();
        const int l = ph < L ? ph : ph - L;
        if (l < ts_base || l >= ts_base + G) {
            ts_base = l;
            build_xweights<NI>(sm.Ts, tb, l, min(G, L - l), jy, ch);
        }
        __syncthreads(); // this phase's rows (every thread's copies) have landed
        xs_first<NF, SP, S>(cur, sm.S0);
        __syncthreads();
        const float *Tl = sm.Ts + (l - ts_base) * A * CL;
        auto sink = [&](int it, int r, int c, int pos, float2 v) {
            if (!XM::kept(r)) return;
            const int mx = r < XM::R / 4 ? pos : pos - NF;
            const float Mv = Tl[(mx < 0 ? -mx : mx) * CL + c];
            F[it][r] = make_float2(fmaf(Mv, v.x, F[it][r].x), fmaf(Mv, v.y, F[it][r].y));
        };
        rr_rest<NF, false, CL, TB, S>(sm.S0, sm.S1, sm.twF, sink);
        __syncthreads();
        if (l == L - 1) { // this instance's level sum is complete: restore its box origin
            const int px = plan[inst_of(ph)].pos0[0];
            const bool isA = hasA && ph < L;
            for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) {
                const int mx = jx < N / 2 ? jx : jx - N;
                const float2 v = cmul(F[i2][r], box_phase<NF>(sm.twF, mx, px));
                if (isA) sm.FAt[jx * CL + c] = v;
                else F[i2][r] = v;
            });
            if (isA) zero_f();
        }
    }
    if (!hasB) {
        for_kept<NF, NI, S>([&](int, int, int c, int jx) {
            fa_out[((long long)jx * N + jy) * H + ch * CL + c] = sm.FAt[jx * CL + c];
        });
        return;
    }
    for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) {
        const int mx = mode_of(jx, N), mz = ch * CL + c;
        float2 v = make_float2(0.f, 0.f);
        if (jx != N / 2 && jy != N / 2) {
            v = cmulc(sm.FAt[jx * CL + c], F[i2][r]);
            v = cscale(v, ((mx + my + mz) & 1) ? -g.inv_P3 : g.inv_P3);
        }
        sm.S0[jx * CL + c] = v;
    });
    __syncthreads();
    const float2 *res = il_fft<NI, true, CL, TB>(sm.S0, sm.S1, sm.twI);
    float2 *Hp = h + pr.h_off + (long long)jy * H + ch * CL + 2 * part;
    for (int kx = r8; kx < N; kx += TB / 8)
        *reinterpret_cast<float4 *>(Hp + (long long)kx * N * H) = *reinterpret_cast<const float4 *>(res + kx * CL + 2 * part);
    __syncthreads();
}

// One x-pass item of pair `pr`: row j_y and z-modes 16 ch .. 16 ch + 15.
//   F_s(m) = sum_l T_l(|m|^2) D(m) FFT_x[Y_{s,l}](m)    (s = A, B)
//   g'(m)  = P^-3 (-1)^(m_x+m_y+m_z) F_A(m) conj(F_B(m)), zero on the Nyquist planes
//   H(k_x, j_y, m_z) = sum_{j_x} g'(m) exp(+2 pi i j_x k_x / N)
// D(m) = deconv[j_x] deconv[j_y] deconv[m_z].  The sign moves the origin of the
// translation grid to t = -P/2: exp(2 pi i m (-P/2) / P) = (-1)^m.
// With pr.a < 0, F_A comes from the cached spectrum; with pr.b < 0, F_A is
// written to `fa_out` and nothing else happens.  All threads call it; it ends
// with a block barrier except when pr.b < 0.
template <int NF, int NI, bool SP, int S>
__device__ __forceinline__ void x_item(const Geometry &g, const Tables &tb, const InstDesc *__restrict__ inst,
                                       const InstPlan *__restrict__ plan, const PairDesc &pr, int jy, int ch,
                                       const float2 *__restrict__ y1, const float2 *__restrict__ fa_cache,
                                       float2 *fa_out, float2 *h, int G, const typename XSmem<NF, NI, SP, S>::Ptr &sm)
{
    if constexpr (XStage<NF, SP, S>::on) {
        constexpr int MAXR = XStage<NF, SP, S>::MAXR;
        if ((pr.a < 0 || plan[pr.a].b[0] <= MAXR) && (pr.b < 0 || plan[pr.b].b[0] <= MAXR)) {
            x_item_staged<NF, NI, SP, S>(g, tb, inst, plan, pr, jy, ch, y1, fa_cache, fa_out, h, G, sm);
            return;
        }
    }
    using XM = XModes<NF, S>;
    constexpr int H = NI / 2, N = NI;
    const float2 *twF = sm.twF, *twI = sm.twI;
    float2 *S0 = sm.S0, *S1 = sm.S1, *FAt = sm.FAt;
    float *Ts = sm.Ts;
    const int part = threadIdx.x & 7, r8 = threadIdx.x >> 3;
    const int my = mode_of(jy, N);
    int ts_base = INT_MIN / 2; // no level weights built for this item yet
    // F_A waits in its own tile (each thread reads back only what it wrote)
    // while F_B is accumulated in registers.
    {
        float2 FA[XM::IT][XM::R];
        if (pr.a < 0) {
            for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) {
                FAt[jx * CL + c] = fa_cache[((long long)jx * N + jy) * H + ch * CL + c];
            });
        } else {
            spectrum_x<NF, NI, SP, S>(FA, g, tb, inst, plan, pr.a, y1, jy, ch, twF, S0, S1, Ts, G, ts_base);
            for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) { FAt[jx * CL + c] = FA[i2][r]; });
        }
    }
    if (pr.b < 0) {
        for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) {
            fa_out[((long long)jx * N + jy) * H + ch * CL + c] = FAt[jx * CL + c];
        });
        return;
    }
    float2 FB[XM::IT][XM::R];
    spectrum_x<NF, NI, SP, S>(FB, g, tb, inst, plan, pr.b, y1, jy, ch, twF, S0, S1, Ts, G, ts_base);
    for_kept<NF, NI, S>([&](int i2, int r, int c, int jx) {
        const int mx = mode_of(jx, N), mz = ch * CL + c;
        float2 v = make_float2(0.f, 0.f);
        if (jx != N / 2 && jy != N / 2) {
            v = cmulc(FAt[jx * CL + c], FB[i2][r]);
            v = cscale(v, ((mx + my + mz) & 1) ? -g.inv_P3 : g.inv_P3);
        }
        S0[jx * CL + c] = v;
    });
    __syncthreads();
    const float2 *res = il_fft<NI, true, CL, TB>(S0, S1, twI);
    float2 *Hp = h + pr.h_off + (long long)jy * H + ch * CL + 2 * part;
    for (int kx = r8; kx < N; kx += TB / 8)
        *reinterpret_cast<float4 *>(Hp + (long long)kx * N * H) = *reinterpret_cast<const float4 *>(res + kx * CL + 2 * part);
    __syncthreads();
}

// Peak keys: an order-preserving map of the FP32 value to the high 32 bits
// (negative values bit-inverted, non-negative ones with the sign bit set) and
// the complement of the linear grid index in the low 32 bits, so that the
// maximum key is the largest value and, among equal values, the lowest index.
__device__ __forceinline__ unsigned long long peak_key(float v, unsigned idx)
{
    unsigned u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

} // namespace bc
